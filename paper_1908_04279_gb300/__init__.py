"""GB300-native microscale kinetic step of the micro-macro gliding-assay model
(Cook & Shinar, arXiv:1908.04279): hand-written sm_103a CUDA kernels behind a
C ABI (include/mm.h), with a thin Python binding (`mm`).

Importing the package loads nothing; `paper_1908_04279_gb300.mm` loads the
CUDA library on first use and raises if it is missing.
"""
__all__ = ["inputs", "mm", "build"]
