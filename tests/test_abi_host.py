"""C-ABI library: builds for sm_103a, loads, exports every symbol the public
header declares, and rejects bad arguments on the host before touching CUDA.
No compute call is made here (no GPU in this environment)."""
import ctypes as C
import math
import os
import re

import pytest

from paper_1908_04279_gb300 import build as B
from paper_1908_04279_gb300 import mm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mm.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:mm_status|const\s+char\s*\*|void|int)\s+\**\s*(mm_\w+)\s*\(",
                                 src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mm.load_library()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("mm_create", "mm_destroy", "mm_set_state", "mm_get_state", "mm_set_velocity",
              "mm_micro_step", "mm_moments", "mm_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    raw = C.CDLL(B.LIB)
    missing = [s for s in declared_symbols() if not hasattr(raw, s)]
    assert not missing, missing
    # and the binding declares a prototype for each of them
    assert set(declared_symbols()) <= set(mm.PROTOTYPES)


def _create(lib, grid=(4, 4, 4, 4, 1.0), rates=None, prec=mm.MM_FP64):
    g = mm.mm_grid(*grid)
    r = rates or mm.mm_rates(1.0, 1.0, 0.5, 0.05, 0.0, 1.0, 1.0, 0.4)
    h = C.c_void_p()
    st = lib.mm_create(C.byref(g), C.byref(r), prec, None, C.byref(h))
    return st, h


@pytest.mark.parametrize("grid,code", [
    ((0, 4, 4, 4, 1.0), 1), ((4, -1, 4, 4, 1.0), 1), ((4, 4, 0, 4, 1.0), 1),
    ((4, 4, 4, 0, 1.0), 1), ((4, 4, 4, 4, 0.0), 1), ((4, 4, 4, 4, float("nan")), 1),
    ((4, 4, 2000, 4, 1.0), 4), ((4, 4, 4, 65, 1.0), 4)])
def test_create_rejects_bad_grid(lib, grid, code):
    st, h = _create(lib, grid)
    assert st == code and not h.value
    assert lib.mm_last_error(None)


def test_create_rejects_bad_rates(lib):
    bad = [mm.mm_rates(-1.0, 1, 0.5, 0, 0, 1, 1, 0.4),          # v_walk < 0: unsupported
           mm.mm_rates(1, -1, 0.5, 0, 0, 1, 1, 0.4),            # k_on < 0
           mm.mm_rates(1, 1, math.nan, 0, 0, 1, 1, 0.4),        # NaN
           mm.mm_rates(1, 1, 0.5, 0, 0, 1, 1, 0.0)]             # cfl = 0
    codes = [4, 1, 1, 1]
    for r, code in zip(bad, codes):
        st, h = _create(lib, rates=r)
        assert st == code and not h.value


def test_ns_limit_depends_on_precision(lib):
    st, _ = _create(lib, (4, 4, 4, 129, 1.0), prec=mm.MM_FP32_MIXED)
    assert st == 4
    st, _ = _create(lib, (4, 4, 4, 100, 1.0), prec=mm.MM_FP64)
    assert st == 4


def test_null_handle_calls_are_invalid(lib):
    assert lib.mm_destroy(None) == 1
    assert lib.mm_micro_step(None, 1) == 1
    assert lib.mm_set_dt(None, 1.0) == 1
    assert lib.mm_motor_local(None, 0.1, None, None, 0) == 1
    assert lib.mm_set_anchors(None, 1) == 1
    assert lib.mm_fluid_setup(None, 0.1, 0.1) == 1
    assert lib.mm_fluid_solve(None, None, 0, 0, None, 0) == 1
    assert lib.mm_fluid_response(None, None, 0) == 1
    assert lib.mm_diffuse(None, 0.1, 0.1, 0.1) == 1
    assert lib.mm_sync(None) == 1
    assert lib.mm_build_info().startswith(b"libmm sm_103a")
