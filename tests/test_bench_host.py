"""The benchmark's byte accounting and its use of the committed ncu summaries,
on CPU: the algorithmic bytes per substep launch against the per-unit figures
of the fused substep (each motor value read and written once; psi and n_b of
each (cell, theta) read and written once; a few scalars per cell), and the rule
that a summary's DRAM traffic is reported only when it was taken on the current
kernel sources."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1908_04279_gb300.inputs import Grid  # noqa: E402


@pytest.fixture()
def bench():
    import bench as b
    return b


@pytest.mark.parametrize("dims,tsize,expected", [
    # float32, 512^2 x 64^2: 8 B per motor value (read + write), 24 B per
    # (cell, theta) (psi and n_b read + written), 40 B per cell (Mf read and
    # written, C written, M read, the velocity block)
    ((512, 512, 64, 64), 4, 262144 * 4096 * 8 + 262144 * 64 * 24 + 262144 * 40),
    # float32, 128^2 x 32^2: the 147.456 MB per launch of the L2-resident case
    ((128, 128, 32, 32), 4, 147456000),
    # float64: 16 B per motor value, 32 B per (cell, theta), 48 B per cell
    ((64, 64, 32, 32), 8, 4096 * 1024 * 16 + 4096 * 32 * 32 + 4096 * 48),
])
def test_algorithmic_bytes_per_launch(bench, dims, tsize, expected):
    assert bench.algorithmic_bytes_per_launch(Grid(*dims), tsize) == expected


def test_large512_bytes_equal_the_headline_figure(bench):
    assert bench.algorithmic_bytes_per_launch(Grid(512, 512, 64, 64), 4) == 9003073536


def _summary(path, sha, dram=None):
    lines = ["# k_substep (float32 form)", "", f"kernel_source_sha256: {sha}"]
    if dram is not None:
        lines.append(f"| dram_bytes_per_launch: {dram} | (read + write) |")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def test_profile_traffic_only_for_the_current_sources(bench, tmp_path, monkeypatch):
    """A summary's DRAM bytes are used (scaled) when its source hash is the
    current one, and ignored when the hash differs, the summary is missing or
    it carries no traffic line."""
    current, stale = "a" * 64, "b" * 64
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sha", lambda kernel: current)
    prof = tmp_path / "profiles"
    prof.mkdir()
    _summary(prof / "k_substep_large512_fp32.md", current, 8683460000)
    assert bench.read_profile_traffic("k_substep", "large512", "fp32") == 8683460000.0
    assert bench.read_profile_traffic("k_substep", "large512", "fp32", 4.0) == 4 * 8683460000.0
    _summary(prof / "k_substep_large512_fp32.md", stale, 8683460000)
    assert bench.read_profile_traffic("k_substep", "large512", "fp32") is None
    assert bench.read_profile_traffic("k_substep", "precision128", "fp32") is None
    _summary(prof / "k_substep_precision128_fp32.md", current)
    assert bench.read_profile_traffic("k_substep", "precision128", "fp32") is None


def test_kernel_hash_covers_every_listed_source(bench, tmp_path, monkeypatch):
    """Changing any one file of a kernel's source list changes its hash."""
    src = tmp_path / "csrc"
    src.mkdir()
    files = bench.KERNEL_SRCS["k_substep"]
    for f in files:
        (src / f).write_text(f"// {f}\n")
    monkeypatch.setattr(bench, "CSRC", str(src))
    base = bench.kernel_sha("k_substep")
    for f in files:
        (src / f).write_text(f"// {f} changed\n")
        assert bench.kernel_sha("k_substep") != base, f
        (src / f).write_text(f"// {f}\n")
    assert bench.kernel_sha("k_substep") == base


def test_float64_operation_split(bench):
    """The float64 roofline counts the scheme's operations per cell-update; of
    them, the sign transfers, minima and maximum of both stages (10) run on the
    integer pipe and the rest on the float64 pipe."""
    assert bench.SUBSTEP_OPS == 2 * 11 + 1
    assert bench.SUBSTEP_FP64_PIPE_OPS == bench.SUBSTEP_OPS - 2 * 5
