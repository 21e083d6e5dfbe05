"""The CUDA library's per-mode fluid response (fl_mode_response in
mm_fluid.cu, compiled for the host by nvcc) against the fluid oracle
(oracle/fluid.py), without a GPU: the two solve the transformed Eq. 7-9 by
different routes (an 8 x 8 system for w with bounded exponential bases, and
multiple shooting of the u, w, q system). Relative agreement <= 1e-13 over
eps from 0.05 to 3 (through eps = 1, where the bases' divided difference
takes over), z0 from 0.02 to 0.9 and kappa up to 700; beyond, against the
closed free-space limits where the walls are far (kappa up to 1e5)."""
import math
import os
import shutil
import subprocess

import pytest

from oracle import fluid as FL

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("fluid_host") / "fluid_mode_host")
    subprocess.check_call([nvcc, "-std=c++17", "-O2", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_1908_04279_gb300", "csrc"),
                           "-gencode", "arch=compute_103a,code=sm_103a",
                           os.path.join(HERE, "fluid_mode_host.cu"), "-o", exe, "-lcufft"])
    return exe


def run(exe, eps, z0, kappas):
    out = subprocess.check_output([exe, repr(eps), repr(z0)] + [repr(k) for k in kappas], text=True)
    return [tuple(map(float, line.split()[1:])) for line in out.split("\n") if line]


@pytest.mark.parametrize("eps", [0.05, 0.1, 0.5, 0.999, 1.0, 1.001, 1.3, 3.0])
@pytest.mark.parametrize("z0", [0.02, 0.1, 0.37, 0.5, 0.9])
def test_cuda_response_matches_oracle(harness, eps, z0):
    kappas = [0.0, 2 * math.pi, 2 * math.pi * math.sqrt(2), 30.0, 150.0, 700.0]
    for k, (gT, gL) in zip(kappas, run(harness, eps, z0, kappas)):
        oT, oL = FL.mode_response(k, eps, z0)
        assert abs(gT - oT) <= 1e-13 * oT and abs(gL - oL) <= 1e-13 * oL, (k, gT, oT, gL, oL)


@pytest.mark.parametrize("eps", [0.1, 1.0, 2.0])
def test_cuda_response_free_space_limit(harness, eps):
    z0 = 0.3
    kappas = [1e3, 1e4, 1e5]
    for k, (gT, gL) in zip(kappas, run(harness, eps, z0, kappas)):
        assert eps * k * z0 > 20
        assert abs(gT - eps / (2 * k)) <= 1e-13 * gT
        assert abs(gL - eps * eps / (2 * k * (1 + eps))) <= 1e-13 * gL
