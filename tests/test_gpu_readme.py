"""The README's Alg. 1 loop (fluid solve, substeps, filament diffusion, moments)
through the C ABI at 32^2 x 16^2, float32: it runs, and the filament number and
the motor number stay fixed (the per-substep mass correction; bound + free = M)."""
import math

import pytest

from paper_1908_04279_gb300.inputs import Grid, Rates, psi_isotropic_perturbed

pytestmark = pytest.mark.gpu


def test_readme_macro_loop():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_04279_gb300 import build as B
    B.build()
    from paper_1908_04279_gb300 import mm
    g = Grid(32, 32, 16, 16)
    sim = mm.Simulation(g, Rates(), "fp32")
    sim.set_state(psi_isotropic_perturbed(g, 0))
    sim.fluid_setup(eps=0.1, z0=0.1)
    for _ in range(3):
        sim.fluid_solve(dipole=True, u_out=None)
        sim.step(50)
        sim.diffuse(1e-3, 0.1, 50 * sim.dt)
    fields, scalars = sim.moments()
    sim.close()
    assert all(math.isfinite(v) for v in scalars.values())
    assert abs(scalars["N_psi"] - 1.0) <= 1e-6
    assert abs(scalars["motors"] - 1.0) <= 1e-6
    assert scalars["bound"] > 0.0
