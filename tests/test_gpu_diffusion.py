"""Filament diffusion (mm_diffuse): Crank-Nicolson per direction against the
float64 oracle's dense solves, then the re-derived C, scale-down and Mf.

* float64 to 1e-12 and float32 to 1e-5 on ragged grids (directions of 2, 5,
  6, 7, 9 points), with bound motors from earlier substeps (n_b != 0), a
  forced scale-down, and in float32 a pending mass-correction factor;
* a Fourier mode decays by the closed-form factor on the GPU;
* a direction of one point is left alone; zero diffusivity is the identity;
* diffusion is refused during an adjoint recording.
"""
import math

import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import Grid, Rates, psi_isotropic_perturbed, random_divfree_flow

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_04279_gb300 import build as B
    B.build()
    from paper_1908_04279_gb300 import mm
    return mm


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("dims", [(9, 7, 6, 8), (5, 12, 16, 4), (2, 6, 5, 4)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_diffuse_matches_oracle(mmod, oracle_mod, dims, precision, tol):
    g = Grid(*dims, L=1.0)
    r = Rates(k_on=2.0, k_off=0.5, glide=0.3)
    psi0 = psi_isotropic_perturbed(g, 51, amp=0.4)
    u = random_divfree_flow(g, 52, 4, 0.3)
    D_t, D_r, dt = 0.004, 0.6, 0.07
    with mmod.Simulation(g, r, precision) as sim:
        sim.set_state(psi0)
        sim.set_velocity(u)
        sim.step(7)  # bound motors and, in float32, a pending correction factor
        before = sim.get_state()
        sim.diffuse(D_t, D_r, dt)
        after = sim.get_state()
        sim.step(3)  # the state stays usable
        sim.sync()
    psi_ref = oracle_mod.diffuse(g, before["psi"], D_t, D_r, dt)
    o = oracle_mod.make_state(g, psi_ref, before["mb"])
    assert rel(after["psi"], psi_ref) <= tol, rel(after["psi"], psi_ref)
    assert rel(after["mb"], o.mb) <= tol
    assert rel(after["mf"], o.mf) <= tol
    assert rel(after["c"], o.c) <= tol


def test_diffuse_forced_scale_down(mmod, oracle_mod):
    """Few total motors: after diffusion the coarse density exceeds M in some
    cells and the rows are scaled down (Alg. 2), as in the oracle."""
    g = Grid(8, 6, 8, 8, L=1.0)
    psi0 = psi_isotropic_perturbed(g, 53, amp=0.6)
    rng = np.random.default_rng(54)
    mb = 0.05 * rng.random((g.ny, g.nx, g.ntheta, g.ns))
    dth, ds = 2 * math.pi / g.ntheta, g.L / g.ns
    C0 = np.einsum("yxk,yxkj->yx", psi0, mb) * dth * ds
    mtot = C0 * 1.0000001  # just above the coarse density: diffusion pushes some cells over
    with mmod.Simulation(g, Rates(), "fp64") as sim:
        sim.set_state(psi0, mb, mtot)
        before = sim.get_state()
        sim.diffuse(0.02, 2.0, 0.1)
        after = sim.get_state()
    psi_ref = oracle_mod.diffuse(g, before["psi"], 0.02, 2.0, 0.1)
    o = oracle_mod.make_state(g, psi_ref, before["mb"], mtot)
    assert np.any(o.mf == 0.0)  # some cells clipped
    for k, ref in (("psi", psi_ref), ("mb", o.mb), ("mf", o.mf), ("c", o.c)):
        assert rel(after[k], ref) <= 1e-12, (k, rel(after[k], ref))


def test_diffuse_fourier_mode_and_degenerate_directions(mmod):
    g = Grid(10, 12, 16, 4, L=1.0)
    x = (np.arange(g.nx) + 0.5) / g.nx
    y = (np.arange(g.ny) + 0.5) / g.ny
    th = np.arange(g.ntheta) * 2 * np.pi / g.ntheta
    psi = 1.0 + 0.1 * (np.cos(2 * np.pi * 3 * y)[:, None, None] * np.cos(2 * np.pi * 2 * x)[None, :, None]
                       * np.cos(5 * th)[None, None, :])
    D_t, D_r, dt = 0.003, 0.7, 0.05

    def amp(n, h, D, m):
        q = D * dt / h ** 2 * (1 - np.cos(2 * np.pi * m / n))
        return (1 - q) / (1 + q)
    fac = amp(g.nx, 1 / g.nx, D_t, 2) * amp(g.ny, 1 / g.ny, D_t, 3) * amp(
        g.ntheta, 2 * np.pi / g.ntheta, D_r, 5)
    with mmod.Simulation(g, Rates(), "fp64") as sim:
        sim.set_state(psi)
        sim.diffuse(D_t, D_r, dt)
        got = sim.get_state()["psi"]
        sim.set_state(psi)
        sim.diffuse(0.0, 0.0, dt)
        same = sim.get_state()["psi"]
    assert np.max(np.abs(got - (1.0 + fac * (psi - 1.0)))) <= 1e-13
    assert np.array_equal(same, psi)
    g1 = Grid(1, 6, 8, 4, L=1.0)  # one column in x: that direction is a single point
    p1 = psi_isotropic_perturbed(g1, 55, amp=0.3)
    with mmod.Simulation(g1, Rates(), "fp64") as sim:
        sim.set_state(p1)
        sim.diffuse(0.01, 0.2, 0.1)
        got1 = sim.get_state()["psi"]
    from oracle import oracle as O
    assert rel(got1, O.diffuse(g1, p1, 0.01, 0.2, 0.1)) <= 1e-12


def test_diffuse_refused_while_recording(mmod):
    g = Grid(6, 6, 8, 8, L=1.0)
    with mmod.Simulation(g, Rates(), "fp64") as sim:
        sim.set_state(psi_isotropic_perturbed(g, 56))
        sim.set_velocity(random_divfree_flow(g, 57, 4, 0.2))
        sim.set_checkpointing(2, 4)
        with pytest.raises(mmod.MMError) as ei:
            sim.diffuse(0.01, 0.1, 0.1)
        assert ei.value.status == 7
        with pytest.raises(mmod.MMError):
            sim.diffuse(-1.0, 0.1, 0.1)
