"""GPU parity of the thin-gap fluid solve (mm_fluid_setup / mm_fluid_solve,
Eq. 7-9) against the float64 fluid oracle (oracle/fluid.py) fed with the
oracle's own moments of the same state (oracle.moments: the motor force of
Eq. 10, the dipole stress sigma_a).

Tolerances: the per-mode response table <= 1e-12 relative per entry (both
sides solve the same ODE exactly, by different routes: the CUDA table an 8 x 8
system in w, the oracle multiple shooting in u, w, q); the velocity <= 1e-12
relative L2 in float64 (cuFFT and numpy's FFT round differently) and <= 1e-5
in float32 (the force comes from the float32 state).
"""
import math

import numpy as np
import pytest

from oracle import fluid as FL
from paper_1908_04279_gb300.inputs import Grid, Rates, SplitMix64, psi_isotropic_perturbed

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def mmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_04279_gb300 import build as B
    B.build()
    from paper_1908_04279_gb300 import mm
    mm.load_library()
    return mm


def rel_l2(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def seeded(g, seed, mb_scale=0.3):
    rng = SplitMix64(seed)
    psi = psi_isotropic_perturbed(g, seed, amp=0.4)
    mb = mb_scale * rng.uniforms(g.ny * g.nx * g.ntheta * g.ns).reshape(g.ny, g.nx, g.ntheta, g.ns)
    return psi, mb


def oracle_velocity(O, g, r, psi, mb, eps, z0, dipole=False, sigma=None, anchors=False):
    if anchors:
        st = O.make_state_anchor(g, r, psi, mb)
        F = O.anchor_force(g, r, st)
        S = None
    else:
        st = O.make_state(g, psi, mb)
        f, _ = O.moments(g, r, st)
        F = np.stack([f["Fx"], f["Fy"]])
        S = -np.stack([f["Sxx"], f["Sxy"], f["Syy"]]) if dipole else None
    if sigma is not None:
        S = sigma if S is None else S + sigma
    return FL.velocity(eps, z0, F, S), st


@pytest.mark.parametrize("nx,ny,eps,z0", [(12, 10, 0.1, 0.1), (9, 7, 0.5, 0.3), (24, 20, 1.0, 0.05),
                                          (16, 15, 2.0, 0.5), (2, 2, 0.3, 0.2)])
def test_response_table_matches_oracle(mmod, nx, ny, eps, z0):
    g = Grid(nx, ny, 8, 8)
    with mmod.Simulation(g, Rates(), "fp64") as sim:
        sim.fluid_setup(eps, z0)
        tab = sim.fluid_response()
    ref = FL.response_table(nx, ny, eps, z0)
    assert tab.shape == ref.shape
    assert np.max(np.abs(tab - ref) / ref) <= 1e-12


def test_response_table_samples_large_grid(mmod):
    """512 x 512: sampled modes up to the largest |k| (2 pi 256 sqrt 2)."""
    g = Grid(512, 512, 4, 4)
    eps, z0 = 0.1, 0.1
    with mmod.Simulation(g, Rates(), "fp32") as sim:
        sim.fluid_setup(eps, z0)
        tab = sim.fluid_response()
    rng = np.random.default_rng(5)
    picks = [(0, 0), (256, 256), (1, 0), (0, 1), (511, 3), (256, 0)] + \
        [(int(a), int(b)) for a, b in zip(rng.integers(0, 512, 10), rng.integers(0, 257, 10))]
    for jy, jx in picks:
        my = jy if jy <= 256 else jy - 512
        ref = FL.mode_response(2 * math.pi * math.hypot(jx, my), eps, z0)
        assert np.max(np.abs(tab[jy, jx] - ref) / np.asarray(ref)) <= 1e-12, (jy, jx)


@pytest.mark.parametrize("dims,eps,z0", [((12, 10, 8, 16), 0.1, 0.1), ((9, 7, 16, 8), 0.5, 0.3),
                                         ((24, 20, 8, 8), 1.0, 0.05), ((16, 15, 12, 10), 2.0, 0.5)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_velocity_matches_oracle(mmod, oracle_mod, dims, eps, z0, precision):
    g = Grid(*dims)
    r = Rates(ell=0.2)
    psi, mb = seeded(g, 301 + sum(dims))
    ref, _ = oracle_velocity(oracle_mod, g, r, psi, mb, eps, z0)
    with mmod.Simulation(g, r, precision) as sim:
        sim.set_state(psi, np.ascontiguousarray(mb))
        sim.fluid_setup(eps, z0)
        u = sim.fluid_solve()
    assert np.abs(ref).max() > 0
    assert rel_l2(u, ref) <= TOL[precision], rel_l2(u, ref)


@pytest.mark.parametrize("dims", [(12, 10, 8, 16), (9, 8, 16, 8)])
def test_dipole_and_extra_stress(mmod, oracle_mod, dims):
    g = Grid(*dims)
    r = Rates(ell=0.3)
    eps, z0 = 0.2, 0.15
    psi, mb = seeded(g, 311 + sum(dims))
    sigma = np.random.default_rng(312).standard_normal((3, g.ny, g.nx)) * 0.05
    with mmod.Simulation(g, r, "fp64") as sim:
        sim.set_state(psi, np.ascontiguousarray(mb))
        sim.fluid_setup(eps, z0)
        u_d = sim.fluid_solve(dipole=True)
        u_s = sim.fluid_solve(sigma=sigma)
        u_ds = sim.fluid_solve(sigma=sigma, dipole=True)
    ref_d, _ = oracle_velocity(oracle_mod, g, r, psi, mb, eps, z0, dipole=True)
    ref_s, _ = oracle_velocity(oracle_mod, g, r, psi, mb, eps, z0, sigma=sigma)
    ref_ds, _ = oracle_velocity(oracle_mod, g, r, psi, mb, eps, z0, dipole=True, sigma=sigma)
    for got, ref in ((u_d, ref_d), (u_s, ref_s), (u_ds, ref_ds)):
        assert rel_l2(got, ref) <= TOL["fp64"], rel_l2(got, ref)


def test_solved_velocity_is_in_effect(mmod, oracle_mod):
    """The solved u_2 becomes the velocity: the adaptive dt and the next
    substeps are those of mm_set_velocity with the same field."""
    g = Grid(12, 10, 16, 16)
    r = Rates(ell=0.2, k_on=2.0)
    psi, mb = seeded(g, 321)
    eps, z0 = 0.3, 0.1
    with mmod.Simulation(g, r, "fp64") as sim:
        sim.set_state(psi, np.ascontiguousarray(mb))
        sim.fluid_setup(eps, z0)
        u = sim.fluid_solve()
        dt = sim.dt
        sim.step(5)
        got = sim.get_state()
    ref_u, st = oracle_velocity(oracle_mod, g, r, psi, mb, eps, z0)
    dt_ref = oracle_mod.dt(g, r, st, ref_u)
    assert abs(dt - dt_ref) <= 1e-12 * dt_ref
    oracle_mod.run(g, r, st, np.ascontiguousarray(u), dt, 5)
    for k in ("psi", "mb", "mf", "c"):
        assert rel_l2(got[k], getattr(st, k)) <= 1e-12, k


def test_macro_loop_against_oracle(mmod, oracle_mod):
    """Alg. 1 end to end on the device: per macro step the fluid solve from the
    current state, then substeps at the new adaptive dt; three macro steps."""
    g = Grid(10, 8, 16, 16)
    r = Rates(ell=0.25, k_on=1.5, glide=0.2)
    psi, mb = seeded(g, 331)
    eps, z0 = 0.5, 0.2
    st = oracle_mod.make_state(g, psi, mb)
    with mmod.Simulation(g, r, "fp64") as sim:
        sim.set_state(psi, np.ascontiguousarray(mb))
        sim.fluid_setup(eps, z0)
        for _ in range(3):
            u = sim.fluid_solve(dipole=True)
            f, _ = oracle_mod.moments(g, r, st)
            uo = FL.velocity(eps, z0, np.stack([f["Fx"], f["Fy"]]),
                             -np.stack([f["Sxx"], f["Sxy"], f["Syy"]]))
            assert rel_l2(u, uo) <= 1e-11
            dto = oracle_mod.dt(g, r, st, uo)
            assert abs(sim.dt - dto) <= 1e-11 * dto
            sim.step(4)
            oracle_mod.run(g, r, st, uo, dto, 4)
        got = sim.get_state()
    for k in ("psi", "mb", "mf", "c"):
        assert rel_l2(got[k], getattr(st, k)) <= 1e-11, k


def test_anchor_force_drives_the_fluid(mmod, oracle_mod):
    g = Grid(12, 10, 8, 16)
    r = Rates(ell=0.3)
    psi, mb = seeded(g, 341)
    eps, z0 = 0.2, 0.1
    with mmod.Simulation(g, r, "fp64") as sim:
        sim.set_anchors(True)
        sim.set_state(psi, np.ascontiguousarray(mb))
        sim.fluid_setup(eps, z0)
        u = sim.fluid_solve()
        with pytest.raises(mmod.MMError) as e:
            sim.fluid_solve(dipole=True)
        assert e.value.status == 4
    ref, _ = oracle_velocity(oracle_mod, g, r, psi, mb, eps, z0, anchors=True)
    assert rel_l2(u, ref) <= TOL["fp64"]


def test_device_output_and_large_grid_consistency(mmod):
    """128 x 128 (the throughput workload's grid), float32: the device copy
    equals the host copy, and u is the per-mode map of the force's DFT with the
    device table (numpy FFT on the host; the table itself is checked against
    the oracle above)."""
    import torch
    g = Grid(128, 128, 8, 8)
    r = Rates(ell=0.1)
    psi, mb = seeded(g, 351)
    eps, z0 = 0.1, 0.1
    with mmod.Simulation(g, r, "fp32") as sim:
        sim.set_state(psi, np.ascontiguousarray(mb))
        sim.fluid_setup(eps, z0)
        u_dev = torch.empty((2, g.ny, g.nx), dtype=torch.float64, device="cuda")
        sim.fluid_solve(u_out=u_dev)
        u = sim.fluid_solve()
        tab = sim.fluid_response()
        f, _ = sim.moments()
    assert np.array_equal(u_dev.cpu().numpy(), u)
    Fh = np.fft.rfft2(np.stack([f["Fx"], f["Fy"]]), axes=(-2, -1))
    jy = np.arange(g.ny)
    ky = 2 * np.pi * np.where(jy <= g.ny // 2, jy, jy - g.ny)[:, None] * np.ones((1, g.nx // 2 + 1))
    kx = 2 * np.pi * np.arange(g.nx // 2 + 1)[None, :] * np.ones((g.ny, 1))
    k2 = kx * kx + ky * ky
    gT, gL = tab[..., 0], tab[..., 1]
    with np.errstate(invalid="ignore", divide="ignore"):
        c = np.where(k2 > 0, (gL - gT) / k2, 0.0)
    # Nyquist rows/columns: the +-k mean drops the cross terms kx ky
    nyq = (np.arange(g.nx // 2 + 1)[None, :] == g.nx // 2) | (jy[:, None] == g.ny // 2)
    cxy = np.where(nyq, 0.0, c)
    ux = gT * Fh[0] + c * kx * kx * Fh[0] + cxy * kx * ky * Fh[1]
    uy = gT * Fh[1] + cxy * ky * kx * Fh[0] + c * ky * ky * Fh[1]
    ref = np.fft.irfft2(np.stack([ux, uy]), s=(g.ny, g.nx), axes=(-2, -1))
    assert rel_l2(u, ref) <= 1e-12


def test_fluid_refusals(mmod):
    g = Grid(6, 6, 8, 8)
    with mmod.Simulation(g, Rates(), "fp64") as sim:
        with pytest.raises(mmod.MMError) as e:
            sim.fluid_solve()
        assert e.value.status == 7  # no set-up
        for eps, z0 in ((0.0, 0.1), (float("nan"), 0.1), (0.1, 0.0), (0.1, 1.0)):
            with pytest.raises(mmod.MMError) as e:
                sim.fluid_setup(eps, z0)
            assert e.value.status == 1
        sim.fluid_setup(0.2, 0.1)
        with pytest.raises(mmod.MMError) as e:
            sim.fluid_solve()
        assert e.value.status == 7  # no state
        psi, mb = seeded(g, 361)
        sim.set_state(psi, np.ascontiguousarray(mb))
        sim.set_velocity(np.zeros((2, g.ny, g.nx)))
        sim.set_checkpointing(2, 4)
        with pytest.raises(mmod.MMError) as e:
            sim.fluid_solve()
        assert e.value.status == 7  # recording
    with mmod.Simulation(Grid(1, 6, 8, 8), Rates(), "fp64") as sim:
        with pytest.raises(mmod.MMError) as e:
            sim.fluid_setup(0.2, 0.1)
        assert e.value.status == 4
    with mmod.Batch([g, g], [Rates(), Rates()], "fp64") as b:
        with pytest.raises(mmod.MMError) as e:
            b.members[0].fluid_setup(0.2, 0.1)
        assert e.value.status == 4
