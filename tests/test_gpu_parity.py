"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (relative L2 per output field, ||gpu - oracle|| / ||oracle||):
  float64 path  <= 1e-12  (same arithmetic up to rounding order and fma)
  float32 path  <= 1e-5   (float32 storage and arithmetic, float64 sums)
Both sides take the same dt (the oracle's, passed with mm_set_dt) after the
GPU's own dt has been checked against the oracle's.
"""
import math

import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import (Grid, Rates, SplitMix64, WORKLOADS, cellular_flow,
                                           psi_isotropic_perturbed, psi_uniform,
                                           random_divfree_flow, workload_velocity)

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


def rand_state(g, seed, mb_scale=0.3):
    rng = SplitMix64(seed)
    psi = psi_isotropic_perturbed(g, seed, amp=0.3)
    mb = mb_scale * rng.uniforms(g.ny * g.nx * g.ntheta * g.ns).reshape(g.ny, g.nx, g.ntheta, g.ns)
    return psi, mb


def run_both(mmod, O, g, r, psi, mb, mtot, u, nsub, precision, check_dt=True, dt=None):
    st = O.make_state(g, psi, mb, mtot)
    dt_o = O.dt(g, r, st, u) if dt is None else dt
    check_dt = check_dt and dt is None
    with mmod.Simulation(g, r, precision) as sim:
        sim.set_state(np.ascontiguousarray(psi), None if mb is None else np.ascontiguousarray(mb),
                      None if mtot is None else np.ascontiguousarray(mtot))
        sim.set_velocity(np.ascontiguousarray(u))
        if check_dt:
            assert abs(sim.dt - dt_o) <= (1e-14 if precision == "fp64" else 1e-6) * dt_o
        sim.set_dt(dt_o)
        sim.step(nsub)
        gs = sim.get_state()
        gf, gsc = sim.moments()
    O.run(g, r, st, u, dt_o, nsub)
    of, osc = O.moments(g, r, st)
    return st, gs, (of, osc), (gf, gsc)


def assert_state_close(st, gs, tol):
    for name in ("psi", "mb", "mf", "c"):
        err = rel_l2(gs[name], getattr(st, name))
        assert err <= tol, (name, err)


def assert_moments_close(om, gm, tol, st=None):
    """Fields by relative L2. Global sums that cancel (sum psi cos, sum psi sin
    and the polar order built from them, the mean active stress) are compared
    against the sum of the magnitudes of their terms, the scale their
    round-off is proportional to."""
    of, osc = om
    gf, gsc = gm
    for k in of:
        err = rel_l2(gf[k], of[k])
        assert err <= tol or np.abs(gf[k] - of[k]).max() <= tol * 1e-3, (k, err)
    spsi = st.psi.sum() if st is not None else 1.0
    stress_scale = np.mean(np.abs(of["Sxx"]) + np.abs(of["Syy"]))
    scale = {"sum_psi_cos": spsi, "sum_psi_sin": spsi, "polar_order": 1.0,
             "mean_stress": stress_scale}
    for k in osc:
        s_k = max(abs(osc[k]), scale.get(k, 0.0), 1e-300)
        assert abs(gsc[k] - osc[k]) <= tol * s_k, (k, gsc[k], osc[k])


def test_fp64_cellular_flow_matches_oracle(mmod, oracle_mod):
    """32x32 grid, 16 orientations, 16 arclength nodes, cellular flow, 200
    substeps at cfl 0.4 from a perturbed isotropic start."""
    w = WORKLOADS["cellular32"]
    g, r = w["grid"], Rates()
    psi = psi_isotropic_perturbed(g, w["seed"])
    u = cellular_flow(g, w["amp"])
    st, gs, om, gm = run_both(mmod, oracle_mod, g, r, psi, None, None, u, w["substeps"], "fp64")
    assert_state_close(st, gs, TOL["fp64"])
    assert_moments_close(om, gm, TOL["fp64"], st)


@pytest.mark.parametrize("dims", [(37, 29, 6, 6), (64, 48, 40, 16), (5, 3, 3, 7), (12, 10, 33, 64),
                                  (1, 1, 1, 1), (70, 9, 17, 10)])
def test_fp64_ragged_shapes_match_oracle(mmod, oracle_mod, dims):
    """Shapes that leave ragged tails: odd ns (scalar lanes), ns not filling a
    warp segment, more orientations than a CTA pass, single cells."""
    g = Grid(*dims, L=1.2)
    r = Rates(v_walk=0.9, k_on=1.3, k_off=0.7, glide=0.4, v_sp=0.15)
    psi, mb = rand_state(g, 5)
    u = random_divfree_flow(g, 6, 6, 0.3)
    st, gs, om, gm = run_both(mmod, oracle_mod, g, r, psi, mb, None, u, 12, "fp64")
    assert_state_close(st, gs, TOL["fp64"])
    assert_moments_close(om, gm, TOL["fp64"], st)


def test_fp64_scale_down_clip_matches_oracle(mmod, oracle_mod):
    """Large binding rate and little motor supply with a substep above the
    adaptive one: the Alg. 2 scale-down triggers on alternate substeps."""
    g = Grid(16, 12, 8, 8)
    r = Rates(k_on=300.0, k_off=0.5, glide=0.5, v_sp=0.1)
    psi, mb = rand_state(g, 9, mb_scale=0.02)
    mtot = np.full((g.ny, g.nx), 0.08)
    u = random_divfree_flow(g, 10, 6, 0.3)
    st, gs, om, gm = run_both(mmod, oracle_mod, g, r, psi, mb, mtot, u, 9, "fp64", dt=0.01)
    assert np.count_nonzero(st.mf == 0.0) > 0
    assert_state_close(st, gs, TOL["fp64"])


def test_fp64_isotropic_state_stays_uniform(mmod):
    """Uniform isotropic psi with zero flow: psi bitwise unchanged and every
    cell's rows identical (the GPU reproduces the exact cancellation)."""
    g = Grid(8, 6, 8, 8)
    with mmod.Simulation(g, Rates(glide=0.5, v_sp=0.3), "fp64") as sim:
        p0 = psi_uniform(g)
        sim.set_state(p0)
        sim.set_velocity(np.zeros((2, g.ny, g.nx)))
        sim.step(50)
        s = sim.get_state()
    assert np.array_equal(s["psi"], p0)
    assert np.array_equal(s["mb"], np.broadcast_to(s["mb"][0, 0], s["mb"].shape))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_conservation_on_gpu(mmod, precision, tol):
    """Total filament number (Eq. 1 telescopes) and motor number (Eq. 5-6)."""
    g = Grid(48, 40, 16, 16)
    with mmod.Simulation(g, Rates(), precision) as sim:
        sim.set_state(psi_isotropic_perturbed(g, 4))
        sim.set_velocity(random_divfree_flow(g, 5, 8, 0.1))
        _, s0 = sim.moments(fields=False)
        sim.step(150)
        f, s1 = sim.moments()
        st = sim.get_state()
    assert abs(s1["N_psi"] - s0["N_psi"]) <= tol * s0["N_psi"]
    # Mf = M - C per cell in the state precision: exact in float64, to float32
    # rounding in the float32 form
    assert abs(s1["motors"] - 1.0) <= (1e-14 if precision == "fp64" else 1e-7)
    dth, ds = 2 * math.pi / g.ntheta, g.L / g.ns
    C = np.einsum("yxk,yxkj->yx", st["psi"], st["mb"]) * dth * ds
    assert np.abs(st["mf"] + C - 1.0).max() <= (1e-13 if precision == "fp64" else 1e-6)


def test_fp32_cellular_flow_within_tolerance(mmod, oracle_mod):
    """Float32 form on the 32x32x16x16 cellular-flow case, 200 substeps."""
    w = WORKLOADS["cellular32"]
    g, r = w["grid"], Rates()
    psi = psi_isotropic_perturbed(g, w["seed"])
    u = cellular_flow(g, w["amp"])
    st, gs, om, gm = run_both(mmod, oracle_mod, g, r, psi, None, None, u, w["substeps"], "fp32")
    assert_state_close(st, gs, TOL["fp32"])
    assert_moments_close(om, gm, TOL["fp32"], st)


@pytest.mark.parametrize("dims", [(37, 29, 6, 8), (20, 24, 12, 6), (9, 7, 5, 31), (5, 6, 3, 128),
                                  (11, 13, 7, 12)])
def test_fp32_ragged_shapes_within_tolerance(mmod, oracle_mod, dims):
    g = Grid(*dims)
    r = Rates(glide=0.3, v_sp=0.1)
    psi, mb = rand_state(g, 12)
    u = random_divfree_flow(g, 13, 6, 0.3)
    st, gs, om, gm = run_both(mmod, oracle_mod, g, r, psi, mb, None, u, 30, "fp32")
    assert_state_close(st, gs, TOL["fp32"])


def _sampled_full_size(mmod, O, name, precision, n_pre, n_samples=48):
    """Full-size run in the benchmark's launch configuration; then one more
    substep on the GPU, checked cell by cell on sampled cells against the
    oracle's substep of the 3x3 patch around each cell, started from the
    GPU's own pre-step state."""
    import torch
    w = WORKLOADS[name]
    g, r = w["grid"], Rates()
    dev = torch.device("cuda")
    with mmod.Simulation(g, r, precision) as sim:
        sim.set_state(psi_isotropic_perturbed(g, w["seed"]))
        u = workload_velocity(name, 0)
        sim.set_velocity(u)
        dt = sim.dt
        sim.step(n_pre)
        pre = dict(psi=torch.empty((g.ny, g.nx, g.ntheta), dtype=torch.float64, device=dev),
                   mb=torch.empty((g.ny, g.nx, g.ntheta, g.ns), dtype=torch.float64, device=dev),
                   mf=torch.empty((g.ny, g.nx), dtype=torch.float64, device=dev))
        sim.get_state_into(psi=pre["psi"], mb=pre["mb"], mf=pre["mf"])
        sim.step(1)
        post = dict(psi=torch.empty_like(pre["psi"]), mb=torch.empty_like(pre["mb"]),
                    mf=torch.empty_like(pre["mf"]), c=torch.empty_like(pre["mf"]))
        sim.get_state_into(**post)
        torch.cuda.synchronize()
    rng = SplitMix64(99)
    cells = [(int(rng.uniform() * g.ny), int(rng.uniform() * g.nx)) for _ in range(n_samples)]
    cells += [(0, 0), (g.ny - 1, g.nx - 1), (0, g.nx - 1), (g.ny - 1, 0)]
    # gather the 3x3 neighbourhoods on the device, then bring them to the host
    ys = torch.tensor([[(iy + d) % g.ny for d in (-1, 0, 1)] for iy, _ in cells], device=dev)
    xs = torch.tensor([[(ix + d) % g.nx for d in (-1, 0, 1)] for _, ix in cells], device=dev)
    Y, X = ys[:, :, None], xs[:, None, :]
    psi_p = pre["psi"][Y, X].cpu().numpy()
    mb_p = pre["mb"][Y, X].cpu().numpy()
    mf_p = pre["mf"][Y, X].cpu().numpy()
    ut = torch.tensor(u, device=dev)
    u_p = torch.stack([ut[0][Y, X], ut[1][Y, X]], dim=1).cpu().numpy()
    errs = {"psi": [], "mb": [], "mf": [], "c": []}
    refs = {"psi": [], "mb": [], "mf": [], "c": []}
    for q, (iy, ix) in enumerate(cells):
        # a 3x3 patch, then index its centre
        pg_psi, pg_mb, pg_mf = psi_p[q], mb_p[q], mf_p[q]
        st = O.State(O.PatchGrid(3, 3, g.ntheta, g.ns, g.L, 3.0 / g.nx, 3.0 / g.ny),
                     np.ascontiguousarray(pg_psi), np.ascontiguousarray(pg_mb),
                     np.ascontiguousarray(pg_mf), np.zeros((3, 3)), np.ones((3, 3)))
        O.run(st.grid, r, st, np.ascontiguousarray(u_p[q]), dt, 1)
        got = dict(psi=post["psi"][iy, ix].cpu().numpy(), mb=post["mb"][iy, ix].cpu().numpy(),
                   mf=post["mf"][iy, ix].item(), c=post["c"][iy, ix].item())
        exp = dict(psi=st.psi[1, 1], mb=st.mb[1, 1], mf=st.mf[1, 1], c=st.c[1, 1])
        for k in errs:
            errs[k].append(np.ravel(np.asarray(got[k]) - np.asarray(exp[k])))
            refs[k].append(np.ravel(np.asarray(exp[k])))
    return {k: np.linalg.norm(np.concatenate(errs[k])) / np.linalg.norm(np.concatenate(refs[k]))
            for k in errs}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_size_precision128_sampled(mmod, oracle_mod, precision):
    """128x128 grid, 32 orientations, 32 nodes (the benchmark's workload and
    launch configuration): sampled cells after a 50-substep macro step."""
    errs = _sampled_full_size(mmod, oracle_mod, "precision128", precision, 50)
    for k, e in errs.items():
        assert e <= TOL[precision], (k, e)


def test_full_size_large512_sampled(mmod, oracle_mod):
    """512x512 grid, 64 orientations, 64 nodes (1.07e9 motor cells, float32)."""
    errs = _sampled_full_size(mmod, oracle_mod, "large512", "fp32", 5, n_samples=24)
    for k, e in errs.items():
        assert e <= TOL["fp32"], (k, e)
