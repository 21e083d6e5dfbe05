"""GPU parity of mm_motor_local (motor kinetics over a macro interval with psi
frozen and a local substep per cell: the independent time steps of Sec. 3.1,
Alg. 2's inner loop per anchor) against the float64 oracle (or_motor_local).

Both sides start from the same seeded inputs (set_state / make_state). The
substep count of every cell is an integer decided in float64 from the same
formula on both sides: it must agree exactly. Fields: relative L2 <= 1e-12 in
float64, <= 1e-5 in the float32 form (whose psi is float32-rounded: the test
chooses T so that no cell's T rate / cfl lies within 1e-4 of an integer, where
the rounding of psi could move the ceiling).
"""
import math

import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import (Grid, Rates, SplitMix64, WORKLOADS,
                                           psi_isotropic_perturbed)

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


def seeded(g, seed, mb_scale=0.3, amp=0.3):
    rng = SplitMix64(seed)
    psi = psi_isotropic_perturbed(g, seed, amp=amp)
    mb = mb_scale * rng.uniforms(g.ny * g.nx * g.ntheta * g.ns).reshape(g.ny, g.nx, g.ntheta, g.ns)
    return psi, mb


def count_margin(g, r, psi, T):
    """Smallest distance of T rate_i / cfl above the integer below it, and
    below the integer above it, over the cells (float64, the oracle's
    formula)."""
    rho = (psi * (2 * math.pi / g.ntheta)).sum(-1)
    q = T * np.maximum(r.v_walk / (g.L / g.ns), r.k_off + r.k_on * g.L * rho) / r.cfl
    frac = q - np.floor(q)
    return float(np.min(np.minimum(frac, 1.0 - frac)))


def run_both(mmod, O, g, r, psi, mb, mtot, T, precision, nsteps=None):
    st = O.make_state(g, psi, mb, mtot)
    with mmod.Simulation(g, r, precision) as sim:
        sim.set_state(np.ascontiguousarray(psi), np.ascontiguousarray(mb),
                      None if mtot is None else np.ascontiguousarray(mtot))
        n_gpu = sim.motor_local(T, nsteps)
        gs = sim.get_state()
    n_or = O.motor_local(g, r, st, T, nsteps)
    return st, gs, n_or, n_gpu


def assert_close(st, gs, tol, psi):
    for name in ("mb", "mf", "c"):
        err = rel_l2(gs[name], getattr(st, name))
        assert err <= tol, (name, err)
    # psi is frozen
    assert rel_l2(gs["psi"], psi) <= (0.0 if tol < 1e-9 else 1e-7)


SHAPES = [
    (8, 6, 16, 16),    # one pass per warp, bulk copies
    (5, 3, 7, 10),     # ragged: 7 orientations, 10 nodes
    (4, 4, 5, 7),      # odd ns (one node per lane), cell not a whole 16-byte vector
    (3, 2, 40, 32),    # more row groups than warps: several passes per warp
    (2, 3, 64, 64),    # the large workload's cell (64 x 64 rows)
    (1, 1, 3, 2),      # one cell, tiny rows
]


@pytest.mark.parametrize("dims", SHAPES)
def test_fp64_local_matches_oracle(mmod, oracle_mod, dims):
    g = Grid(*dims)
    r = Rates()
    psi, mb = seeded(g, 11 + sum(dims))
    st, gs, n_or, n_gpu = run_both(mmod, oracle_mod, g, r, psi, mb, None, 0.37, "fp64")
    assert np.array_equal(n_gpu, n_or)
    assert n_or.min() >= 2
    assert_close(st, gs, TOL["fp64"], psi)


def test_fp64_local_varied_counts(mmod, oracle_mod):
    """No walking: every cell's count comes from its own density, so the cells
    take different numbers of substeps (the independent time steps)."""
    g = Grid(9, 7, 16, 16)
    r = Rates(v_walk=0.0, k_on=1.3, k_off=0.7)
    psi, mb = seeded(g, 31, amp=0.9)
    st, gs, n_or, n_gpu = run_both(mmod, oracle_mod, g, r, psi, mb, None, 4.3, "fp64")
    assert np.array_equal(n_gpu, n_or)
    assert len(np.unique(n_or)) >= 3
    assert_close(st, gs, TOL["fp64"], psi)


def test_fp64_local_scale_down(mmod, oracle_mod):
    """Few total motors, fast binding and imposed long substeps (1 to 3 per
    cell): the binding overshoots and the Alg. 2 scale-down acts (C = M in the
    cells whose single substep ended with it)."""
    g = Grid(6, 5, 12, 16)
    r = Rates(k_on=40.0, k_off=0.1)
    psi, mb = seeded(g, 41, mb_scale=0.05)
    mtot = 0.1 * np.ones((g.ny, g.nx))
    nsteps = np.random.default_rng(42).integers(1, 4, size=(g.ny, g.nx)).astype(np.int32)
    st, gs, n_or, n_gpu = run_both(mmod, oracle_mod, g, r, psi, mb, mtot, 0.5, "fp64", nsteps)
    assert np.array_equal(n_gpu, nsteps) and np.array_equal(n_or, nsteps)
    assert np.all(st.c[nsteps == 1] == mtot[nsteps == 1])  # the clip was taken
    assert np.sum(nsteps == 1) > 0
    assert_close(st, gs, TOL["fp64"], psi)


def test_fp64_local_imposed_counts(mmod, oracle_mod):
    g = Grid(7, 5, 16, 16)
    r = Rates()
    psi, mb = seeded(g, 51)
    rng = np.random.default_rng(52)
    nsteps = rng.integers(1, 9, size=(g.ny, g.nx)).astype(np.int32)
    st, gs, n_or, n_gpu = run_both(mmod, oracle_mod, g, r, psi, mb, None, 0.05, "fp64", nsteps)
    assert np.array_equal(n_gpu, nsteps) and np.array_equal(n_or, nsteps)
    assert_close(st, gs, TOL["fp64"], psi)


@pytest.mark.parametrize("dims", [(8, 6, 16, 16), (5, 3, 7, 12), (3, 2, 64, 64), (4, 4, 6, 7)])
def test_fp32_local_within_tolerance(mmod, oracle_mod, dims):
    g = Grid(*dims)
    r = Rates(v_walk=0.09)  # binding and unbinding set the count on some grids
    psi, mb = seeded(g, 61 + sum(dims))
    T = next(t for t in (2.41, 2.43, 2.47, 2.53, 2.59, 2.61) if count_margin(g, r, psi, t) > 1e-4)
    st, gs, n_or, n_gpu = run_both(mmod, oracle_mod, g, r, psi, mb, None, T, "fp32")
    assert np.array_equal(n_gpu, n_or)
    assert_close(st, gs, TOL["fp32"], psi)


def test_local_then_global_substeps_consistent(mmod, oracle_mod):
    """n_b, C and Mf left by the local update feed the next global substeps:
    local update then 5 global substeps equal the oracle's same sequence."""
    g = Grid(8, 8, 16, 16)
    r = Rates()
    psi, mb = seeded(g, 71)
    rng = SplitMix64(72)
    u = 0.1 * (2 * rng.uniforms(2 * g.ny * g.nx) - 1).reshape(2, g.ny, g.nx)
    st = oracle_mod.make_state(g, psi, mb)
    with mmod.Simulation(g, r, "fp64") as sim:
        sim.set_state(psi, np.ascontiguousarray(mb))
        n_gpu = sim.motor_local(0.2)
        sim.set_velocity(u)
        n_or = oracle_mod.motor_local(g, r, st, 0.2)
        dt = oracle_mod.dt(g, r, st, u)
        assert abs(sim.dt - dt) <= 1e-14 * dt  # the rule sees the new n_b
        sim.step(5)
        gs = sim.get_state()
    oracle_mod.run(g, r, st, u, dt, 5)
    assert np.array_equal(n_gpu, n_or)
    for name in ("psi", "mb", "mf", "c"):
        assert rel_l2(gs[name], getattr(st, name)) <= TOL["fp64"], name


def test_local_full_size_precision128_sampled(mmod, oracle_mod):
    """The 128x128 x 32 x 32 workload in float32 after 50 global substeps, then
    one local update over the macro interval of 50 substeps; sampled cells
    against the oracle on one-cell grids started from the GPU's state before
    the call (with psi frozen the cells are independent)."""
    import torch
    w = WORKLOADS["precision128"]
    g, r = w["grid"], Rates()
    from paper_1908_04279_gb300.inputs import workload_velocity
    dev = torch.device("cuda")
    with mmod.Simulation(g, r, "fp32") as sim:
        sim.set_state(psi_isotropic_perturbed(g, w["seed"]))
        sim.set_velocity(workload_velocity("precision128", 0))
        T = 50 * sim.dt
        sim.step(50)
        pre = dict(psi=torch.empty((g.ny, g.nx, g.ntheta), dtype=torch.float64, device=dev),
                   mb=torch.empty((g.ny, g.nx, g.ntheta, g.ns), dtype=torch.float64, device=dev),
                   mf=torch.empty((g.ny, g.nx), dtype=torch.float64, device=dev))
        sim.get_state_into(**pre)
        n_gpu = sim.motor_local(T)
        post = dict(mb=torch.empty_like(pre["mb"]), mf=torch.empty_like(pre["mf"]),
                    c=torch.empty_like(pre["mf"]))
        sim.get_state_into(**post)
    rng = SplitMix64(73)
    cells = [(int(rng.uniform() * g.ny), int(rng.uniform() * g.nx)) for _ in range(40)]
    cells += [(0, 0), (g.ny - 1, g.nx - 1)]
    err2 = {"mb": 0.0, "mf": 0.0, "c": 0.0}
    ref2 = dict(err2)
    g1 = Grid(1, 1, g.ntheta, g.ns, g.L)
    for iy, ix in cells:
        st = oracle_mod.State(g1, pre["psi"][iy, ix].cpu().numpy().reshape(1, 1, -1).copy(),
                              pre["mb"][iy, ix].cpu().numpy().reshape(1, 1, g.ntheta, g.ns).copy(),
                              pre["mf"][iy, ix].cpu().numpy().reshape(1, 1).copy(),
                              np.zeros((1, 1)), np.ones((1, 1)))
        n = oracle_mod.motor_local(g1, r, st, T)
        assert n[0, 0] == n_gpu[iy, ix]
        got = dict(mb=post["mb"][iy, ix].cpu().numpy(), mf=post["mf"][iy, ix].item(),
                   c=post["c"][iy, ix].item())
        for k in err2:
            exp = getattr(st, k).reshape(np.shape(got[k]))
            err2[k] += float(np.sum((np.asarray(got[k]) - exp) ** 2))
            ref2[k] += float(np.sum(np.asarray(exp) ** 2))
    for k in err2:
        assert math.sqrt(err2[k] / ref2[k]) <= TOL["fp32"], k


def test_local_errors(mmod):
    g = Grid(4, 4, 8, 8)
    with mmod.Simulation(g, Rates(), "fp64") as sim:
        with pytest.raises(mmod.MMError) as e:
            sim.motor_local(0.1)
        assert e.value.status == 7  # no state yet
        psi, mb = seeded(g, 81)
        sim.set_state(psi, np.ascontiguousarray(mb))
        before = sim.get_state()
        for bad in (0.0, -1.0, float("nan"), float("inf")):
            with pytest.raises(mmod.MMError) as e:
                sim.motor_local(bad)
            assert e.value.status == 1
        with pytest.raises(mmod.MMError) as e:
            sim.motor_local(0.1, np.zeros((g.ny, g.nx), dtype=np.int32))
        assert e.value.status == 1
        # a count beyond 2^20: reported, the state left as it was
        with pytest.raises(mmod.MMError) as e:
            sim.motor_local(1e9)
        assert e.value.status == 1
        after = sim.get_state()
        for k in ("mb", "mf", "c", "psi"):
            assert np.array_equal(before[k], after[k]), k
        # the handle works afterwards
        sim.motor_local(0.05)
        sim.set_velocity(np.zeros((2, g.ny, g.nx)))
        sim.set_checkpointing(2, 4)
        with pytest.raises(mmod.MMError) as e:
            sim.motor_local(0.05)
        assert e.value.status == 7  # not differentiated


def test_local_bounded_wait_timeout(mmod, oracle_mod):
    """The test knob makes every bounded wait of the kernel run out: the call
    reports MM_ERR_TIMEOUT (the GPU is left usable), and with the knob off the
    same handle gives the oracle's answer."""
    g = Grid(6, 4, 16, 16)
    r = Rates()
    psi, mb = seeded(g, 91)
    with mmod.Simulation(g, r, "fp64") as sim:
        sim.set_state(psi, np.ascontiguousarray(mb))
        sim.debug_set(2000, 1)
        with pytest.raises(mmod.MMError) as e:
            sim.motor_local(0.2)
        assert e.value.status == 5
        sim.debug_set(1 << 22, 0)
        sim.set_state(psi, np.ascontiguousarray(mb))
        n_gpu = sim.motor_local(0.2)
        gs = sim.get_state()
    st = oracle_mod.make_state(g, psi, mb)
    n_or = oracle_mod.motor_local(g, r, st, 0.2)
    assert np.array_equal(n_gpu, n_or)
    assert_close(st, gs, TOL["fp64"], psi)
