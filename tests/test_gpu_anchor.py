"""GPU parity of the non-local motor anchors (mm_set_anchors: every bound
configuration anchored in the cell under its motor head, x + (l/L) s p) against
the float64 oracle's anchor substep (or_substep_anchor), its set-up and its
force field. Both sides start from the same seeded inputs and take the same dt
(the oracle's). Relative L2 per field: <= 1e-12 in float64 (the coarse density
is accumulated by float64 atomics, so only its rounding order differs),
<= 1e-5 in float32.
"""
import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import (Grid, Rates, SplitMix64, psi_isotropic_perturbed,
                                           random_divfree_flow)

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


def run_both(mmod, O, g, r, psi, mb, mtot, u, nsub, precision, dt_scale=1.0):
    st = O.make_state_anchor(g, r, psi, mb, mtot)
    dt = O.dt(g, r, st, u) * dt_scale
    with mmod.Simulation(g, r, precision) as sim:
        sim.set_anchors(True)
        sim.set_state(np.ascontiguousarray(psi), np.ascontiguousarray(mb),
                      None if mtot is None else np.ascontiguousarray(mtot))
        s0 = sim.get_state()
        sim.set_velocity(np.ascontiguousarray(u))
        sim.set_dt(dt)
        sim.step(nsub)
        gs = sim.get_state()
        gf, _ = sim.moments()
    init = O.make_state_anchor(g, r, psi, mb, mtot)
    O.run_anchor(g, r, st, u, dt, nsub)
    F = O.anchor_force(g, r, st)
    return init, s0, st, gs, F, gf


def check(init, s0, st, gs, F, gf, tol):
    for k in ("mb", "mf", "c"):
        assert rel_l2(s0[k], getattr(init, k)) <= tol, ("set-up", k, rel_l2(s0[k], getattr(init, k)))
    for k in ("psi", "mb", "mf", "c"):
        err = rel_l2(gs[k], getattr(st, k))
        assert err <= tol, (k, err)
    assert rel_l2(gf["Fx"], F[0]) <= tol and rel_l2(gf["Fy"], F[1]) <= tol


@pytest.mark.parametrize("dims", [(8, 6, 16, 16), (5, 3, 7, 10), (4, 4, 5, 7), (3, 2, 40, 32),
                                  (16, 12, 8, 24)])
def test_fp64_anchor_matches_oracle(mmod, oracle_mod, dims):
    g = Grid(*dims)
    r = Rates(ell=0.3, k_on=2.0, glide=0.1)
    psi, mb = seeded(g, 201 + sum(dims))
    u = random_divfree_flow(g, 202, 4, 0.1)
    out = run_both(mmod, oracle_mod, g, r, psi, mb, None, u, 12, "fp64")
    check(*out, TOL["fp64"])


def test_fp64_anchor_long_filaments(mmod, oracle_mod):
    """Filaments longer than the grid (l/L = 1.5 on 40 x 36 cells): the anchors
    of a cell spread over more cells than the shared-memory window holds, so the
    kernel gathers and scatters in global memory; and offsets wrap the grid."""
    g = Grid(40, 36, 8, 16)
    r = Rates(ell=1.5, k_on=1.2)
    psi, mb = seeded(g, 205)
    u = random_divfree_flow(g, 206, 4, 0.1)
    ox, oy = oracle_mod.anchor_offsets(g, r)
    assert (ox.max() - ox.min() + 1) * (oy.max() - oy.min() + 1) > 1024
    assert ox.max() > g.nx // 2 and ox.min() < -(g.nx // 2)
    check(*run_both(mmod, oracle_mod, g, r, psi, mb, None, u, 4, "fp64"), TOL["fp64"])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_anchor_wide_window(mmod, oracle_mod, precision):
    """A block's window of 25 x 21 anchor cells (48 x 40 cells, l/L = 0.5, 32 x 32):
    a cell's 832 slot runs (888 in float64) lie in 27 (29) places per lane, the
    sums of the 289 window entries span up to 64 places and so several lanes
    (joined by the scan over the lanes), and the shared window holds every
    anchor; the row length is a multiple of 4, so 4 cells share one window."""
    g = Grid(48, 40, 32, 32)
    r = Rates(ell=0.5, k_on=1.4, glide=0.2)
    ox, oy = oracle_mod.anchor_offsets(g, r)
    w = (ox.max() - ox.min() + 1) * (oy.max() - oy.min() + 1)
    assert 512 < w <= 1024 and g.nx % 4 == 0
    psi, mb = seeded(g, 231)
    u = random_divfree_flow(g, 232, 4, 0.1)
    check(*run_both(mmod, oracle_mod, g, r, psi, mb, None, u, 6, precision), TOL[precision])


@pytest.mark.parametrize("dims,precision,ell", [((8, 6, 12, 20), "fp32", 0.3),
                                                ((8, 6, 10, 9), "fp32", 0.3),
                                                ((8, 8, 16, 16), "fp64", 0.9)])
def test_anchor_block_window_lane_widths(mmod, oracle_mod, dims, precision, ell):
    """The block-window form with 4 values per lane (ns = 20) and with one
    (ns = 9) in float32, whose window entries and run places load as 8- and
    2-byte pieces; and in float64 a 7 x 7 window on an 8 x 8 grid (l/L = 0.9),
    so that the block's 10 window columns wrap the grid and some cells appear
    twice in the window."""
    g = Grid(*dims)
    r = Rates(ell=ell, k_on=1.5, glide=0.1)
    ox, oy = oracle_mod.anchor_offsets(g, r)
    wx, wy = ox.max() - ox.min() + 1, oy.max() - oy.min() + 1
    assert g.nx % 4 == 0 and wx <= g.nx and wy <= g.ny
    psi, mb = seeded(g, 251 + sum(dims))
    u = random_divfree_flow(g, 252, 4, 0.1)
    check(*run_both(mmod, oracle_mod, g, r, psi, mb, None, u, 8, precision), TOL[precision])


def test_fp64_anchor_scale_down_shared_window(mmod, oracle_mod):
    """The forced scale-down on a grid whose row length is a multiple of 4 (the
    block's 4 cells share one window and sum their runs per window entry)."""
    g = Grid(8, 6, 12, 16)
    r = Rates(ell=0.25, k_on=80.0, k_off=0.2)
    psi, mb = seeded(g, 241, mb_scale=0.05)
    mtot = 0.03 + 0.1 * np.random.default_rng(242).random((g.ny, g.nx))
    u = random_divfree_flow(g, 243, 3, 0.05)
    init, s0, st, gs, F, gf = run_both(mmod, oracle_mod, g, r, psi, mb, mtot, u, 6, "fp64",
                                       dt_scale=4.0)
    check(init, s0, st, gs, F, gf, TOL["fp64"])
    clipped = st.c == mtot
    assert np.any(clipped) and not np.all(clipped)


def test_fp64_anchor_scale_down(mmod, oracle_mod):
    """Few total motors and fast binding with a long step: the binding
    overshoots and the per-anchor scale-down (and the fix-up of the rows and
    their n_b) acts in some substeps."""
    g = Grid(6, 5, 12, 16)
    r = Rates(ell=0.25, k_on=80.0, k_off=0.2)
    psi, mb = seeded(g, 211, mb_scale=0.05)
    mtot = 0.03 + 0.1 * np.random.default_rng(212).random((g.ny, g.nx))
    u = random_divfree_flow(g, 213, 3, 0.05)
    init, s0, st, gs, F, gf = run_both(mmod, oracle_mod, g, r, psi, mb, mtot, u, 6, "fp64",
                                       dt_scale=4.0)
    check(init, s0, st, gs, F, gf, TOL["fp64"])
    clipped = st.c == mtot
    assert np.any(clipped) and not np.all(clipped)  # some anchors scaled down at the end


def test_fp32_anchor_within_tolerance(mmod, oracle_mod):
    g = Grid(12, 10, 16, 32)
    r = Rates(ell=0.2, k_on=1.5)
    psi, mb = seeded(g, 221)
    u = random_divfree_flow(g, 222, 6, 0.1)
    check(*run_both(mmod, oracle_mod, g, r, psi, mb, None, u, 20, "fp32"), TOL["fp32"])


@pytest.mark.parametrize("nx,precision,tol", [(10, "fp64", 1e-13), (12, "fp64", 1e-13),
                                               (12, "fp32", 1e-5)])
def test_anchor_zero_length_equals_local_path(mmod, nx, precision, tol):
    """With l/L = 0 every anchor is the filament's own cell: the anchor kernels
    give the local kernel's result (to rounding order). With 10 cells a row
    each warp keeps its own window; with 12 the block's 4 cells share one, and
    a cell's run sums all belong to one window entry: every place of every
    lane forms one entry, completed by the scan over all 32 lanes."""
    g = Grid(nx, 8, 16, 16)
    r = Rates(ell=0.0)
    psi, mb = seeded(g, 231)
    u = random_divfree_flow(g, 232, 4, 0.1)
    res = []
    for anchors in (False, True):
        with mmod.Simulation(g, r, precision) as sim:
            sim.set_anchors(anchors)
            sim.set_state(psi, np.ascontiguousarray(mb))
            sim.set_velocity(u)
            sim.step(15)
            res.append(sim.get_state())
    for k in ("psi", "mb", "mf", "c"):
        assert rel_l2(res[1][k], res[0][k]) <= tol, k


def test_anchor_toggle_and_rates(mmod, oracle_mod):
    """Switching anchors on mid-run re-derives C and Mf of the current state;
    a new l/L (mm_set_rates) moves the anchors; switching off returns to the
    local rule."""
    g = Grid(8, 8, 8, 16)
    r = Rates(ell=0.3)
    psi, mb = seeded(g, 241)
    with mmod.Simulation(g, r, "fp64") as sim:
        sim.set_state(psi, np.ascontiguousarray(mb))
        sim.set_anchors(True)
        a = sim.get_state()
        st = oracle_mod.make_state_anchor(g, r, psi, mb)
        for k in ("mb", "mf", "c"):
            assert rel_l2(a[k], getattr(st, k)) <= 1e-12, k
        r2 = Rates(ell=0.15)
        sim.set_rates(r2)
        b = sim.get_state()
        st2 = oracle_mod.make_state_anchor(g, r2, psi, mb)
        for k in ("mf", "c"):
            assert rel_l2(b[k], getattr(st2, k)) <= 1e-12, k
        sim.set_anchors(False)
        c = sim.get_state()
        st3 = oracle_mod.make_state(g, psi, mb)
        for k in ("mf", "c"):
            assert rel_l2(c[k], getattr(st3, k)) <= 1e-12, k


def test_anchor_new_length_between_steps(mmod, oracle_mod):
    """Substeps (captured as a graph), a new l/L through mm_set_rates, the same
    number of substeps again (the graph must not keep the old anchors): the
    oracle's same sequence."""
    g = Grid(10, 8, 16, 16)
    r1, r2 = Rates(ell=0.3), Rates(ell=0.12)
    psi, mb = seeded(g, 261)
    u = random_divfree_flow(g, 262, 4, 0.1)
    st = oracle_mod.make_state_anchor(g, r1, psi, mb)
    dt = oracle_mod.dt(g, r1, st, u)
    with mmod.Simulation(g, r1, "fp64") as sim:
        sim.set_anchors(True)
        sim.set_state(psi, np.ascontiguousarray(mb))
        sim.set_velocity(u)
        sim.set_dt(dt)
        sim.step(3)
        sim.set_rates(r2)
        sim.set_dt(dt)
        sim.step(3)
        gs = sim.get_state()
    oracle_mod.run_anchor(g, r1, st, u, dt, 3)
    st2 = oracle_mod.make_state_anchor(g, r2, st.psi, st.mb, st.mtot)
    oracle_mod.run_anchor(g, r2, st2, u, dt, 3)
    for k in ("psi", "mb", "mf", "c"):
        assert rel_l2(gs[k], getattr(st2, k)) <= TOL["fp64"], k


def test_anchor_refusals(mmod):
    g = Grid(6, 6, 8, 8)
    with mmod.Simulation(g, Rates(ell=0.2), "fp64") as sim:
        psi, mb = seeded(g, 251)
        sim.set_state(psi, np.ascontiguousarray(mb))
        sim.set_velocity(np.zeros((2, g.ny, g.nx)))
        sim.set_anchors(True)
        with pytest.raises(mmod.MMError) as e:
            sim.set_checkpointing(2, 4)
        assert e.value.status == 4
        with pytest.raises(mmod.MMError) as e:
            sim.motor_local(0.1)
        assert e.value.status == 4
        sim.set_anchors(False)
        sim.set_checkpointing(2, 4)
        with pytest.raises(mmod.MMError) as e:
            sim.set_anchors(True)
        assert e.value.status == 7
    with mmod.Batch([g, g], [Rates(), Rates()], "fp64") as b:
        with pytest.raises(mmod.MMError) as e:
            b.members[0].set_anchors(True)
        assert e.value.status == 4


def test_anchor_precision128_full_size(mmod, oracle_mod):
    """The bench's anchor workload at full size (128^2 x 32^2, l/L = 0.05, the
    workload's flow, float32, block window of 4 cells) against the float64
    oracle, element by element, after 3 substeps."""
    from paper_1908_04279_gb300.inputs import WORKLOADS, workload_velocity
    w = WORKLOADS["precision128"]
    g = w["grid"]
    r = Rates(ell=0.05)
    psi = psi_isotropic_perturbed(g, w["seed"])
    mb = np.zeros((g.ny, g.nx, g.ntheta, g.ns))
    u = workload_velocity("precision128", 0)
    check(*run_both(mmod, oracle_mod, g, r, psi, mb, None, u, 3, "fp32"), TOL["fp32"])


def test_anchor_large512_conservation_and_sampled_anchors(mmod, oracle_mod):
    """The bench's large anchor workload (512^2 x 64^2, l/L = 0.05, float32:
    a 27 x 27 window, each cell's 2072 slot runs summed per window entry in 65
    places per lane, three words of end marks): after
    5 substeps the filament number is conserved, bound + free motors equal the
    total, and the coarse density of 32 sampled anchor cells equals the sum of
    psi Mb ds dtheta over the configurations whose heads lie in them,
    recomputed from the exported state (relative 1e-5)."""
    torch = pytest.importorskip("torch")
    from paper_1908_04279_gb300.inputs import WORKLOADS, workload_velocity
    w = WORKLOADS["large512"]
    g = w["grid"]
    r = Rates(ell=0.05)
    dev = torch.device("cuda")
    with mmod.Simulation(g, r, "fp32") as sim:
        sim.set_anchors(True)
        sim.set_state(psi_isotropic_perturbed(g, w["seed"]))
        sim.set_velocity(torch.tensor(workload_velocity("large512", 0), device=dev))
        _, s0 = sim.moments(fields=False)
        sim.step(5)
        _, s1 = sim.moments(fields=False)
        psi = torch.empty((g.ny, g.nx, g.ntheta), dtype=torch.float64, device=dev)
        mb = torch.empty((g.ny, g.nx, g.ntheta, g.ns), dtype=torch.float64, device=dev)
        mf = torch.empty((g.ny, g.nx), dtype=torch.float64, device=dev)
        c = torch.empty((g.ny, g.nx), dtype=torch.float64, device=dev)
        sim.get_state_into(psi, mb, mf, c)
        torch.cuda.synchronize()
    assert abs(s1["N_psi"] - s0["N_psi"]) <= 1e-6 * s0["N_psi"]
    assert abs(s1["motors"] - 1.0) <= 1e-6 and s1["bound"] > 0.0
    ox, oy = oracle_mod.anchor_offsets(g, r)
    ox = torch.tensor(ox, dtype=torch.long, device=dev)
    oy = torch.tensor(oy, dtype=torch.long, device=dev)
    kk = torch.arange(g.ntheta, device=dev)[:, None].expand(g.ntheta, g.ns)
    jj = torch.arange(g.ns, device=dev)[None, :].expand(g.ntheta, g.ns)
    ds, dth = g.L / g.ns, 2.0 * np.pi / g.ntheta
    rng = np.random.default_rng(251)
    for ay, ax in zip(rng.integers(0, g.ny, 32), rng.integers(0, g.nx, 32)):
        cy = (int(ay) - oy) % g.ny
        cx = (int(ax) - ox) % g.nx
        want = float((psi[cy, cx, kk] * mb[cy, cx, kk, jj]).sum() * ds * dth)
        got = float(c[int(ay), int(ax)])
        assert abs(got - want) <= 1e-5 * abs(want), (int(ay), int(ax), got, want)
        assert abs(float(mf[int(ay), int(ax)]) + got - 1.0) <= 1e-6
