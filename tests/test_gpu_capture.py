"""The finite capture radius on the GPU (mm_set_capture) against the oracle's
or_substep_rc / or_moments_rc: the template (lines and binding weights) equal
to the oracle's exactly, the state after substeps with flow, gliding, walking
and a forced scale-down within relative L2 1e-12 in float64 and 1e-5 in
float32, on ragged grids with capture radii of about one to three cells, the
moments (n_b and m1 summed over the anchors, the force at the heads), the
zero-length zero-radius limit against the plain GPU path, and the refusals.
"""
import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import (Grid, Rates, SplitMix64, psi_isotropic_perturbed,
                                           random_divfree_flow)

pytestmark = pytest.mark.gpu

CASES = [  # grid, l/L, r_c (in cells of the x spacing: about 1, 2 and 3 cells)
    ((12, 10, 8, 12), 0.31, 1.1 / 12),
    ((16, 14, 6, 7), 0.27, 2.05 / 16),
    ((20, 18, 8, 16), 0.19, 3.02 / 20),
    ((10, 9, 40, 20), 0.23, 1.3 / 10),   # more orientations than lanes
    ((12, 12, 6, 64), 0.3, 1.2 / 12),    # lines of up to 64 nodes
]


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
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _inputs(O, g, r, rc, seed, mb_scale=1.0, mtot_lo=0.5, mtot_span=0.5):
    tpl = O.rc_template(g, r, rc)
    rng = SplitMix64(seed)
    psi = psi_isotropic_perturbed(g, seed + 1, amp=0.4)
    mb = mb_scale / tpl.nconf * rng.uniforms(g.ny * g.nx * tpl.nconf).reshape(
        g.ny, g.nx, tpl.nconf)
    mtot = mtot_lo + mtot_span * rng.uniforms(g.ny * g.nx).reshape(g.ny, g.nx)
    u = random_divfree_flow(g, seed + 2, 4, 0.25)
    return tpl, psi, mb, mtot, u


def _gpu_run(mmod, g, r, rc, precision, psi, mb, mtot, u, dt, n):
    with mmod.Simulation(g, r, precision) as sim:
        sim.set_capture(rc)
        sim.set_state(psi, mb, mtot)
        sim.set_velocity(u)
        sim.set_dt(dt)
        sim.step(n)
        st = sim.get_state()
        f, sc = sim.moments(fields=True)
    return st, f, sc


@pytest.mark.parametrize("dims,ell,rc", CASES)
def test_capture_template_equals_the_oracle(mmod, oracle_mod, dims, ell, rc):
    g, r = Grid(*dims), Rates(ell=ell)
    tpl = oracle_mod.rc_template(g, r, rc)
    with mmod.Simulation(g, r, "fp64") as sim:
        t = sim.set_capture(rc)
    assert t["nconf"] == tpl.nconf
    assert np.array_equal(t["lines"], tpl.lines)
    assert np.array_equal(t["w"], tpl.w)
    assert tpl.w.min() < 0.5  # several anchors in reach of a node


@pytest.mark.parametrize("dims,ell,rc", CASES)
def test_capture_fp64_equals_the_oracle(mmod, oracle_mod, dims, ell, rc):
    """12 substeps with flow, gliding and walking: psi, Mb (every
    configuration of every anchor), Mf, C and the moments to 1e-12."""
    O = oracle_mod
    g = Grid(*dims)
    r = Rates(ell=ell, k_on=1.6, k_off=0.6, glide=0.3, v_sp=0.05, force_scale=0.8)
    tpl, psi, mb, mtot, u = _inputs(O, g, r, rc, 401 + sum(dims))
    st = O.make_state_rc(g, r, rc, psi, mb, mtot)
    dt = 0.7 * O.dt(g, r, O.make_state(g, psi), u)
    O.run_rc(g, r, rc, st, u, dt, 12)
    got, f, sc = _gpu_run(mmod, g, r, rc, "fp64", psi, mb, mtot, u, dt, 12)
    for k in ("psi", "mb", "mf", "c"):
        assert rel(got[k], getattr(st, k)) <= 1e-12, (k, rel(got[k], getattr(st, k)))
    fo, sco = O.moments_rc(g, r, rc, st)
    for name, field in fo.items():
        assert rel(f[name], field) <= 1e-12, (name, rel(f[name], field))
    for name in ("N_psi", "bound", "free", "motors", "polar_order"):
        assert abs(sc[name] - sco[name]) <= 1e-12 * max(1.0, abs(sco[name])), name


def test_capture_forced_scale_down_fp64(mmod, oracle_mod):
    """Fast binding against scarce motors: the Alg. 2 scale-down at the
    anchors acts (Mf = 0 at some anchors) and the state still equals the
    oracle's."""
    O = oracle_mod
    dims, ell, rc = (10, 9, 6, 10), 0.33, 1.6 / 10
    g = Grid(*dims)
    r = Rates(ell=ell, k_on=60.0, glide=0.2)
    tpl, psi, mb, mtot, u = _inputs(O, g, r, rc, 431, mb_scale=0.05, mtot_lo=0.02, mtot_span=0.03)
    st = O.make_state_rc(g, r, rc, psi, mb, mtot)
    dt = 4.0 * O.dt(g, r, O.make_state(g, psi), u)
    clipped = False
    with mmod.Simulation(g, r, "fp64") as sim:
        sim.set_capture(rc)
        sim.set_state(psi, mb, mtot)
        sim.set_velocity(u)
        sim.set_dt(dt)
        for _ in range(4):
            sim.step(1)
            O.run_rc(g, r, rc, st, u, dt, 1)
            clipped = clipped or bool(np.any(st.mf == 0.0))
        got = sim.get_state()
    assert clipped
    for k in ("psi", "mb", "mf", "c"):
        assert rel(got[k], getattr(st, k)) <= 1e-12, (k, rel(got[k], getattr(st, k)))


@pytest.mark.parametrize("dims,ell,rc", CASES[:2] + CASES[4:])
def test_capture_fp32_close_to_the_oracle(mmod, oracle_mod, dims, ell, rc):
    O = oracle_mod
    g = Grid(*dims)
    r = Rates(ell=ell, k_on=1.6, k_off=0.6, glide=0.3)
    tpl, psi, mb, mtot, u = _inputs(O, g, r, rc, 451 + sum(dims))
    st = O.make_state_rc(g, r, rc, psi, mb, mtot)
    dt = 0.7 * O.dt(g, r, O.make_state(g, psi), u)
    O.run_rc(g, r, rc, st, u, dt, 20)
    got, f, sc = _gpu_run(mmod, g, r, rc, "fp32", psi, mb, mtot, u, dt, 20)
    for k in ("psi", "mb", "mf", "c"):
        assert rel(got[k], getattr(st, k)) <= 1e-5, (k, rel(got[k], getattr(st, k)))
    fo, _ = O.moments_rc(g, r, rc, st)
    for name in ("rho", "C", "Fx", "Fy", "Sxx"):
        assert rel(f[name], fo[name]) <= 1e-5, (name, rel(f[name], fo[name]))


def test_capture_zero_length_zero_radius_is_the_plain_path(mmod):
    """l/L = 0, r_c = 0: one anchor (the filament's cell) and one full walking
    line per row: the capture-radius kernels give the plain substep's state
    (1e-12 in float64; its Mb layout is the plain one)."""
    g = Grid(9, 8, 8, 16)
    r = Rates(ell=0.0, k_on=1.4, glide=0.3)
    rng = SplitMix64(461)
    psi = psi_isotropic_perturbed(g, 462, amp=0.4)
    mb = 0.2 * rng.uniforms(g.ny * g.nx * g.ntheta * g.ns).reshape(g.ny, g.nx, g.ntheta, g.ns)
    u = random_divfree_flow(g, 463, 4, 0.25)
    outs = []
    for rc in (0.0, None):
        with mmod.Simulation(g, r, "fp64") as sim:
            if rc is not None:
                t = sim.set_capture(rc)
                assert t["nconf"] == g.ntheta * g.ns
            sim.set_state(psi, mb.reshape(g.ny, g.nx, -1) if rc is not None else mb)
            sim.set_velocity(u)
            sim.set_dt(0.004)
            sim.step(15)
            outs.append(sim.get_state())
    for k in ("psi", "mf", "c"):
        assert rel(outs[0][k], outs[1][k]) <= 1e-12, k
    assert rel(outs[0]["mb"].reshape(outs[1]["mb"].shape), outs[1]["mb"]) <= 1e-12


def test_capture_refusals_and_switching(mmod):
    g = Grid(8, 8, 4, 8)
    r = Rates(ell=0.2)
    with mmod.Simulation(g, r, "fp32") as sim:
        sim.set_state(psi_isotropic_perturbed(g, 3))
        sim.set_capture(0.15)
        st = sim.get_state()
        assert st["mb"].shape == (g.ny, g.nx, sim.capture_template()["nconf"])
        assert np.all(st["mb"] == 0.0) and np.allclose(st["mf"], 1.0)
        for call in (lambda: sim.set_anchors(True), lambda: sim.set_checkpointing(2, 4),
                     lambda: sim.motor_local(0.1), lambda: sim.snapshot(),
                     lambda: sim.set_rates(Rates(ell=0.3))):
            with pytest.raises(mmod.MMError):
                call()
        sim.set_rates(Rates(ell=0.2, k_on=2.0))  # the same l/L: allowed
        sim.set_velocity(np.zeros((2, g.ny, g.nx)))
        sim.step(3)
        assert np.all(sim.get_state()["mb"] > 0.0)
        sim.set_capture(-1.0)  # back to the plain model, motors discarded
        st = sim.get_state()
        assert st["mb"].shape == (g.ny, g.nx, g.ntheta, g.ns) and np.all(st["mb"] == 0.0)
        with pytest.raises(mmod.MMError):  # a reach wider than the grid
            sim.set_capture(0.6)


def test_capture_precision128_full_size(mmod, oracle_mod):
    """The bench's capture workload at full size (128^2 x 32^2, l/L = 0.05,
    r_c = 1.5 cells: 14422 configurations per anchor, float32, the workload's
    flow) against the float64 oracle, element by element, after one substep
    from a seeded bound state."""
    from paper_1908_04279_gb300.inputs import WORKLOADS, workload_velocity
    O = oracle_mod
    w = WORKLOADS["precision128"]
    g = w["grid"]
    r = Rates(ell=0.05)
    rc = 1.5 / g.nx
    tpl = O.rc_template(g, r, rc)
    assert tpl.nconf == 14422
    rng = SplitMix64(471)
    psi = psi_isotropic_perturbed(g, w["seed"])
    mb = (0.3 / tpl.nconf) * rng.uniforms(g.ny * g.nx * tpl.nconf).reshape(g.ny, g.nx, tpl.nconf)
    mtot = np.ones((g.ny, g.nx))
    u = workload_velocity("precision128", 0)
    st = O.make_state_rc(g, r, rc, psi, mb, mtot)
    dt = O.dt(g, r, O.make_state(g, psi), u)
    O.run_rc(g, r, rc, st, u, dt, 1)
    got, f, sc = _gpu_run(mmod, g, r, rc, "fp32", psi, mb, mtot, u, dt, 1)
    for k in ("psi", "mb", "mf", "c"):
        assert rel(got[k], getattr(st, k)) <= 1e-5, (k, rel(got[k], getattr(st, k)))
