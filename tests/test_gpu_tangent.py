"""The tangent-linear mode (mm_set_tangent): the derivative of the state along
a direction of the rates, advanced with the state by every substep.

* exact tangent: the float64 GPU tangent equals the oracle's tangent substep
  (or_tangent_substep, pinned on the CPU by central differences and the
  adjoint dot-product test) after substeps under two velocity fields, with
  and without the Alg. 2 scale-down, relative 1e-10;
* forward against reverse: the derivative of the polar order and of the mean
  active stress along (dk_off, dv_walk, dk_on) equals the reverse sweep's
  gradient dotted with that direction (relative 1e-10 in float64);
* the state the tangent mode advances is the plain substep's state;
* the float32 tangent against the float64 one, the large case against a
  central difference, and the refusals.
"""
import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import (WORKLOADS, Grid, Rates, SplitMix64,
                                           psi_isotropic_perturbed, random_divfree_flow,
                                           workload_velocity)

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
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


DP = (1.0, 0.3, -0.5)  # d k_off, d v_walk, d k_on


@pytest.mark.parametrize("dims,clip", [((12, 10, 8, 8), False), ((9, 7, 6, 6), False),
                                       ((10, 8, 8, 8), True), ((6, 5, 36, 7), False),
                                       ((5, 4, 6, 64), False)])
def test_tangent_equals_oracle_tangent(mmod, oracle_mod, dims, clip):
    O = oracle_mod
    g = Grid(*dims, L=1.1)
    r = Rates(v_sp=0.1, glide=0.5, k_on=(300.0 if clip else 1.3), k_off=0.7, v_walk=0.9)
    rng = SplitMix64(501)
    psi0 = psi_isotropic_perturbed(g, 502, amp=0.3)
    mb0 = (0.02 if clip else 0.3) * rng.uniforms(g.ny * g.nx * g.ntheta * g.ns).reshape(
        g.ny, g.nx, g.ntheta, g.ns)
    mtot = np.full((g.ny, g.nx), 0.08 if clip else 1.0)
    u1 = random_divfree_flow(g, 503, 6, 0.3)
    u2 = random_divfree_flow(g, 504, 6, 0.3)
    n1, n2 = 5, 6
    dt = 0.01 if clip else 0.006
    with mmod.Simulation(g, r, "fp64") as sim:
        sim.set_tangent(DP)
        sim.set_state(psi0, mb0, mtot)
        sim.set_velocity(u1)
        sim.set_dt(dt)
        sim.step(n1)
        sim.set_velocity(u2)
        sim.set_dt(dt)
        sim.step(n2)
        got = sim.get_tangent()
        st_gpu = sim.get_state()
    st = O.make_state(g, psi0, mb0, mtot)
    tp, tm, tf = np.zeros_like(st.psi), np.zeros_like(st.mb), np.zeros_like(st.mf)
    zero = np.zeros((2, g.ny, g.nx))
    clipped = False
    for u, n in ((u1, n1), (u2, n2)):
        for _ in range(n):
            O.tangent_substep(g, r, dt, u, zero, np.array(DP), st, tp, tm, tf)
            O.run(g, r, st, u, dt, 1)
            clipped = clipped or bool(np.any(st.mf == 0.0))
    assert clipped == clip
    assert rel(st_gpu["psi"], st.psi) <= 1e-12 and rel(st_gpu["mb"], st.mb) <= 1e-12
    assert rel(got["dpsi"], tp) <= 1e-10, rel(got["dpsi"], tp)
    assert rel(got["dmb"], tm) <= 1e-10, rel(got["dmb"], tm)
    assert rel(got["dmf"], tf) <= 1e-10, rel(got["dmf"], tf)


@pytest.mark.parametrize("observable", ["polar_order", "mean_stress"])
def test_tangent_observable_equals_the_reverse_sweep(mmod, observable):
    """Forward mode and reverse mode of the same discrete map: the derivative
    along dp equals dL/drates . dp from mm_adjoint_step."""
    g = Grid(16, 12, 8, 16)
    r = Rates(k_on=1.3, k_off=0.7, glide=0.3)
    psi0 = psi_isotropic_perturbed(g, 511, amp=0.2)
    u = random_divfree_flow(g, 512, 4, 0.3)
    with mmod.Simulation(g, r, "fp64") as sim:
        sim.set_state(psi0)
        sim.set_velocity(u)
        dt = sim.dt
        sim.set_checkpointing(4, 15)
        sim.step(15)
        res = sim.adjoint(15, observable=observable, n_velocities=1, want_du=False,
                          want_dpsi0=False)
        sim.set_checkpointing(0, 1)
        sim.set_tangent(DP)
        sim.set_state(psi0)
        sim.set_velocity(u)
        sim.set_dt(dt)
        sim.step(15)
        val, dval = sim.tangent_observable(observable)
    assert abs(val - res["value"]) <= 1e-13 * abs(res["value"])
    want = float(np.dot(res["dL_drates"], DP))
    assert abs(dval - want) <= 1e-10 * abs(want), (dval, want)


def test_tangent_mode_state_is_the_plain_state(mmod):
    g = Grid(20, 16, 16, 32)
    r = Rates(glide=0.2)
    psi0 = psi_isotropic_perturbed(g, 521, amp=0.2)
    u = random_divfree_flow(g, 522, 6, 0.2)
    outs = []
    for tangent in (False, True):
        with mmod.Simulation(g, r, "fp64") as sim:
            if tangent:
                sim.set_tangent(DP)
            sim.set_state(psi0)
            sim.set_velocity(u)
            sim.step(25)
            outs.append(sim.get_state())
    for k in ("psi", "mb", "mf", "c"):
        assert rel(outs[1][k], outs[0][k]) <= 1e-13, k


def test_tangent_fp32_close_to_fp64(mmod):
    w = WORKLOADS["adjoint64"]
    g, r = w["grid"], Rates()
    psi0 = psi_isotropic_perturbed(g, w["seed"])
    u = workload_velocity("adjoint64", 0)
    got = {}
    for precision in ("fp64", "fp32"):
        with mmod.Simulation(g, r, precision) as sim:
            sim.set_tangent(DP)
            sim.set_state(psi0)
            sim.set_velocity(u)
            sim.set_dt(0.002)
            sim.step(w["substeps"])
            got[precision] = (sim.get_tangent(), sim.tangent_observable("mean_stress"))
    for k in ("dpsi", "dmb", "dmf"):
        assert rel(got["fp32"][0][k], got["fp64"][0][k]) <= 1e-3, k
    assert abs(got["fp32"][1][1] - got["fp64"][1][1]) <= 1e-3 * abs(got["fp64"][1][1])


def test_tangent_large512_matches_fd(mmod):
    """The large case (512x512 x 64 x 64, float32, 20 macro steps x 100
    substeps, a new 16-mode flow each macro step): the derivative of the mean
    active stress with respect to k_off from one run in tangent mode, against
    a central difference (h = 0.005 on k_off = 0.5, the same dt per macro step
    on every run)."""
    w = WORKLOADS["large512"]
    g, nmac, nsub = w["grid"], w["macro"], w["substeps"]
    psi0 = psi_isotropic_perturbed(g, w["seed"])
    vels = [workload_velocity("large512", m) for m in range(nmac)]

    def run(k_off, tangent, dts=None):
        with mmod.Simulation(g, Rates(k_off=k_off), "fp32") as sim:
            if tangent:
                sim.set_tangent((1.0, 0.0, 0.0))
            sim.set_state(psi0)
            got = []
            for m in range(nmac):
                sim.set_velocity(vels[m])
                if dts is not None:
                    sim.set_dt(dts[m])
                got.append(sim.dt)
                sim.step(nsub)
            if tangent:
                return sim.tangent_observable("mean_stress"), got
            return sim.moments(fields=False)[1]["mean_stress"], got

    (val, dval), dts = run(0.5, True)
    h = 0.005
    Lp, _ = run(0.5 + h, False, dts)
    Lm, _ = run(0.5 - h, False, dts)
    fd = (Lp - Lm) / (2 * h)
    print("\nLARGE512_TANGENT", val, dval, fd)
    assert abs(dval - fd) <= 2e-3 * abs(fd), (dval, fd)


def test_tangent_refusals(mmod):
    g = Grid(8, 8, 8, 8)
    with mmod.Simulation(g, Rates(), "fp32") as sim:
        sim.set_state(psi_isotropic_perturbed(g, 3))
        with pytest.raises(mmod.MMError):  # no tangent yet
            sim.tangent_observable()
        sim.set_tangent(DP)
        sim.set_velocity(np.zeros((2, g.ny, g.nx)))
        for call in (lambda: sim.set_checkpointing(2, 4), lambda: sim.diffuse(0.01, 0.1, 0.01),
                     lambda: sim.motor_local(0.1), lambda: sim.set_anchors(True)):
            with pytest.raises(mmod.MMError):
                call()
        sim.set_tangent(None)
        sim.set_checkpointing(2, 4)  # allowed again
    with mmod.Simulation(g, Rates(ell=0.2), "fp32") as sim:
        sim.set_capture(0.1)
        with pytest.raises(mmod.MMError):
            sim.set_tangent(DP)
