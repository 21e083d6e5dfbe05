"""GPU adjoint (mm_set_checkpointing / mm_adjoint_step) against the float64
oracle's adjoint and against central finite differences of the GPU forward.

* exact transpose: random seeds in moment form (dL/dpsi, dL/dn_b, dL/dm1,
  dL/dMf) and on the whole state (dL/dpsi, dL/dMb, dL/dMf), two velocity fields during the recording, segments shorter than the
  run (checkpoint recompute), with and without the Alg. 2 scale-down; the
  float64 GPU sweep equals the oracle's reverse sweep to relative 1e-10;
* central differences (h = 1e-6, dt held fixed) of the polar order after 100
  substeps on the 64x64 x 32 x 32 adjoint workload, for k_off, v_walk, 20
  seeded velocity entries and 5 initial psi entries: relative 1e-6, except
  entries within h of a limiter or upwind switch (detected by disagreeing
  one-sided differences), which must lie between the one-sided differences;
* the float32 sweep against the float64 sweep.
"""
import math

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


@pytest.mark.parametrize("dims,clip", [((12, 10, 8, 8), False), ((9, 7, 6, 5), False),
                                       ((10, 8, 8, 8), True)])
def test_adjoint_equals_oracle_adjoint(mmod, oracle_mod, dims, clip):
    O = oracle_mod
    g = Grid(*dims, L=1.1)
    r = Rates(v_sp=0.1, glide=0.5, k_on=(300.0 if clip else 1.3), k_off=0.7, v_walk=0.9)
    rng = SplitMix64(101)
    psi0 = psi_isotropic_perturbed(g, 102, amp=0.3)
    mb0 = (0.02 if clip else 0.3) * rng.uniforms(g.ny * g.nx * g.ntheta * g.ns).reshape(
        g.ny, g.nx, g.ntheta, g.ns)
    mtot = np.full((g.ny, g.nx), 0.08 if clip else 1.0)
    u1 = random_divfree_flow(g, 103, 6, 0.3)
    u2 = random_divfree_flow(g, 104, 6, 0.3)
    n1, n2, K = 7, 6, 4
    dpsi = rng.uniforms(g.ny * g.nx * g.ntheta).reshape(g.ny, g.nx, g.ntheta) - 0.5
    dnb = rng.uniforms(g.ny * g.nx * g.ntheta).reshape(g.ny, g.nx, g.ntheta) - 0.5
    dm1 = rng.uniforms(g.ny * g.nx * g.ntheta).reshape(g.ny, g.nx, g.ntheta) - 0.5
    dmf = rng.uniforms(g.ny * g.nx).reshape(g.ny, g.nx) - 0.5
    dt_fixed = 0.01 if clip else None
    with mmod.Simulation(g, r, "fp64") as sim:
        sim.set_state(psi0, mb0, mtot)
        sim.set_velocity(u1)
        if dt_fixed:
            sim.set_dt(dt_fixed)
        dt1 = sim.dt
        sim.set_checkpointing(K, n1 + n2)
        sim.step(n1)
        sim.set_velocity(u2)
        if dt_fixed:
            sim.set_dt(dt_fixed)
        dt2 = sim.dt
        sim.step(n2)
        nv = 3 if dt_fixed else 2
        res = sim.adjoint(n1 + n2, dL_dpsi=dpsi, dL_dnb=dnb, dL_dm1=dm1, dL_dmf=dmf,
                          n_velocities=nv)
    # oracle: forward with stored states, then the reverse sweep
    st = O.make_state(g, psi0, mb0, mtot)
    states, vel, dts = [], [], []
    for u, dt, n in ((u1, dt1, n1), (u2, dt2, n2)):
        for _ in range(n):
            states.append(st.copy())
            vel.append(0 if u is u1 else 1)
            dts.append(dt)
            O.run(g, r, st, u, dt, 1)
    ds = g.L / g.ns
    s = -g.L / 2 + (np.arange(g.ns) + 0.5) * ds
    lpsi = dpsi.copy()
    lmb = dnb[..., None] * ds + dm1[..., None] * s * ds
    lmf = dmf.copy()
    lu = [np.zeros((2, g.ny, g.nx)), np.zeros((2, g.ny, g.nx))]
    lp = np.zeros(3)
    for i in range(len(states) - 1, -1, -1):
        O.adjoint_substep(g, r, dts[i], (u1, u2)[vel[i]], states[i], lpsi, lmb, lmf, lu[vel[i]], lp)
    nb0 = (states[0].mb * ds).sum(-1)
    lpsi0 = lpsi - lmf[..., None] * nb0 * (2 * math.pi / g.ntheta)
    gdu = res["dL_du"]
    du1 = gdu[0]
    du2 = gdu[1:].sum(0)  # the second velocity may carry a (u2, auto dt) block with no substeps
    assert rel(du1, lu[0]) <= 1e-10, rel(du1, lu[0])
    assert rel(du2, lu[1]) <= 1e-10, rel(du2, lu[1])
    assert rel(res["dL_drates"], lp) <= 1e-10, (res["dL_drates"], lp)
    assert rel(res["dL_dpsi0"], lpsi0) <= 1e-10, rel(res["dL_dpsi0"], lpsi0)
    if clip:
        assert np.count_nonzero([np.any(x.mf == 0.0) for x in states[1:]]) > 0


def _full_seed_run(mmod, g, r, psi0, mb0, u, n, K, seeds, precision, device=False):
    import torch
    with mmod.Simulation(g, r, precision) as sim:
        sim.set_state(psi0, mb0)
        sim.set_velocity(u)
        dt = sim.dt
        sim.set_checkpointing(K, n)
        sim.step(n)
        if device:
            seeds = {k: torch.tensor(v, device="cuda") for k, v in seeds.items()}
        res = sim.adjoint(n, **seeds, n_velocities=1)
    return res, dt


@pytest.mark.parametrize("dims,moment_seeds", [((12, 10, 8, 8), True), ((9, 7, 6, 5), False),
                                               ((6, 5, 16, 32), True)])
def test_full_state_seed_equals_oracle_adjoint(mmod, oracle_mod, dims, moment_seeds):
    """A seed on the whole final state -- dL/dpsi, dL/dMb (every node of every
    row), dL/dMf, with or without the moment seeds dL/dn_b, dL/dm1 added to the
    rows -- gives the oracle's reverse sweep started from lam_Mb = dL/dMb +
    dL/dn_b ds + dL/dm1 s ds (relative 1e-10 in float64, host and device
    seeds alike); the float32 sweep agrees with the float64 one to 1e-3."""
    O = oracle_mod
    g = Grid(*dims, L=1.1)
    r = Rates(v_sp=0.1, glide=0.5, k_on=1.3, k_off=0.7, v_walk=0.9)
    rng = SplitMix64(301 + sum(dims))
    psi0 = psi_isotropic_perturbed(g, 302, amp=0.3)
    mb0 = 0.3 * rng.uniforms(g.ny * g.nx * g.ntheta * g.ns).reshape(g.ny, g.nx, g.ntheta, g.ns)
    u = random_divfree_flow(g, 303, 6, 0.3)
    n, K = 9, 4
    seeds = dict(
        dL_dpsi=rng.uniforms(g.ny * g.nx * g.ntheta).reshape(g.ny, g.nx, g.ntheta) - 0.5,
        dL_dmb=rng.uniforms(g.ny * g.nx * g.ntheta * g.ns).reshape(g.ny, g.nx, g.ntheta, g.ns)
        - 0.5,
        dL_dmf=rng.uniforms(g.ny * g.nx).reshape(g.ny, g.nx) - 0.5)
    if moment_seeds:
        seeds["dL_dnb"] = rng.uniforms(g.ny * g.nx * g.ntheta).reshape(g.ny, g.nx, g.ntheta) - 0.5
        seeds["dL_dm1"] = rng.uniforms(g.ny * g.nx * g.ntheta).reshape(g.ny, g.nx, g.ntheta) - 0.5
    res, dt = _full_seed_run(mmod, g, r, psi0, mb0, u, n, K, seeds, "fp64")
    res_dev, _ = _full_seed_run(mmod, g, r, psi0, mb0, u, n, K, seeds, "fp64", device=True)
    st = O.make_state(g, psi0, mb0)
    states = O.substep_states(g, r, st, u, dt, n)
    ds = g.L / g.ns
    s = -g.L / 2 + (np.arange(g.ns) + 0.5) * ds
    lpsi = seeds["dL_dpsi"].copy()
    lmb = seeds["dL_dmb"].copy()
    if moment_seeds:
        lmb += seeds["dL_dnb"][..., None] * ds + seeds["dL_dm1"][..., None] * s * ds
    lmf = seeds["dL_dmf"].copy()
    lu, lp = np.zeros((2, g.ny, g.nx)), np.zeros(3)
    for i in range(n - 1, -1, -1):
        O.adjoint_substep(g, r, dt, u, states[i], lpsi, lmb, lmf, lu, lp)
    nb0 = (states[0].mb * ds).sum(-1)
    lpsi0 = lpsi - lmf[..., None] * nb0 * (2 * math.pi / g.ntheta)
    for rr in (res, res_dev):
        assert rel(rr["dL_du"][0], lu) <= 1e-10, rel(rr["dL_du"][0], lu)
        assert rel(rr["dL_drates"], lp) <= 1e-10, (rr["dL_drates"], lp)
        assert rel(rr["dL_dpsi0"], lpsi0) <= 1e-10, rel(rr["dL_dpsi0"], lpsi0)
    # the motor seed matters: without it the gradients differ
    no_mb = {k: v for k, v in seeds.items() if k != "dL_dmb"}
    res_no, _ = _full_seed_run(mmod, g, r, psi0, mb0, u, n, K, no_mb, "fp64")
    assert rel(res_no["dL_drates"], lp) > 1e-3
    r32, _ = _full_seed_run(mmod, g, r, psi0, mb0, u, n, K, seeds, "fp32")
    assert rel(r32["dL_du"][0], lu) <= 1e-3, rel(r32["dL_du"][0], lu)
    assert rel(r32["dL_drates"], lp) <= 1e-3, (r32["dL_drates"], lp)
    assert rel(r32["dL_dpsi0"], lpsi0) <= 1e-3, rel(r32["dL_dpsi0"], lpsi0)


def _polar_order(mmod, g, r, psi0, u, dt, n, precision="fp64"):
    with mmod.Simulation(g, r, precision) as sim:
        sim.set_state(psi0)
        sim.set_velocity(u)
        sim.set_dt(dt)
        sim.step(n)
        _, sc = sim.moments(fields=False)
    return sc["polar_order"]


def _adjoint_run(mmod, g, r, psi0, u, n, K, precision):
    with mmod.Simulation(g, r, precision) as sim:
        sim.set_state(psi0)
        sim.set_velocity(u)
        dt = sim.dt
        sim.set_dt(dt)
        sim.set_checkpointing(K, n)
        sim.step(n)
        res = sim.adjoint(n, observable="polar_order", n_velocities=2)
    res["dL_du"] = res["dL_du"].sum(0)
    return res, dt


def test_adjoint_matches_central_differences(mmod):
    """Polar order after 100 substeps on the 64x64 x 32 x 32 adjoint workload,
    checkpoint every 10 substeps, central differences with h = 1e-6 at fixed dt.

    The discrete map is piecewise smooth: the Superbee limiter and the upwind
    choice switch branches, and a perturbation of size h can cross a switch.
    An entry passes when the adjoint matches the central difference to 1e-6
    relative; where the two one-sided differences disagree (a switch lies
    within h) it must lie between them instead, and at most 3 of the 27
    entries may need that."""
    w = WORKLOADS["adjoint64"]
    g, r = w["grid"], Rates()
    psi0 = psi_isotropic_perturbed(g, w["seed"])
    u = workload_velocity("adjoint64", 0)
    n = w["substeps"]
    res, dt = _adjoint_run(mmod, g, r, psi0, u, n, 10, "fp64")
    h = 1e-6
    L0 = _polar_order(mmod, g, r, psi0, u, dt, n)
    assert res["value"] == pytest.approx(L0, rel=1e-12)
    # each entry: (name, adjoint, perturbed evaluation L(rates, u, psi0) for a step e)
    entries = []
    for q, name in enumerate(("k_off", "v_walk")):
        def ev(e, name=name):
            return _polar_order(mmod, g, Rates(**{**r.__dict__, name: getattr(r, name) + e}),
                                psi0, u, dt, n)
        entries.append((name, res["dL_drates"][q], ev))
    rng = SplitMix64(7)
    for _ in range(20):
        c, iy, ix = int(rng.uniform() * 2), int(rng.uniform() * g.ny), int(rng.uniform() * g.nx)
        def ev(e, c=c, iy=iy, ix=ix):
            up = u.copy()
            up[c, iy, ix] += e
            return _polar_order(mmod, g, r, psi0, up, dt, n)
        entries.append((f"u[{c},{iy},{ix}]", res["dL_du"][c, iy, ix], ev))
    for _ in range(5):
        iy, ix, k = int(rng.uniform() * g.ny), int(rng.uniform() * g.nx), int(rng.uniform() * g.ntheta)
        def ev(e, iy=iy, ix=ix, k=k):
            pp = psi0.copy()
            pp[iy, ix, k] += e
            return _polar_order(mmod, g, r, pp, u, dt, n)
        entries.append((f"psi0[{iy},{ix},{k}]", res["dL_dpsi0"][iy, ix, k], ev))

    def judge(adj, Lp, Lm, hh, scale):
        fd = (Lp - Lm) / (2 * hh)
        fwd, bwd = (Lp - L0) / hh, (L0 - Lm) / hh
        tol = 1e-6 * max(abs(fd), 1e-2 * scale)
        if abs(adj - fd) <= tol:
            return "ok", fd
        if abs(fwd - bwd) > 4 * tol:  # a switch lies within hh
            inside = min(fwd, bwd) - tol <= adj <= max(fwd, bwd) + tol
            return ("kink-bracketed" if inside else "kink"), fd
        return "bad", fd

    evals = [(nm, adj, ev, ev(h), ev(-h)) for nm, adj, ev in entries]
    scale = max(abs(Lp - Lm) / (2 * h) for _, _, _, Lp, Lm in evals)
    report, kinks, bad = [], [], []
    for nm, adj, ev, Lp, Lm in evals:
        verdict, fd = judge(adj, Lp, Lm, h, scale)
        if verdict == "kink":  # retry closer to the point
            verdict, fd = judge(adj, ev(0.1 * h), ev(-0.1 * h), 0.1 * h, scale)
            verdict = "ok-at-h/10" if verdict == "ok" else verdict
        report.append((nm, float(adj), float(fd), verdict))
        if verdict.startswith("kink") or verdict == "ok-at-h/10":
            kinks.append(nm)
        if verdict in ("bad", "kink"):
            bad.append((nm, adj, fd))
    print("\nFD_CHECKS", report, "KINKS", kinks)
    assert not bad, bad
    assert len(kinks) <= 3, kinks


def test_fp32_adjoint_close_to_fp64(mmod):
    w = WORKLOADS["adjoint64"]
    g, r = w["grid"], Rates()
    psi0 = psi_isotropic_perturbed(g, w["seed"])
    u = workload_velocity("adjoint64", 0)
    r64, _ = _adjoint_run(mmod, g, r, psi0, u, w["substeps"], 10, "fp64")
    r32, _ = _adjoint_run(mmod, g, r, psi0, u, w["substeps"], 10, "fp32")
    print("\nFP32_ADJ", rel(r32["dL_du"], r64["dL_du"]), rel(r32["dL_drates"], r64["dL_drates"]),
          rel(r32["dL_dpsi0"], r64["dL_dpsi0"]))
    assert rel(r32["dL_du"], r64["dL_du"]) <= 1e-3
    assert rel(r32["dL_drates"], r64["dL_drates"]) <= 1e-3
    assert rel(r32["dL_dpsi0"], r64["dL_dpsi0"]) <= 1e-3


def test_recording_reuse_is_repeatable(mmod):
    """A second recording with the same K and max_substeps reuses the first
    one's memory (set_state ends a recording and keeps it) and gives the same
    gradients bit for bit; set_state or set_rates without a new
    mm_set_checkpointing leaves no recording to differentiate."""
    g = Grid(16, 12, 8, 16, L=1.0)
    r = Rates(k_on=1.3, k_off=0.7)
    psi0 = psi_isotropic_perturbed(g, 11, amp=0.2)
    u1 = random_divfree_flow(g, 12, 4, 0.3)
    u2 = random_divfree_flow(g, 13, 4, 0.3)
    outs = []
    with mmod.Simulation(g, r, "fp32") as sim:
        for _ in range(3):
            sim.set_state(psi0)
            sim.set_velocity(u1)
            sim.set_checkpointing(3, 10)
            sim.step(4)
            sim.set_velocity(u2)
            sim.step(5)
            outs.append(sim.adjoint(9, observable="polar_order", n_velocities=2))
        sim.set_state(psi0)
        with pytest.raises(RuntimeError):
            sim.adjoint(9, observable="polar_order", n_velocities=2)
        # new rates end a recording: the substeps taken so far ran with the
        # old ones, so the reverse sweep is refused rather than mixing them
        sim.set_state(psi0)
        sim.set_velocity(u1)
        sim.set_checkpointing(3, 10)
        sim.step(4)
        sim.set_rates(Rates(k_on=1.3, k_off=0.9))
        with pytest.raises(mmod.MMError) as err:
            sim.adjoint(4, observable="polar_order")
        assert mmod.STATUS[err.value.status] == "MM_ERR_STATE"
    for o in outs[1:]:
        assert o["value"] == outs[0]["value"]
        assert np.array_equal(o["dL_du"], outs[0]["dL_du"])
        assert np.array_equal(o["dL_dpsi0"], outs[0]["dL_dpsi0"])
        assert np.array_equal(o["dL_drates"], outs[0]["dL_drates"])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_two_level_checkpoints_equal_one_level(mmod, precision):
    """Outer checkpoints every 10 substeps with inner checkpoints every 3
    rebuilt in the reverse sweep (ragged inner and outer segments, a velocity
    change inside an outer segment) give the same gradients, bit for bit, as
    one level of checkpoints every 10: the recomputed states are the same."""
    g = Grid(12, 10, 8, 16, L=1.0)
    r = Rates(k_on=1.3, k_off=0.7, glide=0.3)
    psi0 = psi_isotropic_perturbed(g, 31, amp=0.2)
    u1 = random_divfree_flow(g, 32, 4, 0.3)
    u2 = random_divfree_flow(g, 33, 4, 0.3)
    out = []
    for K_inner in (10, 3, 1):
        with mmod.Simulation(g, r, precision) as sim:
            sim.set_state(psi0)
            sim.set_velocity(u1)
            sim.set_checkpointing(10, 27, K_inner=K_inner)
            sim.step(14)
            sim.set_velocity(u2)
            sim.step(13)
            out.append(sim.adjoint(27, observable="mean_stress", n_velocities=2))
    for o in out[1:]:
        assert o["value"] == out[0]["value"]
        assert np.array_equal(o["dL_drates"], out[0]["dL_drates"])
        assert np.array_equal(o["dL_du"], out[0]["dL_du"])
        assert np.array_equal(o["dL_dpsi0"], out[0]["dL_dpsi0"])


def test_large512_two_level_adjoint_matches_fd(mmod):
    """The large case (512x512 x 64 x 64, float32, 20 macro steps x 100
    substeps with a new 16-mode flow each macro step): forward plus adjoint of
    the mean active stress with respect to k_off, outer checkpoints every 100
    substeps and inner ones every 10 (40 states of 4.4 GB on the device, where
    one level would need about 90), against a central difference
    (h = 0.005 on k_off = 0.5, the same dt per macro step on every run)."""
    w = WORKLOADS["large512"]
    g, nmac, nsub = w["grid"], w["macro"], w["substeps"]
    psi0 = psi_isotropic_perturbed(g, w["seed"])
    vels = [workload_velocity("large512", m) for m in range(nmac)]

    def run(k_off, record, dts=None):
        with mmod.Simulation(g, Rates(k_off=k_off), "fp32") as sim:
            sim.set_state(psi0)
            got = []
            for m in range(nmac):
                sim.set_velocity(vels[m])
                if dts is not None:
                    sim.set_dt(dts[m])
                got.append(sim.dt)
                if m == 0 and record:
                    sim.set_checkpointing(100, nmac * nsub, K_inner=10)
                sim.step(nsub)
            if record:
                res = sim.adjoint(nmac * nsub, observable="mean_stress", n_velocities=2 * nmac,
                                  want_du=False, want_dpsi0=False)
                return res, got
            return sim.moments(fields=False)[1]["mean_stress"], got

    res, dts = run(0.5, True)
    h = 0.005
    Lp, _ = run(0.5 + h, False, dts)
    Lm, _ = run(0.5 - h, False, dts)
    fd = (Lp - Lm) / (2 * h)
    print("\nLARGE512_ADJ", res["value"], res["dL_drates"][0], fd)
    assert abs(res["dL_drates"][0] - fd) <= 2e-3 * abs(fd), (res["dL_drates"][0], fd)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_recorded_tail_segment(mmod, precision):
    """With one level of checkpoints the recording writes its last segment
    straight into the slots (split over calls here, with a velocity change
    inside it): the live state after the recording, the observable and the
    gradients equal, bit for bit, those of a recording whose reservation is
    longer (so that every segment is recomputed in the reverse sweep)."""
    g = Grid(10, 12, 8, 16, L=1.0)
    r = Rates(k_on=1.3, k_off=0.7, glide=0.3)
    psi0 = psi_isotropic_perturbed(g, 41, amp=0.2)
    u1 = random_divfree_flow(g, 42, 4, 0.3)
    u2 = random_divfree_flow(g, 43, 4, 0.3)
    outs, states = [], []
    for reserve in (23, 40):
        with mmod.Simulation(g, r, precision) as sim:
            sim.set_state(psi0)
            sim.set_velocity(u1)
            sim.set_checkpointing(5, reserve)
            sim.step(21)
            sim.set_velocity(u2)
            sim.step(1)
            sim.step(1)
            states.append(sim.get_state())
            outs.append(sim.adjoint(23, observable="mean_stress", n_velocities=2))
    for k in ("psi", "mb", "mf", "c"):
        assert np.array_equal(states[0][k], states[1][k]), k
    assert outs[0]["value"] == outs[1]["value"]
    assert np.array_equal(outs[0]["dL_drates"], outs[1]["dL_drates"])
    assert np.array_equal(outs[0]["dL_du"], outs[1]["dL_du"])
    assert np.array_equal(outs[0]["dL_dpsi0"], outs[1]["dL_dpsi0"])
