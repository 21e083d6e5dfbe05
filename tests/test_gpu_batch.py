"""Batched ensemble (mm_create_batch): one launch per substep over members
with uneven grids, rates and dt.

* float64: every member equals the float64 oracle run of that member to
  relative 1e-12 and the same member stepped alone by the single-instance
  kernel bit for bit (same arithmetic; float64 applies no mass correction);
* float32: every member within 1e-5 of the oracle and 1e-6 of the member
  stepped alone (the mass-correction sums are grouped by tile instead of by
  warp);
* graph and direct launches, members stepped alone in between (their
  parities diverge), odd and even substep counts;
* members with at most 16 orientations and an even row length go two cells
  to a warp (8 and 16 orientations), one with an odd row length one;
* the autotuner leaves the state as it found it;
* a member recording an adjoint during batched substeps gives the adjoint of
  the same member recorded alone;
* a bounded wait that runs out is reported per batch and the batch recovers.
"""
import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import (Grid, Member, Rates, ensemble_members,
                                           member_inputs)

pytestmark = pytest.mark.gpu

# uneven members: grids, angle and arclength counts, rates; members 0, 1, 3
# and 6 go two cells to a warp (at most 16 orientations, even nx), member 2
# (32 x 16) in float32 in units of two cells taken in turn, member 5 (odd nx)
# one cell per warp
SHAPES = [((8, 8, 16, 16), 0.3, 1.0), ((12, 10, 16, 32), 2.0, 0.6), ((6, 7, 32, 16), 0.07, 1.7),
          ((16, 16, 16, 16), 0.5, 1.0), ((9, 5, 32, 32), 4.0, 1.2), ((7, 6, 16, 16), 1.1, 0.8),
          ((10, 6, 8, 32), 0.9, 1.4)]


@pytest.fixture(scope="module")
def mmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_04279_gb300 import build as B
    B.build()
    from paper_1908_04279_gb300 import mm
    return mm


def members():
    out = []
    for i, (dims, koff, vw) in enumerate(SHAPES):
        out.append(Member(Grid(*dims), Rates(k_off=koff, v_walk=vw, glide=0.3), 500 + i))
    return out


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def setup(batch, ms):
    for sim, m in zip(batch.members, ms):
        psi0, u = member_inputs(m, modes=4, amp=0.3)
        sim.set_state(psi0)
        sim.set_velocity(u)


def alone(mmod, m, precision, n_list):
    psi0, u = member_inputs(m, modes=4, amp=0.3)
    with mmod.Simulation(m.grid, m.rates, precision) as sim:
        sim.set_state(psi0)
        sim.set_velocity(u)
        for n in n_list:
            sim.step(n)
        return sim.get_state()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_members_and_oracle(mmod, oracle_mod, precision):
    ms = members()
    with mmod.Batch([m.grid for m in ms], [m.rates for m in ms], precision) as b:
        setup(b, ms)
        dts = [s.dt for s in b.members]
        b.step(7)      # graph, odd
        b.step(4)      # graph, even
        b.members[1].step(1)  # one member alone: parities diverge
        b.step(3)
        b.sync()
        states = [s.get_state() for s in b.members]
    for i, m in enumerate(ms):
        n_i = 14 + (1 if i == 1 else 0)
        st = alone(mmod, m, precision, [n_i])
        o = oracle_mod.make_state(m.grid, *member_inputs(m, modes=4, amp=0.3)[:1])
        _, u = member_inputs(m, modes=4, amp=0.3)
        oracle_mod.run(m.grid, m.rates, o, u, dts[i], n_i)
        tol_o = 1e-12 if precision == "fp64" else 1e-5
        assert rel(states[i]["psi"], o.psi) <= tol_o, (i, rel(states[i]["psi"], o.psi))
        assert rel(states[i]["mb"], o.mb) <= tol_o, (i, rel(states[i]["mb"], o.mb))
        assert rel(states[i]["mf"], o.mf) <= tol_o, (i, rel(states[i]["mf"], o.mf))
        if precision == "fp64":
            for k in ("psi", "mb", "mf", "c"):
                assert np.array_equal(states[i][k], st[k]), (i, k)
        else:
            for k in ("psi", "mb", "mf"):
                assert rel(states[i][k], st[k]) <= 1e-6, (i, k, rel(states[i][k], st[k]))


def test_batch_autotune_restores_state(mmod):
    ms = members()
    with mmod.Batch([m.grid for m in ms], [m.rates for m in ms], "fp32") as b:
        setup(b, ms)
        b.step(3)
        before = [s.get_state() for s in b.members]
        res = b.autotune(substeps=2)
        info = b.launch_info()
        after = [s.get_state() for s in b.members]
        b.step(2)
        b.sync()
    # 6 tile sizes x 3 chunk sizes, with two cells per warp where possible and without
    assert len(res) == 36 and all(r["ms_per_substep"] > 0 for r in res)
    assert sorted({r["cells_per_warp"] for r in res}) == [1, 2]
    assert info["tuned"] == 1
    best = min(res, key=lambda r: r["ms_per_substep"])
    assert (info["tile_work"], info["chunk_bytes"], info["pair_cells"]) == (
        best["tile_work"], best["chunk_bytes"], int(best["cells_per_warp"] == 2))
    for x, y in zip(before, after):
        for k in ("psi", "mb", "mf", "c"):
            assert np.array_equal(x[k], y[k]), k


def test_batch_member_adjoint(mmod):
    """Member 3 records an adjoint while the batch steps; the gradients equal
    those of the same recording made alone (float64: identical forward)."""
    ms = members()
    K, n = 4, 10
    with mmod.Batch([m.grid for m in ms], [m.rates for m in ms], "fp64") as b:
        setup(b, ms)
        b.members[3].set_checkpointing(K, n)
        b.step(6)
        b.step(4)
        got = b.members[3].adjoint(n, observable="polar_order", n_velocities=1)
    m = ms[3]
    psi0, u = member_inputs(m, modes=4, amp=0.3)
    with mmod.Simulation(m.grid, m.rates, "fp64") as sim:
        sim.set_state(psi0)
        sim.set_velocity(u)
        sim.set_checkpointing(K, n)
        sim.step(n)
        ref = sim.adjoint(n, observable="polar_order", n_velocities=1)
    assert got["value"] == ref["value"]
    assert np.array_equal(got["dL_du"], ref["dL_du"])
    assert np.array_equal(got["dL_drates"], ref["dL_drates"])
    assert np.array_equal(got["dL_dpsi0"], ref["dL_dpsi0"])


def test_batch_timeout_is_reported_and_recovers(mmod):
    ms = members()
    with mmod.Batch([m.grid for m in ms], [m.rates for m in ms], "fp32") as b:
        setup(b, ms)
        b.debug_set(64, 1)  # every bounded wait gives up after 64 polls
        b.step(2)
        with pytest.raises(mmod.MMError) as ei:
            b.sync()
        assert ei.value.status == 5
        b.debug_set(1 << 22, 0)
        setup(b, ms)
        b.step(5)
        b.sync()
        psi = b.members[0].get_state()["psi"]
    ref = alone(mmod, ms[0], "fp32", [5])
    assert rel(psi, ref["psi"]) <= 1e-6


def test_batch_rejects_single_instance_calls(mmod):
    ms = members()[:2]
    with mmod.Batch([m.grid for m in ms], [m.rates for m in ms], "fp32") as b:
        lib = b.lib
        import ctypes as C
        assert lib.mm_set_dt(b.h, C.c_double(0.01)) == 1
        assert lib.mm_destroy(b.members[0].h) == 1
        with pytest.raises(mmod.MMError):
            b.step(1)  # members have no state yet
    bad = [Grid(8, 8, 16, 18)]
    with pytest.raises(mmod.MMError):
        mmod.Batch(bad, [Rates()], "fp32")


def test_ensemble64_shapes_step(mmod):
    """The 64-member detachment-rate sweep: one graph of 10 substeps runs and
    conserves each member's filament number (float32 form: to 1e-6, as for a
    single instance)."""
    ms = ensemble_members()
    with mmod.Batch([m.grid for m in ms], [m.rates for m in ms], "fp32") as b:
        for sim, m in zip(b.members, ms):
            psi0, u = member_inputs(m)
            sim.set_state(psi0)
            sim.set_velocity(u)
        n0 = [s.moments(fields=False)[1]["N_psi"] for s in b.members]
        b.step(10)
        b.sync()
        n1 = [s.moments(fields=False)[1]["N_psi"] for s in b.members]
    for a, c in zip(n0, n1):
        assert abs(c - a) <= 1e-6 * abs(a)


def test_ensemble64_members_match_alone(mmod):
    """The 64-member detachment-rate sweep in one batch (the bench's plan:
    autotuned, two cells per warp where possible), 10 substeps: four members --
    two with 16 orientations (two cells per warp) and two with 32 -- equal the
    same members stepped alone (float32: 1e-6, the mass sums being grouped by
    tile)."""
    ms = ensemble_members()
    picks = [next(i for i, m in enumerate(ms) if (m.grid.ntheta, m.grid.ns) == key)
             for key in ((16, 16), (16, 32), (32, 16), (32, 32))]
    with mmod.Batch([m.grid for m in ms], [m.rates for m in ms], "fp32") as b:
        for sim, m in zip(b.members, ms):
            psi0, u = member_inputs(m)
            sim.set_state(psi0)
            sim.set_velocity(u)
        b.autotune(substeps=2)
        assert b.launch_info()["pair_cells"] in (0, 1)
        b.step(10)
        b.sync()
        got = {i: b.members[i].get_state() for i in picks}
    for i in picks:
        m = ms[i]
        psi0, u = member_inputs(m)
        with mmod.Simulation(m.grid, m.rates, "fp32") as sim:
            sim.set_state(psi0)
            sim.set_velocity(u)
            sim.step(10)
            ref = sim.get_state()
        for k in ("psi", "mb", "mf"):
            assert rel(got[i][k], ref[k]) <= 1e-6, (i, k, rel(got[i][k], ref[k]))
