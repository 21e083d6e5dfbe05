"""Bitwise checkpoint and restart (mm_save_snapshot / mm_load_snapshot).

A run interrupted after some substeps, saved, loaded into a fresh handle and
continued (more substeps, a new velocity, more substeps) must end in the same
state, bit for bit, as the run that was never interrupted -- in float64 and in
the float32 form, whose pending mass-correction factor and reference filament
number the snapshot carries. Host and device snapshot buffers both; wrong
grids, precisions and sizes are refused.
"""
import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import (Grid, Rates, SplitMix64, psi_isotropic_perturbed,
                                           random_divfree_flow)

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


def _final(sim):
    out = sim.get_state()
    _, sc = sim.moments(fields=False)
    return dict(out, sc=np.array(list(sc.values())), dt=sim.dt)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("device", [False, True])
def test_restart_continues_bit_for_bit(mmod, precision, device):
    import torch
    g = Grid(24, 20, 16, 24, L=1.0)
    r = Rates(k_on=1.4, k_off=0.6, glide=0.2)
    rng = SplitMix64(71)
    psi0 = psi_isotropic_perturbed(g, 72, amp=0.3)
    mb0 = 0.2 * rng.uniforms(g.ny * g.nx * g.ntheta * g.ns).reshape(g.ny, g.nx, g.ntheta, g.ns)
    u1 = random_divfree_flow(g, 73, 6, 0.3)
    u2 = random_divfree_flow(g, 74, 6, 0.3)
    with mmod.Simulation(g, r, precision) as a:
        a.set_state(psi0, mb0)
        a.set_velocity(u1)
        a.step(7)  # odd: the snapshot is taken from the second ping-pong buffer
        if device:
            snap = torch.empty(a.snapshot_bytes(), dtype=torch.uint8, device="cuda")
            a.snapshot(snap)
        else:
            snap = a.snapshot()
        a.step(5)
        a.set_velocity(u2)
        a.step(6)
        ref = _final(a)
    with mmod.Simulation(g, r, precision) as b:
        b.load_snapshot(snap)
        b.step(5)
        b.set_velocity(u2)
        b.step(6)
        got = _final(b)
    for k in ("psi", "mb", "mf", "c", "sc"):
        assert np.array_equal(got[k], ref[k]), (precision, k)
    assert got["dt"] == ref["dt"]


def test_snapshot_refusals(mmod):
    g = Grid(8, 6, 8, 8)
    with mmod.Simulation(g, Rates(), "fp32") as a:
        with pytest.raises(mmod.MMError):  # no state yet
            a.snapshot()
        a.set_state(psi_isotropic_perturbed(g, 5))
        snap = a.snapshot()
        with pytest.raises(mmod.MMError):  # too small
            a.load_snapshot(snap[: snap.nbytes // 2].copy())
        bad = snap.copy()
        bad[:8] = 0
        with pytest.raises(mmod.MMError):  # not a snapshot
            a.load_snapshot(bad)
    with mmod.Simulation(g, Rates(), "fp64") as b:  # other precision
        with pytest.raises(mmod.MMError):
            b.load_snapshot(snap)
    with mmod.Simulation(Grid(8, 6, 8, 16), Rates(), "fp32") as c:  # other grid
        big = np.zeros(snap.nbytes * 4, dtype=np.uint8)
        big[:snap.nbytes] = snap
        with pytest.raises(mmod.MMError):
            c.load_snapshot(big)
