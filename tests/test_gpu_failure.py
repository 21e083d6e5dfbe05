"""Failure detection on the GPU without faulting it: the substep kernel's
mbarrier waits are bounded; a test knob makes every wait run out (the warp
waits on a barrier that nothing completes). The kernel must record the
failure, drain its in-flight bulk copies and return, the host must report
MM_ERR_TIMEOUT, and the context must stay usable."""
import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import Grid, Rates, cellular_flow, psi_isotropic_perturbed

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


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_bounded_wait_times_out_and_context_survives(mmod, precision):
    g = Grid(16, 16, 32, 32)
    psi = psi_isotropic_perturbed(g, 0)
    u = cellular_flow(g)
    with mmod.Simulation(g, Rates(), precision) as ref:
        ref.set_state(psi)
        ref.set_velocity(u)
        ref.step(5)
        want = ref.get_state()
    with mmod.Simulation(g, Rates(), precision) as sim:
        assert sim.launch_info()["tma"] == 1
        sim.set_state(psi)
        sim.set_velocity(u)
        sim.debug_set(2000, 1)
        sim.step(2)
        with pytest.raises(mmod.MMError) as e:
            sim.sync()
        assert e.value.status == 5  # MM_ERR_TIMEOUT
        # back to normal: the same handle and context compute the same answer
        sim.debug_set(1 << 22, 0)
        sim.set_state(psi)
        sim.set_velocity(u)
        sim.step(5)
        sim.sync()
        got = sim.get_state()
    for k in ("psi", "mb", "mf", "c"):
        assert np.array_equal(got[k], want[k]), k


@pytest.mark.parametrize("dims,precision,tma", [
    ((128, 128, 32, 32), "fp32", 1), ((512, 8, 64, 64), "fp32", 1), ((64, 64, 32, 32), "fp64", 1),
    ((9, 7, 5, 31), "fp32", 0), ((5, 3, 3, 7), "fp64", 0), ((4, 4, 1024, 4), "fp64", 1)])
def test_launch_plan(mmod, dims, precision, tma):
    """Bulk copies are used exactly when an s-row is whole 16-byte vectors, and
    the shared-memory plan fits for large orientation counts."""
    g = Grid(*dims)
    with mmod.Simulation(g, Rates(), precision) as sim:
        info = sim.launch_info()
    assert info["tma"] == tma
    assert info["smem"] <= 200 * 1024
    assert info["block"] % 32 == 0 and info["grid"] >= 1
    assert info["chunk_rows"] * info["chunks_per_cell"] == g.ntheta


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_reverse_sweep_timeout_is_reported_and_recovers(mmod, precision):
    """The knob on during a reverse sweep: the replays and both reverse kernels
    (bulk-copy rings) give up their waits, drain their copies and return; the
    sweep reports MM_ERR_TIMEOUT. With the knob off, a new recording on the
    same handle gives the gradients of a clean handle, bit for bit."""
    g = Grid(12, 10, 16, 16)
    psi = psi_isotropic_perturbed(g, 3)
    u = cellular_flow(g)

    def record(sim):
        sim.set_state(psi)
        sim.set_velocity(u)
        sim.set_checkpointing(4, 12)
        sim.step(12)

    with mmod.Simulation(g, Rates(), precision) as ref:
        record(ref)
        want = ref.adjoint(12, observable="polar_order")
    with mmod.Simulation(g, Rates(), precision) as sim:
        record(sim)
        sim.debug_set(2000, 1)
        with pytest.raises(mmod.MMError) as e:
            sim.adjoint(12, observable="polar_order")
        assert e.value.status == 5  # MM_ERR_TIMEOUT
        sim.debug_set(1 << 22, 0)
        record(sim)
        got = sim.adjoint(12, observable="polar_order")
    assert np.array_equal(got["dL_drates"], want["dL_drates"])
    assert np.array_equal(got["dL_du"], want["dL_du"])
    assert np.array_equal(got["dL_dpsi0"], want["dL_dpsi0"])
