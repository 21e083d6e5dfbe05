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
