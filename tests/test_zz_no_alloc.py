"""The allocation-free moments entry point, mm_moments_static.

It is meant for callers that cannot call cudaMalloc -- an application that
reserved the GPU's memory for its own pool and forbids allocations it does
not manage, or a time-critical loop that must not pay the synchronisation an
allocation may imply. Its only scratch is a file-scope device array shared by
every call, so these checks run it twice in a row on two different states and
compare each result with the handle's own mm_moments of that state, within
the float64 tolerance the parity tests use (relative 1e-12).

This file is named to be collected last: it also passes when run alone in a
fresh process (the array's device address is set up on the first call).
"""
import math

import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import Grid, Rates, SplitMix64, psi_isotropic_perturbed, random_divfree_flow

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_04279_gb300 import build as B
    B.build()
    from paper_1908_04279_gb300 import mm
    return torch, mm


def _state_and_reference(torch, mm, g, r, seed):
    """A state stepped on a handle, exported to caller-held device arrays, and
    the handle's own moments of it (fields [12][cells] and scalars)."""
    rng = SplitMix64(seed)
    psi0 = psi_isotropic_perturbed(g, seed + 2, amp=0.2)
    mb0 = 0.3 * rng.uniforms(g.ny * g.nx * g.ntheta * g.ns).reshape(g.ny, g.nx, g.ntheta, g.ns)
    dev = torch.device("cuda")
    with mm.Simulation(g, r, "fp64") as sim:
        sim.set_state(psi0, mb0)
        sim.set_velocity(random_divfree_flow(g, seed + 3, 6, 0.2))
        sim.step(15)
        state = dict(psi=torch.empty((g.ny, g.nx, g.ntheta), dtype=torch.float64, device=dev),
                     mb=torch.empty((g.ny, g.nx, g.ntheta, g.ns), dtype=torch.float64, device=dev),
                     mf=torch.empty((g.ny, g.nx), dtype=torch.float64, device=dev),
                     c=torch.empty((g.ny, g.nx), dtype=torch.float64, device=dev))
        sim.get_state_into(**state)
        ref_fields = torch.empty(12 * g.ny * g.nx, dtype=torch.float64, device=dev)
        _, ref_scalars = sim.moments(fields=ref_fields)
    return state, ref_fields.cpu().numpy().reshape(12, -1), ref_scalars


def _check(g, state, ref_f, ref_scalars, fields, scalars, call):
    spsi = float(state["psi"].sum())
    stress_scale = float(np.mean(np.abs(ref_f[9]) + np.abs(ref_f[11])))
    scale = [max(abs(v), 1e-300) for v in ref_scalars.values()]
    scale[6] = scale[7] = spsi          # sums of psi cos / psi sin cancel
    scale[4] = 1.0                      # polar order is built from them
    scale[5] = max(scale[5], stress_scale)
    f = fields.cpu().numpy().reshape(12, -1)
    for q in range(12):
        nrm = np.linalg.norm(ref_f[q])
        err = np.linalg.norm(f[q] - ref_f[q]) / (nrm if nrm > 0 else 1.0)
        assert err <= TOL, (call, q, err)
    got = scalars.cpu().numpy()
    for q, (name, want) in enumerate(ref_scalars.items()):
        assert abs(got[q] - want) <= TOL * scale[q], (call, name, got[q], want)


def test_static_moments_match_handle_moments_twice(env):
    """Two calls in a row on two different states -- the second on a smaller
    grid, so that records the first call left behind in the shared scratch
    would show up if the second call read any it had not rewritten -- each
    against the handle's mm_moments of its own state. The second call must
    not change the device's free memory: the scratch array is placed on the
    device by the first call (lazy module loading) and never grows."""
    torch, mm = env
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(Grid(64, 48, 16, 12, L=1.1), Rates(glide=0.3, v_sp=0.1, force_scale=1.3, ell=0.7), 5),
             (Grid(40, 30, 8, 20, L=0.9), Rates(glide=0.1, force_scale=0.6, ell=1.2), 17)]
    refs = [_state_and_reference(torch, mm, g, r, seed) for g, r, seed in cases]
    outs = [(torch.full((12 * g.ny * g.nx,), math.nan, dtype=torch.float64, device=dev),
             torch.full((8,), math.nan, dtype=torch.float64, device=dev)) for g, _, _ in cases]
    torch.cuda.synchronize()
    free = []
    for call, ((g, r, _), (state, ref_f, ref_s), (fields, scalars)) in enumerate(
            zip(cases, refs, outs)):
        mm.moments_static(g, r, state["psi"], state["mb"], state["mf"], state["c"], fields,
                          scalars, stream)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        _check(g, state, ref_f, ref_s, fields, scalars, call)
    assert free[1] == free[0], free


def test_static_moments_reject_oversize_grid(env):
    torch, mm = env
    g = Grid(257, 256, 4, 4)  # 65792 cells, above the 65536-cell scratch
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(mm.MMError) as e:
        mm.moments_static(g, Rates(), t, t, t, t, None, t)
    assert e.value.status == 4
    assert "65536" in str(e.value)
