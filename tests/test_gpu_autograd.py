"""torch.autograd binding (paper_1908_04279_gb300.autograd.micro_steps):
its backward returns the discrete-adjoint gradients of mm_adjoint_step,
scaled by the incoming gradient, and agrees with a central difference along
a random direction of (u, k_off, v_walk, psi0)."""
import numpy as np
import pytest

from paper_1908_04279_gb300.inputs import (Grid, Rates, SplitMix64, psi_isotropic_perturbed,
                                           random_divfree_flow)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_04279_gb300 import build as B
    B.build()
    from paper_1908_04279_gb300 import autograd as AG
    from paper_1908_04279_gb300 import mm
    return torch, mm, AG


def _case(torch):
    g = Grid(16, 12, 8, 16, L=1.0)
    psi0 = torch.tensor(psi_isotropic_perturbed(g, 21, amp=0.2), device="cuda")
    u = torch.tensor(random_divfree_flow(g, 22, 4, 0.3), device="cuda")
    return g, psi0, u


def test_autograd_matches_raw_adjoint(env):
    torch, mm, AG = env
    g, psi0, u = _case(torch)
    r = Rates(k_on=1.3, k_off=0.7, v_walk=0.9)
    with mm.Simulation(g, r, "fp64") as sim:
        u_ = u.clone().requires_grad_(True)
        p_ = psi0.clone().requires_grad_(True)
        koff = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
        vw = torch.tensor(0.9, dtype=torch.float64, requires_grad=True)
        L = AG.micro_steps(sim, p_, u_, koff, vw, n_substeps=12, K=5, observable="polar_order")
        (3.0 * L).backward()
        dt = sim.dt
        # the same recording through the raw binding
        sim.set_rates(r)
        sim.set_state(psi0)
        sim.set_velocity(u)
        sim.set_dt(dt)
        sim.set_checkpointing(5, 12)
        sim.step(12)
        raw = sim.adjoint(12, observable="polar_order", n_velocities=2)
    assert L.item() == pytest.approx(raw["value"], rel=1e-14)
    assert koff.grad.item() == pytest.approx(3.0 * raw["dL_drates"][0], rel=1e-12)
    assert vw.grad.item() == pytest.approx(3.0 * raw["dL_drates"][1], rel=1e-12)
    np.testing.assert_allclose(u_.grad.cpu().numpy(), 3.0 * raw["dL_du"].sum(0), rtol=1e-12,
                               atol=1e-18)
    np.testing.assert_allclose(p_.grad.cpu().numpy(), 3.0 * raw["dL_dpsi0"], rtol=1e-12,
                               atol=1e-18)


def test_autograd_directional_derivative(env):
    """<grad L, d> against (L(x + h d) - L(x - h d)) / 2h at a fixed dt, h = 1e-6,
    for a random direction d of all four inputs at once."""
    torch, mm, AG = env
    g, psi0, u = _case(torch)
    r = Rates(k_on=1.3, k_off=0.7, v_walk=0.9)
    rng = SplitMix64(23)
    du = torch.tensor(rng.uniforms(u.numel()).reshape(tuple(u.shape)) - 0.5, device="cuda")
    dp = torch.tensor(rng.uniforms(psi0.numel()).reshape(tuple(psi0.shape)) - 0.5, device="cuda")
    dk, dv = 0.3, -0.2
    with mm.Simulation(g, r, "fp64") as sim:
        sim.set_state(psi0)
        sim.set_velocity(u)
        dt = sim.dt

        def L(e, grad=False):
            u_ = (u + e * du).requires_grad_(grad)
            p_ = (psi0 + e * dp).requires_grad_(grad)
            k_ = torch.tensor(0.7 + e * dk, dtype=torch.float64, requires_grad=grad)
            v_ = torch.tensor(0.9 + e * dv, dtype=torch.float64, requires_grad=grad)
            out = AG.micro_steps(sim, p_, u_, k_, v_, n_substeps=20, K=4,
                                 observable="mean_stress", dt=dt)
            if not grad:
                return out.item()
            out.backward()
            return (out.item(), (u_.grad * du).sum().item() + (p_.grad * dp).sum().item() +
                    k_.grad.item() * dk + v_.grad.item() * dv)

        L0, dd = L(0.0, grad=True)
        h = 1e-6
        fd = (L(h) - L(-h)) / (2 * h)
    assert abs(dd - fd) <= 1e-5 * abs(fd), (dd, fd)


def test_autograd_state_outputs(env):
    """observable=None: (psi, Mf) of the final state; a loss built from them
    seeds the reverse sweep with its gradients."""
    torch, mm, AG = env
    g, psi0, u = _case(torch)
    r = Rates(k_on=1.3, k_off=0.7)
    rng = SplitMix64(24)
    wpsi = torch.tensor(rng.uniforms(psi0.numel()).reshape(tuple(psi0.shape)), device="cuda")
    wmf = torch.tensor(rng.uniforms(g.ny * g.nx).reshape(g.ny, g.nx), device="cuda")
    with mm.Simulation(g, r, "fp64") as sim:
        u_ = u.clone().requires_grad_(True)
        koff = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
        psi, mf = AG.micro_steps(sim, psi0, u_, koff, 1.0, n_substeps=9, K=3, observable=None)
        ((psi * wpsi).sum() + (mf * wmf).sum()).backward()
        dt = sim.dt
        sim.set_rates(r)
        sim.set_state(psi0)
        sim.set_velocity(u)
        sim.set_dt(dt)
        sim.set_checkpointing(3, 9)
        sim.step(9)
        raw = sim.adjoint(9, dL_dpsi=wpsi.cpu().numpy(), dL_dmf=wmf.cpu().numpy(),
                          n_velocities=2)
        # a second forward drops the first recording
        L1 = AG.micro_steps(sim, psi0, u_, koff, 1.0, n_substeps=3, K=3)
        AG.micro_steps(sim, psi0, u, 0.7, 1.0, n_substeps=3, K=3)
        with pytest.raises(RuntimeError):
            L1.backward()
    assert koff.grad.item() == pytest.approx(raw["dL_drates"][0], rel=1e-12)
    np.testing.assert_allclose(u_.grad.cpu().numpy(), raw["dL_du"].sum(0), rtol=1e-12,
                               atol=1e-18)
