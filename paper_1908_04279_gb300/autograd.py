"""torch.autograd binding of the microscale substeps.

`micro_steps(sim, psi0, u, k_off, v_walk, ...)` advances a Simulation by
n_substeps under an adjoint recording (checkpoint every K substeps) and
returns a macroscopic observable of the final state: the polar order
|sum psi e^{i theta}| / sum psi or the mean over cells of tr sigma_a (the
moments of Eq. 5 and the active stress), or, with observable=None, the final
psi and free-motor density Mf as tensors. Its backward runs the discrete
adjoint of the substeps (mm_adjoint_step) and returns the gradients with
respect to the initial psi, the velocity field u, and the rates k_off, v_walk
and k_on. The time step is held fixed (not differentiated): pass `dt` to fix
it explicitly, otherwise the CFL step of the forward's rates and velocity is
used on both passes.

All arithmetic runs in libmm's CUDA kernels; this module only moves pointers
and scalars. Tensors are float64 on the Simulation's CUDA device, and the
Simulation's stream is torch's current stream when it was created.
"""
from __future__ import annotations

import dataclasses

import torch

from .mm import Simulation

_OBS = ("polar_order", "mean_stress")


class _MicroSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sim: Simulation, n: int, K: int, observable, dt, psi0, u, k_off, v_walk,
                k_on):
        dev = torch.device("cuda", torch.cuda.current_device())
        sim.set_rates(dataclasses.replace(sim.rates, k_off=float(k_off), v_walk=float(v_walk),
                                          k_on=float(k_on)))
        sim.set_state(psi0.detach().to(device=dev, dtype=torch.float64).contiguous())
        sim.set_velocity(u.detach().to(device=dev, dtype=torch.float64).contiguous())
        if dt is not None:
            sim.set_dt(float(dt))
        sim.set_checkpointing(K, n)
        sim.step(n)
        sim._recording_id = getattr(sim, "_recording_id", 0) + 1
        ctx.sim, ctx.n, ctx.obs, ctx.rec = sim, n, observable, sim._recording_id
        ctx.shape_u = tuple(u.shape)
        ctx.psi_dtype, ctx.u_dtype = psi0.dtype, u.dtype
        ctx.psi_dev, ctx.u_dev = psi0.device, u.device
        ctx.rate_like = [(x.device, x.dtype) for x in (k_off, v_walk, k_on)]
        if observable in _OBS:
            _, sc = sim.moments(fields=False)
            return torch.tensor(sc[observable], dtype=torch.float64, device=dev)
        g = sim.grid
        psi = torch.empty((g.ny, g.nx, g.ntheta), dtype=torch.float64, device=dev)
        mf = torch.empty((g.ny, g.nx), dtype=torch.float64, device=dev)
        sim.get_state_into(psi=psi, mf=mf)
        return psi, mf

    @staticmethod
    def backward(ctx, *grads):
        sim = ctx.sim
        if getattr(sim, "_recording_id", None) != ctx.rec:
            raise RuntimeError("micro_steps: the Simulation was stepped or recorded again after "
                               "this forward; its recording is gone")
        g = sim.grid
        dev = torch.device("cuda", torch.cuda.current_device())
        du = torch.empty((2, 2, g.ny, g.nx), dtype=torch.float64, device=dev)
        dpsi0 = torch.empty((g.ny, g.nx, g.ntheta), dtype=torch.float64, device=dev)
        if ctx.obs in _OBS:
            res = sim.adjoint(ctx.n, observable=ctx.obs, out_du=du, out_dpsi0=dpsi0)
            scale = grads[0].to(device=dev, dtype=torch.float64)
        else:
            gpsi, gmf = grads
            gpsi = (torch.zeros((g.ny, g.nx, g.ntheta), dtype=torch.float64, device=dev)
                    if gpsi is None else gpsi.to(device=dev, dtype=torch.float64).contiguous())
            gmf = (torch.zeros((g.ny, g.nx), dtype=torch.float64, device=dev)
                   if gmf is None else gmf.to(device=dev, dtype=torch.float64).contiguous())
            res = sim.adjoint(ctx.n, dL_dpsi=gpsi, dL_dmf=gmf, out_du=du, out_dpsi0=dpsi0)
            scale = torch.ones((), dtype=torch.float64, device=dev)
        dr = torch.as_tensor(res["dL_drates"], dtype=torch.float64, device=dev) * scale
        # a set_dt during the recording adds a (velocity, dt) block: both blocks
        # belong to the same u here
        du_total = du[: res["n_velocities"]].sum(0) * scale
        drates = [dr[i].to(device=d, dtype=t) for i, (d, t) in enumerate(ctx.rate_like)]
        return (None, None, None, None, None,
                (dpsi0 * scale).to(device=ctx.psi_dev, dtype=ctx.psi_dtype),
                du_total.reshape(ctx.shape_u).to(device=ctx.u_dev, dtype=ctx.u_dtype), *drates)


def micro_steps(sim: Simulation, psi0: torch.Tensor, u: torch.Tensor, k_off, v_walk, k_on=None,
                n_substeps: int = 100, K: int = 10, observable: str | None = "polar_order",
                dt: float | None = None):
    """Differentiable n_substeps of `sim` from the initial psi0 [ny][nx][ntheta]
    (bound motors zero, total motors one per cell) under the velocity
    u [2][ny][nx], with k_off, v_walk and k_on as 0-d tensors (or floats).
    Returns the observable (0-d tensor) or, for observable=None, (psi, Mf) of
    the final state."""
    if observable is not None and observable not in _OBS:
        raise ValueError(f"observable must be one of {_OBS} or None")
    if k_on is None:
        k_on = sim.rates.k_on

    def t(x):
        return x if torch.is_tensor(x) else torch.tensor(float(x), dtype=torch.float64)

    return _MicroSteps.apply(sim, int(n_substeps), int(K), observable, dt, psi0, u, t(k_off),
                             t(v_walk), t(k_on))
