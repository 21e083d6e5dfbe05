"""Run one synthetic case of the library's kernels, for profilers.

    python bench_profile.py
        [--case single|batch|adjoint|moments|local|fluid]
        [--grid NX NY NTHETA NS] [--precision fp32|fp64] [--substeps N]
        [--repeat R] [--K K] [--members M] [--autotune] [--anchors ELL]
        [--capture ELL RC_CELLS] [--tangent]

single:  the perturbed isotropic state under a seeded 8-mode divergence-free
         flow (amplitude 0.1); R calls of N substeps (with --anchors ELL: motor
         anchors under the motor heads, l/L = ELL; with --capture ELL RC_CELLS:
         the finite capture radius r_c = RC_CELLS cell widths, l/L = ELL; with
         --tangent: the tangent-linear mode along d k_off, every substep
         advancing the state and its tangent).
batch:   the first M members of the detachment-rate ensemble (64 by default)
         as one batch; R calls of N batched substeps (after mm_batch_autotune
         with --autotune).
adjoint: a recording of N substeps (checkpoint every K) on the single case,
         then the reverse sweep for the polar order; R times.
moments: N substeps of the single case, then R calls of mm_moments.
local:   the single case's state, then R calls of mm_motor_local over the
         interval of N substeps of the adaptive dt (psi frozen, local steps).
fluid:   N substeps of the single case, then R macro steps of Alg. 1: the
         thin-gap fluid solve (eps = 0.1, z0 = 0.1, dipole term on), then N
         substeps at the solved velocity.
Prints the times measured with CUDA events on the handle's stream.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main():
    import torch

    from paper_1908_04279_gb300 import build as B
    from paper_1908_04279_gb300 import mm
    from paper_1908_04279_gb300.inputs import (Grid, Rates, ensemble_members, member_inputs,
                                               psi_isotropic_perturbed, random_divfree_flow)

    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="single",
                    choices=["single", "batch", "adjoint", "moments", "local", "fluid"])
    ap.add_argument("--grid", type=int, nargs=4, default=[256, 256, 64, 64])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--substeps", type=int, default=10)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--K", type=int, default=10)
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--anchors", type=float, default=None)
    ap.add_argument("--capture", type=float, nargs=2, default=None)
    ap.add_argument("--tangent", action="store_true")
    args = ap.parse_args()
    B.build()
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    if args.case == "batch":
        ms = ensemble_members()[: args.members]
        with mm.Batch([m.grid for m in ms], [m.rates for m in ms], args.precision,
                      stream=stream.cuda_stream) as b:
            for sim, m in zip(b.members, ms):
                psi0, u = member_inputs(m)
                sim.set_state(psi0)
                sim.set_velocity(u)
            if args.autotune:
                b.autotune(substeps=3)
            times = [timed(lambda: b.step(args.substeps)) / args.substeps
                     for _ in range(args.repeat)]
            b.sync()
            cells = b.cell_updates_per_substep
            print(json.dumps({"case": "batch", "members": len(ms), "ms_per_substep": times,
                              "launch": b.launch_info(),
                              "cell_updates_per_s": cells / (min(times) * 1e-3)}))
        return

    g = Grid(*args.grid)
    rates = Rates() if args.anchors is None else Rates(ell=args.anchors)
    if args.capture is not None:
        rates = Rates(ell=args.capture[0])
    with mm.Simulation(g, rates, args.precision, stream=stream.cuda_stream) as sim:
        if args.anchors is not None:
            sim.set_anchors(True)
        if args.capture is not None:
            sim.set_capture(args.capture[1] / g.nx)
        if args.tangent:
            sim.set_tangent((1.0, 0.0, 0.0))
        psi0 = psi_isotropic_perturbed(g, 0)
        u = random_divfree_flow(g, 1, 8, 0.1)
        sim.set_state(psi0)
        sim.set_velocity(u)
        if args.case == "moments":
            sim.step(args.substeps)
            fields = torch.empty(12 * g.nx * g.ny, dtype=torch.float64, device="cuda")
            times = [timed(lambda: sim.moments(fields=fields)) for _ in range(args.repeat)]
            print(json.dumps({"case": "moments", "grid": args.grid, "precision": args.precision,
                              "ms_per_call": times}))
            return
        if args.case == "fluid":
            sim.step(args.substeps)
            sim.fluid_setup(0.1, 0.1)
            solve, macro = [], []
            for _ in range(args.repeat):
                solve.append(timed(lambda: sim.fluid_solve(dipole=True, u_out=None)))
                macro.append(timed(lambda: sim.step(args.substeps)))
            sim.sync()
            print(json.dumps({"case": "fluid", "grid": args.grid, "precision": args.precision,
                              "ms_per_solve": solve, "ms_substeps_after": macro}))
            return
        if args.case == "local":
            T = args.substeps * sim.dt
            nst = sim.motor_local(T)
            times = [timed(lambda: sim.motor_local_device(T)) for _ in range(args.repeat)]
            sim.sync()
            upd = int(nst.sum()) * g.ntheta * g.ns
            print(json.dumps({"case": "local", "grid": args.grid, "precision": args.precision,
                              "T": T, "substeps_per_cell": [int(nst.min()), int(nst.max())],
                              "ms_per_call": times,
                              "cell_updates_per_s": upd / (min(times) * 1e-3)}))
            return
        if args.case == "single":
            times = [timed(lambda: sim.step(args.substeps)) / args.substeps
                     for _ in range(args.repeat)]
            sim.sync()
            print(json.dumps({"case": "single", "grid": args.grid, "precision": args.precision,
                              "ms_per_substep": times, "launch": sim.launch_info(),
                              "cell_updates_per_s": g.micro_cells / (min(times) * 1e-3)}))
            return
        fwd, adj = [], []
        for _ in range(args.repeat):
            sim.set_state(psi0)
            sim.set_velocity(u)
            sim.set_checkpointing(args.K, args.substeps)
            fwd.append(timed(lambda: sim.step(args.substeps)))
            adj.append(timed(lambda: sim.adjoint(args.substeps, observable="polar_order",
                                                 want_dpsi0=False)))
        print(json.dumps({"case": "adjoint", "grid": args.grid, "precision": args.precision,
                          "recorded_forward_ms": fwd, "reverse_sweep_ms": adj}))


if __name__ == "__main__":
    main()
