"""Run the substep path on one synthetic case, for profilers.

    python -m paper_1908_04279_gb300.profile_case --grid NX NY NTHETA NS \
        [--precision fp32|fp64] [--substeps N] [--repeat R]

Sets the perturbed isotropic state and a seeded 8-mode divergence-free flow
(amplitude 0.1), then runs R calls of N substeps each and prints the kernel
time per substep measured with CUDA events on the handle's stream.
"""
from __future__ import annotations

import argparse
import json


def main():
    import torch

    from . import build as B
    from . import mm
    from .inputs import Grid, Rates, psi_isotropic_perturbed, random_divfree_flow

    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, nargs=4, default=[256, 256, 64, 64])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--substeps", type=int, default=10)
    ap.add_argument("--repeat", type=int, default=3)
    args = ap.parse_args()
    B.build()
    g = Grid(*args.grid)
    stream = torch.cuda.current_stream()
    with mm.Simulation(g, Rates(), args.precision, stream=stream.cuda_stream) as sim:
        sim.set_state(psi_isotropic_perturbed(g, 0))
        sim.set_velocity(random_divfree_flow(g, 1, 8, 0.1))
        times = []
        for _ in range(args.repeat):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(args.substeps)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / args.substeps)
        sim.sync()
        print(json.dumps({"grid": args.grid, "precision": args.precision,
                          "ms_per_substep": times, "launch": sim.launch_info(),
                          "cell_updates_per_s": g.micro_cells / (min(times) * 1e-3)}))


if __name__ == "__main__":
    main()
