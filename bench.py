"""Benchmark of the microscale kinetic step on GB300.

A step is one macro step of the workload: prescribe that macro step's
velocity (mm_set_velocity, which also recomputes the adaptive substep), run its
substeps (mm_micro_step) and reduce the macroscale moments (mm_moments).
Metric: micro-state cell-updates per second = nx*ny*ntheta*ns*substeps / time.

Default workload "large512": 512x512 periodic grid, 64 orientations, 64
arclength nodes (1.07e9 motor cells, 4.29 GB of float32 motor density, 33x the
L2), 100 substeps per macro step, velocity from a seeded random
divergence-free field (16 Fourier modes, amplitude 0.2) refreshed every macro
step, mixed precision (float32 Mb/psi, float64 sums); the default 20 timed
steps are the workload's 20 macro steps. The float64 path is timed on the same
workload and reported beside it, with its roofline against the measured
float64 fused multiply-add rate. Beside the main line: the L2-resident
precision128 case (128x128 x 32 x 32), the adjoint/forward time ratio
(adjoint64 and large512), the batched ensemble (ensemble64, 64 uneven members,
500 substeps per graph), and the next rows (diffusion, anchors, fluid solve,
local substeps). The last keys of the line are flat summaries of every leg.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large512|precision128|adjoint64|cellular32]

Under torchrun (N > 1) every rank advances its own instance of the workload
(weak scaling, no collective in the data path); the time is the maximum over
ranks. --impl reference times the float64 CPU oracle on the host cores (rank 0
only) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1908_04279_gb300.inputs import (WORKLOADS, Rates, psi_isotropic_perturbed,  # noqa: E402
                                           workload_velocity)

METRIC = "micro-state cell-updates/s"
UNIT = "cell-updates/s"
CSRC = os.path.join(ROOT, "paper_1908_04279_gb300", "csrc")
# sources of each kernel a committed profile summary may describe
KERNEL_SRCS = {
    "k_substep": ("mm_step.cu", "mm_async.cuh", "mm_cell.cuh", "mm_walk.cuh", "mm_internal.cuh"),
    "k_substep_batch": ("mm_batch.cu", "mm_cell.cuh", "mm_walk.cuh", "mm_internal.cuh"),
    "k_adjoint": ("mm_adjoint.cu", "mm_async.cuh", "mm_cell.cuh", "mm_walk.cuh",
                  "mm_internal.cuh"),
    "k_motor_local": ("mm_local.cu", "mm_cell.cuh", "mm_walk.cuh", "mm_internal.cuh"),
    "k_substep_anchor": ("mm_anchor.cu", "mm_async.cuh", "mm_cell.cuh", "mm_walk.cuh",
                         "mm_internal.cuh"),
    "k_substep_tl": ("mm_tangent.cu", "mm_cell.cuh", "mm_walk.cuh", "mm_internal.cuh"),
    "k_rc_motor": ("mm_capture.cu", "mm_async.cuh", "mm_cell.cuh", "mm_walk.cuh",
                   "mm_internal.cuh"),
}


def kernel_sha(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SRCS[kernel]:
        h.update(open(os.path.join(CSRC, f), "rb").read())
    return h.hexdigest()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(vals, device=None):
    """Element-wise maximum over the ranks of a list of floats (the timing rule:
    the slowest rank decides); the identity at world size 1."""
    import torch
    world, _, _ = dist_env()
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_value(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: every rank advances its own instance (weak
    scaling), so the job processes world x units in the slowest rank's time."""
    return world * units_per_rank / seconds


def algorithmic_bytes_per_launch(g, tsize: int) -> int:
    """Bytes one substep launch must move at minimum, with tsize the state
    precision's size (4 in the float32 form, 8 in float64): Mb read and written
    once (2 * tsize per motor cell); per (cell, theta) psi read and written
    (2 * tsize) and n_b read and written (2 * tsize), counted as
    2 * tsize + 16, which is exact in the float32 form (16 = 4 * 4) and
    undercounts n_b by 16 bytes per (cell, theta) in float64; per cell 32 bytes
    for Mf read and written, C written and M read, and 2 * tsize for the
    cell's velocity."""
    cells = g.nx * g.ny
    return (cells * g.ntheta * g.ns * 2 * tsize + cells * g.ntheta * (2 * tsize + 16)
            + cells * (32 + 2 * tsize))


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Arithmetic operations per motor value and substep of the row update, counted
# from the scheme: per RK2 stage the backward difference, its half, two sign
# transfers, two minima, the maximum with zero, the flux fma, the flux
# difference and two fmas of the stage update (11); two stages, plus one add of
# the n_b sum. The local-step kernel runs them on the float32 pipe. The float64
# substep runs 13 of them on the float64 pipe (difference, half, flux, flux
# difference, two stage fmas; the n_b add) and the sign transfers, minima and
# maximum (10) on the integer pipe, on the values' bit patterns; its per-(cell,
# theta) transport work, about 40 operations per row, adds under 1 per motor
# value at 64 nodes and is left out.
LOCAL_OPS = 23
SUBSTEP_OPS = 23
SUBSTEP_FP64_PIPE_OPS = 13


def wname_of(leg: dict) -> str:
    """Workload name of a bench leg from its description."""
    return leg["workload"].split(" ")[0]


def read_profile_traffic(kernel: str, workload: str, precision: str, scale: float = 1.0):
    """DRAM bytes per launch of a kernel from its committed ncu summary, if it
    was taken on the current kernel sources (sha256 match); `scale` converts a
    capture of a smaller case to the timed launch (traffic in proportion to
    the motor cells)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}_{precision}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", txt)
    if not m or not h:
        return None
    return float(m.group(1)) * scale if h.group(1) == kernel_sha(kernel) else None


class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = list(csv.reader(open(self.path)))
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample_grid(name: str):
    """Grid on which the float64 CPU oracle is timed for a workload: the
    workload's own grid, or for workloads above 2e8 motor cells (large512) a
    64x64-cell periodic grid with the workload's orientations and arclength
    nodes (the substep's cost per motor cell does not depend on the number of
    cells). Returns (grid, label, velocity of macro step 0 on that grid)."""
    from paper_1908_04279_gb300.inputs import Grid, random_divfree_flow, velocity_seed
    w = WORKLOADS[name]
    g = w["grid"]
    if g.micro_cells <= 2e8:
        return g, "", workload_velocity(name, 0)
    gs = Grid(64, 64, g.ntheta, g.ns, g.L)
    return gs, " on a 64x64-cell sub-grid", random_divfree_flow(gs, velocity_seed(w["seed"], 0),
                                                                w["modes"], w["amp"])


def time_oracle_sample(name: str, budget_s: float = 12.0, max_sub: int = 40):
    """Float64 CPU oracle on a bounded sample of the workload: the workload's
    initial state and first velocity, as many substeps as fit in budget_s."""
    from oracle import oracle as O
    w = WORKLOADS[name]
    r = Rates()
    g, sub, u = oracle_sample_grid(name)
    st = O.make_state(g, psi_isotropic_perturbed(g, w["seed"]))
    dt = O.dt(g, r, st, u)
    t0 = time.perf_counter()
    O.run(g, r, st, u, dt, 1)
    t1 = time.perf_counter() - t0
    n = max(1, min(max_sub, int(budget_s / max(t1, 1e-9)) - 1))
    t0 = time.perf_counter()
    O.run(g, r, st, u, dt, n)
    el = time.perf_counter() - t0
    return {"value": g.micro_cells * n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{name}: {n} substeps of the float64 oracle on 1 host core "
                      f"({g.nx}x{g.ny}x{g.ntheta}x{g.ns}{sub})"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    name = args.workload
    w = WORKLOADS[name]
    r = Rates()
    g, sub, u = oracle_sample_grid(name)
    st = O.make_state(g, psi_isotropic_perturbed(g, w["seed"]))
    dt = O.dt(g, r, st, u)
    # a step of the reference arm: one substep of the workload (a bounded
    # sample of its macro step), timed on one host core
    per_step = 1
    for _ in range(args.warmup):
        O.run(g, r, st, u, dt, per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.run(g, r, st, u, dt, per_step)
    el = time.perf_counter() - t0
    units = g.micro_cells * per_step * args.steps
    value = units / el
    wg = w["grid"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": name, "grid": f"{wg.nx}x{wg.ny}", "ntheta": wg.ntheta,
                       "ns": wg.ns, "substeps_per_step": per_step,
                       "sampled_grid": f"{g.nx}x{g.ny}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} steps of {per_step} oracle substep(s) of "
                                       f"{name}{sub} ({g.nx}x{g.ny}x{g.ntheta}x{g.ns}) on 1 "
                                       f"host core"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the benchmark needs the GPU path")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1908_04279_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1908_04279_gb300 import mm

    name = args.workload
    r = Rates()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def inputs_of(wname):
        w = WORKLOADS[wname]
        n_vel = max(w["macro"], 1)
        vh = [np.ascontiguousarray(workload_velocity(wname, m)) for m in range(n_vel)]
        return w, vh, psi_isotropic_perturbed(w["grid"], w["seed"])

    def device_run(wname, precision, steps, warmup):
        """Inputs resident in HBM: a step = set_velocity (device array, the
        macro step's flow) + the workload's substeps + moments into a device
        buffer. CUDA events per step on the handle's stream; L2 flushed
        between steps outside the events. Returns (step ms total, substep
        graph ms total)."""
        w, vh, psi0 = inputs_of(wname)
        g, nsub, n_vel = w["grid"], w["substeps"], len(vh)
        vels = [torch.tensor(v, device=dev) for v in vh]
        fields = torch.empty(12 * g.nx * g.ny, dtype=torch.float64, device=dev)
        sim = mm.Simulation(g, r, precision, stream=stream.cuda_stream)
        sim.set_state(psi0)
        m = 0
        for _ in range(warmup):
            sim.set_velocity(vels[m % n_vel]); m += 1
            sim.step(nsub)
            sim.moments(fields=fields)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        step_ms, kern_ms = [], []
        for _ in range(steps):
            flush.zero_()  # L2 flush between timed steps, outside the timed events
            e0, e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
            e0.record(stream)
            sim.set_velocity(vels[m % n_vel]); m += 1
            e1.record(stream)
            sim.step(nsub)
            e2.record(stream)
            sim.moments(fields=fields)
            e3.record(stream)
            e3.synchronize()
            step_ms.append(e0.elapsed_time(e3))
            kern_ms.append(e1.elapsed_time(e2))
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        sim.sync()
        sim.close()
        del vels, fields
        return sum(step_ms), sum(kern_ms)

    def e2e_run(wname, precision, steps, warmup):
        """Through the public API with host buffers: every step copies its
        velocity from pinned host memory and reads the moments back."""
        w, vh, psi0 = inputs_of(wname)
        g, nsub, n_vel = w["grid"], w["substeps"], len(vh)
        sim = mm.Simulation(g, r, precision, stream=stream.cuda_stream)
        sim.set_state(psi0)
        pinned = [torch.from_numpy(v).pin_memory() for v in vh]
        out = torch.empty(12 * g.nx * g.ny, dtype=torch.float64).pin_memory()
        m = 0
        for _ in range(warmup):
            sim.set_velocity(pinned[m % n_vel]); m += 1
            sim.step(nsub)
            sim.moments(fields=out)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            sim.set_velocity(pinned[m % n_vel]); m += 1
            sim.step(nsub)
            sim.moments(fields=out)
        torch.cuda.synchronize(dev)
        el = time.perf_counter() - t0
        sim.close()
        return el, pinned[0].numel() * 8, out.numel() * 8 + 64

    def adjoint_ratio(precision):
        """Adjoint workload (64x64 x 32 x 32, 100 substeps, checkpoint every
        10): time of the start of the recording (checkpoint 0 into memory
        reserved once, before the timed runs), the recorded forward and the
        reverse sweep (gradients of the polar order w.r.t. k_off, v_walk, k_on
        and the velocity field, copied to the host) over the time of the plain
        forward (graph replay), CUDA events on the handle's stream; best of 4."""
        wa = WORKLOADS["adjoint64"]
        ga, na = wa["grid"], wa["substeps"]
        pa = psi_isotropic_perturbed(ga, wa["seed"])
        ua = workload_velocity("adjoint64", 0)
        sim = mm.Simulation(ga, r, precision, stream=stream.cuda_stream)
        best_f, best_a = 1e30, 1e30
        # the checkpoint memory is reserved once (a first recording outside the
        # timed region); each timed recording reuses it, as a training loop would
        sim.set_state(pa)
        sim.set_velocity(ua)
        sim.set_checkpointing(10, na)
        for rep in range(4):
            sim.set_state(pa)
            sim.set_velocity(ua)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(na)
            e1.record(stream)
            e1.synchronize()
            best_f = min(best_f, e0.elapsed_time(e1))
            sim.set_state(pa)
            sim.set_velocity(ua)
            e0.record(stream)
            sim.set_checkpointing(10, na)
            sim.step(na)
            sim.adjoint(na, observable="polar_order", n_velocities=1, want_dpsi0=False)
            e1.record(stream)
            e1.synchronize()
            best_a = min(best_a, e0.elapsed_time(e1))
        sim.set_checkpointing(0, 1)
        sim.close()
        return {"forward_ms": best_f, "forward_plus_adjoint_ms": best_a,
                "adjoint_over_forward": (best_a - best_f) / best_f}

    def large_adjoint_run():
        """large512 forward + adjoint: 20 macro steps x 100 substeps (a new
        16-mode flow each macro step), gradient of the mean active stress
        with respect to k_off, outer checkpoints every 100 substeps and inner
        ones every 10 (two levels: about 40 states of 4.4 GB held). Times the
        plain forward, the recorded forward + reverse sweep, and the same
        derivative in tangent-linear mode (one forward pass carrying the
        tangent along d k_off, wall clock to the derivative on the host)."""
        wl = WORKLOADS["large512"]
        gl, nmac, nsl = wl["grid"], wl["macro"], wl["substeps"]
        psi_l = psi_isotropic_perturbed(gl, wl["seed"])
        vl = [torch.tensor(workload_velocity("large512", m), device=dev) for m in range(nmac)]
        sim = mm.Simulation(gl, r, "fp32", stream=stream.cuda_stream)
        out = {}
        # reserve the checkpoint memory once, before the timed runs
        sim.set_state(psi_l)
        sim.set_velocity(vl[0])
        sim.set_checkpointing(100, nmac * nsl, K_inner=10)
        for rec in (False, True):
            sim.set_state(psi_l)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for m in range(nmac):
                sim.set_velocity(vl[m])
                if m == 0 and rec:
                    sim.set_checkpointing(100, nmac * nsl, K_inner=10)
                sim.step(nsl)
            if rec:
                res = sim.adjoint(nmac * nsl, observable="mean_stress", n_velocities=nmac,
                                  want_du=False, want_dpsi0=False)
                out["dL_dk_off"] = float(res["dL_drates"][0])
            sim.sync()
            out["forward_plus_adjoint_s" if rec else "forward_s"] = time.perf_counter() - t0
        # the same derivative in tangent-linear mode: one pass carrying the
        # state and its tangent along d k_off, no checkpoints
        sim.set_checkpointing(0, 1)
        sim.set_tangent((1.0, 0.0, 0.0))
        sim.set_state(psi_l)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for m in range(nmac):
            sim.set_velocity(vl[m])
            sim.step(nsl)
        _, out["dL_dk_off_tangent"] = sim.tangent_observable("mean_stress")
        out["forward_plus_tangent_s"] = time.perf_counter() - t0
        sim.close()
        out["adjoint_over_forward"] = (out["forward_plus_adjoint_s"] - out["forward_s"]) / out[
            "forward_s"]
        out["tangent_over_forward"] = (out["forward_plus_tangent_s"] - out["forward_s"]) / out[
            "forward_s"]
        out["checkpoints"] = "outer every 100 substeps (21), inner every 10 (9), 10 slots"
        return out

    def diffusion_run():
        """Filament diffusion (mm_diffuse, Crank-Nicolson per direction) on the
        large512 state, float32: events around one call (the three directions
        and the re-derived coarse density, which reads the motor density),
        and around the psi solves alone."""
        wl = WORKLOADS["large512"]
        gl = wl["grid"]
        sim = mm.Simulation(gl, r, "fp32", stream=stream.cuda_stream)
        sim.set_state(psi_isotropic_perturbed(gl, wl["seed"]))
        sim.set_velocity(torch.tensor(workload_velocity("large512", 0), device=dev))
        sim.step(2)
        sim.diffuse(1e-3, 0.1, 0.01)
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.diffuse(1e-3, 0.1, 0.01)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        sim.sync()
        sim.close()
        psi_bytes = gl.nx * gl.ny * gl.ntheta * 4
        return {"workload": "large512 psi (512x512 x 64, float32), D_t = 1e-3, D_r = 0.1",
                "ms_per_call": min(ts),
                "algorithmic_bytes_psi_solves": 3 * 3 * 2 * psi_bytes,
                "algorithmic_bytes_reinit": gl.micro_cells * 4 + 3 * psi_bytes}

    def local_run(wname, precision="fp32", reps=5):
        """Local substeps with psi frozen (mm_motor_local) over the macro
        interval of the workload (its substeps x the global dt): CUDA events
        around each call; the cell-updates are sum_i n_i x ntheta x ns with n_i
        the substeps cell i took. Beside it, the global substeps over the same
        interval."""
        wl = WORKLOADS[wname]
        gl = wl["grid"]
        sim = mm.Simulation(gl, r, precision, stream=stream.cuda_stream)
        sim.set_state(psi_isotropic_perturbed(gl, wl["seed"]))
        sim.set_velocity(torch.tensor(workload_velocity(wname, 0), device=dev))
        T = wl["substeps"] * sim.dt
        nst = sim.motor_local(T)
        updates = int(nst.astype(np.int64).sum()) * gl.ntheta * gl.ns
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.motor_local_device(T)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(wl["substeps"])
        e1.record(stream)
        e1.synchronize()
        sim.sync()
        sim.close()
        ms = sum(ts) / len(ts)
        return {"workload": f"{wname} ({gl.nx}x{gl.ny} x {gl.ntheta} x {gl.ns}, {precision}), "
                            f"T = {wl['substeps']} global substeps",
                "substeps_per_cell": [int(nst.min()), int(nst.max())],
                "value": world * updates / (ms * 1e-3), "unit": UNIT, "ms_per_call": ms,
                "global_substeps_ms_same_interval": e0.elapsed_time(e1),
                "cell_updates_per_call": updates}

    def anchors_run(wname, substeps, ell=0.05):
        """Non-local motor anchors (mm_set_anchors, l/L = ell: the filament
        spans ell of the domain, 6.4 cells at 128^2): a captured graph of
        `substeps` anchor substeps (three launches each: the substep, the
        per-anchor close, the scale-down fix-up) after a warm-up graph."""
        wl = WORKLOADS[wname]
        gl = wl["grid"]
        sim = mm.Simulation(gl, Rates(ell=ell), "fp32", stream=stream.cuda_stream)
        sim.set_anchors(True)
        sim.set_state(psi_isotropic_perturbed(gl, wl["seed"]))
        sim.set_velocity(torch.tensor(workload_velocity(wname, 0), device=dev))
        sim.step(substeps)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(substeps)
        e1.record(stream)
        e1.synchronize()
        sim.sync()
        sim.close()
        ms = e0.elapsed_time(e1) / substeps
        algo = algorithmic_bytes_per_launch(gl, 4)
        peak_, src_ = read_peaks()
        return {"workload": f"{wname} ({gl.nx}x{gl.ny} x {gl.ntheta} x {gl.ns}, fp32), l/L = {ell}",
                "value": world * gl.micro_cells / (ms * 1e-3), "unit": UNIT,
                "ms_per_substep": ms, "algorithmic_bytes_per_substep": algo,
                "roofline": {"bound": "hbm", "achieved": algo / (ms * 1e-3) / 1e9, "peak": peak_,
                             "unit": "GB/s", "frac": algo / (ms * 1e-3) / 1e9 / peak_,
                             "kernel": "k_substep_anchor + k_anchor_close + k_anchor_fix (float32)",
                             "peak_source": src_, "traffic": None}}

    def capture_run(wname, substeps, ell=0.05, rc_cells=1.5):
        """Finite capture radius (mm_set_capture, r_c = rc_cells x the cell
        width, l/L = ell): a captured graph of `substeps` substeps (three
        launches each: psi transport, Alg. 2 per anchor, the n_b gather)
        after a warm-up graph, on the workload's grid with the motors bound
        to their anchors from a seeded random state. Algorithmic bytes per
        substep: the motor density read and written (2 t per configuration),
        the line sums written and read (2 t per (anchor, line)), per
        (cell, theta) psi read and written, n_b written and read and psi^{n+1}
        read once for the coarse density (5 t), per cell Mf read and
        written, C written and M read (4 t)."""
        wl = WORKLOADS[wname]
        gl = wl["grid"]
        rc = rc_cells / gl.nx
        sim = mm.Simulation(gl, Rates(ell=ell), "fp32", stream=stream.cuda_stream)
        sim.set_state(psi_isotropic_perturbed(gl, wl["seed"]))
        tpl = sim.set_capture(rc)
        nconf, nlines = tpl["nconf"], len(tpl["lines"])
        sim.set_velocity(torch.tensor(workload_velocity(wname, 0), device=dev))
        sim.step(substeps)  # the motors bind from Mb = 0
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(substeps)
        e1.record(stream)
        e1.synchronize()
        sim.sync()
        sim.close()
        ms = e0.elapsed_time(e1) / substeps
        cells, t = gl.nx * gl.ny, 4
        algo = (cells * nconf * 2 * t + cells * nlines * 2 * t + cells * gl.ntheta * 5 * t
                + cells * 4 * t)
        peak_, src_ = read_peaks()
        return {"workload": f"{wname} ({gl.nx}x{gl.ny} x {gl.ntheta} x {gl.ns}, fp32), "
                            f"l/L = {ell}, r_c = {rc_cells} cells",
                "configurations_per_anchor": nconf, "lines_per_anchor": nlines,
                "value": world * cells * nconf / (ms * 1e-3), "unit": "configuration-updates/s",
                "ms_per_substep": ms, "algorithmic_bytes_per_substep": algo,
                "roofline": {"bound": "hbm", "achieved": algo / (ms * 1e-3) / 1e9, "peak": peak_,
                             "unit": "GB/s", "frac": algo / (ms * 1e-3) / 1e9 / peak_,
                             "kernel": "k_rc_psi + k_rc_motor + k_rc_nb (float32)",
                             "peak_source": src_, "traffic": None}}

    def fluid_run(wname, reps=5):
        """Thin-gap fluid solve (mm_fluid_solve, eps = 0.1, z0 = 0.1, with the
        dipole term) on the workload's state, float32: CUDA events around each
        solve (the moments of the state, three batched float64 transforms, the
        per-mode map, the velocity update and the substep rule), and around one
        Alg. 1 macro step (the solve, then the workload's substeps)."""
        wl = WORKLOADS[wname]
        gl = wl["grid"]
        sim = mm.Simulation(gl, r, "fp32", stream=stream.cuda_stream)
        sim.set_state(psi_isotropic_perturbed(gl, wl["seed"]))
        sim.set_velocity(torch.tensor(workload_velocity(wname, 0), device=dev))
        sim.step(2)
        sim.fluid_setup(0.1, 0.1)
        sim.fluid_solve(dipole=True, u_out=None)
        sim.step(wl["substeps"])
        ts, tm = [], []
        for _ in range(reps):
            flush.zero_()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            sim.fluid_solve(dipole=True, u_out=None)
            e1.record(stream)
            sim.step(wl["substeps"])
            e2.record(stream)
            e2.synchronize()
            ts.append(e0.elapsed_time(e1))
            tm.append(e0.elapsed_time(e2))
        sim.sync()
        sim.close()
        ms, mac = sum(ts) / len(ts), sum(tm) / len(tm)
        return {"workload": f"{wname} ({gl.nx}x{gl.ny} x {gl.ntheta} x {gl.ns}, fp32), "
                            f"eps = 0.1, z0 = 0.1, macro step = solve + {wl['substeps']} substeps",
                "ms_per_solve": ms, "macro_step_ms": mac, "solve_share_of_macro_step": ms / mac,
                "macro_value": world * gl.micro_cells * wl["substeps"] / (mac * 1e-3),
                "unit": UNIT}

    def ensemble_run(steps):
        """ensemble64: 64 members with uneven grids (N in {32..128}, Ntheta and
        Ns in {16, 32}), k_off log-uniform in [0.05, 5], v_walk in [0.5, 2];
        after mm_batch_autotune, a step is one graph of 500 batched substeps
        (one launch per substep over all members)."""
        from paper_1908_04279_gb300.inputs import ensemble_members, member_inputs
        ms_ = ensemble_members()
        b = mm.Batch([m.grid for m in ms_], [m.rates for m in ms_], "fp32",
                     stream=stream.cuda_stream)
        for sim, m in zip(b.members, ms_):
            psi_m, u_m = member_inputs(m)
            sim.set_state(psi_m)
            sim.set_velocity(u_m)
        tune = b.autotune(substeps=3)
        ne = WORKLOADS["ensemble64"]["substeps"]
        b.step(ne)
        b.sync()
        times = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(ne)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        b.sync()
        info = b.launch_info()
        cells = b.cell_updates_per_substep
        algo_e = sum(algorithmic_bytes_per_launch(m.grid, 4) for m in ms_)
        b.close()
        ms_step = sum(times) / len(times)
        launch = ms_step / ne
        best = min(tune, key=lambda x: x["ms_per_substep"])
        return {"workload": "ensemble64 (64 members, 500 substeps per step in one CUDA graph, "
                            "float32)",
                "value": world * cells * ne / (ms_step * 1e-3), "unit": UNIT, "steps": steps,
                "ms_per_step": ms_step, "kernel_ms_per_launch": launch,
                "motor_cells_per_substep": cells, "algorithmic_bytes_per_launch": algo_e,
                "achieved_gbs": algo_e / (launch * 1e-3) / 1e9,
                "plan": {k: info[k] for k in ("grid", "block", "tiles", "V", "tile_work",
                                              "chunk_bytes", "pair_cells")},
                "autotune_best_ms_per_substep": best["ms_per_substep"],
                "autotune_candidates": len(tune)}

    w = WORKLOADS[name]
    g, nsub = w["grid"], w["substeps"]
    big = g.micro_cells > 2e8
    units_per_step = g.micro_cells * nsub
    peak, peak_src = read_peaks()

    # ---- headline: the workload in the float32 form
    clocks = ClockSampler(local)
    clocks.start()
    total_ms, kern_ms = device_run(name, "fp32", args.steps, args.warmup)
    clk = clocks.stop()
    # the float64 form on the same workload (one macro step after one warm-up
    # macro step on the large case: 100 substeps of about 65 ms)
    fp64_steps = 1 if big else max(2, min(args.steps, 3))
    fp64_ms, fp64_kern = device_run(name, "fp64", fp64_steps, 1)
    e2e_s, h2d, d2h = e2e_run(name, "fp32", args.steps, args.warmup)

    # ---- the other single-instance workload: the L2-resident precision128
    # case beside a large headline (or large512 beside a small one)
    other = "precision128" if name != "precision128" else "large512"
    wo = WORKLOADS[other]
    go, nso = wo["grid"], wo["substeps"]
    o_steps = 10 if other == "precision128" else 3
    o_ms, o_kern = device_run(other, "fp32", o_steps, 3)

    adj = {"workload": "adjoint64 (64x64 x 32 x 32, 100 substeps, checkpoint every 10, polar order)",
           "fp32": adjoint_ratio("fp32"), "fp64": adjoint_ratio("fp64")}
    ens = ensemble_run(10)
    large_adj = large_adjoint_run()
    diff = diffusion_run()
    anchors = {"precision128": anchors_run("precision128", 50),
               "large512": anchors_run("large512", 5)}
    fluid = {"precision128": fluid_run("precision128"), "large512": fluid_run("large512", reps=3)}
    capture = {"precision128": capture_run("precision128", 20),
               "large512": capture_run("large512", 3)}
    local = {"precision128": local_run("precision128"),
             "large512": local_run("large512", reps=3)}
    # measured arithmetic roofs (fused multiply-adds per second)
    alu = {k: mm.alu_peak(k, stream.cuda_stream) for k in ("fp64", "fp32", "fp32x2")}
    packed_tops = alu["fp32x2"]["fma_per_s"] / 1e12
    for v in local.values():
        # LOCAL_OPS float32 operations per motor value and substep against the
        # measured packed float32 rate (the kernel's element-wise arithmetic is
        # packed; its minima and maxima are scalar, so this is the roof it can
        # approach, not exceed)
        ops = v["cell_updates_per_call"] * LOCAL_OPS / (v["ms_per_call"] * 1e-3) / 1e12
        v["roofline"] = {"bound": "alu", "achieved": ops, "peak": packed_tops,
                         "unit": "Tops/s", "frac": ops / packed_tops,
                         "peak_source": "measured (mm_alu_peak, packed float32 fma)",
                         "kernel": "k_motor_local (float32)",
                         "traffic": read_profile_traffic("k_motor_local", wname_of(v), "fp32")}

    total_ms, kern_ms, fp64_ms, fp64_kern, e2e_s, o_ms, o_kern = reduce_max(
        [total_ms, kern_ms, fp64_ms, fp64_kern, e2e_s, o_ms, o_kern], dev)

    value = whole_job_value(world, units_per_step * args.steps, total_ms * 1e-3)
    launch_ms = kern_ms / (args.steps * nsub)
    algo = algorithmic_bytes_per_launch(g, 4)
    achieved = algo / (launch_ms * 1e-3) / 1e9
    # the large case's capture is taken at a quarter of its cells (256x256 x
    # 64 x 64) and scaled to a full launch by the motor cells
    traffic = (read_profile_traffic("k_substep", "large512", "fp32") if name == "large512"
               else read_profile_traffic("k_substep", name, "fp32"))
    fp64_value = whole_job_value(world, units_per_step * fp64_steps, fp64_ms * 1e-3)
    fp64_launch_ms = fp64_kern / (fp64_steps * nsub)
    fp64_ops = g.micro_cells * SUBSTEP_OPS / (fp64_launch_ms * 1e-3) / 1e12
    fp64_peak = alu["fp64"]["fma_per_s"] / 1e12
    o_launch = o_kern / (o_steps * nso)
    o_algo = algorithmic_bytes_per_launch(go, 4)
    o_traffic = read_profile_traffic("k_substep", other, "fp32")
    o_leg = {"workload": f"{other} ({go.nx}x{go.ny} x {go.ntheta} x {go.ns}, {nso} substeps per "
                         f"macro step, float32)",
             "value": whole_job_value(world, go.micro_cells * nso * o_steps, o_ms * 1e-3),
             "unit": UNIT, "steps": o_steps, "ms_per_step": o_ms / o_steps,
             "kernel_ms_per_launch": o_launch, "algorithmic_bytes_per_launch": o_algo,
             "roofline": {"bound": "hbm", "peak": peak, "unit": "GB/s",
                          "achieved": o_algo / (o_launch * 1e-3) / 1e9,
                          "frac": o_algo / (o_launch * 1e-3) / 1e9 / peak,
                          "kernel": "k_substep (float32)", "peak_source": peak_src,
                          "traffic": o_traffic,
                          "dram_frac": (None if o_traffic is None
                                        else o_traffic / (o_launch * 1e-3) / 1e9 / peak)}}
    if other == "precision128":
        o_leg["note"] = ("L2-resident: the 67 MB motor density stays in the 129 MB L2 within a "
                         "macro step, so frac compares an L2-fed kernel with the HBM copy peak; "
                         "dram_frac is its measured DRAM traffic over the same time")
    if rank == 0:
        cpu = time_oracle_sample(name)
        ens_frac = ens["achieved_gbs"] / peak
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": name, "grid": f"{g.nx}x{g.ny}", "ntheta": g.ntheta, "ns": g.ns,
                       "substeps_per_step": nsub, "precision": "float32 Mb/psi, float64 sums",
                       "l2": (f"inputs larger than L2 ({g.micro_cells * 4 / 1e9:.2f} GB of motor "
                              "density) and L2 flushed between timed steps (256 MiB write "
                              "outside the timed events)") if big else
                             "flushed between timed steps (256 MiB write outside the timed events)",
                       "parallelism": f"{world} independent instance(s), one per GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_substep (float32)", "peak_source": peak_src,
                         "kernel_ms_per_launch": launch_ms,
                         "algorithmic_bytes_per_launch": algo},
            "cpu_baseline": cpu,
            "e2e": {"value": whole_job_value(world, units_per_step * args.steps, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "fp64": {"value": fp64_value, "unit": UNIT, "steps": fp64_steps,
                     "ms_per_step": fp64_ms / fp64_steps, "kernel_ms_per_launch": fp64_launch_ms,
                     "roofline": {"bound": "alu", "achieved": fp64_ops, "peak": fp64_peak,
                                  "unit": "Tops/s", "frac": fp64_ops / fp64_peak,
                                  "kernel": "k_substep (float64)",
                                  "ops_per_cell_update": SUBSTEP_OPS,
                                  "peak_source": "measured (mm_alu_peak, float64 fma)",
                                  "fp64_pipe_ops_per_cell_update": SUBSTEP_FP64_PIPE_OPS,
                                  "fp64_pipe_frac": fp64_ops * SUBSTEP_FP64_PIPE_OPS
                                  / SUBSTEP_OPS / fp64_peak}},
            other: o_leg,
            "alu_peaks": {k: {"fma_per_s": v["fma_per_s"], "ms_per_launch": v["ms_per_launch"]}
                          for k, v in alu.items()},
            "adjoint": adj,
            "large512_adjoint": dict(
                large_adj, workload="large512, 2000 substeps, float32, mean active stress vs k_off"),
            "diffusion": diff,
            "local": local,
            "anchors": anchors,
            "fluid": fluid,
            "capture": capture,
            "ensemble": dict(ens, roofline={"bound": "hbm", "peak": peak, "unit": "GB/s",
                                            "achieved": ens["achieved_gbs"], "frac": ens_frac,
                                            "kernel": "k_substep_batch (float32)",
                                            "peak_source": peak_src,
                                            "traffic": read_profile_traffic(
                                                "k_substep_batch", "ensemble64", "fp32")}),
            # per macro step: set_velocity (precision conversion, per-cell velocity
            # block, the two substep-rule kernels), nsub substeps, moments
            "gpu_launches": args.steps * (nsub + 5),
            "clocks": clk,
            # flat summaries of every leg (fractions of the measured peaks)
            "hbm_frac": achieved / peak,
            "fp64_value": fp64_value,
            "fp32_over_fp64": value / fp64_value,
            "fp64_alu_frac": fp64_ops / fp64_peak,
            "adjoint_over_forward": {"adjoint64_fp32": adj["fp32"]["adjoint_over_forward"],
                                     "adjoint64_fp64": adj["fp64"]["adjoint_over_forward"],
                                     "large512_fp32": large_adj["adjoint_over_forward"],
                                     "large512_fp32_tangent": large_adj["tangent_over_forward"]},
            "ensemble_frac": ens_frac,
            "anchors_frac": {k: v["roofline"]["frac"] for k, v in anchors.items()},
            "capture_frac": {k: v["roofline"]["frac"] for k, v in capture.items()},
            "local_alu_frac": {k: v["roofline"]["frac"] for k, v in local.items()},
            f"{other}_frac": o_leg["roofline"]["frac"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large512", choices=sorted(WORKLOADS))
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
