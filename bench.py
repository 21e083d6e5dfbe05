"""Benchmark of the microscale kinetic step on GB300.

A step is one macro step of the workload: prescribe that macro step's
velocity (mm_set_velocity, which also recomputes the adaptive substep), run its
substeps (mm_micro_step) and reduce the macroscale moments (mm_moments).
Metric: micro-state cell-updates per second = nx*ny*ntheta*ns*substeps / time.

Default workload "precision128": 128x128 periodic grid, 32 orientations, 32
arclength nodes, 50 substeps per macro step, velocity from a seeded random
divergence-free field (8 Fourier modes, amplitude 0.1) refreshed every macro
step, mixed precision (float32 Mb/psi, float64 sums). The float64 path is timed
on the same workload and reported beside it. Beside the main line: the
adjoint/forward time ratio (adjoint64), the substep on large512 (4.3 GB of
motor state, the HBM roofline case) in float32 and float64, and the batched
ensemble (ensemble64, 64 uneven members, 500 substeps per graph).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload precision128|large512|adjoint64|cellular32]

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
    "k_substep": ("mm_step.cu", "mm_cell.cuh", "mm_walk.cuh", "mm_internal.cuh"),
    "k_substep_batch": ("mm_batch.cu", "mm_cell.cuh", "mm_walk.cuh", "mm_internal.cuh"),
    "k_adjoint": ("mm_adjoint.cu", "mm_walk.cuh", "mm_internal.cuh"),
    "k_motor_local": ("mm_local.cu", "mm_cell.cuh", "mm_walk.cuh", "mm_internal.cuh"),
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
    """Bytes one substep launch must move at minimum: Mb read and written once
    (2 * tsize per motor cell); per (cell, theta) psi read and written
    (2 * tsize) and n_b read and written (2 * 8); per cell Mf read and written,
    C written, M read and u read (4 * 8 + 2 * tsize)."""
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


# Float32 operations per motor value and substep of the local-step kernel,
# counted from the scheme: per RK2 stage the backward difference, its half,
# two sign transfers, two minima, the maximum with zero, the flux fma, the flux
# difference and two fmas of the stage update (11); two stages, plus one add
# of the n_b sum.
LOCAL_OPS = 23


def wname_of(leg: dict) -> str:
    """Workload name of a bench leg from its description."""
    return leg["workload"].split(" ")[0]


def alu_peak_tops(sm_mhz: float = 2070.0, sms: int = 152, lanes: int = 128) -> float:
    """Float32 operations per second of GB300 in Tops/s: 152 SMs x 128 float32
    lanes x the maximum SM clock (one fma, add, mul, min or max per lane and
    clock)."""
    return sms * lanes * sm_mhz * 1e6 / 1e12


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


def time_oracle_sample(name: str, budget_s: float = 12.0, max_sub: int = 40):
    """Float64 CPU oracle on a bounded sample of the workload: the workload's
    initial state and first velocity, as many substeps as fit in budget_s.
    Workloads above 2e8 motor cells are sampled on a 64x64-cell periodic grid
    with the workload's orientations and arclength nodes."""
    from oracle import oracle as O
    from paper_1908_04279_gb300.inputs import Grid
    w = WORKLOADS[name]
    g, r = w["grid"], Rates()
    sub = ""
    if g.micro_cells > 2e8:
        g = Grid(64, 64, g.ntheta, g.ns, g.L)
        sub = " on a 64x64-cell sub-grid"
    st = O.make_state(g, psi_isotropic_perturbed(g, w["seed"]))
    if sub:
        from paper_1908_04279_gb300.inputs import random_divfree_flow, velocity_seed
        u = random_divfree_flow(g, velocity_seed(w["seed"], 0), w["modes"], w["amp"])
    else:
        u = workload_velocity(name, 0)
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
    g, r = w["grid"], Rates()
    st = O.make_state(g, psi_isotropic_perturbed(g, w["seed"]))
    u = workload_velocity(name, 0)
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
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": name, "grid": f"{g.nx}x{g.ny}", "ntheta": g.ntheta, "ns": g.ns,
                       "substeps_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} steps of {per_step} oracle substep(s) of "
                                       f"{name} on 1 host core"},
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
    w = WORKLOADS[name]
    g, r = w["grid"], Rates()
    nsub = w["substeps"]
    n_vel = max(w["macro"], 1)
    stream = torch.cuda.current_stream(dev)
    vels_host = [np.ascontiguousarray(workload_velocity(name, m)) for m in range(n_vel)]
    vels_dev = [torch.tensor(v, device=dev) for v in vels_host]
    psi0 = psi_isotropic_perturbed(g, w["seed"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    fields_dev = torch.empty(12 * g.nx * g.ny, dtype=torch.float64, device=dev)

    def device_run(precision, steps, warmup, timed_kernel=True):
        sim = mm.Simulation(g, r, precision, stream=stream.cuda_stream)
        sim.set_state(psi0)
        m = 0
        for _ in range(warmup):
            sim.set_velocity(vels_dev[m % n_vel]); m += 1
            sim.step(nsub)
            sim.moments(fields=fields_dev)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        step_ms, kern_ms = [], []
        for _ in range(steps):
            flush.zero_()  # L2 flush between timed steps, outside the timed events
            e0, e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
            e0.record(stream)
            sim.set_velocity(vels_dev[m % n_vel]); m += 1
            e1.record(stream)
            sim.step(nsub)
            e2.record(stream)
            sim.moments(fields=fields_dev)
            e3.record(stream)
            e3.synchronize()
            step_ms.append(e0.elapsed_time(e3))
            kern_ms.append(e1.elapsed_time(e2))
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        sim.close()
        return sum(step_ms), sum(kern_ms)

    def e2e_run(precision, steps, warmup):
        """Through the public API with host buffers: every step copies its
        velocity from pinned host memory and reads the moments back."""
        sim = mm.Simulation(g, r, precision, stream=stream.cuda_stream)
        sim.set_state(psi0)
        pinned = [torch.from_numpy(v).pin_memory() for v in vels_host]
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

    def large_run(precision, substeps):
        """large512 (512x512 x 64 x 64, 4.3 GB of float32 Mb): far beyond L2,
        so its substep launch gives the HBM roofline fraction. Timed as one
        graph of `substeps` launches after a warm-up graph."""
        wl = WORKLOADS["large512"]
        gl = wl["grid"]
        sim = mm.Simulation(gl, r, precision, stream=stream.cuda_stream)
        sim.set_state(psi_isotropic_perturbed(gl, wl["seed"]))
        sim.set_velocity(torch.tensor(workload_velocity("large512", 0), device=dev))
        sim.step(substeps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(substeps)
        e1.record(stream)
        e1.synchronize()
        sim.sync()
        sim.close()
        ms = e0.elapsed_time(e1) / substeps
        tsz = 4 if precision == "fp32" else 8
        algo_l = algorithmic_bytes_per_launch(gl, tsz)
        return {"value": world * gl.micro_cells / (ms * 1e-3), "unit": UNIT,
                "kernel_ms_per_launch": ms, "algorithmic_bytes_per_launch": algo_l,
                "achieved_gbs": algo_l / (ms * 1e-3) / 1e9}

    def large_adjoint_run():
        """large512 forward + adjoint: 20 macro steps x 100 substeps (a new
        16-mode flow each macro step), gradient of the mean active stress
        with respect to k_off, outer checkpoints every 100 substeps and inner
        ones every 10 (two levels: about 40 states of 4.4 GB held). Times the
        plain forward and the recorded forward + reverse sweep."""
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
        sim.close()
        out["adjoint_over_forward"] = (out["forward_plus_adjoint_s"] - out["forward_s"]) / out[
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
                                              "chunk_bytes")},
                "autotune_best_ms_per_substep": best["ms_per_substep"],
                "autotune_candidates": len(tune)}

    units_per_step = g.micro_cells * nsub
    clocks = ClockSampler(local)
    clocks.start()
    total_ms, kern_ms = device_run("fp32", args.steps, args.warmup)
    clk = clocks.stop()
    fp64_steps = max(2, min(args.steps, 3))
    fp64_ms, fp64_kern = device_run("fp64", fp64_steps, 1)
    e2e_s, h2d, d2h = e2e_run("fp32", args.steps, args.warmup)
    adj = {"workload": "adjoint64 (64x64 x 32 x 32, 100 substeps, checkpoint every 10, polar order)",
           "fp32": adjoint_ratio("fp32"), "fp64": adjoint_ratio("fp64")}
    large = {"workload": "large512 (512x512 x 64 x 64, 1.07e9 motor cells)",
             "fp32": large_run("fp32", 10), "fp64": large_run("fp64", 3)}
    ens = ensemble_run(max(2, min(args.steps, 3)))
    large_adj = large_adjoint_run()
    diff = diffusion_run()
    anchors = {"precision128": anchors_run("precision128", 50),
               "large512": anchors_run("large512", 5)}
    fluid = {"precision128": fluid_run("precision128"), "large512": fluid_run("large512", reps=3)}
    local = {"precision128": local_run("precision128"),
             "large512": local_run("large512", reps=3)}
    for v in local.values():
        # ALU roofline: LOCAL_OPS float32 operations per motor value and
        # substep against 128 float32 lanes per SM at the maximum SM clock
        ops = v["cell_updates_per_call"] * LOCAL_OPS / (v["ms_per_call"] * 1e-3) / 1e12
        v["roofline"] = {"bound": "alu", "achieved": ops, "peak": alu_peak_tops(),
                         "unit": "Tops/s", "frac": ops / alu_peak_tops(),
                         "kernel": "k_motor_local (float32)",
                         "traffic": read_profile_traffic("k_motor_local", wname_of(v), "fp32")}

    total_ms, kern_ms, fp64_ms, e2e_s = reduce_max([total_ms, kern_ms, fp64_ms, e2e_s], dev)

    value = whole_job_value(world, units_per_step * args.steps, total_ms * 1e-3)
    launch_ms = kern_ms / (args.steps * nsub)
    peak, peak_src = read_peaks()
    algo = algorithmic_bytes_per_launch(g, 4)
    achieved = algo / (launch_ms * 1e-3) / 1e9
    traffic = read_profile_traffic("k_substep", name, "fp32")
    fp64_value = whole_job_value(world, units_per_step * fp64_steps, fp64_ms * 1e-3)
    if rank == 0:
        cpu = time_oracle_sample(name) if world == 1 or rank == 0 else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": name, "grid": f"{g.nx}x{g.ny}", "ntheta": g.ntheta, "ns": g.ns,
                       "substeps_per_step": nsub, "precision": "float32 Mb/psi, float64 sums",
                       "l2": "flushed between timed steps (256 MiB write outside the timed events)",
                       "parallelism": f"{world} independent instance(s), one per GPU"},
            "fp64": {"value": fp64_value, "unit": UNIT, "steps": fp64_steps,
                     "ms_per_step": fp64_ms / fp64_steps,
                     "kernel_ms_per_launch": fp64_kern / (fp64_steps * nsub),
                     "fp32_over_fp64": value / fp64_value},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_substep (float32)", "peak_source": peak_src,
                         "kernel_ms_per_launch": launch_ms,
                         "algorithmic_bytes_per_launch": algo},
            "cpu_baseline": cpu,
            "e2e": {"value": whole_job_value(world, units_per_step * args.steps, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "adjoint": adj,
            "large512": dict(large, fp32_over_fp64=large["fp32"]["value"] / large["fp64"]["value"],
                             roofline={"bound": "hbm", "peak": peak, "unit": "GB/s",
                                       "achieved": large["fp32"]["achieved_gbs"],
                                       "frac": large["fp32"]["achieved_gbs"] / peak,
                                       "kernel": "k_substep (float32)", "peak_source": peak_src,
                                       "traffic": read_profile_traffic(
                                           "k_substep", "large512", "fp32")}),
            "large512_adjoint": dict(
                large_adj, workload="large512, 2000 substeps, float32, mean active stress vs k_off"),
            "diffusion": diff,
            "local": local,
            "anchors": anchors,
            "fluid": fluid,
            "ensemble": dict(ens, roofline={"bound": "hbm", "peak": peak, "unit": "GB/s",
                                            "achieved": ens["achieved_gbs"],
                                            "frac": ens["achieved_gbs"] / peak,
                                            "kernel": "k_substep_batch (float32)",
                                            "peak_source": peak_src,
                                            "traffic": read_profile_traffic(
                                                "k_substep_batch", "ensemble64", "fp32")}),
            # per macro step: set_velocity (precision conversion, per-cell velocity
            # block, the two substep-rule kernels), nsub substeps, moments
            "gpu_launches": args.steps * (nsub + 5),
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="precision128", choices=sorted(WORKLOADS))
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
