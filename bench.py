"""Benchmark: GDoF/s of the matrix-free SBM operator apply on one workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

A step is one operator apply y = A x (cells, surrogate faces, scatter) of the
workload.  Default workload: 3D continuous Galerkin Q4 on 96^3 cells, sphere
r = 0.71, FP64, x ~ U(-1,1) seed 1.  Prints one JSON line (rank 0).

--impl reference times the CPU FP64 oracle (the element-by-element
definition), on the host cores, on the same workload and metric.
With N > 1 (torchrun) every rank applies its own replica of the problem
(independent work, no collective on the data path); value is the DoFs of all
ranks per second.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as S  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 1.25      # GB300 FP64 (CUDA cores) nominal dense rate
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=S.SPHERE_3D_Q4.name)
    return ap.parse_args()


def workload(name):
    if name in S.WORKLOADS:
        return S.WORKLOADS[name]
    raise SystemExit(f"unknown workload {name}; choose from {sorted(S.WORKLOADS)}")


def flops_per_apply(d, p, n_cells, n_sfaces):
    """Floating-point operations of one apply as the kernels compute it.

    Cell term: 7 (3D) or 4 (2D) one-dimensional sweeps of n^(d+1) FMAs.
    Surrogate face: point evaluation n^(2d-1) + n^(2d-2) + ... FMAs plus
    11 n^d FMAs of sum-factorised traces and integration (counted per face).
    """
    n = p + 1
    sweeps = 7 if d == 3 else 4
    cell = 2 * sweeps * n ** (d + 1)
    pe = n ** (2 * d - 1) + n ** (2 * d - 2) + (n ** d if d == 3 else 0)
    face = 2 * (pe + 11 * n ** d)
    return cell * n_cells + face * n_sfaces


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_init(n):
    import torch
    if n <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch.distributed as dist
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend)
    return dist.get_rank(), dist.get_world_size(), dist


def cpu_baseline(w, O=None, x=None):
    """The oracle's apply on the host cores: one full apply of the workload."""
    from oracle.operator import Problem as OracleProblem
    if O is None:
        O = OracleProblem.from_workload(w)
        x = S.random_vector(w.seed, O.n_dofs, w.dist)
    t = time.perf_counter()
    O.apply(x)
    dt = time.perf_counter() - t
    return {"value": O.n_dofs / dt / 1e9, "unit": "GDoF/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"one full EBE apply of {w.name} ({O.n_dofs} DoFs), {dt:.1f} s"}


def run_reference(args, w):
    rank, world, dist = dist_init(args.gpus)
    if rank != 0:
        return
    from oracle.operator import Problem as OracleProblem
    O = OracleProblem.from_workload(w)
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    times = []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        O.apply(x)
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
    total = sum(times)
    v = O.n_dofs * len(times) / total / 1e9
    line = {
        "impl": "reference", "metric": "GDoF/s per operator apply (FP64)", "value": v,
        "unit": "GDoF/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_dofs": O.n_dofs},
        "cpu_baseline": {"value": v, "unit": "GDoF/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{len(times)} full EBE applies of {w.name}"},
        "e2e": {"value": v, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, w):
    import torch

    import paper_2507_17053_gb300 as G
    rank, world, dist = dist_init(args.gpus)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P = G.Problem.from_workload(w)
    x_host = S.random_vector(w.seed, P.n_dofs, w.dist)
    x = torch.from_numpy(x_host).to(dev)
    y = torch.empty_like(x)
    st = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        P.apply_f64(x, y)
    torch.cuda.synchronize()
    G.sbm_profile_read(P.handle)
    G.sbm_profile_enable(P.handle, True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        P.apply_f64(x, y)
    e1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms = e0.elapsed_time(e1)
    kern_ms, launches = G.sbm_profile_read(P.handle)
    G.sbm_profile_enable(P.handle, False)
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # end to end through the C ABI with host buffers (H2D + apply + D2H per step)
    xh = torch.from_numpy(x_host).pin_memory()
    yh = torch.empty(P.n_dofs, dtype=torch.float64).pin_memory()
    e2e_steps = max(3, min(50, args.steps // 10))
    P.apply_f64_host(xh, yh)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        P.apply_f64_host(xh, yh)
    e2e_s = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    if rank != 0:
        return
    n = P.n_dofs
    value = world * n * args.steps / (ms * 1e-3) / 1e9
    pk, pk_src = peaks()
    flops = flops_per_apply(w.dim, w.degree, P.n_cells, P.n_sfaces)
    per_launch_ms = kern_ms / launches
    per_apply_kern_ms = kern_ms / args.steps
    achieved_tf = flops / (per_apply_kern_ms * 1e-3) / 1e12
    alg_bytes = 16 * n
    line = {
        "metric": "GDoF/s per operator apply (FP64)",
        "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_dofs": n, "n_cells": P.n_cells,
                   "n_sfaces": P.n_sfaces, "degree": w.degree, "dim": w.dim,
                   "l2": f"inputs larger than L2: x and y {2 * 8 * n / 1e6:.0f} MB > 129 MB"},
        "e2e": {"value": world * n * e2e_steps / e2e_s / 1e9, "unit": "GDoF/s",
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": FP64_NOMINAL_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved_tf / FP64_NOMINAL_TFLOPS,
                     "traffic": None,
                     "kernel": "cg_apply_f64_kernel (all colour launches of one apply)",
                     "flops_per_apply": flops, "kernel_ms_per_apply": per_apply_kern_ms,
                     "kernel_ms_per_launch": per_launch_ms,
                     "peak_note": "FP64 nominal 1.25 TFLOP/s (FMA microbenchmark: 1.007)",
                     "hbm": {"achieved_gbs": alg_bytes / (ms / args.steps * 1e-3) / 1e9,
                             "peak_gbs": pk.get("hbm_gbs"), "peak_src": pk_src,
                             "frac": alg_bytes / (ms / args.steps * 1e-3) / 1e9 / pk["hbm_gbs"],
                             "bytes_per_dof": 16}},
        "clocks": clk,
    }
    if world == 1 or rank == 0:
        try:
            line["cpu_baseline"] = cpu_baseline(w)
        except MemoryError:
            line["cpu_baseline"] = None
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    w = workload(args.workload)
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
