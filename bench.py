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
# The FP64 pipe issues 2 lane-operations (DFMA, DADD or DMUL alike) per SM
# per clock: 152 SMs x 2070 MHz x 2 = 629.3 G operations/s (x 2 flops per
# FMA = the nominal 1.25 TFLOP/s).  The FP64 apply is bound by this pipe.
SMS, SM_MAX_MHZ, FP64_LANES_PER_SM_CLK = 152, 2070, 2
FP64_PIPE_GOPS = SMS * SM_MAX_MHZ * 1e6 * FP64_LANES_PER_SM_CLK / 1e9
# DRAM bytes (read + write) of one launch of the FP64 cell kernel: constants
# from one ncu capture per (workload, tile shape, store mode) of the kernel as
# it stood when captured (dram__bytes_read.sum + dram__bytes_write.sum), not
# measured by this run; other shapes and modes: not captured
CELL_TRAFFIC = {("sphere3d_cg_q4_n96", 0, 0): 127.09e6 + 106.99e6,
                ("sphere3d_cg_q4_n96", 1, 0): 157.950720e6 + 133.191680e6}
L2_BYTES = 129 * 1024 * 1024
REF_BUDGET_S = 90.0              # wall-clock budget of the --impl reference run


def cell_kernel_name(w, shape, ordered):
    """The FP64 cell-term kernel that tile shape and store mode launch."""
    n = w.degree + 1
    if shape == 2:
        return f"cg_cell_reg_kernel<double,{n}> (cell kernel, tile shape 2)"
    name = ("cg_direct" if shape == 3 else "cg_chunk") + ("_ord" if ordered else "")
    dims = f"{n}" if shape == 3 else f"{w.dim},{n}"
    return (f"{name}_kernel<double,{dims}> (cell kernel, tile shape {shape}, "
            f"{'colour-ordered stores' if ordered else 'colour buffers'})")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=S.SPHERE_3D_Q4.name)
    ap.add_argument("--skip-cpu-baseline", action="store_true",
                    help="leave out the oracle timing (profiling runs)")
    ap.add_argument("--skip-extras", action="store_true",
                    help="only the headline workload (no other workloads, batch, solves)")
    ap.add_argument("--profile-applies", choices=["f64", "f32", "tf32", "bf16"], default=None,
                    help="run --steps applies of the workload in this precision and exit "
                         "(a fixed launch sequence for ncu captures; prints no JSON)")
    ap.add_argument("--profile-batch", choices=["f64", "f32"], default=None,
                    help="run --steps persistent batched applies of 24 rotated ellipsoids x 4 "
                         "right-hand sides (a fixed launch sequence for ncu captures; no JSON)")
    ap.add_argument("--tile-shape", type=int, choices=[-1, 0, 1, 2, 3], default=-1,
                    help="with --profile-applies: pin the cell kernel's tile shape "
                         "(-1 keeps the default, 0)")
    ap.add_argument("--ordered-stores", type=int, choices=[-1, 0, 1], default=-1,
                    help="with --profile-applies: pin the store mode of the shared DoFs "
                         "(1: colour-ordered stores, 0: colour buffers + assembly)")
    return ap.parse_args()


def workload(name):
    if name in S.WORKLOADS:
        return S.WORKLOADS[name]
    raise SystemExit(f"unknown workload {name}; choose from {sorted(S.WORKLOADS)}")


def cell_ops(d, p, n_cells):
    """FP64/FP32 operations the cell kernel executes per apply: (FMAs, other).

    3D: the exact cell operator in the eigenbasis of the 1D pencil (K, M),
    A_K = h (V x V x V) diag(lam_i + lam_j + lam_k) (V x V x V)^T, with the
    x-direction's transform, scaling and transform back merged into the
    matrix h K + mu M of each x-line: per line of the tile 5 one-dimensional
    products in even/odd form, ((n+1)/2)^2 + (n/2)^2 FMAs each, and 3 folds +
    3 unfolds of 2 (n/2) additions each (p = 4: 1625 FMAs + 600 other per
    cell).
    2D: 4 one-dimensional matrix applications per line (Algorithm 1 in
    tensor-product form), even/odd split for n >= 5 with 3 folds and 3
    unfolds per line pair."""
    n = p + 1
    lines = n ** (d - 1)
    h, he = n // 2, (n + 1) // 2
    if d == 3:
        fma = 5 * (he * he + h * h)
        other = 12 * h
    elif n >= 5:
        fma = 4 * (he * he + h * h)
        other = 6 * 2 * h
    else:
        fma, other = 4 * n * n, 0
    return fma * lines * n_cells, other * lines * n_cells


def face_flops(d, p, n_sfaces):
    """FLOPs of the surrogate-face kernel per apply (exact extension): point
    evaluation per face (Algorithm 3's dominant step) n^(2d-1) + n^d FMAs in
    3D (with the stored products of two axes' values), n^3 + n^2 in 2D; plus
    7 n^d FMAs: the normal-derivative trace, its mass product (2 sweeps), one
    transposed interpolation (2 sweeps) and the fold of the face result into
    the cell."""
    n = p + 1
    point = n ** 5 + n ** 3 if d == 3 else n ** 3 + n ** 2
    return 2 * (point + 7 * n ** d) * n_sfaces


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


def max_over_ranks(v, dist, dev):
    """The largest of every rank's v (the job's time is its slowest rank's)."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank in `seconds` (the max over ranks): weak scaling."""
    return world * units_per_rank / seconds


def dist_init(n):
    import torch
    if n <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
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
    """The oracle (element-by-element FP64 definition) on the host cores.

    Each step applies a bounded sample of the workload: a contiguous block of
    active cells (with their faces), sized so that the whole --steps/--warmup
    run takes about REF_BUDGET_S seconds; the blocks cycle through the mesh.
    GDoF/s counts the sample's share of the DoFs (cells in the sample / all
    cells x n_dofs).
    """
    rank, world, dist = dist_init(args.gpus)
    if rank != 0:
        return
    from oracle.operator import Problem as OracleProblem
    O = OracleProblem.from_workload(w)
    x = S.random_vector(w.seed, O.n_dofs, w.dist)
    nc = len(O.mesh.cells)
    # calibrate: time one block of 1/64 of the cells
    blk = max(1, nc // 64)
    t = time.perf_counter()
    O.apply_cells(x, np.arange(blk))
    per_cell = (time.perf_counter() - t) / blk
    total_steps = args.warmup + args.steps
    m = int(max(1, min(nc, REF_BUDGET_S / total_steps / per_cell)))
    times = []
    start = 0
    for i in range(total_steps):
        cells = (np.arange(m) + start) % nc
        start = (start + m) % nc
        t = time.perf_counter()
        O.apply_cells(x, cells)
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
    total = sum(times)
    units = O.n_dofs * m / nc
    v = units * len(times) / total / 1e9
    line = {
        "impl": "reference", "metric": "GDoF/s per operator apply (FP64)", "value": v,
        "unit": "GDoF/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_dofs": O.n_dofs},
        "cpu_baseline": {"value": v, "unit": "GDoF/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"each step: {m} of {nc} active cells (with their faces) "
                                   f"of {w.name}, EBE"},
        "e2e": {"value": v, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_applies(P, fn, x, y, steps, warmup, st, dist=None, dev=None, clocks=None):
    """CUDA-event time of `steps` applies (after `warmup`), per-phase kernel
    times from the library's profiler, max over ranks."""
    import torch

    import paper_2507_17053_gb300 as G
    for _ in range(max(3, warmup)):
        fn(x, y)
    torch.cuda.synchronize()
    G.sbm_profile_read(P.handle)
    G.sbm_profile_enable(P.handle, True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        fn(x, y)
    e1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks is not None else None
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    phases, launches = G.sbm_profile_read(P.handle)
    G.sbm_profile_enable(P.handle, False)
    ms = max_over_ranks(ms, dist, dev)
    return ms, [p / steps for p in phases], launches, clk


def time_plain(fn, x, y, steps, warmup, st, dist=None, dev=None):
    """CUDA-event time of `steps` applies (after `warmup`) with the library's
    profiler off: no events between an apply's kernels, so FP32 applies keep
    their programmatic dependent launches (the call a user makes), max over
    ranks."""
    import torch

    for _ in range(max(3, warmup)):
        fn(x, y)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        fn(x, y)
    e1.record(st)
    torch.cuda.synchronize()
    return max_over_ranks(e0.elapsed_time(e1), dist, dev)


def solve_times(G, torch):
    """Time-to-1e-10 (true FP64 relative residual; b from u = prod sin(pi x_i)).

    2D disk (CG Q2, N = 32): CG as named (it diverges: the operator is
    nonsymmetric), GMRES(100) and BiCGStab in FP64, and FP64 iterative
    refinement around FP32 GMRES / FP32 BiCGStab / BiCGStab on FP64 vectors
    with FP32 applies (short inner solves: 1e-2, at most 300 iterations; an
    FP64 BiCGStab finish when they stall).  3D sphere, Q2, N = 64 (413,013
    DoFs): BiCGStab and GMRES(200) in FP64, and the two BiCGStab refinements.
    The disk also: BiCGStab on the FP32 apply with FP64 reliable updates (on
    the sphere it stalls near 2e-5; see the solver notes).  Each time is the median of 3 solves after a warm-up solve (the solves are
    deterministic: the same iterations every time).  (At p >= 3 in 3D no
    unpreconditioned Krylov method reaches 1e-10 on this operator; see the
    solver notes.)"""

    def timed(b, f):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = f(x)
        torch.cuda.synchronize()
        return r, time.perf_counter() - t

    def run(b, f, reps=3):
        timed(b, f)                 # the first call builds graphs / warms the path
        res = [timed(b, f) for _ in range(reps)]
        return res[-1][0], sorted(dt for _, dt in res)[reps // 2]      # median time

    out = {"rtol": 1e-10}
    w = S.DISK_2D_Q2
    P = G.Problem.from_workload(w)
    b = torch.from_numpy(P.rhs(0)).cuda()
    d2 = {"workload": w.name, "n_dofs": P.n_dofs}
    (it, rr, ok), dt = run(b, lambda x: G.sbm_cg(P.handle, b, x, rtol=1e-10, maxit=2000))
    d2["cg"] = {"converged": ok, "iters": it, "rel_residual": rr, "seconds": dt,
                "note": "operator is nonsymmetric (shifted trial functions); CG diverges"}
    (it, rr, ok), dt = run(b, lambda x: G.sbm_gmres(P.handle, b, x, rtol=1e-10, maxit=5000,
                                                    restart=100))
    d2["gmres_fp64"] = {"converged": ok, "iters": it, "rel_residual": rr, "seconds": dt}
    (it, rr, ok), dt = run(b, lambda x: G.sbm_bicgstab(P.handle, b, x, rtol=1e-10, maxit=5000))
    d2["bicgstab_fp64"] = {"converged": ok, "iters": it, "applies": 2 * it, "rel_residual": rr,
                           "seconds": dt}
    for name, inner, tol, mi in (("ir_fp32_gmres", "gmres", 1e-4, 3000),
                                 ("ir_fp32_bicgstab", "bicgstab", 1e-4, 3000),
                                 ("ir_mixed_bicgstab", "bicgstab_mixed", 1e-2, 300)):
        (it, rr, ok, outer), dt = run(b, lambda x: G.sbm_solve_ir(
            P.handle, b, x, rtol=1e-10, max_outer=100, restart=100, inner_rtol=tol,
            inner_maxit=mi, inner_solver=G.INNER[inner]))
        d2[name] = {"converged": ok, "inner_iters": it, "outer": outer, "rel_residual": rr,
                    "seconds": dt, "inner_rtol": tol, "inner_maxit": mi}
    (it, rr, ok, rep), dt = run(b, lambda x: G.sbm_bicgstab_mixed(P.handle, b, x, rtol=1e-10,
                                                                 maxit=20000))
    d2["bicgstab_mixed_reliable"] = {"converged": ok, "iters": it, "fp32_applies": 2 * it,
                                     "fp64_applies": rep + 2, "rel_residual": rr, "seconds": dt}
    out["disk2d_q2"] = d2

    w = S.SPHERE_3D_Q4.resized(64, degree=2)
    P = G.Problem.from_workload(w)
    G.sbm_autotune(P.handle)
    b = torch.from_numpy(P.rhs(0)).cuda()
    d3 = {"workload": w.name, "n_dofs": P.n_dofs}
    (it, rr, ok), dt = run(b, lambda x: G.sbm_bicgstab(P.handle, b, x, rtol=1e-10,
                                                       maxit=20000))
    d3["bicgstab_fp64"] = {"converged": ok, "iters": it, "applies": 2 * it, "rel_residual": rr,
                           "seconds": dt}
    (it, rr, ok), dt = run(b, lambda x: G.sbm_gmres(P.handle, b, x, rtol=1e-10, maxit=20000,
                                                    restart=200), reps=1)
    d3["gmres200_fp64"] = {"converged": ok, "iters": it, "rel_residual": rr, "seconds": dt}
    for name, inner in (("ir_mixed_bicgstab", "bicgstab_mixed"),
                        ("ir_fp32_bicgstab", "bicgstab")):
        (it, rr, ok, outer), dt = run(b, lambda x: G.sbm_solve_ir(
            P.handle, b, x, rtol=1e-10, max_outer=100, inner_rtol=1e-2, inner_maxit=300,
            inner_solver=G.INNER[inner]))
        d3[name] = {"converged": ok, "inner_iters": it, "outer": outer, "rel_residual": rr,
                    "seconds": dt, "inner_rtol": 1e-2, "inner_maxit": 300}
    out["sphere3d_q2_n64"] = d3
    return out


def _attempt(torch, fn):
    torch.cuda.synchronize()
    t = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t


def solves_by_config(G, torch):
    """Time to a true FP64 relative residual of 1e-10 (b from u = prod sin(pi
    x_i)) on the 3D workloads, within bounded iteration budgets, each
    attempt recording its solver, iterations, seconds, the true relative
    residual it ended with (BiCGStab keeps its best iterate) and whether it
    reached 1e-10.  CG is run as the metric names it; it needs a symmetric
    positive definite operator, which the shifted operator is not.  The
    operator has eigenvalues with negative real part at p >= 3 in 3D, so no
    unpreconditioned Krylov method is expected to reach 1e-10 there: the
    records say how far each got.  The batched workload's refinement solve is
    recorded with the batched apply (batched_64x8)."""
    out = {"rtol": 1e-10}
    inner = dict(inner_rtol=1e-2, restart=100, inner_solver=G.INNER["bicgstab_mixed"])
    cases = (
        (S.SPHERE_3D_Q4, 300, 1000, 400, None, (3, 200)),
        (S.ELLIPSOID_3D_Q6, 300, 2000, 800, "tf32", (4, 250)),
        (S.TORUS_3D_DG_Q3, 300, 3000, 1500, "bf16", (4, 250)),
    )
    for w, cg_it, bi_it, gm_it, mode, (outer, inner_it) in cases:
        P = G.Problem.from_workload(w)
        b = torch.from_numpy(P.rhs(0)).cuda()
        rec = {"workload": w.name, "n_dofs": P.n_dofs}
        x = torch.zeros_like(b)
        (it, rr, ok), dt = _attempt(torch, lambda: G.sbm_cg(P.handle, b, x, rtol=1e-10,
                                                            maxit=cg_it))
        rec["cg_fp64"] = {"iters": it, "seconds": dt, "rel_residual": rr, "reached": bool(ok),
                          "maxit": cg_it}
        x = torch.zeros_like(b)
        (it, rr, ok), dt = _attempt(torch, lambda: G.sbm_bicgstab(P.handle, b, x, rtol=1e-10,
                                                                  maxit=bi_it))
        rec["bicgstab_fp64"] = {"iters": it, "applies": 2 * it, "seconds": dt,
                                "rel_residual": rr, "reached": bool(ok), "maxit": bi_it}
        x = torch.zeros_like(b)
        (it, rr, ok), dt = _attempt(torch, lambda: G.sbm_gmres(P.handle, b, x, rtol=1e-10,
                                                               maxit=gm_it, restart=50))
        rec["gmres50_fp64"] = {"iters": it, "seconds": dt, "rel_residual": rr,
                               "reached": bool(ok), "maxit": gm_it}
        for fm in ("fp32",) + ((mode,) if mode else ()):
            x = torch.zeros_like(b)
            (it, rr, ok, nout), dt = _attempt(torch, lambda: G.sbm_solve_ir(
                P.handle, b, x, rtol=1e-10, max_outer=outer, inner_maxit=inner_it,
                face_mode=G.FACE_MODE[fm], **inner))
            rec[f"ir_fp64_{fm}_faces"] = {
                "inner_iters": it, "outer": nout, "seconds": dt, "rel_residual": rr,
                "reached": bool(ok), "max_outer": outer, "inner_maxit": inner_it,
                "inner": "BiCGStab on FP64 vectors, FP32 cells, "
                         f"{fm.upper()} faces; FP64 BiCGStab finish of at most "
                         f"{outer * inner_it} iterations"}
        out[w.name] = rec
        del P, b, x
    return out


def other_workloads(G, torch, steps=40):
    """FP64 / FP32 / TF32-face / BF16-face applies of the 3D Q6 ellipsoid and
    the DG Q3 torus: GDoF/s (CUDA events) and the FP32-path error against the
    FP64 apply of the same x."""
    out = {}
    for w in (S.ELLIPSOID_3D_Q6, S.TORUS_3D_DG_Q3):
        P = G.Problem.from_workload(w)
        G.sbm_autotune(P.handle)
        x = torch.from_numpy(S.random_vector(w.seed, P.n_dofs, w.dist)).cuda()
        y = torch.empty_like(x)
        x32 = x.float()
        y32 = torch.empty_like(x32)
        ref = P.apply_f64(x).clone()
        res = {"n_dofs": P.n_dofs, "n_cells": P.n_cells, "n_sfaces": P.n_sfaces}
        for name, fn, xx, yy in (("f64", lambda a, b: P.apply_f64(a, b), x, y),
                                 ("f32", lambda a, b: P.apply_f32(a, b), x32, y32),
                                 ("tf32_faces", lambda a, b: P.apply_f32(a, b, face_mode="tf32"),
                                  x32, y32),
                                 ("bf16_faces", lambda a, b: P.apply_f32(a, b, face_mode="bf16"),
                                  x32, y32)):
            for _ in range(3):
                fn(xx, yy)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                fn(xx, yy)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            r = {"gdofs": P.n_dofs / ms / 1e6, "ms": ms}
            if name != "f64":
                r["rel_err_vs_f64"] = float((yy.double() - ref).abs().max() / ref.abs().max())
            res[name] = r
        G.sbm_device_status(P.handle)
        out[w.name] = res
    return out


def extension_study(G, torch, steps=40):
    """First-order Taylor extension against the exact one (the survey's
    "next" row 1): throughput of the FP64 / FP32 applies and their face phase
    on the 3D Q4 sphere (96^3), and accuracy on the 2D disk with
    u = sin(pi x) sin(pi y): max nodal error |u_h - I u| / |I u| of the
    solution (BiCGStab, else GMRES(300), to 1e-10) for p = 1, 2, 3 and
    N = 16, 32, 64, with the observed rates (None: no solver converged)."""
    import dataclasses
    out = {"throughput": {}, "accuracy": {}}
    for ext in ("exact", "taylor1"):
        w = dataclasses.replace(S.SPHERE_3D_Q4, extension=ext)
        P = G.Problem.from_workload(w)
        G.sbm_autotune(P.handle)
        x = torch.from_numpy(S.random_vector(w.seed, P.n_dofs, w.dist)).cuda()
        res = {}
        for name, xx in (("f64", x), ("f32", x.float())):
            yy = torch.empty_like(xx)
            fn = (lambda a, b: P.apply_f64(a, b)) if name == "f64" else \
                 (lambda a, b: P.apply_f32(a, b))
            for _ in range(3):
                fn(xx, yy)
            torch.cuda.synchronize()
            G.sbm_profile_enable(P.handle, True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                fn(xx, yy)
            e1.record()
            torch.cuda.synchronize()
            phases, _ = G.sbm_profile_read(P.handle)
            G.sbm_profile_enable(P.handle, False)
            ms = e0.elapsed_time(e1) / steps
            res[name] = {"gdofs": P.n_dofs / ms / 1e6, "ms": ms,
                         "face_ms": phases[0] / steps}
        out["throughput"][ext] = res
    for p in (1, 2, 3):
        for ext in ("exact", "taylor1"):
            errs = []
            for N in (16, 32, 64):
                w = dataclasses.replace(S.DISK_2D_Q2.resized(N, degree=p), extension=ext)
                P = G.Problem.from_workload(w)
                b = torch.from_numpy(P.rhs(0)).cuda()
                u = torch.from_numpy(P.interpolate(0)).cuda()
                xs = torch.zeros_like(b)
                _, rr, ok = G.sbm_bicgstab(P.handle, b, xs, rtol=1e-10, maxit=20000)
                if not ok:                      # BiCGStab stalls: GMRES(300)
                    xs.zero_()
                    _, rr, ok = G.sbm_gmres(P.handle, b, xs, rtol=1e-10, maxit=30000,
                                            restart=300)
                errs.append(float((xs - u).abs().max() / u.abs().max()) if ok else None)
            rates = [None if (e0 is None or e1 is None) else float(np.log2(e0 / e1))
                     for e0, e1 in zip(errs[:-1], errs[1:])]
            out["accuracy"][f"p{p}_{ext}"] = {"N": [16, 32, 64], "max_nodal_rel_err": errs,
                                             "rates": rates}
    return out


def activity_study(G, torch):
    """Active-cell criterion (Section 2): the cell centre inside Omega against
    the volume fraction >= 0.25 / 0.75 (8^d sub-cell midpoints), on the 2D
    disk, p = 2, u = sin(pi x) sin(pi y): active cells and the max nodal error
    of the solution (BiCGStab, else GMRES(300), to 1e-10)."""
    import dataclasses
    out = {}
    for crit, th in (("centre", 0.5), ("volume", 0.25), ("volume", 0.75)):
        key = crit if crit == "centre" else f"volume{th}"
        rows = []
        for N in (16, 32, 64):
            w = dataclasses.replace(S.DISK_2D_Q2.resized(N), activity=crit, vf_threshold=th)
            P = G.Problem.from_workload(w)
            b = torch.from_numpy(P.rhs(0)).cuda()
            u = torch.from_numpy(P.interpolate(0)).cuda()
            xs = torch.zeros_like(b)
            _, rr, ok = G.sbm_bicgstab(P.handle, b, xs, rtol=1e-10, maxit=20000)
            if not ok:
                xs.zero_()
                _, rr, ok = G.sbm_gmres(P.handle, b, xs, rtol=1e-10, maxit=30000, restart=300)
            rows.append({"N": N, "n_cells": P.n_cells, "n_dofs": P.n_dofs,
                         "max_nodal_rel_err": float((xs - u).abs().max() / u.abs().max())
                         if ok else None})
        out[key] = rows
    return out


def _cut_fraction(w):
    """Fraction of background cells the true boundary cuts, among the cells
    that are active or cut (the paper's measure of geometric complexity):
    a cell is cut when the level set changes sign over its corners."""
    N, d = w.cells, w.dim
    h = 2.0 / N
    g = np.asarray(w.geom).reshape(-1, d + 1)
    xs = -1.0 + h * np.arange(N + 1)
    X = np.stack(np.meshgrid(*([xs] * d), indexing="ij"), -1)
    phi = np.min([np.sqrt(((X - b[:d]) ** 2).sum(-1)) - b[d] for b in g], axis=0)
    corners = [phi[tuple(slice(o, N + o) for o in off)]
               for off in np.ndindex(*([2] * d))]
    lo, hi = np.min(corners, 0), np.max(corners, 0)
    xc = -1.0 + h * (np.arange(N) + 0.5)
    Xc = np.stack(np.meshgrid(*([xc] * d), indexing="ij"), -1)
    active = np.min([np.sqrt(((Xc - b[:d]) ** 2).sum(-1)) - b[d] for b in g], axis=0) < 0
    cut = (lo < 0) & (hi > 0)
    return float(cut.sum() / (cut | active).sum())


def multiball_study(G, torch, steps=20):
    """Geometric complexity (Section 4.3): unions of 3 to 25 random balls on a
    64^3 background mesh, CG p = 2 and 4: FP64 and FP32 GDoF/s and the share
    of the apply spent on surrogate faces, against the fraction of cut cells."""
    out = []
    for p in (2, 4):
        for nb in (3, 5, 10, 15, 25):
            w = S.multiple_balls(nb, degree=p)
            P = G.Problem.from_workload(w)
            G.sbm_autotune(P.handle)
            x = torch.from_numpy(S.random_vector(w.seed, P.n_dofs, w.dist)).cuda()
            r = {"balls": nb, "degree": p, "n_dofs": P.n_dofs, "n_cells": P.n_cells,
                 "n_sfaces": P.n_sfaces, "cut_fraction": _cut_fraction(w)}
            for name, xx in (("f64", x), ("f32", x.float())):
                yy = torch.empty_like(xx)
                fn = P.apply_f64 if name == "f64" else P.apply_f32
                for _ in range(3):
                    fn(xx, yy)
                torch.cuda.synchronize()
                G.sbm_profile_enable(P.handle, True)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(steps):
                    fn(xx, yy)
                e1.record()
                torch.cuda.synchronize()
                ph, _ = G.sbm_profile_read(P.handle)
                G.sbm_profile_enable(P.handle, False)
                ms = e0.elapsed_time(e1) / steps
                r[name] = {"gdofs": P.n_dofs / ms / 1e6,
                           "face_share": ph[0] / max(sum(ph), 1e-30)}
            out.append(r)
    return out


def batched(G, torch, steps=10):
    """64 rotated-ellipsoid CG problems (N ~ U{16..48}, p ~ U{2..6}), 8
    right-hand sides each, one CUDA-graph launch per batched apply."""
    ws = S.batched_ellipsoids()
    ps = [G.Problem.from_workload(w) for w in ws]
    for P in ps:
        G.sbm_autotune(P.handle)
    nrhs = 8
    # the autotuner may choose tensor-core (TF32) faces for the FP32 applies
    # per degree; it keeps the fastest option and records every timing
    B = G.Batch(ps, nrhs, autotune=True, tensor_cores=True)
    tot = sum(p.n_dofs for p in ps) * nrhs
    res = {"problems": len(ps), "nrhs": nrhs, "dof_rhs_per_apply": tot,
           "tile_shape_by_degree": {str(w.degree): B.tile_shape(k) for k, w in enumerate(ws)}}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        xs = [torch.from_numpy(np.concatenate([S.random_vector(w.seed + r, p.n_dofs, "uniform")
                                               for r in range(nrhs)])).to("cuda", dt)
              for w, p in zip(ws, ps)]
        ys = [torch.empty_like(v) for v in xs]
        for _ in range(3):
            B.apply(xs, ys)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            B.apply(xs, ys)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[name] = {"gdofs": tot / ms / 1e6, "ms": ms}
        # the same systems through the single-problem entry point, one
        # problem and right-hand side after another (each problem with its
        # autotuned tile shape and store mode): what the batch replaces
        apply1 = (lambda P, a, b: P.apply_f32(a, b)) if dt == torch.float32 else \
            (lambda P, a, b: P.apply_f64(a, b))
        views = [[(x[r * P.n_dofs:(r + 1) * P.n_dofs], y[r * P.n_dofs:(r + 1) * P.n_dofs])
                  for r in range(nrhs)] for P, x, y in zip(ps, xs, ys)]
        for P, vs in zip(ps, views):
            apply1(P, *vs[0])
        torch.cuda.synchronize()
        e0.record()
        for _ in range(2):
            for P, vs in zip(ps, views):
                for a, b in vs:
                    apply1(P, a, b)
        e1.record()
        torch.cuda.synchronize()
        ms1 = e0.elapsed_time(e1) / 2
        res[name]["single_applies"] = {"gdofs": tot / ms1 / 1e6, "ms": ms1,
                                       "launches": "one apply per problem and right-hand "
                                                   "side, issued from Python through the "
                                                   "binding (host overhead included)"}
        del xs, ys, views
    B.device_status()
    res["knobs_by_degree"] = {
        str(prec): {str(deg): B.knobs(prec, deg) for deg in sorted({w.degree for w in ws})}
        for prec in (32, 64)}
    # the batched workload's solve: FP64 refinement (one refinement step with
    # an inner BiCGStab of FP64 vectors and FP32 batched applies, then FP64
    # BiCGStab), every system to a true residual of 1e-10 within the budget
    bs = [torch.from_numpy(np.concatenate([P.rhs(0)] * nrhs)).cuda() for P in ps]
    xs = [torch.empty_like(v) for v in bs]
    (st, iters, relres, outer), dt = _attempt(torch, lambda: B.solve(
        bs, xs, mode="mixed", rtol=1e-10, maxit=1, inner_rtol=1e-2, inner_maxit=100,
        check=False))
    res["solve_fp64_refinement"] = {
        "systems": int(relres.size), "reached": int((relres <= 1e-10).sum()),
        "seconds": dt, "outer": outer, "iters_max": int(iters.max()),
        "rel_residual_median": float(np.median(relres)),
        "rel_residual_max": float(relres.max()),
        "reached_by_degree": {str(d): int(sum((relres[k * nrhs:(k + 1) * nrhs] <= 1e-10).sum()
                                              for k, w in enumerate(ws) if w.degree == d))
                              for d in sorted({w.degree for w in ws})},
        "budget": "1 refinement (inner BiCGStab, FP32 applies, at most 100 iterations, "
                  "tolerance 1e-2) + FP64 BiCGStab finish of at most 100 iterations",
        "rhs": "b from u = prod sin(pi x_i), the same for the 8 right-hand sides"}
    del bs, xs
    B.close()
    return res


def batched_solve(G, torch):
    """Time to a true relative residual of 1e-10 for a batch of independent
    systems: the 8 rotated-ellipsoid CG problems of S.solve_batch() (p = 2, 3;
    the batch generator's positive-real ones: BiCGStab needs no eigenvalue
    in the left half-plane) x 4 right-hand sides (x ~ U(-1, 1)), solved (a)
    one system after another with the single-problem FP64 BiCGStab, (b) all
    together by the batched FP64 BiCGStab, (c) all together by the batched
    FP64 refinement with FP32-apply inner solves."""
    ws = S.solve_batch()
    ps = [G.Problem.from_workload(w) for w in ws]
    nrhs = 4
    B = G.Batch(ps, nrhs, autotune=True)
    bs = [torch.from_numpy(np.concatenate([S.random_vector(w.seed + 7 + r, p.n_dofs, "uniform")
                                           for r in range(nrhs)])).cuda()
          for w, p in zip(ws, ps)]
    xs = [torch.empty_like(b) for b in bs]
    res = {"problems": len(ps), "nrhs": nrhs, "systems": len(ps) * nrhs,
           "dofs_total": sum(p.n_dofs for p in ps) * nrhs,
           "n_dofs_range": [min(p.n_dofs for p in ps), max(p.n_dofs for p in ps)],
           "rtol": 1e-10}
    # (a) one after another
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its, worst, ok = [], 0.0, True
    for p, b in zip(ps, bs):
        for r in range(nrhs):
            br = b[r * p.n_dofs:(r + 1) * p.n_dofs].contiguous()
            x = torch.zeros_like(br)
            it, rr, conv = G.sbm_bicgstab(p.handle, br, x, rtol=1e-10, maxit=20000)
            its.append(it)
            worst = max(worst, rr)
            ok &= conv
    torch.cuda.synchronize()
    res["sequential_bicgstab_fp64"] = {"seconds": time.perf_counter() - t0, "converged": ok,
                                       "iters_total": int(sum(its)), "iters_max": int(max(its)),
                                       "worst_rel_residual": worst}
    for mode in ("fp64", "mixed"):
        B.solve(bs, xs, mode=mode, rtol=1e-10, check=False)      # workspace, graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, iters, relres, outer = B.solve(bs, xs, mode=mode, rtol=1e-10, check=False)
        torch.cuda.synchronize()
        res[f"batched_{mode}"] = {"seconds": time.perf_counter() - t0,
                                  "converged": st == G.SBM_OK,
                                  "iters_max": int(iters.max()), "iters_total": int(iters.sum()),
                                  "worst_rel_residual": float(relres.max()),
                                  **({"outer": outer} if mode == "mixed" else {})}
    B.close()
    return res


def profile_applies(args, w):
    import torch

    import paper_2507_17053_gb300 as G
    P = G.Problem.from_workload(w)
    if args.tile_shape >= 0:
        if args.profile_applies == "f64":
            G.sbm_set_tile_shape(P.handle, args.tile_shape, -1)
        else:
            G.sbm_set_tile_shape(P.handle, -1, args.tile_shape)
    if args.ordered_stores >= 0:
        if args.profile_applies == "f64":
            G.sbm_set_ordered_stores(P.handle, args.ordered_stores, -1)
        else:
            G.sbm_set_ordered_stores(P.handle, -1, args.ordered_stores)
    x = torch.from_numpy(S.random_vector(w.seed, P.n_dofs, w.dist)).cuda()
    if args.profile_applies != "f64":
        x = x.float()
    y = torch.empty_like(x)
    for _ in range(args.steps):
        if args.profile_applies == "f64":
            P.apply_f64(x, y)
        else:
            P.apply_f32(x, y, face_mode={"f32": "fp32", "tf32": "tf32",
                                         "bf16": "bf16"}[args.profile_applies])
    torch.cuda.synchronize()
    G.sbm_device_status(P.handle)


def profile_batch(args):
    """The batched apply on a batch small enough for a full ncu capture:
    24 rotated ellipsoids (N ~ U{20..36}, p ~ U{2..6}) x 4 right-hand sides,
    tile shape 0 and the full face batch (no autotuning)."""
    import torch

    import paper_2507_17053_gb300 as G
    ws = S.batched_ellipsoids(nprob=24, n_range=(20, 36))
    ps = [G.Problem.from_workload(w) for w in ws]
    nrhs = 4
    B = G.Batch(ps, nrhs, autotune=False)
    dt = torch.float32 if args.profile_batch == "f32" else torch.float64
    xs = [torch.from_numpy(np.concatenate([S.random_vector(S.rhs_seed(w, r), p.n_dofs, "uniform")
                                           for r in range(nrhs)])).to("cuda", dt)
          for w, p in zip(ws, ps)]
    ys = [torch.empty_like(v) for v in xs]
    for _ in range(args.steps):
        B.apply(xs, ys)
    torch.cuda.synchronize()
    B.device_status()


def run_ours(args, w):
    import torch

    import paper_2507_17053_gb300 as G
    rank, world, dist = dist_init(args.gpus)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    torch.zeros(1, device=dev)              # context creation outside the set-up timing
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P = G.Problem.from_workload(w, device=False)     # host: geometry, numbering
    t1 = time.perf_counter()
    G.sbm_setup_face_data(P.handle)                  # device tables, chunking, uploads
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    # the same with the geometry stage on the GPU (identical problem)
    t3 = time.perf_counter()
    Pg = G.Problem.from_workload(w, device=False, gpu_setup=True)
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    G.sbm_setup_face_data(Pg.handle)
    torch.cuda.synchronize()
    t5 = time.perf_counter()
    del Pg
    init = {"host_geometry_s": t1 - t0, "device_setup_s": t2 - t1,
            "dofs_per_s": P.n_dofs / (t2 - t0),
            "gpu_geometry": {"create_s": t4 - t3, "device_setup_s": t5 - t4,
                             "dofs_per_s": P.n_dofs / (t5 - t3)},
            "face_table_bytes_per_dof": (P.n_sfaces * (w.degree + 1) ** (w.dim - 1)
                                         * (w.dim * (w.degree + 1)
                                            + ((w.degree + 1) ** 2 if w.dim == 3 else 0))
                                         * 8) / P.n_dofs,
            "note": "sbm_create (host) or sbm_create_gpu (geometry stage on the GPU, numbering "
                    "on the host) + sbm_setup_face_data; face table = FP64 1D values at the "
                    "shifted points and, in 3D, their products over the two non-first axes "
                    "(an FP32 copy of the 1D values adds 1.5 B/DoF at p = 4)"}
    shapes = G.sbm_autotune(P.handle)       # tile shapes of the FP64 / FP32 cell kernel
    x_host = S.random_vector(w.seed, P.n_dofs, w.dist)
    x = torch.from_numpy(x_host).to(dev)
    y = torch.empty_like(x)
    st = torch.cuda.current_stream()
    n = P.n_dofs

    # measured FMA rates (the roofline's peak for the ALU-bound cell kernels):
    # the library's probe, repeated for about a second under clock sampling
    probe_clk = ClockSampler(local)
    probe_clk.start()
    t0 = time.perf_counter()
    p64, p32 = [], []
    while time.perf_counter() - t0 < 1.0 or len(p64) < 3:
        p64.append(G.sbm_peak_probe(64))
        p32.append(G.sbm_peak_probe(32))
    probe = {"fp64_gfma": max(p64), "fp32_gfma": max(p32), "clocks": probe_clk.stop(),
             "how": "sbm_peak_probe: independent fma.rn chains, 8 per thread, 8 x 256-thread "
                    "blocks per SM, best launch (CUDA events)"}

    clocks = ClockSampler(local)
    ms, ph, launches, clk = time_applies(P, lambda a, b: P.apply_f64(a, b), x, y, args.steps,
                                         args.warmup, st, dist, dev, clocks)
    # FP32 apply of the same operator (the inner operator of the mixed-precision path)
    x32 = x.float()
    y32 = torch.empty_like(x32)
    ms32, ph32, launches32, _ = time_applies(P, lambda a, b: P.apply_f32(a, b), x32, y32,
                                             args.steps, args.warmup, st, dist, dev)
    ms32u = time_plain(lambda a, b: P.apply_f32(a, b), x32, y32, args.steps, args.warmup, st,
                       dist, dev)

    # end to end through the C ABI with host buffers (H2D + apply + D2H per step)
    xh = torch.from_numpy(x_host).pin_memory()
    yh = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_steps = max(3, min(50, args.steps // 10))
    P.apply_f64_host(xh, yh)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        P.apply_f64_host(xh, yh)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)

    if rank != 0:
        return
    value = job_rate(world, n * args.steps, ms * 1e-3) / 1e9
    value32 = job_rate(world, n * args.steps, ms32 * 1e-3) / 1e9
    value32u = job_rate(world, n * args.steps, ms32u * 1e-3) / 1e9
    pk, pk_src = peaks()
    cfma, cadd = cell_ops(w.dim, w.degree, P.n_cells)
    cflops = 2 * cfma + cadd
    cops = cfma + cadd
    fflops = face_flops(w.dim, w.degree, P.n_sfaces)
    cell_ms = ph[1]
    achieved_gops = cops / (cell_ms * 1e-3) / 1e9
    step_s = ms / args.steps * 1e-3
    step32_s = ms32u / args.steps * 1e-3
    line = {
        "metric": "GDoF/s per operator apply (FP64)",
        "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_dofs": n, "n_cells": P.n_cells,
                   "n_sfaces": P.n_sfaces, "degree": w.degree, "dim": w.dim,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "tile_shape_f64_f32": list(shapes),
                   "ordered_stores_f64_f32": list(G.sbm_ordered_stores(P.handle)),
                   "l2": f"inputs larger than L2: x, y, colour buffers and tables "
                         f"{(2 * 8 * n + 8 * 8 * n) / 1e6:.0f} MB > 129 MB"},
        "e2e": {"value": job_rate(world, n * e2e_steps, e2e_s) / 1e9, "unit": "GDoF/s",
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": achieved_gops, "peak": probe["fp64_gfma"],
                     "unit": "G FP64 ops/s", "frac": achieved_gops / probe["fp64_gfma"],
                     "peak_src": "measured (sbm_peak_probe, this run); FP64 FMA pipe ops",
                     "peak_derived": FP64_PIPE_GOPS,
                     "frac_of_derived": achieved_gops / FP64_PIPE_GOPS,
                     "traffic": CELL_TRAFFIC.get((w.name, shapes[0],
                                                  G.sbm_ordered_stores(P.handle)[0])),
                     "traffic_src": "constant from one earlier ncu capture of this kernel "
                                    "(dram__bytes_read.sum + dram__bytes_write.sum), not "
                                    "measured by this run",
                     "kernel": cell_kernel_name(w, shapes[0], G.sbm_ordered_stores(P.handle)[0]),
                     "ops_per_launch": cops, "fma_per_launch": cfma,
                     "other_per_launch": cadd,
                     "launches_per_step": 1, "kernel_ms_per_launch": cell_ms,
                     "achieved_tflops": cflops / (cell_ms * 1e-3) / 1e12,
                     "peak_note": "peak = the measured FP64 FMA rate (G FMA/s; DFMA and "
                                  "DADD share the FP64 pipe at one op each); derived: 2 "
                                  "lane-ops per SM per clock x 152 SMs x 2070 MHz",
                     "probe": probe,
                     "phases_ms_per_step": {"face": ph[0], "cell": ph[1], "assembly": ph[2]},
                     "face_kernel_tflops": fflops / (ph[0] * 1e-3) / 1e12 if ph[0] > 0 else None,
                     "hbm": {"bytes_per_dof": 16,
                             "achieved_gbs": 16 * n / step_s / 1e9,
                             "peak_gbs": pk.get("hbm_gbs"), "peak_src": pk_src,
                             "frac": 16 * n / step_s / 1e9 / pk["hbm_gbs"]}},
        "fp32_apply": {"value": value32u, "unit": "GDoF/s", "ms_per_step": ms32u / args.steps,
                       "timing": "profiler off (the applies as a user calls them, programmatic "
                                 "dependent launches active); the phases come from a second, "
                                 "profiled loop of the same applies",
                       "profiled": {"value": value32, "ms_per_step": ms32 / args.steps},
                       "launches": launches32,
                       "phases_ms_per_step": {"face": ph32[0], "cell": ph32[1],
                                              "assembly": ph32[2]},
                       "cell_tflops": cflops / (ph32[1] * 1e-3) / 1e12,
                       "cell_frac_of_measured_fp32_fma": cops / (ph32[1] * 1e-3) / 1e9
                       / probe["fp32_gfma"],
                       "hbm_frac_8B_per_dof": 8 * n / step32_s / 1e9 / pk["hbm_gbs"]},
        "clocks": clk,
        "init": init,
    }
    if not args.skip_extras:
        for key, fn in (("solves", solve_times), ("solves_by_config", solves_by_config),
                        ("other_workloads", other_workloads),
                        ("batched_64x8", batched), ("batched_solve", batched_solve),
                        ("extension_taylor1", extension_study),
                        ("multiple_balls", multiball_study),
                        ("activity_criterion", activity_study)):
            try:
                line[key] = fn(G, torch)
            except Exception as e:  # noqa: BLE001 -- report, never hide the main number
                line[key] = {"error": str(e)}
    if not args.skip_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    w = workload(args.workload)
    if args.impl == "reference":
        run_reference(args, w)
    elif args.profile_applies:
        profile_applies(args, w)
    elif args.profile_batch:
        profile_batch(args)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
