#!/usr/bin/env python
"""Benchmark of the Lippmann-Schwinger Nystrom hot path on one B300.

A step is one full left-preconditioned FP64 GMRES solve (tol 1e-8) of the
two-material disk (off-centre inclusion; n_opt = 1.5 + 0.2 exp(-|x|^2/0.1)
outside, 2.2 inside), k = 20, 2,680 curved triangles x 15 nodes = 40,200 nodes,
Cartesian preconditioner on 256^2 over [-1.2, 1.2]^2, one plane wave at pi/4,
plus its far-field pattern at 64 angles.  Setup (correction and preconditioner
factors) is excluded, as the paper excludes it from its solve times.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line.  Under torchrun every rank solves its own incident
direction (independent replicas, no collective); value = all solves / max time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "two-material disk, k=20, 40,200 nodes (2,680 curved P4 triangles), 256^2 Cartesian preconditioner, tol 1e-8"
METRIC = "LS GMRES solves/s (FP64, preconditioned)"
# Preconditioned GMRES iterations of this workload as measured by the GPU arm;
# the reference arm scales its sampled matvec cost by it.
REFERENCE_ITERS = 8


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def rank_direction(rank, world, base=np.pi / 4):
    """Incident angle of rank `rank`: independent replicas, one direction each."""
    return base + 2 * np.pi * rank / world if world > 1 else base


def max_over_ranks(total_ms, dist=None, device="cpu"):
    """Max of the per-rank timed totals (the whole job ends with the slowest rank)."""
    if dist is None:
        return float(total_ms)
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world, steps, max_total_ms):
    """Whole-job throughput: all solves of all ranks over the slowest rank's time."""
    return world * steps / (max_total_ms * 1e-3)


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clocks, throttle reasons)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _oracle_rows_job(job):
    """Worker of the CPU baseline (spawned process): the oracle's pair-sum rows and
    correction rows of one slice of the sample, with their wall times."""
    import numpy as np
    from lsinput.workloads import two_material
    from oracle.nystrom import naive_rows
    from oracle.vdim import correction_matrix
    level, f, ps_rows, corr_rows = job
    wl = two_material(level)
    t0 = time.perf_counter()
    nv = naive_rows(wl.mesh.nodes, wl.mesh.weights, wl.k, f, ps_rows) if len(ps_rows) else np.zeros(0, complex)
    t1 = time.perf_counter()
    dV = correction_matrix(wl.mesh, wl.k, 3.0, rows=corr_rows) if len(corr_rows) else None
    t2 = time.perf_counter()
    return nv, (dV @ f if dV is not None else np.zeros(0, complex)), t1 - t0, t2 - t1


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(wl, u_gpu, Lu_gpu, iters, budget_s=24.0):
    """The oracle as it stands, timed on the host's cores (one spawned process per core,
    each with single-threaded BLAS) on a bounded sample of the same workload: a slice of
    pair-sum rows and of correction rows per process, sized from a short calibration so
    that the whole sample takes about budget_s, plus one apply of the oracle's
    preconditioner (SuperLU solve on the 256^2 grid; its assembly is setup).  The sampled
    rows also give the GPU matvec's error against the oracle.  Solves/s = 1 / (iters x
    (extrapolated L apply + P apply))."""
    import multiprocessing as mp
    from oracle.precond import Grid, Preconditioner
    os.environ["OPENBLAS_NUM_THREADS"] = "1"          # inherited by the spawned workers
    os.environ["OMP_NUM_THREADS"] = "1"
    cores = _host_cores()
    n = wl.mesh.n_nodes
    f = wl.m * u_gpu
    rng = np.random.default_rng(0)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        # calibration: 64 pair-sum rows and 4 correction rows per process
        cal = pool.map(_oracle_rows_job, [("small", f, rng.choice(n, 64, replace=False), rng.choice(n, 4, replace=False))
                                          for _ in range(cores)])
        t_row_ps = np.median([c[2] for c in cal]) / 64
        t_row_corr = np.median([c[3] for c in cal]) / 4
        n_ps = max(64, int(0.5 * budget_s / t_row_ps))
        n_corr = max(4, int(0.5 * budget_s / t_row_corr))
        perm = rng.permutation(n)
        jobs = []
        for c in range(cores):
            ps = perm[(c * n_ps) % n:(c * n_ps) % n + n_ps]
            jobs.append(("small", f, np.sort(ps), np.sort(ps[:n_corr])))   # correction rows among the pair-sum rows
        w0 = time.perf_counter()
        res = pool.map(_oracle_rows_job, jobs)
        wall = time.perf_counter() - w0
    rows_ps = sum(len(j[2]) for j in jobs)
    rows_corr = sum(len(j[3]) for j in jobs)
    t_ps = sum(r[2] for r in res) / rows_ps            # core-seconds per row
    t_corr = sum(r[3] for r in res) / rows_corr
    t_apply = (t_ps + t_corr) * n / cores              # all cores, one full L apply
    # matvec error on the first job's rows that carry both parts
    job0, r0 = jobs[0], res[0]
    common = np.intersect1d(job0[2], job0[3])
    err = None
    if common.size:
        a = np.searchsorted(job0[2], common)
        b = np.searchsorted(job0[3], common)
        ref = u_gpu[common] + wl.k**2 * (r0[0][a] + r0[1][b])
        err = float(np.linalg.norm(Lu_gpu[common] - ref) / np.linalg.norm(ref))
    P = Preconditioner(Grid(wl.box, wl.nx, wl.ny), wl.mesh.nodes, wl.k, wl.m_grid)
    tp0 = time.perf_counter()
    P.apply(u_gpu)
    t_P = time.perf_counter() - tp0
    t_solve = iters * (t_apply + t_P)
    return {
        "value": 1.0 / t_solve, "unit": "solves/s", "cores": cores, "kind": "oracle",
        "sample": f"{rows_ps} pair-sum rows x {n} sources and {rows_corr} correction rows over {cores} processes "
                  f"({wall:.1f} s wall), extrapolated to {n} rows per L apply, plus one timed P apply, "
                  f"x {iters} iterations",
        "seconds": round(wall + t_P, 2), "pairs_per_s": rows_ps * (n - 1) / (t_ps * rows_ps) * cores,
        "t_apply_s": t_apply, "t_precond_s": t_P,
    }, err


def reference_arm(args):
    """--impl reference: the oracle as it stands, each step a bounded sample."""
    from lsinput.workloads import two_material
    from oracle.nystrom import naive_rows
    from oracle.vdim import correction_matrix

    wl = two_material("small")
    n = wl.mesh.n_nodes
    x = np.exp(1j * wl.k * (wl.mesh.nodes @ np.array([np.cos(np.pi / 4), np.sin(np.pi / 4)])))
    f = wl.m * x
    rows = np.arange(0, n, n // 256)[:256]
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        naive_rows(wl.mesh.nodes, wl.mesh.weights, wl.k, f, rows)
        t1 = time.perf_counter()
        correction_matrix(wl.mesh, wl.k, 3.0, rows=rows[:8])
        t2 = time.perf_counter()
        if s >= args.warmup:
            times.append(((t1 - t0) / rows.size + (t2 - t1) / 8) * n * REFERENCE_ITERS)
    t_solve = statistics.mean(times)
    value = 1.0 / t_solve
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_solve * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"per step: 256 pair-sum rows + 8 correction rows of one L apply, "
                                       f"extrapolated to {n} rows x {REFERENCE_ITERS} iterations"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def precision_report(args):
    """--workload precision: the precision form on its own configuration (two-material
    disk at k = 40, 13,042 triangles = 195,630 nodes, 512^2 preconditioner): one FP32
    solve and one FP64-accurate double-float solve (the reference for the error),
    both timed with CUDA events, plus the FP32 matvec against the FP64 oracle on
    sampled rows.  One JSON line; not part of the default run."""
    import torch
    import paper_2608_17615_b300 as L
    from lsinput.workloads import two_material

    torch.cuda.set_device(0)
    wl = two_material("medium", k=40.0, nx=512, ny=512)
    n = wl.mesh.n_nodes
    t0 = time.perf_counter()
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=wl.nx, ny=wl.ny, tol=1e-8, pairsum=2)
    setup_s = time.perf_counter() - t0
    d = np.array([np.cos(np.pi / 4), np.sin(np.pi / 4)])
    b = torch.from_numpy(np.exp(1j * wl.k * (wl.mesh.nodes @ d))).cuda().view(1, -1)
    out = {}
    sols = {}
    for mode, name in ((2, "fp32"), (3, "double_float")):
        op.set_pairsum(mode)
        u = torch.empty_like(b)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it, st = op.solve_dev(b, u)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        sols[name] = u
        out[name] = {"solve_ms": ms, "solves_per_s": 1e3 / ms, "iterations": int(it[0]), "status": int(st),
                     "pairs_per_s": int(it[0]) * n * (n - 1) / (ms * 1e-3)}
        print(f"[precision] setup {setup_s:.1f} s; {name}: {json.dumps(out[name])}", file=sys.stderr, flush=True)
    out["fp32"]["rel_err_vs_double_float_solution"] = (
        torch.linalg.norm(sols["fp32"] - sols["double_float"]) / torch.linalg.norm(sols["double_float"])).item()
    # FP32 matvec against the oracle on sampled rows
    from oracle.operator import Operator as OracleOp
    op.set_pairsum(2)
    x = np.exp(1j * np.arange(n) * 0.37)
    y = torch.empty(n, dtype=torch.complex128, device="cuda")
    op.apply_dev(torch.from_numpy(x).cuda(), y)
    rows = np.arange(0, n, n // 24)[:24]
    ref = OracleOp(wl.mesh, wl.k, wl.m, rows_only=True).apply_rows(x, rows)
    yv = y.cpu().numpy()[rows]
    out["fp32"]["matvec_rel_err_vs_oracle"] = float(np.linalg.norm(yv - ref) / np.linalg.norm(ref))
    line = {"report": "precision form", "config": {"workload": "two-material disk, k=40, 195,630 nodes "
            "(13,042 curved P4 triangles), 512^2 Cartesian preconditioner, tol 1e-8", "nodes": n},
            "setup_s": setup_s, "setup_parts_s": dict(zip(["correction", "grid", "block_lu", "table"],
                                                         [round(float(t), 3) for t in op.setup_times()])),
            "forms": out}
    print(json.dumps(line), flush=True)


def batched_pairsum_report(args):
    """--workload batched: the batched pair sum alone (two-material disk, k = 20, 40,200 nodes,
    64 right-hand sides), tensor-core GEMM (k_pairsum_tc) against the CUDA-core kernel
    (k_pairsum_multi_f32), each timed with CUDA events over --steps launches after
    --warmup, with its error against the FP64 pair sum on 4 sampled right-hand sides.
    Also the launch to profile the tensor-core kernel.  One JSON line."""
    import torch
    import paper_2608_17615_b300 as L
    from lsinput.workloads import random_density, two_material

    torch.cuda.set_device(0)
    wl = two_material("small")
    n = wl.mesh.n_nodes
    R = 64
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, use_precond=0)
    F = torch.from_numpy(np.stack([random_density(n, 900 + r) for r in range(R)])).cuda()
    Y = torch.empty_like(F)
    sample = (0, 21, 42, 63)
    ref = {}
    for r in sample:
        y1 = torch.empty_like(F[r])
        op.pairsum_dev(F[r].contiguous(), y1)
        ref[r] = y1
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")))
    except OSError:
        pass
    tf32_peak = peaks.get("bf16_tflops", 1800.0) * (1.1 / 2.25)
    out = {}
    for kind, name in ((1, "tensor_cores"), (0, "cuda_cores")):
        op.set_batch_kernel(kind, 4)
        for _ in range(max(1, args.warmup)):
            op.pairsum_batch_dev(F, Y)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            op.pairsum_batch_dev(F, Y)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        err = max((torch.linalg.norm(Y[r] - ref[r]) / torch.linalg.norm(ref[r])).item() for r in sample)
        pairs = R * n * (n - 1)
        out[name] = {"ms_per_launch_incl_epilogue": ms, "pair_rhs_interactions_per_s": pairs / (ms * 1e-3),
                     "rel_err_vs_fp64_max_of_4": err}
        if kind == 1:
            flops = 24.0 * pairs                       # 3 split products x 2 K-slots x 2 columns x 2 flops
            out[name]["tensor_pipe"] = {"executed_tf32_tflops": flops / (ms * 1e-3) / 1e12,
                                        "peak_tf32_tflops": tf32_peak,
                                        "peak_source": "measured bf16 burst x nominal tf32/bf16 ratio 1.1/2.25"}
    line = {"report": "batched pair sum", "config": {"workload": "two-material disk, k=20, 40,200 nodes, "
            "64 right-hand sides, tensor-core run length 4 stages", "nodes": n, "rhs": R},
            "speedup_tensor_vs_cuda_cores": out["cuda_cores"]["ms_per_launch_incl_epilogue"]
            / out["tensor_cores"]["ms_per_launch_incl_epilogue"], "forms": out}
    print(json.dumps(line), flush=True)


BATCH_NODES = (5000, 8000, 14000, 22000, 34000, 50000, 72000, 100000)


def batching_report(args):
    """--workload batching: the batching form's configuration, 8 star-shaped scatterers of
    uneven size (5k-100k nodes, k = 10, 20, 40 in turn, grids at k h_C ~ 0.19), 64 incident
    directions each, all solved in lock step with one persistent pair-sum launch per
    iteration (ls_solve_multi_dev), once on the tensor cores and once on the CUDA cores;
    error of direction 0 of every scatterer against its FP64-accurate double-float solve.
    One JSON line; not part of the default run."""
    import torch
    import paper_2608_17615_b300 as L
    from lsinput.workloads import star_scatterer

    torch.cuda.set_device(0)
    R = 64
    ops, B, wls, setup = [], [], [], 0.0
    for s, nn in enumerate(BATCH_NODES):
        k = (10.0, 20.0, 40.0)[s % 3]
        nx = int(round(2.9 * k / 0.19)) + 1
        wl = star_scatterer(s, nn, k=k, nx=nx, ny=nx, n_dirs=R)
        t0 = time.perf_counter()
        op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, box=wl.box, nx=wl.nx, ny=wl.ny, tol=1e-8,
                        max_iter=100)
        setup += time.perf_counter() - t0
        b = torch.empty((R, wl.mesh.n_nodes), dtype=torch.complex128, device="cuda")
        op.incident_dev(wl.directions, b)
        ops.append(op)
        B.append(b)
        wls.append(wl)
        print(f"[batching] scatterer {s}: {wl.mesh.n_nodes} nodes, k={k}, grid {nx}^2", file=sys.stderr, flush=True)
    n_s = [w.mesh.n_nodes for w in wls]
    out = {}
    sols = {}
    for kind, name in ((1, "tensor_cores"), (0, "cuda_cores")):
        for op in ops:
            op.set_batch_kernel(kind)
        U = [torch.empty_like(b) for b in B]
        L.solve_multi_dev(ops, B, U)                   # warm-up (grid autotune, buffers)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        iters, st = L.solve_multi_dev(ops, B, U)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        it = np.asarray(iters)
        pairs = float(sum(int(it[s].max()) * R * n * (n - 1) for s, n in enumerate(n_s)))
        out[name] = {"ms": ms, "solves_per_s": len(ops) * R / (ms * 1e-3), "status": int(st),
                     "iterations_max_per_scatterer": [int(x.max()) for x in it],
                     "pair_interactions_per_s": pairs / (ms * 1e-3)}
        print(f"[batching] setup {setup:.1f} s; {name}: {json.dumps(out[name])}", file=sys.stderr, flush=True)
        sols[name] = [u[0].clone() for u in U]
    errs = []
    for s, op in enumerate(ops):
        op.set_pairsum(3)
        u1 = torch.empty_like(B[s][0]).view(1, -1)
        op.solve_dev(B[s][0].contiguous().view(1, -1), u1)
        ref = u1[0]
        errs.append({name: (torch.linalg.norm(sols[name][s] - ref) / torch.linalg.norm(ref)).item() for name in sols})
    for name in sols:
        out[name]["rel_err_vs_fp64_accurate_dir0_max"] = max(e[name] for e in errs)
    line = {"report": "batching form", "config": {"workload": "8 star scatterers (r = 1 + 0.2 cos(5 theta + phi)), "
            f"nodes {n_s}, k = 10/20/40, 64 directions each, tol 1e-8", "nodes": n_s, "rhs_per_scatterer": R},
            "setup_s": setup, "forms": out}
    print(json.dumps(line), flush=True)


def gradient_report(args):
    """--workload gradient: the differentiation form's configuration (two-material disk,
    k = 40, 32,830 curved triangles = 492,450 nodes, 512^2 preconditioner): gradient of
    the far-field misfit 1/2 sum |u_inf - t|^2 over 16 incident directions and 32
    receivers with respect to every nodal contrast, the target t made by a forward solve
    with a Gaussian blob added to the index; forward and adjoint solves batched over the
    16 directions.  One gradient after a warm-up, timed with the host clock around the
    synchronised forward + backward.  One JSON line; the finite-difference check of the
    gradient runs in the GPU tests on smaller meshes."""
    import torch
    import paper_2608_17615_b300 as L
    from lsinput.workloads import perturbed_contrast, two_material
    from paper_2608_17615_b300.misfit import far_field_misfit

    torch.cuda.set_device(0)
    wl = two_material("large", k=40.0, nx=512, ny=512)
    n = wl.mesh.n_nodes
    t0 = time.perf_counter()
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=512, ny=512, tol=1e-8)
    setup_s = time.perf_counter() - t0
    print(f"[gradient] setup {setup_s:.1f} s {op.setup_times()}", file=sys.stderr, flush=True)
    dirs = 2 * np.pi * np.arange(16) / 16
    ff = 2 * np.pi * np.arange(32) / 32
    B = torch.empty((16, n), dtype=torch.complex128, device="cuda")
    U = torch.empty_like(B)
    uinf_t = torch.empty((16, 32), dtype=torch.complex128, device="cuda")
    op.set_contrast(perturbed_contrast(wl))
    op.incident_dev(dirs, B)
    t1 = time.perf_counter()
    it_t, st_t = op.solve_batch_dev(B, U, ff, uinf_t)
    torch.cuda.synchronize()
    t_target = time.perf_counter() - t1
    op.set_contrast(wl.m)
    m_t = torch.from_numpy(np.ascontiguousarray(np.real(wl.m), np.float64)).cuda().requires_grad_(True)
    (g,) = torch.autograd.grad(far_field_misfit(m_t, op, dirs, ff, uinf_t, batched=True), m_t)   # warm-up
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    J = far_field_misfit(m_t, op, dirs, ff, uinf_t, batched=True)
    (g,) = torch.autograd.grad(J, m_t)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t2
    line = {"report": "differentiation form", "config": {"workload": "two-material disk, k=40, 492,450 nodes "
            "(32,830 curved P4 triangles), 512^2 Cartesian preconditioner, 16 directions x 32 receivers, "
            "target: +0.05 Gaussian blob at (-0.3, -0.2)", "nodes": n},
            "setup_s": setup_s, "setup_parts_s": dict(zip(["correction", "grid", "block_lu", "table"],
                                                         [round(float(t), 3) for t in op.setup_times()])),
            "target_solve_s": t_target, "target_iterations_max": int(np.max(it_t)),
            "value": 1.0 / dt, "unit": "gradients/s", "seconds": dt, "misfit": float(J.item()),
            "grad_norm": float(torch.linalg.norm(g).item())}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="default", choices=["default", "precision", "batching", "batched",
                                                                 "gradient"])
    args = ap.parse_args()
    rank, world, local = _env_rank()
    if args.workload == "precision":
        if rank == 0:
            precision_report(args)
        return
    if args.workload == "batching":
        if rank == 0:
            batching_report(args)
        return
    if args.workload == "batched":
        if rank == 0:
            batched_pairsum_report(args)
        return
    if args.workload == "gradient":
        if rank == 0:
            gradient_report(args)
        return
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return

    import torch
    import paper_2608_17615_b300 as L
    from lsinput.workloads import two_material

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = two_material("small")
    n = wl.mesh.n_nodes
    t0 = time.perf_counter()
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, tol=1e-8)
    setup_s = time.perf_counter() - t0
    fp64_peak = L.probe_fp64()
    setup_parts = {k: round(float(v), 3) for k, v in zip(["correction", "grid", "block_lu", "table"], op.setup_times())}
    print(f"[bench] setup {setup_s:.1f} s {setup_parts}, FP64 probe {fp64_peak:.1f} GFLOP/s", file=sys.stderr, flush=True)
    # each rank solves its own direction (replicas)
    angle = rank_direction(rank, world)
    d = np.array([np.cos(angle), np.sin(angle)])
    b = torch.from_numpy(np.exp(1j * wl.k * (wl.mesh.nodes @ d))).cuda()
    u = torch.empty_like(b)
    n_ff = wl.ff_angles.size
    uinf = torch.empty(n_ff, dtype=torch.complex128, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 512 MB > 126 MB L2
    for _ in range(args.warmup):
        op.solve_dev(b.view(1, -1), u.view(1, -1), wl.ff_angles, uinf.view(1, -1))
    torch.cuda.synchronize()
    op.set_timing(True)
    stream = torch.cuda.current_stream()
    iters_list, step_ms = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it, st = op.solve_dev(b.view(1, -1), u.view(1, -1), wl.ff_angles, uinf.view(1, -1))
            e1.record(stream)
            iters_list.append(int(it[0]))
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    ps_ms, ps_launches, launches = op.stats()
    print(f"[bench] steps ms {step_ms}, iters {iters_list}, pair-sum {ps_ms:.1f} ms / {ps_launches} launches",
          file=sys.stderr, flush=True)
    op.set_timing(False)
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    iters = statistics.mean(iters_list)
    value = aggregate_value(world, args.steps, total_ms)
    pairs_per_solve = iters * n * (n - 1)
    # roofline of the pair-sum kernel (FP64 ALU bound)
    avg_launch_s = ps_ms / max(ps_launches, 1) * 1e-3
    nc_tab, tune_ms = op.tuning()
    flops_per_pair = flops_per_pair_of(op.params.pairsum, nc_tab)
    achieved = flops_per_pair * n * (n - 1) / avg_launch_s / 1e12
    peak = fp64_peak / 1e3
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": TRAFFIC.get(op.params.pairsum), "kernel": KERNEL[op.params.pairsum],
                "flops_per_pair": flops_per_pair, "table_ncoef": nc_tab, "tuning_ms": list(tune_ms),
                "peak_source": "measured FP64 FMA probe (ls_probe_fp64), same run",
                "kernel_ms_per_launch": avg_launch_s * 1e3, "kernel_share_of_step": ps_ms / total_ms}
    # end to end through the host-buffer entry point
    e2e_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        uh, uinfh, hist, it_h, st_h = op.solve([angle], wl.ff_angles)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = {"value": world * args.steps / (sum(e2e_ms) * 1e-3), "unit": "solves/s",
           "h2d_bytes_per_step": 8 * (1 + n_ff), "d2h_bytes_per_step": 16 * n + 16 * n_ff + 8 * (int(it_h[0]) + 1)}
    # precision form on the same operator (FP32 pair sum), timed the same way
    forms = {}
    op.set_pairsum(2)
    u32 = torch.empty_like(u)
    op.solve_dev(b.view(1, -1), u32.view(1, -1))
    ms32, it32 = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it, st = op.solve_dev(b.view(1, -1), u32.view(1, -1), wl.ff_angles, uinf.view(1, -1))
        e1.record(stream)
        torch.cuda.synchronize()
        ms32.append(e0.elapsed_time(e1))
        it32.append(int(it[0]))
    rel32 = (torch.linalg.norm(u32 - u) / torch.linalg.norm(u)).item()
    forms["fp32_pairsum"] = {"value": args.steps / (sum(ms32) * 1e-3), "unit": "solves/s", "iterations": it32[0],
                             "rel_err_vs_fp64_solution": rel32,
                             "pairs_per_s": it32[0] * n * (n - 1) * args.steps / (sum(ms32) * 1e-3)}
    # FP64-accurate double-float pair sum on the same operator
    op.set_pairsum(3)
    op.solve_dev(b.view(1, -1), u32.view(1, -1))
    msd, itd = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it, st = op.solve_dev(b.view(1, -1), u32.view(1, -1), wl.ff_angles, uinf.view(1, -1))
        e1.record(stream)
        torch.cuda.synchronize()
        msd.append(e0.elapsed_time(e1))
        itd.append(int(it[0]))
    reld = (torch.linalg.norm(u32 - u) / torch.linalg.norm(u)).item()
    forms["df_pairsum"] = {"value": args.steps / (sum(msd) * 1e-3), "unit": "solves/s", "iterations": itd[0],
                           "rel_err_vs_fp64_solution": reld,
                           "pairs_per_s": itd[0] * n * (n - 1) * args.steps / (sum(msd) * 1e-3)}
    op.set_pairsum(0)
    # batching form on the same operator: 64 incident directions (the bench direction among
    # them) in one lock-step solve, on the tensor cores (with refinement) and on the CUDA cores
    R64 = 64
    dirs64 = rank_direction(rank, world) + 2 * np.pi * np.arange(R64) / R64
    B64 = torch.empty((R64, n), dtype=torch.complex128, device=u.device)
    op.incident_dev(dirs64, B64)
    U64 = torch.empty_like(B64)
    for kind, name in ((1, "batched_tensor_cores_64rhs"), (0, "batched_cuda_cores_64rhs")):
        op.set_batch_kernel(kind)
        op.solve_batch_dev(B64, U64)                          # warm-up (workspace)
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it64, st64 = op.solve_batch_dev(B64, U64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        forms[name] = {"value": R64 / (ms64 * 1e-3), "unit": "solves/s", "rhs": R64, "status": int(st64),
                       "iterations_max": int(np.max(it64)),
                       "rel_err_vs_fp64_solution": (torch.linalg.norm(U64[0] - u) / torch.linalg.norm(u)).item()}
    op.set_batch_kernel(1)
    # differentiation form on the same operator: gradient of the far-field misfit with respect
    # to the nodal contrast for 16 directions and 32 receivers (batched forward and adjoint
    # solves on the tensor cores, then V^T lambda per direction in FP64), once after a warm-up
    try:
        from paper_2608_17615_b300.misfit import far_field_misfit
        dirs16 = rank_direction(rank, world) + 2 * np.pi * np.arange(16) / 16
        ff32 = 2 * np.pi * np.arange(32) / 32
        m_t = torch.from_numpy(np.ascontiguousarray(np.real(wl.m), np.float64)).to(u.device).requires_grad_(True)
        tg = torch.zeros((16, 32), dtype=torch.complex128, device=u.device)
        (gr,) = torch.autograd.grad(far_field_misfit(m_t, op, dirs16, ff32, tg, batched=True), m_t)   # warm-up
        torch.cuda.synchronize()
        t_g = time.perf_counter()
        Jg = far_field_misfit(m_t, op, dirs16, ff32, tg, batched=True)
        (gr,) = torch.autograd.grad(Jg, m_t)
        torch.cuda.synchronize()
        dt_g = time.perf_counter() - t_g
        forms["gradient_16dirs_32receivers"] = {"value": 1.0 / dt_g, "unit": "gradients/s", "seconds": dt_g,
                                                "misfit": float(Jg.item()),
                                                "grad_norm": float(torch.linalg.norm(gr).item()),
                                                "timing": "host wall clock around forward + backward, synchronised"}
    except Exception as exc:                        # a form's failure must not cost the bench line
        forms["gradient_16dirs_32receivers"] = {"error": f"{type(exc).__name__}: {str(exc)[:200]}"}
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nodes": n, "k": wl.k, "grid": [wl.nx, wl.ny],
                       "l2": "flushed (512 MB write) before every timed step", "parallelism": "replicas"},
            "iterations": iters, "pairs_per_s": world * pairs_per_solve * args.steps / (total_ms * 1e-3),
            "matvecs_per_s": world * iters * args.steps / (total_ms * 1e-3), "setup_s": setup_s, "setup_parts_s": setup_parts,
            "wall_s_timed": wall, "roofline": roofline, "gpu_launches": launches, "clocks": clocks.summary(),
            "e2e": e2e, "forms": forms}
    if rank == 0 and not args.no_cpu_baseline:
        Lu = torch.empty_like(u)
        op.apply_dev(u, Lu)
        cb, err = cpu_baseline(wl, u.cpu().numpy(), Lu.cpu().numpy(), int(round(iters)))
        line["cpu_baseline"] = cb
        if err is not None:
            line["matvec_rel_err_vs_oracle"] = err
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# Floating-point operations per pair of each pair-sum kernel (FMA = 2).
#  0 k_pairsum_tab (FP64): dx, dy 2; t = dx^2 + dy^2 3; u 2; two degree-11
#    Horner chains 44; complex multiply-accumulate 8 -> 59
#  1 k_pairsum (FP64, direct): 89 FP64 instructions per pair measured by ncu
#    (58.5 DFMA, 23.5 DMUL, 7.1 DADD) -> 148
#  2 k_pairsum_f32 (FP32): two double-float differences 22, double-float t 16,
#    u 4, two degree-6 Horner chains 24, complex multiply 6, Kahan sums 8 -> 80
#  3 k_pairsum_df (double-float on FP32): differences 22, t 12, u 8, two degree-11
#    DF Horner chains 2 x 11 x 15 = 330, DF complex multiply-accumulate 60 -> 432
FLOPS_PER_PAIR = {0: 59, 1: 148, 2: 80, 3: 432}


def flops_per_pair_of(mode, nc):
    """Source count for the table degree in use (nc coefficients per cell)."""
    if mode == 0:
        return 15 + 4 * (nc - 1)            # 59 at nc = 12
    if mode == 3:
        return 102 + 30 * (nc - 1)          # 432 at nc = 12
    return FLOPS_PER_PAIR[mode]
KERNEL = {0: "k_pairsum_tab", 1: "k_pairsum", 2: "k_pairsum_f32", 3: "k_pairsum_df"}
# dram__bytes_read + write per launch from ncu captures of the current kernels (None until captured)
TRAFFIC = {}

if __name__ == "__main__":
    main()
