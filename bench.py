#!/usr/bin/env python
"""Benchmark of the Lippmann-Schwinger Nystrom hot path on one B300.

A step is one full left-preconditioned GMRES solve (tol 1e-8) of the two-material
disk (off-centre inclusion; n_opt = 1.5 + 0.2 exp(-|x|^2/0.1) outside, 2.2 inside),
k = 20, 2,680 curved triangles x 15 nodes = 40,200 nodes, Cartesian preconditioner on
256^2 over [-1.2, 1.2]^2, one plane wave at pi/4, plus its far-field pattern at 64
angles, with the FP64-accurate pair sum (the H0 table evaluated in double-float
arithmetic on the FP32 pipe; its matvec agrees with the FP64 oracle to ~1e-12, and the
line states the measured error).  Setup (correction and preconditioner factors) is
excluded, as the paper excludes it from its solve times.  The line also carries, under
"forms", every other form on its own configuration: the FP64-pipe pair sum and the
FP32 precision form on the same workload, the batched 64-direction solves, the
Approach I / II comparison, the precision form at k = 40 on 195,630 nodes, the
batching form (8 star scatterers, 64 directions each) and the differentiation form
(gradient on 492,450 nodes), each with its error and a roofline fraction.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload default|precision|batching|gradient|batched]
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
METRIC = ("LS GMRES solves/s (FP64-accurate: FP32 GMRES refined until the double-float operator's residual "
          "meets tol, preconditioned)")
# Preconditioned GMRES iterations of this workload as measured by the GPU arm;
# the reference arm scales its sampled matvec cost by it.
REFERENCE_ITERS = 8
LS_PREC_FP64_TABLE, LS_PREC_FP64_DIRECT, LS_PREC_FP32, LS_PREC_FP64_DF, LS_PREC_MIXED = range(5)


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


# ---------------------------------------------------------------- peaks and flop counts
def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


# B300 unit counts at 2.032 GHz on 148 SMs: FP32 128 lanes/SM (FMA = 2 flops), FP64 2 DFMA/clk/SM.
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12          # 77.0
FP64_UNIT_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12       # 1.203
FP32_PEAK_SOURCE = "FP32 unit count: 148 SMs x 128 lanes x 2 flops x 2.032 GHz"


# Floating-point operations per pair of each pair-sum kernel (FMA = 2), counted from the source:
#  0 k_pairsum_tab (FP64): dx, dy 2; t 3; u 2; two Horner chains 4 (nc - 1); complex MAC 8
#  1 k_pairsum (FP64, direct): 89 FP64 instructions per pair measured by ncu (58.5 DFMA,
#    23.5 DMUL, 7.1 DADD) -> 148
#  2 FP32 table: H = two double-float differences 22, double-float t 21, u 4, two degree-6
#    Horner chains 24 (71); multiply-add = complex multiply 6 + Kahan sums 8 (14)
#  3 double-float table: H = differences 22, t 21, u 10, normalisation 6, per chain nf FP32
#    Horner steps (2 flops) and nc - 1 - nf compensated double-float steps (15 flops);
#    multiply-add = four products to first order 28 + four TwoSums with residual sums 32 (60);
#    the ordered-pair kernel normalises every sum (84)
# The unordered-pair kernels (k_pairsum_f32s, k_pairsum_dfs, the default) form H once per
# unordered pair and do both multiply-adds: per ordered pair H / 2 plus one multiply-add.
# ncu check (k_pairsum_dfs<10, 2>, 40,200 nodes): FADD 122.0 + FMUL 14.1 + 2 x FFMA 39.3 =
# 214.8 FP32 flops per ordered pair against 198.5 counted here (the rest: the diagonal
# blocks' ordered pairs and the FP64 folds).
def flops_per_pair_of(mode, nc, nf=0, symmetric=True):
    if mode == 0:
        return 15 + 4 * (nc - 1)
    if mode == 3:
        h = 59 + 4 * nf + 30 * (nc - 1 - nf)
        return h / 2 + 60 if symmetric else h + 84
    if mode == 2:
        return 71 / 2 + 14 if symmetric else 85
    return 148


KERNEL = {0: "k_pairsum_tab", 1: "k_pairsum", 2: "k_pairsum_f32s", 3: "k_pairsum_dfs"}
# dram__bytes_read + write per launch (40,200 nodes) from ncu captures of the pair-sum kernels
# (the ordered-pair kernels read the nodes and densities once: 2.4 MB; the unordered-pair
# kernels also write one partial row per block distance: k_pairsum_f32s 2.43 + 46.45 MB,
# k_pairsum_dfs 3.20 + 46.99 MB)
TRAFFIC_BYTES = {0: 2.4e6, 2: 4.889e7, 3: 5.019e7}
# Thread instructions per ordered pair of the unordered-pair kernels (ncu smsp__inst_executed x 32
# / pairs, 40,200 nodes): the FP32-pipe kernels are issue-bound, so their instruction rate
# against the SM's issue limit (148 SMs x 128 lanes x 2.032 GHz) shows how busy they keep it
INSTR_PER_PAIR = {2: 62.5, 3: 200.0}
ISSUE_PEAK = 148 * 128 * 2.032e9


def _timed(fn, stream, reps=1):
    """Run fn reps times between CUDA events on `stream`; returns (ms per run, last result)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def _pairsum_roofline(op, n, peak, peak_source, total_ms=None, kind=None):
    """Roofline of a single-RHS pair-sum kernel from the operator's event-timed launches
    (kind: the arithmetic of the launches to take, LS_PREC_*; default the operator's own)."""
    if kind is None:
        ps_ms, ps_launches, _ = op.stats()
        mode = op.params.prec
    else:
        ps_ms, ps_launches = op.stats_kind(kind)
        mode = kind
    nc, _ = op.tuning()
    nf = op.df_tail() if mode == 3 else 0
    fpp = flops_per_pair_of(mode, nc, nf)
    avg_s = ps_ms / max(ps_launches, 1) * 1e-3
    achieved = fpp * n * (n - 1) / avg_s / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": TRAFFIC_BYTES.get(mode) if n == 40200 else None, "kernel": KERNEL[mode],
           "flops_per_pair": fpp, "table_ncoef": nc, "peak_source": peak_source,
           "kernel_ms_per_launch": avg_s * 1e3, "kernel_launches": ps_launches}
    if mode == 3:
        out["fp32_tail_coefficients"] = nf
    if mode in INSTR_PER_PAIR and n == 40200:
        out["thread_instructions_per_pair"] = INSTR_PER_PAIR[mode]
        out["issue_frac"] = INSTR_PER_PAIR[mode] * n * (n - 1) / avg_s / ISSUE_PEAK
    if total_ms:
        out["kernel_share_of_step"] = ps_ms / total_ms
    return out


# ---------------------------------------------------------------- CPU baselines (the oracle)
def _oracle_rows_job(job):
    """Worker of the CPU baselines (spawned process): the oracle's pair-sum rows and
    correction rows of one slice of the sample, with their wall times."""
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


def _oracle_pool(cores):
    import multiprocessing as mp
    os.environ["OPENBLAS_NUM_THREADS"] = "1"          # inherited by the spawned workers
    os.environ["OMP_NUM_THREADS"] = "1"
    return mp.get_context("spawn").Pool(cores)


def _oracle_sample(pool, cores, wl, f, n_ps, n_corr, seed):
    """One bounded sample on all cores: n_ps pair-sum rows and n_corr correction rows (among
    them) per process.  Returns (core-seconds per pair-sum row, per correction row, wall
    seconds, jobs, results)."""
    n = wl.mesh.n_nodes
    perm = np.random.default_rng(seed).permutation(n)
    jobs = []
    for c in range(cores):
        ps = perm[(c * n_ps) % n:(c * n_ps) % n + n_ps]
        jobs.append(("small", f, np.sort(ps), np.sort(ps[:n_corr])))
    w0 = time.perf_counter()
    res = pool.map(_oracle_rows_job, jobs)
    wall = time.perf_counter() - w0
    rows_ps = sum(len(j[2]) for j in jobs)
    rows_corr = sum(len(j[3]) for j in jobs)
    return sum(r[2] for r in res) / rows_ps, sum(r[3] for r in res) / rows_corr, wall, jobs, res


def cpu_baseline(wl, u_gpu, Lu_gpu, iters, budget_s=24.0):
    """The oracle as it stands, timed on the host's cores (one spawned process per core,
    single-threaded BLAS) on a bounded sample of the same workload: pair-sum rows and
    correction rows per process, sized from a short calibration so the sample takes about
    budget_s, plus one apply of the oracle's preconditioner (SuperLU solve on the 256^2
    grid; its assembly is setup).  The sampled rows also give the GPU matvec's error
    against the oracle.  Solves/s = 1 / (iters x (extrapolated L apply + P apply))."""
    from oracle.precond import Grid, Preconditioner
    cores = _host_cores()
    n = wl.mesh.n_nodes
    f = wl.m * u_gpu
    with _oracle_pool(cores) as pool:
        t_ps, t_corr, _, _, _ = _oracle_sample(pool, cores, wl, f, 64, 4, 1)
        n_ps = max(64, int(0.5 * budget_s / t_ps))
        n_corr = min(n_ps, max(4, int(0.5 * budget_s / t_corr)))
        t_ps, t_corr, wall, jobs, res = _oracle_sample(pool, cores, wl, f, n_ps, n_corr, 0)
    t_apply = (t_ps + t_corr) * n / cores
    job0, r0 = jobs[0], res[0]
    a = np.searchsorted(job0[2], job0[3])
    ref = u_gpu[job0[3]] + wl.k**2 * (r0[0][a] + r0[1])
    err = float(np.linalg.norm(Lu_gpu[job0[3]] - ref) / np.linalg.norm(ref))
    P = Preconditioner(Grid(wl.box, wl.nx, wl.ny), wl.mesh.nodes, wl.k, wl.m_grid)
    tp0 = time.perf_counter()
    P.apply(u_gpu)
    t_P = time.perf_counter() - tp0
    t_solve = iters * (t_apply + t_P)
    return {
        "value": 1.0 / t_solve, "unit": "solves/s", "cores": cores, "kind": "oracle",
        "sample": f"{n_ps * cores} pair-sum rows x {n} sources and {n_corr * cores} correction rows over {cores} "
                  f"processes ({wall:.1f} s wall), extrapolated to {n} rows per L apply, plus one timed P apply, "
                  f"x {iters} iterations",
        "seconds": round(wall + t_P, 2), "pairs_per_s": (n - 1) / t_ps * cores,
        "t_apply_s": t_apply, "t_precond_s": t_P,
    }, err


def reference_arm(args):
    """--impl reference: the oracle as it stands on the host's cores, each step a bounded
    sample (cores x 48 pair-sum rows and cores x 2 correction rows of one L apply,
    extrapolated to the whole apply and REFERENCE_ITERS iterations)."""
    from lsinput.workloads import two_material
    wl = two_material("small")
    n = wl.mesh.n_nodes
    x = np.exp(1j * wl.k * (wl.mesh.nodes @ np.array([np.cos(np.pi / 4), np.sin(np.pi / 4)])))
    f = wl.m * x
    cores = _host_cores()
    times = []
    with _oracle_pool(cores) as pool:
        for s in range(args.warmup + args.steps):
            t_ps, t_corr, _, _, _ = _oracle_sample(pool, cores, wl, f, 48, 2, s)
            if s >= args.warmup:
                times.append((t_ps + t_corr) * n / cores * REFERENCE_ITERS)
    t_solve = statistics.mean(times)
    value = 1.0 / t_solve
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_solve * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"per step: {48 * cores} pair-sum rows + {2 * cores} correction rows of one "
                                       f"L apply over {cores} processes, extrapolated to {n} rows x "
                                       f"{REFERENCE_ITERS} iterations"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- forms on their own configurations
def precision_report(args):
    """The precision form on its own configuration (two-material disk at k = 40, 13,042
    triangles = 195,630 nodes, 512^2 preconditioner): FP32 solves (one warm-up, two timed
    with CUDA events), one FP64-accurate double-float solve for the error, the mixed form
    (FP32 GMRES refined against the double-float operator; one warm-up, one timed), and
    the FP32 matvec against the oracle on sampled rows."""
    import torch
    import paper_2608_17615_b300 as L
    from lsinput.workloads import two_material
    from oracle.operator import Operator as OracleOp

    wl = two_material("medium", k=40.0, nx=512, ny=512)
    n = wl.mesh.n_nodes
    t0 = time.perf_counter()
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=wl.nx, ny=wl.ny, tol=1e-8, prec=LS_PREC_FP32)
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    d = np.array([np.cos(np.pi / 4), np.sin(np.pi / 4)])
    b = torch.from_numpy(np.exp(1j * wl.k * (wl.mesh.nodes @ d))).cuda().view(1, -1)
    u32, udf = torch.empty_like(b), torch.empty_like(b)
    op.solve_dev(b, u32)                                     # warm-up
    op.set_timing(True)
    ms32, (it32, st32) = _timed(lambda: op.solve_dev(b, u32), stream, reps=2)
    rl = _pairsum_roofline(op, n, FP32_PEAK_TFLOPS, FP32_PEAK_SOURCE, ms32 * 2)
    op.set_timing(False)
    op.set_pairsum(LS_PREC_FP64_DF)
    msdf, (itdf, stdf) = _timed(lambda: op.solve_dev(b, udf), stream)
    err = (torch.linalg.norm(u32 - udf) / torch.linalg.norm(udf)).item()
    op.set_pairsum(LS_PREC_MIXED)
    umx = torch.empty_like(b)
    op.solve_dev(b, umx)                                     # warm-up
    msmx, (itmx, stmx) = _timed(lambda: op.solve_dev(b, umx), stream)
    mixed = {"ms": msmx, "solves_per_s": 1e3 / msmx, "iterations_all_inner": int(itmx[0]), "status": int(stmx),
             "explicit_exit_residual_accurate_operator": op.last_residual(),
             "rel_err_vs_fp64_accurate_solution": (torch.linalg.norm(umx - udf) / torch.linalg.norm(udf)).item()}
    op.set_pairsum(LS_PREC_FP32)
    x = np.exp(1j * np.arange(n) * 0.37)
    y = torch.empty(n, dtype=torch.complex128, device="cuda")
    op.apply_dev(torch.from_numpy(x).cuda(), y)
    rows = np.arange(0, n, n // 24)[:24]
    ref = OracleOp(wl.mesh, wl.k, wl.m, rows_only=True).apply_rows(x, rows)
    mv_err = float(np.linalg.norm(y.cpu().numpy()[rows] - ref) / np.linalg.norm(ref))
    return {"config": {"workload": "two-material disk, k=40, 195,630 nodes (13,042 curved P4 triangles), 512^2 "
                                   "Cartesian preconditioner, tol 1e-8, FP32 pair sum", "nodes": n},
            "value": 1e3 / ms32, "unit": "solves/s", "ms": ms32, "iterations": int(it32[0]), "status": int(st32),
            "pairs_per_s": int(it32[0] + 1) * n * (n - 1) / (ms32 * 1e-3),
            "rel_err_vs_fp64_accurate_solution": err, "matvec_rel_err_vs_oracle_24_rows": mv_err,
            "fp64_accurate_solve": {"ms": msdf, "iterations": int(itdf[0]), "status": int(stdf)},
            "mixed_fp32_refined_against_double_float": mixed,
            "roofline": rl, "setup_s": setup_s,
            "setup_parts_s": dict(zip(["correction", "grid", "preconditioner_factors", "table"],
                                      [round(float(t), 3) for t in op.setup_times()]))}


def batched_pairsum_report(args):
    """The batched pair sum alone (two-material disk, k = 20, 40,200 nodes, 64 right-hand
    sides): tensor-core GEMM (k_pairsum_tc), the CUDA-core FP32 kernel (k_pairsum_multi_f32)
    and the double-float one (k_pairsum_multi_df), each timed with CUDA events over
    max(1, --steps) launches after a warm-up, with its error against the FP64-accurate
    single-RHS pair sum on 4 sampled right-hand sides."""
    import torch
    import paper_2608_17615_b300 as L
    from lsinput.workloads import random_density, two_material

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
    tf32_peak = _peaks().get("bf16_tflops", 1800.0) * (1.1 / 2.25)
    out = {}
    stream = torch.cuda.current_stream()
    for kind, name in ((1, "tensor_cores"), (0, "cuda_cores"), (2, "cuda_cores_double_float")):
        op.set_batch_kernel(kind, 4)
        op.pairsum_batch_dev(F, Y)
        ms, _ = _timed(lambda: op.pairsum_batch_dev(F, Y), stream, reps=max(1, min(args.steps, 5)))
        err = max((torch.linalg.norm(Y[r] - ref[r]) / torch.linalg.norm(ref[r])).item() for r in sample)
        pairs = R * n * (n - 1)
        out[name] = {"ms_per_launch_incl_epilogue": ms, "pair_rhs_interactions_per_s": pairs / (ms * 1e-3),
                     "rel_err_vs_fp64_max_of_4": err}
        if kind == 1:
            flops = 24.0 * pairs
            out[name]["roofline"] = {"bound": "tensor", "achieved": flops / (ms * 1e-3) / 1e12, "peak": tf32_peak,
                                     "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / 1e12 / tf32_peak,
                                     "peak_source": "measured bf16 burst x nominal tf32/bf16 ratio 1.1/2.25"}
    return {"config": {"workload": "two-material disk, k=20, 40,200 nodes, 64 right-hand sides", "nodes": n,
                       "rhs": R}, "forms": out}


BATCH_NODES = (5000, 8000, 14000, 22000, 34000, 50000, 72000, 100000)
# k in {10, 20, 40} assigned by size, so that every scatterer keeps >= 2 P4 elements per
# interior wavelength (by index, k = 40 would fall on the 14k-node mesh: 0.9 per wavelength)
BATCH_K = (10.0, 10.0, 10.0, 20.0, 20.0, 20.0, 40.0, 40.0)


def batching_report(args):
    """The batching form's configuration: 8 star-shaped scatterers of uneven size (5k-100k
    nodes, k = 10, 20, 40 by size, grids at k h_C ~ 0.19), 64 incident directions each, all
    solved in lock step with one persistent pair-sum launch per iteration
    (ls_solve_multi_dev) on the tensor cores, refined against the batched FP32 operator and
    against the single-RHS double-float operator; error of direction 0 of every scatterer
    against its single-RHS double-float solve."""
    import torch
    import paper_2608_17615_b300 as L
    from lsinput.workloads import star_scatterer

    R = 64
    ops, B, wls, setup = [], [], [], 0.0
    for s, nn in enumerate(BATCH_NODES):
        k = BATCH_K[s]
        nx = int(round(2.9 * k / 0.19)) + 1
        wl = star_scatterer(s, nn, k=k, nx=nx, ny=nx, n_dirs=R)
        t0 = time.perf_counter()
        op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, box=wl.box, nx=wl.nx, ny=wl.ny, tol=1e-8,
                        max_iter=100, prec=LS_PREC_FP64_DF)
        setup += time.perf_counter() - t0
        b = torch.empty((R, wl.mesh.n_nodes), dtype=torch.complex128, device="cuda")
        op.incident_dev(wl.directions, b)
        ops.append(op)
        B.append(b)
        wls.append(wl)
        print(f"[batching] scatterer {s}: {wl.mesh.n_nodes} nodes, k={k}, grid {nx}^2, setup {setup:.1f} s",
              file=sys.stderr, flush=True)
    n_s = [w.mesh.n_nodes for w in wls]
    stream = torch.cuda.current_stream()
    for op in ops:
        op.set_batch_kernel(1)
    U = [torch.empty_like(b) for b in B]
    # reference: direction 0 of every scatterer by the single-RHS double-float solve
    ref = []
    for s, op in enumerate(ops):
        u1 = torch.empty_like(B[s][0]).view(1, -1)
        op.solve_dev(B[s][0].contiguous().view(1, -1), u1)
        ref.append(u1[0].clone())
    forms = {}
    for accurate, name in ((False, "fp32_refined"), (True, "fp64_refined")):
        for op in ops:
            op.set_batch_refine(accurate)
        if not accurate:
            L.solve_multi_dev(ops, B, U)                   # warm-up (workspace)
        ms, (iters, st) = _timed(lambda: L.solve_multi_dev(ops, B, U), stream)
        it = np.asarray(iters)
        pairs = float(sum(int(it[s].max()) * R * n * (n - 1) for s, n in enumerate(n_s)))
        errs = [(torch.linalg.norm(U[s][0] - ref[s]) / torch.linalg.norm(ref[s])).item() for s in range(len(ops))]
        forms[name] = {"value": len(ops) * R / (ms * 1e-3), "unit": "solves/s", "ms": ms, "status": int(st),
                       "iterations_max_per_scatterer": [int(x.max()) for x in it],
                       "pair_rhs_interactions_per_s": pairs / (ms * 1e-3),
                       "rel_err_vs_fp64_accurate_dir0_per_scatterer": errs,
                       "rel_err_vs_fp64_accurate_dir0_max": max(errs)}
        print(f"[batching] {name}: {json.dumps(forms[name])}", file=sys.stderr, flush=True)
    best = forms["fp64_refined"]
    return {"config": {"workload": "8 star scatterers (r = 1 + 0.2 cos(5 theta + phi)), nodes "
                                   f"{n_s}, k = {list(BATCH_K)}, 64 directions each, tol 1e-8, tensor-core batched, "
                                   "refined against the single-RHS double-float operator",
                       "nodes": n_s, "rhs_per_scatterer": R},
            "value": best["value"], "unit": "solves/s", "ms": best["ms"], "status": best["status"],
            "rel_err_vs_fp64_accurate_dir0_max": best["rel_err_vs_fp64_accurate_dir0_max"],
            "forms": forms, "setup_s": setup}


def gradient_report(args):
    """The differentiation form's configuration (two-material disk, k = 40, 32,830 curved
    triangles = 492,450 nodes, 512^2 preconditioner): gradient of the far-field misfit
    1/2 sum |u_inf - t|^2 over 16 incident directions and 32 receivers with respect to
    every nodal contrast, the target t made by a forward solve with a Gaussian blob added
    to the index; forward and adjoint solves batched over the 16 directions.  One
    gradient, timed with the host clock around the synchronised forward + backward (the
    target solve is the warm-up).  The finite-difference check of the gradient runs in the
    GPU tests on smaller meshes."""
    import torch
    import paper_2608_17615_b300 as L
    from lsinput.workloads import perturbed_contrast, two_material
    from paper_2608_17615_b300.misfit import far_field_misfit

    wl = two_material("large", k=40.0, nx=512, ny=512)
    n = wl.mesh.n_nodes
    t0 = time.perf_counter()
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=512, ny=512, tol=1e-8)
    setup_s = time.perf_counter() - t0
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
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    J = far_field_misfit(m_t, op, dirs, ff, uinf_t, batched=True)
    (g,) = torch.autograd.grad(J, m_t)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t2
    return {"config": {"workload": "two-material disk, k=40, 492,450 nodes (32,830 curved P4 triangles), 512^2 "
                                   "Cartesian preconditioner, 16 directions x 32 receivers, target: +0.05 Gaussian "
                                   "blob at (-0.3, -0.2)", "nodes": n},
            "value": 1.0 / dt, "unit": "gradients/s", "seconds": dt, "misfit": float(J.item()),
            "grad_norm": float(torch.linalg.norm(g).item()), "target_solve_s": t_target,
            "target_iterations_max": int(np.max(it_t)), "setup_s": setup_s,
            "setup_parts_s": dict(zip(["correction", "grid", "preconditioner_factors", "table"],
                                      [round(float(t), 3) for t in op.setup_times()])),
            "timing": "host wall clock around the synchronised forward + backward"}


def correction_report(args):
    """The VDIM correction setup on the device (double-double k_vdim) against the host build
    (long double), on the tiny (120 triangles) and small (2,680 triangles, 40,200 nodes)
    two-material meshes, with the largest entry difference between the two builds."""
    import paper_2608_17615_b300 as L
    from lsinput.workloads import two_material

    out = {}
    for level, k in (("tiny", 8.0), ("small", 20.0)):
        wl = two_material(level, k=k)
        mesh = L.Mesh(wl.mesh)
        t0 = time.perf_counter()
        rp_d, ci_d, va_d, n_host = L.correction_dev(mesh, k, 3.0)
        t_dev = time.perf_counter() - t0
        row = {"nodes": wl.mesh.n_nodes, "k": k, "device_s": t_dev, "blocks_on_host": int(n_host)}
        if level == "tiny" or args.steps > 1:
            t0 = time.perf_counter()
            rp_h, ci_h, va_h = L.correction_host(mesh, k, 3.0)
            row["host_s"] = time.perf_counter() - t0
            assert np.array_equal(rp_d, rp_h) and np.array_equal(ci_d, ci_h)
            row["max_abs_diff_over_max_abs"] = float(np.max(np.abs(va_d - va_h)) / np.max(np.abs(va_h)))
        out[level] = row
        print(f"[correction] {level}: {json.dumps(row)}", file=sys.stderr, flush=True)
    return {"config": {"workload": "two-material disk, VDIM correction setup (patch radius 3 h), tiny k=8 and "
                                   "small k=20 meshes"}, "forms": out}


def _form(forms, key, fn):
    """Run one form; its failure is recorded instead of costing the bench line."""
    t0 = time.perf_counter()
    try:
        forms[key] = fn()
    except Exception as exc:
        forms[key] = {"error": f"{type(exc).__name__}: {str(exc)[:300]}"}
    forms[key]["wall_s"] = round(time.perf_counter() - t0, 1)
    print(f"[bench] {key}: {json.dumps(forms[key])[:600]}", file=sys.stderr, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forms", default="standard", choices=["none", "standard", "all"],
                    help="none: the headline only; standard: + the 40k-node forms and the 195k-node precision "
                         "configuration; all: + the 8-scatterer batching and 492k-node differentiation "
                         "configurations (about 10 minutes more)")
    ap.add_argument("--workload", default="default", choices=["default", "precision", "batching", "batched",
                                                                 "gradient", "correction"])
    args = ap.parse_args()
    rank, world, local = _env_rank()
    reports = {"precision": precision_report, "batching": batching_report, "batched": batched_pairsum_report,
               "gradient": gradient_report, "correction": correction_report}
    if args.workload in reports:
        if rank == 0:
            import torch
            torch.cuda.set_device(0)
            print(json.dumps({"report": args.workload, **reports[args.workload](args)}), flush=True)
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
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, tol=1e-8, prec=LS_PREC_MIXED)
    setup_s = time.perf_counter() - t0
    fp64_probe = L.probe_fp64()
    setup_parts = {k: round(float(v), 3) for k, v in
                   zip(["correction", "grid", "preconditioner_factors", "table"], op.setup_times())}
    print(f"[bench] setup {setup_s:.1f} s {setup_parts}, FP64 probe {fp64_probe:.1f} GFLOP/s", file=sys.stderr,
          flush=True)
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
    exit_res = op.last_residual()
    print(f"[bench] steps ms {step_ms}, iters {iters_list}, pair-sum {ps_ms:.1f} ms / {ps_launches} launches",
          file=sys.stderr, flush=True)
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    iters = statistics.mean(iters_list)
    value = aggregate_value(world, args.steps, total_ms)
    pairs_per_solve = ps_launches / args.steps * n * (n - 1)
    # the mixed form launches the FP32 kernel (inner GMRES) and the double-float one (accurate
    # residuals); the roofline is the dominant one's, the other's share is listed beside it
    by_kind = {kd: op.stats_kind(kd) for kd in (LS_PREC_FP32, LS_PREC_FP64_DF)}
    dominant = max(by_kind, key=lambda kd: by_kind[kd][0])
    roofline = _pairsum_roofline(op, n, FP32_PEAK_TFLOPS, FP32_PEAK_SOURCE, total_ms, kind=dominant)
    other = LS_PREC_FP64_DF if dominant == LS_PREC_FP32 else LS_PREC_FP32
    roofline["other_kernel"] = _pairsum_roofline(op, n, FP32_PEAK_TFLOPS, FP32_PEAK_SOURCE, total_ms, kind=other)
    op.set_timing(False)
    # end to end through the host-buffer entry point
    e2e_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        uh, uinfh, hist, it_h, st_h = op.solve([angle], wl.ff_angles)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = {"value": world * args.steps / (sum(e2e_ms) * 1e-3), "unit": "solves/s",
           "h2d_bytes_per_step": 8 * (1 + n_ff), "d2h_bytes_per_step": 16 * n + 16 * n_ff + 8 * (op.params.max_iter + 1)}
    # reference: the double-float GMRES solve (every pair sum FP64-accurate) of the same system
    op.set_pairsum(LS_PREC_FP64_DF)
    u_ref = torch.empty_like(u)
    it_ref, _ = op.solve_dev(b.view(1, -1), u_ref.view(1, -1))
    iters_fp64 = int(it_ref[0])
    err_headline = (torch.linalg.norm(u - u_ref) / torch.linalg.norm(u_ref)).item()
    forms = {}

    def pipe_form(mode, label, peak, peak_source):
        op.set_pairsum(mode)
        uu = torch.empty_like(u)
        op.solve_dev(b.view(1, -1), uu.view(1, -1))
        op.set_timing(True)
        reps = 3
        ms, (it_, st_) = _timed(lambda: op.solve_dev(b.view(1, -1), uu.view(1, -1), wl.ff_angles, uinf.view(1, -1)),
                                stream, reps=reps)
        rl = _pairsum_roofline(op, n, peak, peak_source, ms * reps) if peak else None
        op.set_timing(False)
        return {"config": {"workload": WORKLOAD + ", " + label}, "value": 1e3 / ms, "unit": "solves/s", "ms": ms,
                "iterations": int(it_[0]), "status": int(st_), "explicit_exit_residual": op.last_residual(),
                "rel_err_vs_fp64_accurate_solution": (torch.linalg.norm(uu - u_ref) / torch.linalg.norm(u_ref)).item(),
                "pairs_per_s": (int(it_[0]) + 1) * n * (n - 1) / (ms * 1e-3), "roofline": rl}

    run_forms = args.forms != "none"
    if run_forms:
        _form(forms, "double_float_40k", lambda: pipe_form(LS_PREC_FP64_DF, "double-float pair sum in every GMRES "
                                                            "iteration", FP32_PEAK_TFLOPS, FP32_PEAK_SOURCE))
        _form(forms, "fp64_pipe_40k",
              lambda: dict(pipe_form(LS_PREC_FP64_TABLE, "FP64-pipe table pair sum", fp64_probe / 1e3,
                                     "measured FP64 FMA probe (ls_probe_fp64), same run"),
                           fp64_unit_count_peak_tflops=FP64_UNIT_PEAK_TFLOPS))
        _form(forms, "fp32_40k", lambda: pipe_form(LS_PREC_FP32, "FP32 precision-form pair sum", FP32_PEAK_TFLOPS,
                                                    FP32_PEAK_SOURCE))
        op.set_pairsum(LS_PREC_FP64_DF)

        def batched_forms():
            R64 = 64
            dirs64 = rank_direction(rank, world) + 2 * np.pi * np.arange(R64) / R64
            B64 = torch.empty((R64, n), dtype=torch.complex128, device=u.device)
            op.incident_dev(dirs64, B64)
            U64 = torch.empty_like(B64)
            out = {}
            for kind, accurate, name in ((1, False, "tensor_cores"), (1, True, "tensor_cores_fp64_refined"),
                                         (0, False, "cuda_cores"), (2, False, "cuda_cores_double_float")):
                op.set_batch_kernel(kind)
                op.set_batch_refine(accurate)
                op.solve_batch_dev(B64, U64)                              # warm-up (workspace)
                ms64, (it64, st64) = _timed(lambda: op.solve_batch_dev(B64, U64), stream)
                out[name] = {"value": R64 / (ms64 * 1e-3), "unit": "solves/s", "ms": ms64, "status": int(st64),
                             "iterations_max": int(np.max(it64)),
                             "rel_err_vs_fp64_accurate_solution":
                                 (torch.linalg.norm(U64[0] - u_ref) / torch.linalg.norm(u_ref)).item()}
            op.set_batch_kernel(1)
            op.set_batch_refine(False)
            out["config"] = {"workload": WORKLOAD + ", 64 incident directions in lock step"}
            return out

        _form(forms, "batched_64rhs_40k", batched_forms)
        _form(forms, "batched_pairsum_64rhs_40k", lambda: batched_pairsum_report(args))

        def approach_form():
            out = {}
            for approach in (2, 1):
                opa = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, tol=1e-8, prec=LS_PREC_FP32,
                                 approach=approach)
                ua = torch.empty_like(u)
                opa.solve_dev(b.view(1, -1), ua.view(1, -1))
                ms, (it_, st_) = _timed(lambda: opa.solve_dev(b.view(1, -1), ua.view(1, -1)), stream)
                out[f"approach_{approach}"] = {"iterations": int(it_[0]), "status": int(st_), "ms": ms,
                                               "rel_err_vs_fp64_accurate_solution":
                                                   (torch.linalg.norm(ua - u_ref) / torch.linalg.norm(u_ref)).item()}
                del opa
            out["config"] = {"workload": WORKLOAD + ", FP32 pair sum, Approach I vs II transfer "
                                             "(Table bakeoff context)"}
            return out

        _form(forms, "approach_I_vs_II_40k", approach_form)
    del flush
    if run_forms and rank == 0:
        _form(forms, "precision_195k_k40", lambda: precision_report(args))
    if args.forms == "all" and rank == 0:
        _form(forms, "batching_8_stars", lambda: batching_report(args))
        _form(forms, "gradient_492k_k40", lambda: gradient_report(args))
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64-accurate (mixed): FP32 pair sum inside GMRES, double-float (FP64-accurate) pair sum for the "
                     "residuals that decide convergence; FP64 correction, preconditioner and Krylov",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nodes": n, "k": wl.k, "grid": [wl.nx, wl.ny],
                       "l2": "flushed (512 MB write) before every timed step", "parallelism": "replicas"},
            "iterations_all_inner": iters, "iterations_fp64_gmres": iters_fp64, "explicit_exit_residual": exit_res,
            "rel_err_vs_double_float_gmres_solution": err_headline,
            "pairs_per_s": world * pairs_per_solve * args.steps / (total_ms * 1e-3),
            "matvecs_per_s": world * ps_launches / (total_ms * 1e-3), "setup_s": setup_s,
            "setup_parts_s": setup_parts, "wall_s_timed": wall, "roofline": roofline, "gpu_launches": launches,
            "clocks": clocks.summary(), "e2e": e2e, "forms": forms}
    if rank == 0 and not args.no_cpu_baseline:
        Lu = torch.empty_like(u)
        op.set_pairsum(LS_PREC_FP64_DF)
        op.apply_dev(u, Lu)
        cb, err = cpu_baseline(wl, u.cpu().numpy(), Lu.cpu().numpy(), iters_fp64)
        line["cpu_baseline"] = cb
        line["matvec_rel_err_vs_oracle"] = err
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
