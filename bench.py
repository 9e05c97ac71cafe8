#!/usr/bin/env python
"""Benchmark of the HSS-ULV factor + solve on GB300.

Workload: the N = 262,144 HSS matrix of the Yukawa kernel exp(-d)/(d + 1e-3)
plus 64 I on points uniform on the unit sphere (leaf 512, rank 128, 9 levels),
16 N(0,1) right-hand sides; seeded synthetic data in place of the paper's
grids.  One step = one factorization (Alg. 2) + one solve of all right-hand
sides.  The headline step factors in FP32 and refines to a 1e-12 relative
residual with the residual HSS matvec, the update and the root Cholesky in
FP64.  ``variants`` holds the same step with the pair-of-FP32 residual, the
tensor-core TF32 / BF16 factors, and ``fp64`` the all-FP64 path.  ``value`` is
the canonical-model TFLOP/s of the step (the paper's dense formulation:
explicit Q, QᵀDQ as 4b³ per node), with inputs resident in HBM; ``e2e`` is the
same metric through the C ABI from pinned host buffers, copies included.
Under torchrun each rank factors its own independent matrix (different seed)
-- weak scaling, no collective on the data path.

``--impl reference`` times the CPU oracle (NumPy/SciPy FP64, as it stands) on a
bounded sample of the same workload per step: the subtree of one level-4 node
(an HSS matrix of order 16,384 with the same leaf size, rank and kernel).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HSS-ULV factor+solve time & TFLOP/s, N=2^18: FP64 vs mixed+IR to 1e-12 residual"
WORKLOAD = "sphere_yukawa_256k"
SAMPLE_LEVEL = 3        # cpu baseline: subtree of one node of this level (N = 32,768)
REFERENCE_LEVEL = 4     # --impl reference: per-step sample (N = 16,384), so that
                        # K + W steps of the oracle end within a few minutes


# ---------------------------------------------------------------- flop model
def node_flops_canonical(b, r):
    """Canonical per-node flops of the paper's dense formulation: Householder QR
    of the basis, forming Q, QᵀDQ as two dense products, partial Cholesky."""
    c = b - r
    return (2 * b * r * r - 2.0 / 3 * r ** 3 + 4 * b * b * r - 4 * b * r * r + 4.0 / 3 * r ** 3
            + 4 * b ** 3 + c ** 3 / 3.0 + r * c * c + r * (r + 1) * c)


def factor_flops(levels, leaf, r):
    f = (2 ** levels) * node_flops_canonical(leaf, r)
    for l in range(1, levels):
        f += (2 ** l) * node_flops_canonical(2 * r, r)
    return f + (2 * r) ** 3 / 3.0


def solve_flops(levels, leaf, r, nrhs):
    def node(b):
        c = b - r
        return (4 * b * b + 2 * c * c + 4 * r * c) * nrhs
    f = (2 ** levels) * node(leaf)
    for l in range(1, levels):
        f += (2 ** l) * node(2 * r)
    return f + 2 * (2 * r) ** 2 * nrhs


def tree_flops(h, nrhs):
    """Canonical factor + solve flops of an HSS matrix on its own node orders
    and ranks (uneven trees included): leaf i has order b_i and rank r_i, an
    upper node order r_c1 + r_c2 and its rank, the root order r_1 + r_2."""
    L = h.levels
    fl = 0.0
    for i, b in enumerate(h.sizes):
        r = int(h.ranks[L][i])
        fl += node_flops_canonical(int(b), r)
        c = int(b) - r
        fl += (4 * b * b + 2 * c * c + 4 * r * c) * nrhs
    for l in range(L - 1, 0, -1):
        for i, r in enumerate(h.ranks[l]):
            b = int(h.ranks[l + 1][2 * i] + h.ranks[l + 1][2 * i + 1])
            r = int(r)
            c = b - r
            fl += node_flops_canonical(b, r) + (4 * b * b + 2 * c * c + 4 * r * c) * nrhs
    b0 = int(h.ranks[1][0] + h.ranks[1][1])
    return fl + b0 ** 3 / 3.0 + 2 * b0 * b0 * nrhs


# ---------------------------------------------------------------- helpers
def subtree(h, l0, p):
    """The HSS generators of the subtree under node p of level l0 (the principal
    submatrix A(I_p, I_p)); pure slicing."""
    from paper_2311_00921_gb300.inputs import HSSMatrix
    L = h.levels
    Ls = L - l0
    lo, hi = p * 2 ** Ls, (p + 1) * 2 ** Ls
    E = {m: h.E[l0 + m][p * 2 ** m:(p + 1) * 2 ** m] for m in range(1, Ls)}
    S = {m: h.S[l0 + m][p * 2 ** (m - 1):(p + 1) * 2 ** (m - 1)] for m in range(1, Ls + 1)}
    ranks = {m: h.ranks[l0 + m][p * 2 ** m:(p + 1) * 2 ** m] for m in range(1, Ls + 1)}
    return HSSMatrix(levels=Ls, sizes=h.sizes[lo:hi], ranks=ranks, D=h.D[lo:hi], U=h.U[lo:hi],
                     E=E, S=S)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_fp64_peak(torch):
    """cuBLAS DGEMM 8192^3 throughput (TFLOP/s), best of 3, in this run."""
    a = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    b = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    a @ b
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2 * 8192 ** 3 / best / 1e12


def traffic_record(kernel, prec):
    """(DRAM bytes per full-size launch, the launch they describe, its
    algorithmic bytes) of `kernel` in arithmetic `prec` from the committed ncu
    summary, or None if the kernel source changed since those counters were
    taken."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kv = dict(x.split("=", 1) for x in line.split())
        if kv.get("kernel") != kernel or kv.get("prec", "f64") != prec:
            continue
        src = os.path.join(ROOT, "paper_2311_00921_gb300", "csrc", kv["src"])
        if not os.path.exists(src):
            return None
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if sha != kv.get("src_sha"):
            return None
        scale = float(kv.get("scale", 1.0))
        algo = kv.get("algo_bytes_per_launch")
        return (float(kv["bytes_per_launch"]) * scale, kv.get("case", "").replace("_", " "),
                float(algo) * scale if algo else None)
    return None


KERNEL_SOURCES = {"tc_gemm": "tc_gemm_kernel", "tc_syr2k": "tc_gemm_kernel",
                  "gemm": "gemm_tile_kernel", "syr2k": "syr2k_lower_kernel",
                  "pchol": "pchol_kernel", "ql": "ql_basis_kernel",
                  "gemm_skinny": "gemm_n16_kernel", "trsv_fwd": "trsv_fwd_kernel",
                  "trsv_bwd": "trsv_bwd_kernel", "other": "logdet_reduce_kernel",
                  "pair_gemm": "df_gemm_kernel", "basis_gemm": "basis_gemm_kernel",
                  "basis_node": "recon_lu_kernel"}
# pair-of-FP32 arithmetic: 12 FP32 instructions per multiply-add (2 flops) plus a
# 3-instruction renormalisation every 4 terms
PAIR_OPS_PER_FLOP = 12.75 / 2


def workload(args):
    from paper_2311_00921_gb300 import inputs as I
    w = I.WORKLOADS[args.workload]
    if args.n and args.n != w.n:
        w = I.scaled(w, args.n)
    return w


# ---------------------------------------------------------------- CPU oracle arm
def oracle_sample(h, nrhs, seed, level):
    """Time the oracle's factor + solve on the subtree under node 0 of `level`
    (level 0: the whole matrix); returns (seconds, canonical flops, order)."""
    from oracle import ulv as O
    from paper_2311_00921_gb300 import inputs as I
    hs = subtree(h, level, 0) if level > 0 else h
    b = I.rhs(hs.n, nrhs, seed)
    t0 = time.perf_counter()
    F = O.factor(hs)
    O.solve(F, b)
    dt = time.perf_counter() - t0
    fl = factor_flops(hs.levels, h.leaf, h.rank) + solve_flops(hs.levels, h.leaf, h.rank, nrhs)
    return dt, fl, hs.n


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2311_00921_gb300 import inputs as I
    w = workload(args)
    h = I.cached_build(w, os.environ.get("HSS_INPUT_CACHE"))
    for _ in range(args.warmup):
        oracle_sample(h, w.nrhs, w.seed + 1, REFERENCE_LEVEL)
    tot_t, tot_f = 0.0, 0.0
    n_s = 0
    for _ in range(args.steps):
        dt, fl, n_s = oracle_sample(h, w.nrhs, w.seed + 1, REFERENCE_LEVEL)
        tot_t += dt
        tot_f += fl
    val = tot_f / tot_t / 1e12
    sample = (f"oracle factor+solve of the subtree under one level-{REFERENCE_LEVEL} node "
              f"(N={n_s}, leaf {w.leaf}, rank {w.rank}, {w.nrhs} rhs) of the {w.name} matrix")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * tot_t / max(1, args.steps), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "n": w.n, "leaf": w.leaf, "rank": w.rank,
                      "levels": w.levels, "nrhs": w.nrhs, "precision": "fp64"},
           "cpu_baseline": dict({"value": val, "unit": "TFLOP/s", "cores": os.cpu_count(),
                                 "kind": "oracle", "sample": sample}, **host_description()),
           "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def measured_peaks(torch):
    """cuBLAS FP64 and FP32 (no TF32) GEMM throughput, TFLOP/s, in this run."""
    peaks = {"f64": measured_fp64_peak(torch)}
    torch.backends.cuda.matmul.allow_tf32 = False
    a = torch.randn(8192, 8192, dtype=torch.float32, device="cuda")
    b = torch.randn(8192, 8192, dtype=torch.float32, device="cuda")
    a @ b
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    peaks["f32"] = 2 * 8192 ** 3 / best / 1e12
    for name, dt, tf32 in (("tf32", torch.float32, True), ("bf16", torch.bfloat16, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(8192, 8192, dtype=dt, device="cuda")
        b = torch.randn(8192, 8192, dtype=dt, device="cuda")
        a @ b
        torch.cuda.synchronize()
        best = 1e9
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        peaks[name] = 2 * 8192 ** 3 / best / 1e12
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = False
    return peaks


PEAK_SOURCE = {"pair32": "cuBLAS SGEMM 8192^3 without TF32 (FP32 SIMT) measured in this run, "
                         "/ 6.375: the pair arithmetic spends 12.75 FP32 instructions per "
                         "multiply-add",
               "f64": "cuBLAS DGEMM 8192^3 (FP64 pipe) measured in this run",
               "f32": "cuBLAS SGEMM 8192^3 without TF32 (FP32 SIMT) measured in this run",
               "tf32": "cuBLAS TF32 GEMM 8192^3 measured in this run (x3 split: 3 MMAs per "
                       "algorithmic product, so frac <= 1/3)",
               "bf16": "cuBLAS BF16 GEMM 8192^3 measured in this run (x3 split: 3 MMAs per "
                       "algorithmic product, so frac <= 1/3)"}


def timed_steps(torch, dev, b, x, prec, steps, clocks=None, residual="fp64", serialize=False,
                trace=False):
    """K timed factor+solve steps on the current stream (basis method, solve
    schedule and sweep staging as the autotuner chose them); returns a dict.
    trace: log every launch with CUDA events (two events a launch: instrumented
    passes only, never the headline's timed steps)."""
    def step():
        dev.factorize(prec, residual=residual, basis="auto", schedule="auto")
        dev.solve(b, x)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    dev.trace(trace or serialize, serialize=serialize)
    l0 = dev.launch_count()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        step()
    t1.record()
    torch.cuda.synchronize()
    out = {"ms": t0.elapsed_time(t1), "launches": dev.launch_count() - l0,
           "trace": dev.trace_read(), "info": dev.last_info()}
    dev.trace(False)
    out["clocks"] = clocks.stop() if clocks else None
    # factor / solve split (one untimed pass)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    dev.factorize(prec, residual=residual, basis="auto", schedule="auto")
    e[1].record()
    dev.solve(b, x)
    e[2].record()
    torch.cuda.synchronize()
    out["factor_ms"], out["solve_ms"] = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    return out


PREC_LABEL = {"f64": "FP64", "f32": "FP32", "tf32": "TF32 x3", "bf16": "BF16 x3",
              "pair32": "pair-of-FP32"}


def roofline_of(tr, peaks, steps, prec_mode="fp64", overlapped=None, overlapped_steps=None):
    """Roofline of the dominant kernel class of trace `tr` (a serialized pass:
    every logged duration is the kernel's own).  `overlapped` is the trace of the
    run as timed (basis chain concurrent on a second stream), reported beside it."""
    dom = max(tr, key=lambda k: tr[k][0])
    dms, dn, dfl = tr[dom]
    kind, prec = dom.split(".")
    if kind.startswith("tc_"):
        prec = prec_mode   # tensor-core kernels: the MMA input type's peak
    achieved = dfl / (dms / 1e3) / 1e12 if dms > 0 else 0.0
    kname = KERNEL_SOURCES[kind]
    peak = peaks.get(prec) if peaks else None
    if kind == "pair_gemm":
        prec = "pair32"
        peak = peaks["f32"] / PAIR_OPS_PER_FLOP if peaks else None
    total = sum(v[0] for v in tr.values())
    traffic = traffic_record(kname, prec)
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": (achieved / peak) if peak else None,
           "traffic": traffic[0] if traffic else None,
           "traffic_launch": traffic[1] if traffic else None,
           "traffic_algorithmic_bytes": traffic[2] if traffic else None,
           "kernel": f"{kname} ({PREC_LABEL.get(prec, prec)})",
           "peak_source": PEAK_SOURCE.get(prec),
           "timing": "serialized pass (basis chain on the main stream), CUDA events per launch",
           "kernel_ms_per_launch": dms / max(1, dn), "kernel_launches_per_step": dn / steps,
           "kernel_share": dms / total,
           "per_kernel_ms_per_step": {k: v[0] / steps for k, v in sorted(tr.items())},
           "per_kernel_tflops": {k: (v[2] / (v[0] / 1e3) / 1e12 if v[0] else 0.0)
                                 for k, v in sorted(tr.items())}}
    if overlapped:
        out["per_kernel_ms_per_step_overlapped"] = {k: v[0] / (overlapped_steps or steps)
                                                    for k, v in sorted(overlapped.items())}
    return out


def replica_workload(base, rank):
    """Rank `rank`'s matrix under --gpus N: the same workload shape with its own
    seed (the ranks run independent replicas; there is no data exchange)."""
    import dataclasses
    return dataclasses.replace(base, seed=base.seed + 10 * rank)


def max_over_ranks(value, dist, device):
    """The largest `value` over all ranks (the slowest rank's step time); the
    value itself when there is no process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_tflops(world, flops_per_step, ms_per_step):
    """Whole-job throughput: every rank's step of flops_per_step in ms_per_step."""
    return world * flops_per_step / (ms_per_step / 1e3) / 1e12


def host_description():
    """CPU model (lscpu / /proc/cpuinfo) and NumPy's BLAS, for the CPU baseline."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    blas = None
    try:
        cfg = np.__config__.CONFIG["Build Dependencies"]["blas"]
        blas = f"{cfg.get('name')} {cfg.get('version')}".strip()
    except Exception:
        pass
    return {"cpu_model": model, "blas": blas, "numpy": np.__version__}


def run_ours(args):
    import torch
    from paper_2311_00921_gb300 import hss, inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = replica_workload(workload(args), rank)
    h = I.cached_build(w, os.environ.get("HSS_INPUT_CACHE"))
    dev = hss.HSS(h)
    b_host = I.rhs(w.n, w.nrhs, w.seed + 1)
    b = hss.colmajor(b_host)
    x = torch.empty((w.nrhs, w.n), dtype=torch.float64, device="cuda").t()
    prec = args.precision
    fl_step = factor_flops(w.levels, w.leaf, w.rank) + solve_flops(w.levels, w.leaf, w.rank,
                                                                    w.nrhs)

    def rel_residual(xv):
        r = b - dev.matvec(xv)
        return (torch.linalg.vector_norm(r, dim=0)
                / torch.linalg.vector_norm(b, dim=0)).max().item()

    resid = args.residual if prec != "fp64" else "fp64"
    tune_cache = os.environ.get("HSS_TUNE_CACHE") or os.path.join(
        tempfile.gettempdir(), f"hss_tune_{os.getpid()}.txt")
    choice = None
    if prec == "auto":
        # the mixed arithmetic of the factor is a tuned choice too: the tuner's
        # factor + solve time of each (all refine to the same 1e-12 with the
        # same residual)
        cand = {p: dev.tune(p, w.nrhs, resid, cache=tune_cache) for p in ("fp32", "tf32", "bf16")}
        prec = min(cand, key=lambda p: cand[p]["factor_ms"] + cand[p]["solve_ms"])
        choice = {"chosen": prec, "tuned_factor_plus_solve_ms": {
            p: t["factor_ms"] + t["solve_ms"] for p, t in cand.items()}}
    tuning = {prec: dev.tune(prec, w.nrhs, resid, cache=tune_cache)}
    for _ in range(args.warmup):
        dev.factorize(prec, residual=resid, basis="auto", schedule=args.schedule)
        dev.solve(b, x)
    if args.profile_step:
        # one step inside the profiler window (ncu --profile-from-start off):
        # the launch list of exactly one factorization + solve
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        l0 = dev.launch_count()
        dev.factorize(prec, residual=resid, basis="auto", schedule=args.schedule)
        dev.solve(b, x)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_step": True, "precision": prec, "residual": resid,
                          "workload": w.name, "gpu_launches": dev.launch_count() - l0,
                          "max_rel_residual": rel_residual(x)}), flush=True)
        return 0
    peaks = measured_peaks(torch) if rank == 0 else None
    if dist:
        dist.barrier()
    head = timed_steps(torch, dev, b, x, prec, args.steps, ClockSampler(local), resid)
    ms = max_over_ranks(head["ms"], dist, "cuda")
    # the same steps once more with every launch logged (per-kernel times as
    # they overlap in the timed configuration), outside the timed steps
    traced = timed_steps(torch, dev, b, x, prec, min(args.steps, 5), residual=resid, trace=True)
    ms_step = ms / args.steps
    value = job_tflops(world, fl_step, ms_step)
    # correctness of the timed result: FP64 residual through the HSS matvec
    rel = rel_residual(x)
    logdet = dev.logdet()
    x_head = x.clone()
    # the same configuration once more with the basis chain serialized, so that
    # every kernel's logged time is its own (the roofline's denominator)
    nser = min(args.steps, 5)
    ser = timed_steps(torch, dev, b, x, prec, nser, residual=resid, serialize=True)

    def variant(p, r_mode):
        tuning[f"{p}_{r_mode}"] = dev.tune(p, w.nrhs, r_mode, cache=tune_cache)
        for _ in range(2):
            dev.factorize(p, residual=r_mode, basis="auto", schedule="auto")
            dev.solve(b, x)
        g = timed_steps(torch, dev, b, x, p, args.steps, residual=r_mode)
        if p == "fp64":
            g["trace"] = timed_steps(torch, dev, b, x, p, min(args.steps, 3), residual=r_mode,
                                     trace=True)["trace"]
            g["trace_steps"] = min(args.steps, 3)
        m = g["ms"] / args.steps
        out = {"precision": p, "residual": r_mode, "ms_per_step": m,
               "value": fl_step / (m / 1e3) / 1e12, "unit": "TFLOP/s",
               "factor_ms": g["factor_ms"], "solve_ms": g["solve_ms"],
               "max_rel_residual": rel_residual(x)}
        if p != "fp64":
            out["ir_iterations"] = g["info"]["ir_iters"]
        out["max_rel_diff_vs_headline_x"] = (
            torch.linalg.vector_norm(x_head - x, dim=0)
            / torch.linalg.vector_norm(x_head, dim=0)).max().item()
        return out, g

    variants = {}
    fp64 = None
    if not args.no_variants:
        if prec != "fp64":
            other = "pair32" if resid == "fp64" else "fp64"
            variants[f"{prec}_{other}_residual"] = variant(prec, other)[0]
            for p in ("tf32", "bf16", "fp32"):
                if p != prec:
                    variants[f"{p}_fp64_residual"] = variant(p, "fp64")[0]
        if prec != "fp64":
            v64, g64 = variant("fp64", "fp64")
            ser64 = timed_steps(torch, dev, b, x, "fp64", min(args.steps, 3), serialize=True)
            v64["logdet"] = dev.logdet()
            v64["headline_speedup_vs_fp64"] = v64["ms_per_step"] / ms_step
            v64["roofline"] = roofline_of(ser64["trace"], peaks, min(args.steps, 3), "fp64",
                                          overlapped=g64["trace"],
                                          overlapped_steps=g64["trace_steps"])
            fp64 = v64

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, h, w, b_host, prec, fl_step, world, dist, tune_cache)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        dt, fl, n_s = oracle_sample(h, w.nrhs, w.seed + 1, SAMPLE_LEVEL)
        cpu = {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"oracle FP64 factor+solve of the subtree under one level-{SAMPLE_LEVEL}"
                         f" node (N={n_s}, same leaf/rank/kernel, {w.nrhs} rhs), "
                         f"{dt:.1f} s"}
        cpu.update(host_description())
    if rank == 0 and args.cpu_full and world == 1:
        dt, fl, n_s = oracle_sample(h, w.nrhs, w.seed + 1, 0)
        cpu = dict(cpu or {}, full_matrix={"seconds": dt, "value": fl / dt / 1e12,
                                           "unit": "TFLOP/s", "n": n_s})

    if rank == 0:
        info = head["info"]
        out = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if prec == "fp64" else f"{prec}+f64",
               "data": "synthetic",
               "config": {"workload": w.name, "n": w.n, "leaf": w.leaf, "rank": w.rank,
                          "levels": w.levels, "nrhs": w.nrhs,
                          "precision": prec if prec == "fp64" else
                          f"{prec} factor + iterative refinement to 1e-12 (residual HSS "
                          f"matvec, update and test in "
                          f"{'pair-of-FP32 (48-bit) / FP64' if resid == 'pair32' else 'FP64'}"
                          f"; root Cholesky FP64)",
                          "residual": resid,
                          "parallelism": f"replicas{world}" if world > 1 else "single",
                          "l2": "HSS data (1.54 GB) and factors exceed L2; no flush",
                          "flop_model": "canonical dense-QtDQ model per node (4b^3 + form-Q "
                                        "+ QR + partial Cholesky) + solve (4b^2+2c^2+4rc) "
                                        "per rhs"},
               "factor_ms": head["factor_ms"], "solve_ms": head["solve_ms"],
               "check": {"max_rel_residual": rel, "logdet": logdet,
                         "ir_iterations": info["ir_iters"], "ir_resid": info["ir_resid"]},
               "fp64": fp64, "variants": variants,
               "roofline": roofline_of(ser["trace"], peaks, nser, prec,
                                       overlapped=traced["trace"],
                                       overlapped_steps=min(args.steps, 5)),
               "cpu_baseline": cpu, "e2e": e2e, "clocks": head["clocks"],
               "autotune": tuning, "precision_choice": choice,
               "gpu_launches": head["launches"]}
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """Batched uneven workload: `--batch` matrices of the batched-workload
    distribution (N log-uniform in [4096, 65536] rounded to a multiple of the
    leaf size, so the trees are uneven; leaf in {128, 256, 512}, rank in {32,
    64, 128}; kernel half 1/(d + 1e-3) on the unit cube, half exp(-d/0.1) on a
    jittered grid, built by the generator; one right-hand side each), factored
    and solved by the batch path (plain and CUDA-graph replay) and by a loop of
    single-matrix calls."""
    import torch
    from paper_2311_00921_gb300 import hss, inputs as I
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ws = I.batch_workloads(args.batch, seed=1003)
    cache = os.environ.get("HSS_INPUT_CACHE")
    mats = [I.cached_build(w, cache) for w in ws]
    bs = [hss.colmajor(I.rhs(h.n, 1, i)) for i, h in enumerate(mats)]
    out = {}
    # canonical flops of each tree on its own (uneven) node orders and ranks
    fl = sum(tree_flops(h, 1) for h in mats)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    bt = hss.HSSBatch(mats)
    xs = [torch.empty_like(b) for b in bs]
    out["batch_ms"] = timed(lambda: (bt.factorize(), bt.solve(bs, xs)))
    bt.use_graph(True)
    out["batch_graph_ms"] = timed(lambda: (bt.factorize(), bt.solve(bs, xs)))
    lds = bt.logdet()
    del bt
    torch.cuda.empty_cache()
    objs = [hss.HSS(h) for h in mats]

    def loop():
        for o, b, x in zip(objs, bs, xs):
            o.factorize("fp64")
            o.solve(b, x)
    out["loop_ms"] = timed(loop)
    lds_loop = np.array([o.logdet() for o in objs])
    ms = min(out["batch_ms"], out["batch_graph_ms"])
    res = {"metric": f"batched uneven HSS-ULV factor+solve, {args.batch} matrices (FP64)",
           "value": fl / (ms / 1e3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (the generator's cube 1/r and grid exponential kernels)",
           "config": {"workload": f"batch{args.batch}_uneven", "matrices": args.batch,
                      "total_n": int(sum(w.n for w in ws)),
                      "uneven_trees": int(sum(not h.uniform for h in mats)),
                      "groups": len({(w.leaf, w.rank) for w in ws})},
           "batch_ms": out["batch_ms"], "batch_graph_ms": out["batch_graph_ms"],
           "loop_of_single_calls_ms": out["loop_ms"],
           "speedup_vs_loop": out["loop_ms"] / ms,
           "max_logdet_rel_diff_vs_loop": float(np.max(np.abs(lds - lds_loop) /
                                                       np.abs(lds_loop)))}
    print(json.dumps(res), flush=True)
    return 0


def run_sweep(args):
    """The paper's two scaling experiments on one GPU (Sec. 5: problem size with
    constant resources, and the impact of the leaf size): factor + solve time of
    the FP64 path and of the headline mixed path (FP32 factor, FP64-residual
    refinement to 1e-12) over N = 2^14 .. 2^18 at leaf 512 / rank 128, and over
    leaf sizes 128 .. 768 at N = 2^17 with rank 96 (the paper's leaf study uses
    rank 100).  16 right-hand sides.  Random generators with these shapes (SPD
    by a diagonal shift): the values do not change the work.  One JSON line per
    point, then a summary line."""
    import torch
    from paper_2311_00921_gb300 import hss, inputs as I
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    nrhs = 16
    points = [("n", 2 ** k, 512, 128) for k in range(14, 19)]
    points += [("leaf", 2 ** 17, leaf, 96) for leaf in (128, 192, 256, 384, 512, 768)]
    out = []
    for kind, n, leaf, r in points:
        L = int(round(math.log2(n / leaf)))
        if leaf * 2 ** L != n:
            L = int(math.ceil(math.log2(n / leaf)))
        h = I.random_hss(L, leaf, r, seed=L * 1000 + leaf, orthonormal=False, fast_bound=True)
        dev = hss.HSS(h)
        b = hss.colmajor(I.rhs(h.n, nrhs, 1))
        x = torch.empty_like(b)
        rec = {"sweep": kind, "n": h.n, "leaf": leaf, "rank": r, "levels": L}
        fl = factor_flops(L, leaf, r) + solve_flops(L, leaf, r, nrhs)
        for prec in ("fp64", "fp32"):
            dev.tune(prec, nrhs, "fp64")
            for _ in range(args.warmup):
                dev.factorize(prec, basis="auto", schedule="auto")
                dev.solve(b, x)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                dev.factorize(prec, basis="auto", schedule="auto")
                dev.solve(b, x)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            rec[prec] = {"ms_per_step": ms, "tflops": fl / (ms / 1e3) / 1e12}
        rec["mixed_speedup"] = rec["fp64"]["ms_per_step"] / rec["fp32"]["ms_per_step"]
        print(json.dumps(rec), flush=True)
        out.append(rec)
        del dev
        torch.cuda.empty_cache()
    nrec = [r for r in out if r["sweep"] == "n"]
    # growth of the time per unknown from the smallest to the largest N (1.0 = O(N))
    growth = {p: (nrec[-1][p]["ms_per_step"] / nrec[-1]["n"]) /
                 (nrec[0][p]["ms_per_step"] / nrec[0]["n"]) for p in ("fp64", "fp32")}
    print(json.dumps({"metric": "HSS-ULV factor+solve time vs N and leaf size (1 GPU)",
                      "points": len(out), "time_per_unknown_growth_n14_to_n18": growth,
                      "best_leaf_fp32": min((r for r in out if r["sweep"] == "leaf"),
                                            key=lambda r: r["fp32"]["ms_per_step"])["leaf"],
                      "best_leaf_fp64": min((r for r in out if r["sweep"] == "leaf"),
                                            key=lambda r: r["fp64"]["ms_per_step"])["leaf"]}),
          flush=True)
    return 0


def run_large(args):
    """The largest workload's shape on one GPU: N = 2^21, leaf 1024, rank 256, 11
    levels, 4 right-hand sides, mixed factor (FP32, TF32 x3, BF16 x3; the
    autotuner's basis, panel and schedule) refined to 1e-12 with the FP64
    residual, against the FP64 HSS matvec of the result.  The generators are
    seeded random ones with that shape, built on the GPU (orthonormal nested
    bases, SPD by a diagonal shift, random_hss_device): the kernel-valued
    construction of this N is O(N^2 r) on the host.  One JSON line."""
    import torch
    from paper_2311_00921_gb300 import hss, inputs as I
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    L, leaf, r, nrhs = 11, 1024, 256, 4
    t0 = time.time()
    shape, D, U, E, S, shift = I.random_hss_device(L, leaf, r, seed=1004)
    dev = hss.HSS.from_device(shape, D, U, E, S)
    del D, U, E, S
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    n = shape[0]
    bh = I.rhs(n, nrhs, 1005)
    b = hss.colmajor(bh)
    x = torch.empty_like(b)
    fl = factor_flops(L, leaf, r) + solve_flops(L, leaf, r, nrhs)
    out = {"metric": "HSS-ULV factor+solve at N=2^21, leaf 1024, rank 256 (1 GPU)",
           "n": n, "leaf": leaf, "rank": r, "levels": L, "nrhs": nrhs,
           "data": "seeded random generators of this shape built on the GPU (SPD by shift "
                   f"{shift:g}); the exponential-covariance construction is not run at this N",
           "generation_s": gen_s}
    for prec in args.large_precisions.split(","):
        tune = dev.tune(prec, nrhs, "fp64")
        for _ in range(args.warmup):
            dev.factorize(prec, basis="auto", schedule="auto")
            dev.solve(b, x)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fms = sms = 0.0
        for _ in range(args.steps):
            e[0].record()
            dev.factorize(prec, basis="auto", schedule="auto")
            e[1].record()
            dev.solve(b, x)
            e[2].record()
            torch.cuda.synchronize()
            fms += e[0].elapsed_time(e[1])
            sms += e[1].elapsed_time(e[2])
        fms, sms = fms / args.steps, sms / args.steps
        info = dev.last_info()
        res = b - dev.matvec(x)
        rel = (torch.linalg.vector_norm(res, dim=0) / torch.linalg.vector_norm(b, dim=0)).max()
        # one more step with the launches logged one after the other: where the time goes
        dev.trace(True, serialize=True)
        dev.factorize(prec, basis="auto", schedule="auto")
        dev.solve(b, x)
        torch.cuda.synchronize()
        per_class = {k: round(v[0], 3) for k, v in sorted(dev.trace_read().items())}
        dev.trace(False)
        out[prec] = {"factor_ms": fms, "solve_ms": sms, "ms_per_step": fms + sms,
                     "tflops": fl / ((fms + sms) / 1e3) / 1e12, "ir_iterations": info["ir_iters"],
                     "max_rel_residual_fp64_matvec": rel.item(),
                     "autotune": {k: tune[k] for k in ("basis", "ql_panel", "schedule", "staging",
                                                       "ir_lanes")},
                     "serialized_ms_by_kernel_class": per_class}
    out["device_memory_gb"] = torch.cuda.max_memory_allocated() / 1e9
    free, total = torch.cuda.mem_get_info()
    out["device_memory_in_use_gb"] = (total - free) / 1e9
    print(json.dumps(out), flush=True)
    return 0


def run_e2e(args, h, w, b_host, prec, fl_step, world, dist, tune_cache):
    """One user call sequence per step from pinned host memory: create the object
    (H2D of the generators), factor (hss_tune with the cached choice of the
    autotuner, which factors once with it), upload b, solve, read x back,
    destroy."""
    import torch
    from paper_2311_00921_gb300 import hss
    import ctypes

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t

    D = pinned(hss._colmajor_blocks(h.D))
    U = pinned(hss._colmajor_blocks(h.U))
    E = pinned(np.concatenate([hss._colmajor_blocks(h.E[l]).ravel()
                               for l in range(1, h.levels)]))
    S = pinned(np.concatenate([hss._colmajor_blocks(h.S[l]).ravel()
                               for l in range(1, h.levels + 1)]))
    bh = pinned(np.asfortranarray(b_host).T.copy())     # (nrhs, n) rows = columns of b
    xh = torch.empty_like(bh).pin_memory()
    lib = hss.load()
    h2d = (D.numel() + U.numel() + E.numel() + S.numel() + bh.numel()) * 8
    d2h = xh.numel() * 8
    bd = torch.empty_like(bh, device="cuda")
    xd = torch.empty_like(bh, device="cuda")
    steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        shape = hss.Shape(w.n, w.leaf, w.rank, w.levels)
        out = ctypes.c_void_p()
        hss._check(lib.hss_create(ctypes.byref(shape), D.data_ptr(), U.data_ptr(), E.data_ptr(),
                                  S.data_ptr(), 0, ctypes.byref(out)), "hss_create")
        st = torch.cuda.current_stream()
        opt = hss.Options(hss.PRECISIONS[prec], 30, 1e-12,
                          hss.RESIDUALS[args.residual if prec != "fp64" else "fp64"],
                          hss.BASIS_METHODS["auto"], 0, hss.SCHEDULES["auto"], 0)
        hss._check(lib.hss_tune(out, ctypes.byref(opt), w.nrhs, tune_cache.encode(),
                                st.cuda_stream, None), "hss_tune")
        bd.copy_(bh, non_blocking=True)
        hss._check(lib.hss_solve(out, bd.data_ptr(), xd.data_ptr(), w.nrhs, w.n, st.cuda_stream),
                   "hss_solve")
        xh.copy_(xd, non_blocking=True)
        torch.cuda.synchronize()
        lib.hss_destroy(out)
    dt = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    return {"value": job_tflops(world, fl_step, 1e3 * dt / steps), "unit": "TFLOP/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": 1e3 * dt / steps, "steps": steps,
            "includes": "hss_create from pinned host (generators H2D), factorize (hss_tune with the "
                        "cached choice), b H2D, "
                        "solve, x D2H, hss_destroy"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="auto",
                    choices=["auto", "fp64", "tf32", "bf16", "fp32"],
                    help="factor arithmetic; non-fp64 modes refine in FP64 to 1e-12")
    ap.add_argument("--residual", default="fp64", choices=["fp64", "pair32"],
                    help="arithmetic of the refinement residual of the mixed modes")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the other precisions / residuals and the FP64 path")
    ap.add_argument("--schedule", default="auto", choices=["auto", "async", "levels"],
                    help="solve schedule of --profile-step (default: the autotuner's)")
    ap.add_argument("--profile-step", action="store_true",
                    help="run W warm-up steps, then one step between cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off) and exit")
    ap.add_argument("--cpu-full", action="store_true",
                    help="also time the oracle once on the whole matrix (about 100 s at N=2^18)")
    ap.add_argument("--sweep", action="store_true",
                    help="time the FP64 and mixed paths over N and over the leaf size instead")
    ap.add_argument("--batch", type=int, default=0,
                    help="run the batched uneven workload with this many matrices instead")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--n", type=int, default=0,
                    help="scale the workload to this order (same leaf, rank, kernel)")
    ap.add_argument("--large", action="store_true",
                    help="N = 2^21, leaf 1024, rank 256 with random generators of that shape")
    ap.add_argument("--large-precisions", default="fp32,tf32",
                    help="factor precisions of --large (comma-separated)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    if args.batch:
        return run_batch(args)
    if args.sweep:
        return run_sweep(args)
    if args.large:
        return run_large(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
