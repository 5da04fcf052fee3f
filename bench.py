#!/usr/bin/env python
"""Benchmark: per-fold preprocessed X^T X + X^T Y, effective TFLOP/s.

Workload (the largest single-GPU configuration): N = 1,000,000 rows,
K = 1024 X columns, M = 16 Y columns, P = 20 random balanced folds, FP32
storage with large offsets (mu_k = 1e3, sigma_k ~ U(0.5, 2)) that stress the
cancellation in X^T X - N mu mu^T, Y = X B / sqrt(K) + 0.1 eps; X and Y both
centered and scaled over each training partition (flags = 15), ddof = 1.
Synthetic seeded data (workloads.py).  ``--workload wide_range`` runs the
paper's own benchmark shape instead (Section 7: N = 100,000, K = 500, M = 10,
P = 10 contiguous folds); the default line also reports it under
``other_workloads``.

One step is one cv_products call: shift estimate, conversion of W = [X-s|Y-s|1]
into FP16 hi/lo operand tiles, fold-grouped tcgen05 Gram (exact integer hi*hi
accumulator plus an FP32 remainder accumulator), fold sums, fold statistics and
the fused epilogue, writing all P x K x K and P x K x M FP64 outputs.

Metric: effective TFLOP/s = 2 N K (K + M) / step time (the algorithmic work of
one pass of X^T [X | Y], counted once; the P-fold work the method avoids and the
four-MMA split overhead are not counted).  The inputs (4.2 GB) are larger than
the 129 MB L2, so every step reads them from HBM.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) the folds are sharded over the ranks: each rank
contracts only its folds' rows, one all-reduce (NCCL) sums the partial totals
of the contraction, and each rank writes its folds' products (strong scaling
of one problem).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

FLAGS = 15
DDOF = 1
METRIC = "per-fold preprocessed XtX+XtY eff. TFLOP/s"
UNIT = "TFLOP/s"
WORKLOADS = {
    "offset": ("cv_products N=1000000 K=1024 M=16 P=20 random balanced folds, fp32 storage, mu_k=1e3, "
               "sigma_k~U(0.5,2), center+scale X and Y, ddof=1", workloads.offset_case),
    "wide_range": ("cv_products N=100000 K=500 M=10 P=10 contiguous folds, fp32 storage, mu_k~U(-100,100), "
                   "sigma_k log-uniform [1e-2,1e2], center+scale X and Y, ddof=1", workloads.wide_range_case),
    # profiling workloads: the small-fold strategy and rows that are not 16-byte aligned
    "many_folds": ("cv_products N=50000 K=256 M=4 P=N/10 random folds of 10 rows, fp32 storage, X ~ N(0,1)+50, "
                   "center+scale X and Y, ddof=1", workloads.many_folds_case),
    "odd_k": ("cv_products N=400000 K=1021 M=16 P=20 random folds, fp32 storage, offset 10, center+scale X and Y, "
              "ddof=1", workloads.odd_k_case),
}
BAD_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")
# arithmetic of the Gram contraction per precision (statistics are FP64 in all)
DTYPES = {"fp16x3": "f16x3->f32 (tcgen05) / f64 stats / f32 epilogue",
          "auto": "f16x3->f32 (tcgen05) / f64 stats / f32 epilogue",
          "bf16x3": "bf16x3->f32 (tcgen05) / f64 stats / f32 epilogue",
          "tf32": "tf32->f32 (tcgen05) / f64 stats / f32 epilogue",
          "tf32x3": "tf32x3->f32 (tcgen05) / f64 stats / f32 epilogue",
          "fp64": "f64"}
# seconds of GPU work the clock sampler watches before the timed steps
CLOCK_SOAK_S = 1.5


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="offset")
    ap.add_argument("--rows", type=int, default=0,
                    help="profiling: the workload with this many rows instead of its own (same K, M, P and "
                         "value distributions); not the benchmark line's workload")
    ap.add_argument("--precision", default="fp16x3")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true")
    ap.add_argument("--p-sweep", action="store_true",
                    help="time per call against the number of folds P on N=1e5, K=500, M=10 (the paper's "
                         "Section 7 experiment, FP64 and the split path; prints one JSON line)")
    ap.add_argument("--batched-report", action="store_true",
                    help="256 independent problems of uneven shape: cv_batch_products (batched launches for "
                         "the split precision, a graph for FP64) against per-problem cv_products calls "
                         "(prints one JSON line; not the benchmark line)")
    ap.add_argument("--p-sweep-values", default="3,5,10,100,1000,10000,100000",
                    help="--p-sweep: the fold counts (100000 = N is leave-one-out, FP32 outputs)")
    ap.add_argument("--tune-report", action="store_true",
                    help="the plan tuner on the P-sweep's shapes: default and tuned options and times (one JSON "
                         "line; not the benchmark line)")
    ap.add_argument("--tune-values", default="10,100,1000,2000,10000",
                    help="--tune-report: the fold counts P")
    ap.add_argument("--ridge-report", action="store_true",
                    help="per-fold ridge models on the bench workload's products: time of cv_ridge and "
                         "cv_ridge_press, with the CPU oracle timed beside them (prints one JSON line; not the "
                         "benchmark line)")
    ap.add_argument("--batched-count", type=int, default=256,
                    help="--batched-report: number of problems (the first ones of the same seeded draw)")
    ap.add_argument("--batched-split-only", action="store_true",
                    help="--batched-report: skip the FP64 batch")
    ap.add_argument("--precision-report", action="store_true",
                    help="error and speed of every precision on the N=1e6, K=1024, M=16, P=20 offset workload "
                         "(prints one JSON line; not the benchmark line)")
    return ap.parse_args()


def max_over_ranks(ms, world, device=None):
    """The slowest rank's time: every rank's value all-reduced with MAX over
    the default process group (unchanged for a single process)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_tflops(flops_per_step, ms_per_step):
    """Whole-job rate: one problem per step, its folds sharded over every rank,
    timed by the slowest rank."""
    return flops_per_step / (ms_per_step * 1e-3) / 1e12


def algorithmic_flops(N, K, M):
    return 2.0 * N * K * (K + M)


def issued_mma_flops(N, K, M, tile=128, terms=4):
    """Tensor-core flops one Gram launch issues on the split path: every
    upper-triangle 128 x 128 tile of W^T W (W has K + M + 1 columns), four FP16
    MMA terms (hi*hi, hi*lo, lo*hi, lo*lo) per row; the zero rows that pad each
    segment to a 64-row block are not counted."""
    nb = -(-(K + M + 1) // tile)
    return terms * 2.0 * tile * tile * (nb * (nb + 1) // 2) * N


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def naive_cost(K, M):
    """Dot products of length |T| the naive oracle forms for one fold."""
    return K * (K + 1) / 2 + K * M


def time_oracle_sample(pr, X64, Y64, K_s):
    """Wall time of the naive oracle (Algorithm 6 generalised) on fold 0,
    every training row, the first K_s columns of X and every column of Y."""
    import oracle
    Xs = np.ascontiguousarray(X64[:, :K_s])
    t0 = time.perf_counter()
    oracle.naive_subset(Xs, Y64, pr.folds, pr.P, FLAGS, DDOF, [0])
    return time.perf_counter() - t0


def oracle_rate(pr, K_s, dt):
    """Effective TFLOP/s of the naive oracle on the whole workload, from the
    time dt it took for fold 0 restricted to the first K_s columns of X: the
    naive cost of one fold scales with K(K+1)/2 + K M (dot products of length
    |T|) and every fold costs the same for balanced folds."""
    scale = naive_cost(pr.K, pr.M) / naive_cost(K_s, pr.M)
    t_full = dt * scale * pr.P
    return algorithmic_flops(pr.N, pr.K, pr.M) / t_full / 1e12


def sample_columns(pr, X64, Y64, seconds):
    """The largest power-of-two column count K_s <= K whose oracle sample
    should take about `seconds` at the current thread count (from a timed
    32-column sample)."""
    dt32 = time_oracle_sample(pr, X64, Y64, 32)
    per_dot = dt32 / naive_cost(32, pr.M)
    K_s = 32
    while K_s < pr.K and per_dot * naive_cost(K_s * 2, pr.M) <= seconds:
        K_s *= 2
    return min(K_s, pr.K), dt32


def sample_text(pr, K_s, threads):
    nt = pr.N - int(np.bincount(pr.folds, minlength=pr.P)[0])
    return (f"naive oracle (Algorithm 6 generalised, plain C FP64), fold 0 of {pr.P}: all {nt} training rows, "
            f"the first {K_s} of {pr.K} X columns and all {pr.M} Y columns, {threads} host thread(s); rate "
            f"scaled by the naive cost K(K+1)/2+KM and x P folds")


def cpu_baseline(pr, X64, Y64, seconds_all=12.0):
    """The oracle as it stands, timed on this host at one thread and at every
    host thread (bounded samples of the workload; see sample_text)."""
    import oracle
    oracle.build()
    prev = oracle.get_threads()
    try:
        oracle.set_threads(1)
        dt1 = time_oracle_sample(pr, X64, Y64, 32)
        rate1 = oracle_rate(pr, 32, dt1)
        threads = oracle.set_threads(0)
        K_s, _ = sample_columns(pr, X64, Y64, seconds_all)
        dt = time_oracle_sample(pr, X64, Y64, K_s)
        rate = oracle_rate(pr, K_s, dt)
    finally:
        oracle.set_threads(prev)
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "host_cpus": os.cpu_count(), "sample": sample_text(pr, K_s, threads) + f" ({dt:.1f} s)",
            "one_thread": {"value": rate1, "cores": 1, "sample": sample_text(pr, 32, 1) + f" ({dt1:.1f} s)"}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    desc, make = WORKLOADS[args.workload]
    pr = make()
    X64 = pr.X.astype(np.float64)
    Y64 = pr.Y.astype(np.float64)
    import oracle
    oracle.build()
    threads = oracle.set_threads(0)
    budget_s = 150.0
    t_step = min(15.0, budget_s / max(1, args.steps + args.warmup))
    K_s, _ = sample_columns(pr, X64, Y64, t_step)
    for _ in range(args.warmup):
        time_oracle_sample(pr, X64, Y64, K_s)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        time_oracle_sample(pr, X64, Y64, K_s)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = oracle_rate(pr, K_s, dt)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "l2": "host CPU run"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "host_cpus": os.cpu_count(), "sample": sample_text(pr, K_s, threads)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.5)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return summarize_clocks(lines)


def summarize_clocks(lines):
    """The clocks record of the JSON line from nvidia-smi CSV rows of
    ClockSampler.FIELDS: median SM clock over the samples under load (power
    above 30 % of the largest sample), the largest reported maximum clock, and
    every throttle reason seen active.  None when no row parses."""
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 7:
            continue
        try:
            rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[3:7]))
        except ValueError:
            continue
    if not rows:
        return None
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
    loaded = [r for r in rows if r[2] > 0.3 * max(x[2] for x in rows)] or rows
    return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
            "reasons": reasons, "samples": len(rows)}


def traffic_for(kernel_src, path=None, workload="offset"):
    """DRAM bytes per launch of the dominant kernel on `workload` from the
    committed ncu summary (profiles/traffic.json, one record per workload),
    only while the kernel source is unchanged since the capture."""
    path = path or os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(workload)
        h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
        if rec and rec.get("source_sha256_16") == h:
            return rec.get("bytes_per_launch")
    except Exception:
        return None
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("bf16_tflops"), d.get("hbm_gbs"), "measured"
    return 1900.0, 6800.0, "fallback"


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def split_issued_flops(plan_nb_widths, N, terms=4):
    """Tensor-core flops one split-path Gram launch issues: for every
    upper-triangle tile (bi, bj) of W^T W, terms x 2 x 128 x width(bj) x N,
    with width the number of columns the kernel computes for block bj."""
    w = plan_nb_widths
    return sum(terms * 2.0 * 128 * w[bj] * N for bi in range(len(w)) for bj in range(bi, len(w)))


def narrow_last_block(precision, N, P):
    """Whether the library cuts the last column block to its used columns: it
    does so for contraction segments of at most 4096 rows, which the
    FP32-accumulating precisions always have and the FP16X3 path only when
    its folds are that short."""
    return precision not in ("fp16x3", "auto") or N / P <= 4096


def column_block_widths(K, M, narrow=True):
    """Columns the contraction computes per 128-column block of W = [X|Y|1]:
    128 for full blocks; with `narrow`, the last block is cut to the used
    columns rounded up to a multiple of 16 (the MMA's N granularity)."""
    D = K + M + 1
    nb = -(-D // 128)
    last = D - 128 * (nb - 1)
    return [128] * (nb - 1) + [min(128, -(-last // 16) * 16) if narrow else 128]


def _gpu_uuid(torch, dev):
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if uuid and not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
        return uuid
    except Exception:
        return None


def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist

    import paper_2401_13185_gb300 as cvx

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    desc, make = WORKLOADS[args.workload]
    pr = make(N=args.rows) if args.rows else make()
    if args.rows:
        desc += f" (profiling run with N={args.rows})"
    N, K, M, P = pr.N, pr.K, pr.M, pr.P
    F = algorithmic_flops(N, K, M)
    in_bytes = pr.X.nbytes + pr.Y.nbytes
    # inputs larger than L2 are read from HBM every step as they are; smaller
    # ones rotate over enough resident copies to exceed it
    copies = 1 if in_bytes > 512e6 else 3
    Xs = [torch.from_numpy(pr.X).to(dev) for _ in range(copies)]
    Ys = [torch.from_numpy(pr.Y).to(dev) for _ in range(copies)]
    folds = torch.from_numpy(pr.folds).to(dev)
    stream = torch.cuda.current_stream(dev)
    if world > 1:
        # fold sharding: this rank contracts its folds' rows, one all-reduce
        # (NCCL) sums the partial totals, this rank writes its folds' products
        from paper_2401_13185_gb300 import shard
        plan = shard.shard_plan(N, K, M, P, folds, world, rank, torch.float32, torch.float64, args.precision,
                                stream=stream)
        XTX, XTY = shard.output_tensors(plan, dev, torch.float64)
        bufs = shard.exchange_buffers(plan, dev)

        def run(Xd, Yd):
            shard.sharded_products(plan, Xd, Yd, FLAGS, DDOF, XTX, XTY, stream=stream, buffers=bufs)
    else:
        plan = cvx.cv_plan(N, K, M, P, folds, torch.float32, torch.float64, args.precision, stream)
        XTX = torch.empty((P, K, K), dtype=torch.float64, device=dev)
        XTY = torch.empty((P, K, M), dtype=torch.float64, device=dev)

        def run(Xd, Yd):
            cvx.cv_products(plan, Xd, Yd, FLAGS, DDOF, XTX, XTY, stream=stream)

    def step(k):
        run(Xs[k % copies], Ys[k % copies])

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(nsteps):
        barrier()
        torch.cuda.synchronize(dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(nsteps):
            step(k)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        return max_over_ranks(t0.elapsed_time(t1), world, dev)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize(dev)
    # one more step timed alone sizes the clock soak
    t_one = timed(1)
    soak_steps = int(CLOCK_SOAK_S * 1e3 / max(t_one, 1e-3)) + 1

    clocks = None
    for attempt in range(2):
        sampler = ClockSampler(_gpu_uuid(torch, dev))
        sampler.start()
        for k in range(soak_steps):   # untimed: keeps the GPU loaded while the sampler runs
            step(k)
        launches0 = cvx.cv_plan_launches(plan)
        ms = timed(args.steps)
        launches = cvx.cv_plan_launches(plan) - launches0
        clocks = sampler.stop()
        if clocks is not None:
            clocks["window"] = (f"{soak_steps} untimed steps (~{CLOCK_SOAK_S} s) directly before the timed "
                                f"steps, then the timed steps")
        if not clocks or not any(r in clocks["reasons"] for r in BAD_REASONS):
            break
    status = cvx.cv_plan_status(plan, stream)
    if status != 0:
        raise RuntimeError(f"device error after the timed region: {cvx.cv_status_string(status)}")
    ms_per_step = ms / args.steps
    value = job_tflops(F, ms_per_step)

    # Per-kernel durations over a second pass of the same steps (CUDA events
    # recorded by the library on the launching stream around each phase).
    prof_steps = max(args.steps, soak_steps)
    cvx.cv_plan_profile(plan, True)
    timed(prof_steps)
    phase_ms, ncalls = cvx.cv_plan_phase_ms(plan)
    cvx.cv_plan_profile(plan, False)
    gram_ms = phase_ms["gram"] / ncalls
    peak_tf, hbm_gbs, peak_src = measured_peaks()
    achieved = F / (gram_ms * 1e-3) / 1e12
    widths = column_block_widths(K, M, narrow_last_block(args.precision, N, P))
    terms = 4 if args.precision in ("fp16x3", "auto") else 3 if args.precision == "bf16x3" else \
        6 if args.precision == "tf32x3" else 2   # FP16-rate products per row (a TF32 product costs two)
    issued = split_issued_flops(widths, N, terms) / (gram_ms * 1e-3) / 1e12
    convert_ms = phase_ms["convert"] / ncalls
    # Operand conversion: reads X and Y once (FP32), writes the hi and lo FP16
    # tiles of the computed columns of every 128-column block of W once.
    convert_bytes = 4.0 * N * (K + M) + 4.0 * N * sum(widths) * (2 if args.precision == "tf32x3" else 1)

    # Error against the plain FP64 GPU path on the same inputs, and its speed.
    if world > 1:
        err_xtx = err_xty = ms64 = None
    else:
        err_xtx, err_xty, ms64 = fp64_comparison(cvx, torch, dev, stream, N, K, M, P, folds, Xs, Ys, copies,
                                                 args.steps, XTX, XTY)

    run_e2e_and_report(args, rank, world, cvx, torch, dev, stream, pr, desc, F, plan, run, Xs, Ys, XTX, XTY,
                       copies, in_bytes, value, ms_per_step, launches, clocks, phase_ms, ncalls, achieved, issued,
                       peak_tf, hbm_gbs, peak_src, convert_ms, convert_bytes, err_xtx, err_xty, ms64)


def fp64_comparison(cvx, torch, dev, stream, N, K, M, P, folds, Xs, Ys, copies, steps, XTX, XTY):
    """Relative Frobenius error of the split products (the last timed step's
    outputs) against the plain FP64 GPU path on the same inputs, and the FP64
    path's time per call."""
    split_xtx = XTX.clone()
    split_xty = XTY.clone()
    plan64 = cvx.cv_plan(N, K, M, P, folds, torch.float32, torch.float64, "fp64", stream)
    X64o = torch.empty_like(XTX)
    Y64o = torch.empty_like(XTY)
    cvx.cv_products(plan64, Xs[(steps - 1) % copies], Ys[(steps - 1) % copies], FLAGS, DDOF,
                    X64o, Y64o, stream=stream)
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    n64 = 1 if N * K * K > 1e11 else 3
    t0.record(stream)
    for k in range(n64):
        cvx.cv_products(plan64, Xs[k % copies], Ys[k % copies], FLAGS, DDOF, X64o, Y64o, stream=stream)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    ms64 = t0.elapsed_time(t1) / n64
    assert cvx.cv_plan_status(plan64, stream) == 0

    def rel_fro(a, b):
        d = torch.linalg.vector_norm((a - b).reshape(P, -1), dim=1)
        n = torch.linalg.vector_norm(b.reshape(P, -1), dim=1)
        return float((d / n).max())

    err_xtx = rel_fro(split_xtx, X64o)
    err_xty = rel_fro(split_xty, Y64o)
    del plan64, X64o, Y64o, split_xtx, split_xty
    torch.cuda.empty_cache()
    return err_xtx, err_xty, ms64


def run_e2e_and_report(args, rank, world, cvx, torch, dev, stream, pr, desc, F, plan, run, Xs, Ys, XTX, XTY,
                       copies, in_bytes, value, ms_per_step, launches, clocks, phase_ms, ncalls, achieved, issued,
                       peak_tf, hbm_gbs, peak_src, convert_ms, convert_bytes, err_xtx, err_xty, ms64):
    import torch.distributed as dist

    def barrier():
        if world > 1:
            dist.barrier()

    # End to end through the public API with host buffers: every step uploads
    # X and Y from pinned memory, runs the products and reads both outputs
    # back.  The upload of step k + 1 runs on a copy stream while step k
    # computes (two device input buffers), which is how a caller streaming
    # problems through the library would issue it.
    Xh = torch.from_numpy(pr.X).pin_memory()
    Yh = torch.from_numpy(pr.Y).pin_memory()
    XTXh = torch.empty(XTX.shape, dtype=XTX.dtype).pin_memory()
    XTYh = torch.empty(XTY.shape, dtype=XTY.dtype).pin_memory()
    Xd = [Xs[0], torch.empty_like(Xs[0])]
    Yd = [Ys[0], torch.empty_like(Ys[0])]
    copy_stream = torch.cuda.Stream(dev)
    uploaded = [torch.cuda.Event(), torch.cuda.Event()]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(b):
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(consumed[b])
            Xd[b].copy_(Xh, non_blocking=True)
            Yd[b].copy_(Yh, non_blocking=True)
            uploaded[b].record(copy_stream)

    def e2e_run(nsteps):
        for b in range(2):
            consumed[b].record(stream)
        upload(0)
        for k in range(nsteps):
            b = k % 2
            if k + 1 < nsteps:
                upload(1 - b)
            stream.wait_event(uploaded[b])
            run(Xd[b], Yd[b])
            consumed[b].record(stream)
            XTXh.copy_(XTX, non_blocking=True)
            XTYh.copy_(XTY, non_blocking=True)

    e2e_run(3)
    barrier()
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    e2e_run(args.e2e_steps)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    # every upload waits on an event recorded after t0, and the last step's
    # outputs are read back before t1: every step's copies are inside the span
    e2e_ms = max_over_ranks(t0.elapsed_time(t1) / args.e2e_steps, world, dev)
    e2e_value = job_tflops(F, e2e_ms)

    # The paper's own benchmark shape, measured the same way (kernel time).
    other = {}
    if args.workload == "offset" and world == 1 and not args.no_other_workloads:
        del Xd, Yd, Xs, Ys
        torch.cuda.empty_cache()
        other["wide_range"] = measure_workload(cvx, torch, dev, stream, "wide_range", args.precision, 200)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(pr, pr.X.astype(np.float64), pr.Y.astype(np.float64))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": DTYPES.get(args.precision, args.precision), "data": "synthetic",
            "config": {"workload": desc, "precision": args.precision,
                       "l2": (f"inputs {in_bytes / 1e9:.2f} GB (> 129 MB L2), read from HBM every step"
                              if copies == 1 else
                              f"inputs rotated over {copies} resident copies of {in_bytes / 1e6:.0f} MB (> L2)"),
                       "parallelism": (f"fold sharding x{world}: one NCCL all-reduce of the partial totals per "
                                       f"step" if world > 1 else "1 GPU")},
            "error_vs_fp64_gpu": {"xtx_rel_fro_max_fold": err_xtx, "xty_rel_fro_max_fold": err_xty},
            "fp64_gpu_path": ({"ms_per_step": ms64, "value": F / (ms64 * 1e-3) / 1e12, "unit": UNIT,
                               "speedup_of_split_path": ms64 / ms_per_step} if ms64 else None),
            "phases_ms_per_step": {k: v / ncalls for k, v in phase_ms.items()},
            "roofline": {"kernel": "k_gram_tc", "bound": "tensor", "achieved": achieved, "peak": peak_tf,
                         "unit": UNIT, "frac": achieved / peak_tf if peak_tf else None,
                         "peak_source": f"{peak_src} bf16 dense burst (fp16 runs at the bf16 rate)",
                         "achieved_basis": "algorithmic 2NK(K+M) flops / k_gram_tc time",
                         "issued_mma_tflops": issued,
                         "issued_frac": issued / peak_tf if peak_tf else None,
                         "traffic": traffic_for(os.path.join(ROOT, "paper_2401_13185_gb300", "csrc",
                                                             "gram_tc.cu"), workload=args.workload)},
            "convert_roofline": {"kernel": "k_convert_bulk", "bound": "hbm",
                                 "achieved": convert_bytes / (convert_ms * 1e-3) / 1e9, "peak": hbm_gbs,
                                 "unit": "GB/s",
                                 "frac": convert_bytes / (convert_ms * 1e-3) / 1e9 / hbm_gbs if hbm_gbs else None},
            "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": int(pr.X.nbytes + pr.Y.nbytes),
                    "d2h_bytes_per_step": int(XTX.numel() * 8 + XTY.numel() * 8),
                    "overlap": "H2D of step k+1 on a copy stream during step k (two device input buffers)"},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        if other:
            line["other_workloads"] = other
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)


def measure_workload(cvx, torch, dev, stream, name, precision, nsteps):
    """Kernel-only effective TFLOP/s of another workload (inputs rotated over
    three resident copies when they are smaller than L2)."""
    desc, make = WORKLOADS[name]
    pr = make()
    N, K, M, P = pr.N, pr.K, pr.M, pr.P
    copies = 1 if pr.X.nbytes + pr.Y.nbytes > 512e6 else 3
    Xs = [torch.from_numpy(pr.X).to(dev) for _ in range(copies)]
    Ys = [torch.from_numpy(pr.Y).to(dev) for _ in range(copies)]
    folds = torch.from_numpy(pr.folds).to(dev)
    plan = cvx.cv_plan(N, K, M, P, folds, torch.float32, torch.float64, precision, stream)
    XTX = torch.empty((P, K, K), dtype=torch.float64, device=dev)
    XTY = torch.empty((P, K, M), dtype=torch.float64, device=dev)
    for k in range(10):
        cvx.cv_products(plan, Xs[k % copies], Ys[k % copies], FLAGS, DDOF, XTX, XTY, stream=stream)
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(nsteps):
        cvx.cv_products(plan, Xs[k % copies], Ys[k % copies], FLAGS, DDOF, XTX, XTY, stream=stream)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    assert cvx.cv_plan_status(plan, stream) == 0
    ms = t0.elapsed_time(t1) / nsteps
    cvx.cv_plan_profile(plan, True)
    for k in range(nsteps):
        cvx.cv_products(plan, Xs[k % copies], Ys[k % copies], FLAGS, DDOF, XTX, XTY, stream=stream)
    phase_ms, ncalls = cvx.cv_plan_phase_ms(plan)
    F = algorithmic_flops(N, K, M)
    return {"workload": desc, "steps": nsteps, "ms_per_step": ms, "value": F / (ms * 1e-3) / 1e12, "unit": UNIT,
            "gram_ms": phase_ms["gram"] / ncalls,
            "gram_frac_of_measured_bf16": F / (phase_ms["gram"] / ncalls * 1e-3) / 1e12 / measured_peaks()[0],
            "phases_ms_per_step": {k: v / ncalls for k, v in phase_ms.items()}}


# ---------------------------------------------------------------------------
# Precision report: N=1e6, K=1024, M=16, P=20 random folds, FP32, mu = 1e3
# ---------------------------------------------------------------------------
# The 12 distinct flag combinations of Table 1 (with X centered, centering Y
# changes nothing): every combination without CV_CENTER_X, and those with it
# but without CV_CENTER_Y.
DISTINCT_FLAGS = [f for f in range(16) if not (f & 1) or not (f & 4)]


def xty_reference_flags(flags):
    """Lemma 9: X^T Y centered on either side equals the product with both sides
    centered; the oracle's literal one-sided form loses digits to cancellation
    when a side's |mean| >> std, so the X^T Y reference uses both sides."""
    return flags | 5 if flags & 5 else flags


def run_precision_report(args):
    import torch

    import oracle
    import paper_2401_13185_gb300 as cvx

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    pr = workloads.offset_case()
    N, K, M, P = pr.N, pr.K, pr.M, pr.P
    F = algorithmic_flops(N, K, M)
    X = torch.from_numpy(pr.X).to(dev)
    Y = torch.from_numpy(pr.Y).to(dev)
    folds = torch.from_numpy(pr.folds).to(dev)
    stream = torch.cuda.current_stream(dev)

    def outputs():
        return (torch.empty((P, K, K), dtype=torch.float64, device=dev),
                torch.empty((P, K, M), dtype=torch.float64, device=dev))

    def rel_fro(a, b):
        d = torch.linalg.vector_norm((a - b).reshape(P, -1), dim=1)
        n = torch.linalg.vector_norm(b.reshape(P, -1), dim=1)
        return float((d / n).max())

    def corr_err(a, b):
        dg = torch.sqrt(torch.diagonal(b, dim1=1, dim2=2).abs())
        den = dg[:, :, None] * dg[:, None, :]
        return float(((a - b).abs() / torch.where(den > 0, den, torch.ones_like(den))).max())

    def timed_call(plan, flags, reps=5):
        o = outputs()
        cvx.cv_products(plan, X, Y, flags, 1, *o, stream=stream)
        torch.cuda.synchronize(dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            cvx.cv_products(plan, X, Y, flags, 1, *o, stream=stream)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        return t0.elapsed_time(t1) / reps

    plans = {p: cvx.cv_plan(N, K, M, P, folds, torch.float32, torch.float64, p, stream)
             for p in ("fp64", "fp16x3", "bf16x3", "tf32x3", "tf32")}
    ms = {p: timed_call(plans[p], 15, 2 if p == "fp64" else 10) for p in plans}
    # every precision's products for the 12 combinations: one contraction,
    # then cv_finalize per combination
    for p in plans:
        o = outputs()
        cvx.cv_products(plans[p], X, Y, 0, 1, *o, stream=stream)
    report = {p: {} for p in plans if p != "fp64"}
    fp64_vs_oracle = 0.0
    fp64_per_flags = {}
    rng = np.random.default_rng(7)
    for flags in DISTINCT_FLAGS:
        ref = outputs()
        cvx.cv_finalize(plans["fp64"], flags, 1, *ref, stream=stream)
        # the FP64 GPU path against the oracle on sampled entries
        samples = [(int(rng.integers(P)), 0, int(rng.integers(K)), int(rng.integers(K))) for _ in range(6)]
        ysamples = [(int(rng.integers(P)), 1, int(rng.integers(K)), int(rng.integers(M))) for _ in range(2)]
        want = list(oracle.naive_entries(pr.X, pr.Y, pr.folds, P, flags, 1, samples))
        want += list(oracle.naive_entries(pr.X, pr.Y, pr.folds, P, xty_reference_flags(flags), 1, ysamples))
        samples += ysamples
        worst = 0.0
        r0, r1 = ref[0].cpu().numpy(), ref[1].cpu().numpy()
        for (fp, w, i, j), v in zip(samples, want):
            # X^T X on the correlation scale sqrt(|O_ii O_jj|), X^T Y relative to
            # the fold's largest |X^T Y| entry (entries near zero would turn
            # rounding into large relative errors)
            if w == 0:
                got, scale = r0[fp, i, j], np.sqrt(abs(r0[fp, i, i]) * abs(r0[fp, j, j]))
            else:
                got, scale = r1[fp, i, j], float(np.abs(r1[fp]).max())
            worst = max(worst, abs(got - v) / max(scale, 1e-300))
        fp64_vs_oracle = max(fp64_vs_oracle, worst)
        fp64_per_flags[str(flags)] = worst
        for p in report:
            got = outputs()
            cvx.cv_finalize(plans[p], flags, 1, *got, stream=stream)
            report[p][str(flags)] = {"xtx_rel_fro": rel_fro(got[0], ref[0]), "xty_rel_fro": rel_fro(got[1], ref[1]),
                                     "xtx_corr_scale": corr_err(got[0], ref[0])}
    for p in plans:
        assert cvx.cv_plan_status(plans[p], stream) == 0
    line = {
        "report": "precision", "workload": f"cv_products N={N} K={K} M={M} P={P} random folds, fp32 storage, "
                                          f"mu_k = 1e3, sigma_k ~ U(0.5, 2), ddof=1",
        "fp64_gpu_vs_oracle_sampled": {"max_err": fp64_vs_oracle, "entries": 8 * len(DISTINCT_FLAGS),
                                        "per_flags": fp64_per_flags,
                                        "scale": "X^T X: sqrt(|O_ii O_jj|); X^T Y: fold's max |X^T Y|"},
        "ms_per_call_flags15": ms,
        "eff_tflops_flags15": {p: F / (ms[p] * 1e-3) / 1e12 for p in ms},
        "speedup_vs_fp64_gpu": {p: ms["fp64"] / ms[p] for p in ms},
        "errors_vs_fp64_gpu": {p: {"max_xtx_rel_fro": max(v["xtx_rel_fro"] for v in report[p].values()),
                                   "max_xty_rel_fro": max(v["xty_rel_fro"] for v in report[p].values()),
                                   "max_xtx_corr_scale": max(v["xtx_corr_scale"] for v in report[p].values()),
                                   "per_flags": report[p]} for p in report},
    }
    print(json.dumps(line), flush=True)


def run_p_sweep(args):
    """Section 7 measures the method against P (3 .. N, leave-one-out) on
    N=1e5, K=500, M=10 balanced folds, centered and scaled; its claim is that
    the fast algorithm's time is nearly independent of P while the naive one
    grows linearly.  Here: time per cv_products call for P = 3 .. N, FP32
    storage, flags 15, for the split path, and for the FP64 path up to
    P = 1000 (its contraction alone takes ~30 ms; larger P adds only output
    writes).  The output bytes grow with P, so the rate of output writes is
    reported beside the time.  Leave-one-out (P = N) writes P K (K + M) =
    2.55e10 values: FP32 outputs there (102 GB), FP64 below.  The split path
    runs twice: X^T X in full and as its packed upper triangle (Props 19 and
    22: the output bytes dominate once P >= 100)."""
    import torch

    import paper_2401_13185_gb300 as cvx

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    N, K, M = 100_000, 500, 10
    rng = np.random.default_rng(workloads.SEED_BASE + 7)
    pr = workloads.wide_range_case()
    X = torch.from_numpy(pr.X).to(dev)
    Y = torch.from_numpy(pr.Y).to(dev)
    F = algorithmic_flops(N, K, M)
    out = {}
    values = [int(v) for v in args.p_sweep_values.split(",")]
    fold_ids = {P: workloads.folds_balanced_random(N, P, rng) for P in values}
    runs = [(args.precision, cvx.CV_XTX_FULL), (args.precision, cvx.CV_XTX_PACKED_UPPER), ("fp64", cvx.CV_XTX_FULL)]
    for prec, layout in runs:
        rows = []
        for P in values:
            if prec == "fp64" and P > 1000:
                continue
            out_dtype = torch.float32 if P == N else torch.float64
            folds = torch.from_numpy(fold_ids[P]).to(dev)
            plan = cvx.cv_plan_ex(N, K, M, P, folds, torch.float32, out_dtype, prec, {"xtx_layout": layout}, stream)
            XTX = torch.empty(cvx.xtx_shape(plan), dtype=out_dtype, device=dev)
            XTY = torch.empty((P, K, M), dtype=out_dtype, device=dev)
            reps = 1 if prec == "fp64" else (20 if P <= 1000 else 3)
            cvx.cv_products(plan, X, Y, 15, 1, XTX, XTY, stream=stream)
            torch.cuda.synchronize(dev)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(reps):
                cvx.cv_products(plan, X, Y, 15, 1, XTX, XTY, stream=stream)
            t1.record(stream)
            torch.cuda.synchronize(dev)
            assert cvx.cv_plan_status(plan, stream) == 0
            ms = t0.elapsed_time(t1) / reps
            out_bytes = float(XTX.element_size()) * (XTX.numel() + XTY.numel())
            rows.append({"P": P, "ms": ms, "eff_tflops": F / (ms * 1e-3) / 1e12, "out_dtype": str(out_dtype),
                         "output_GB": out_bytes / 1e9, "output_GBps": out_bytes / (ms * 1e-3) / 1e9})
            del plan, XTX, XTY
            torch.cuda.empty_cache()
        out[prec + ("_packed_xtx" if layout == cvx.CV_XTX_PACKED_UPPER else "")] = rows
    print(json.dumps({"report": "p_sweep", "workload": f"N={N} K={K} M={M} balanced random folds, fp32 storage, "
                      "flags 15, ddof 1", "results": out}), flush=True)


def run_tune_report(args):
    """The plan tuner (cv_plan_tune) on the P-sweep's shapes: N=1e5, K=500,
    M=10, random balanced folds, FP32 storage, flags 15.  For each P it
    reports the default options' time (cv_plan's rule), the options the tuner
    chose and their time; the tuner measures without a cache here."""
    import torch

    import paper_2401_13185_gb300 as cvx

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    N, K, M = 100_000, 500, 10
    rng = np.random.default_rng(workloads.SEED_BASE + 7)
    pr = workloads.wide_range_case()
    X = torch.from_numpy(pr.X).to(dev)
    Y = torch.from_numpy(pr.Y).to(dev)
    rows = []
    for P in [int(v) for v in args.tune_values.split(",")]:
        folds = torch.from_numpy(workloads.folds_balanced_random(N, P, rng)).to(dev)
        plan = cvx.cv_plan_ex(N, K, M, P, folds, torch.float32, torch.float64, args.precision, None, stream)
        XTX = torch.empty((P, K, K), dtype=torch.float64, device=dev)
        XTY = torch.empty((P, K, M), dtype=torch.float64, device=dev)
        for _ in range(2):
            cvx.cv_products(plan, X, Y, 15, 1, XTX, XTY, stream=stream)
        torch.cuda.synchronize(dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        reps = 10
        t0.record(stream)
        for _ in range(reps):
            cvx.cv_products(plan, X, Y, 15, 1, XTX, XTY, stream=stream)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        default_ms = t0.elapsed_time(t1) / reps
        del plan, XTX, XTY
        torch.cuda.empty_cache()
        best, ms = cvx.cv_plan_tune(N, K, M, P, folds, X, Y, 15, 1, torch.float32, torch.float64, args.precision,
                                    stream=stream)
        rows.append({"P": P, "default_ms": default_ms, "tuned": {"strategy": best.strategy, "ctas": best.ctas},
                     "tuned_ms": ms})
        torch.cuda.empty_cache()
    print(json.dumps({"report": "tune", "workload": f"N={N} K={K} M={M} random balanced folds, fp32 storage, "
                      f"flags 15, {args.precision}", "strategies": {"0": "auto", "1": "fold-grouped",
                                                                      "2": "small-fold"}, "results": rows}),
          flush=True)


def run_ridge_report(args):
    """Per-fold ridge regression on the bench workload's products (N=1e5,
    K=500, M=10, P=10 contiguous, flags 15, lambda = 1): device time of the
    factorisation + solves (cv_ridge) and of the validation error
    (cv_ridge_press), the oracle's time for the same on the host, and the
    largest relative difference between the two."""
    import torch

    import paper_2401_13185_gb300 as cvx

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    pr = workloads.wide_range_case()
    N, K, M, P, flags, lam = pr.N, pr.K, pr.M, pr.P, 15, 1.0
    X = torch.from_numpy(pr.X).to(dev)
    Y = torch.from_numpy(pr.Y).to(dev)
    folds = torch.from_numpy(pr.folds).to(dev)
    plan = cvx.cv_plan(N, K, M, P, folds, torch.float32, torch.float64, args.precision, stream)
    XTX = torch.empty((P, K, K), dtype=torch.float64, device=dev)
    XTY = torch.empty((P, K, M), dtype=torch.float64, device=dev)
    mean = torch.empty((P, K + M), dtype=torch.float64, device=dev)
    std = torch.empty_like(mean)
    Lw = torch.empty((P, K, K), dtype=torch.float64, device=dev)
    B = torch.empty((P, K, M), dtype=torch.float64, device=dev)
    info = torch.empty(P, dtype=torch.int32, device=dev)
    press = torch.empty((P, M), dtype=torch.float64, device=dev)
    cvx.cv_products(plan, X, Y, flags, 1, XTX, XTY, mean, std, stream=stream)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize(dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize(dev)
        return t0.elapsed_time(t1) / reps

    ms_ridge = timed(lambda: cvx.cv_ridge(XTX, XTY, lam, Lw, B, info, stream=stream))
    ms_press = timed(lambda: cvx.cv_ridge_press(plan, X, Y, flags, mean, std, B, press, stream=stream))
    assert (info.cpu().numpy() == 0).all() and cvx.cv_plan_status(plan, stream) == 0
    # CPU baseline: the oracle on the host's cores, on the same products
    import oracle
    oracle.build()
    xtx, xty, mn, sd = (t.cpu().numpy() for t in (XTX, XTY, mean, std))
    t0 = time.perf_counter()
    oracle.ridge(xtx, xty, lam)
    cpu_ridge = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.press(pr.X, pr.Y, pr.folds, P, flags, mn, sd, B.cpu().numpy())
    cpu_press = time.perf_counter() - t0
    line = {"report": "ridge", "workload": f"N={N} K={K} M={M} P={P} contiguous folds, fp32 storage, flags 15, "
                                           f"ddof 1, lambda {lam}, products in {args.precision}",
            "ms_cv_ridge": ms_ridge, "ms_cv_ridge_press": ms_press,
            "cpu_baseline": {"kind": "oracle", "cores": 1, "ridge_s": cpu_ridge, "press_s": cpu_press},
            "speedup_over_cpu_baseline": {"ridge": cpu_ridge * 1e3 / ms_ridge, "press": cpu_press * 1e3 / ms_press}}
    print(json.dumps(line), flush=True)


def run_batched_report(args):
    import torch

    import paper_2401_13185_gb300 as cvx

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    prs = workloads.batched_cases(count=args.batched_count)
    F = sum(algorithmic_flops(pr.N, pr.K, pr.M) for pr in prs)
    ds = []
    for pr in prs:
        ds.append({"X": torch.from_numpy(pr.X).to(dev), "Y": torch.from_numpy(pr.Y).to(dev),
                   "folds": torch.from_numpy(pr.folds).to(dev), "P": pr.P, "flags": pr.flags, "ddof": pr.ddof,
                   "XTX": torch.empty((pr.P, pr.K, pr.K), dtype=torch.float64, device=dev),
                   "XTY": torch.empty((pr.P, pr.K, pr.M), dtype=torch.float64, device=dev)})
    out = {}
    for prec in (args.precision,) if args.batched_split_only else (args.precision, "fp64"):
        batch = cvx.cv_batch_plan(ds, torch.float32, torch.float64, prec, stream)
        plans = [cvx.cv_plan(pr.N, pr.K, pr.M, pr.P, d["folds"], torch.float32, torch.float64, prec, stream)
                 for pr, d in zip(prs, ds)]
        reps = 20 if prec != "fp64" else 2

        def timed(fn):
            fn()
            torch.cuda.synchronize(dev)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(reps):
                fn()
            t1.record(stream)
            torch.cuda.synchronize(dev)
            return t0.elapsed_time(t1) / reps

        def run_batch():
            cvx.cv_batch_products(batch, ds, stream)

        def run_each():
            for pl, d in zip(plans, ds):
                cvx.cv_products(pl, d["X"], d["Y"], d["flags"], d["ddof"], d["XTX"], d["XTY"], stream=stream)

        ms_batch = timed(run_batch)
        ms_each = timed(run_each)
        assert cvx.cv_batch_status(batch, stream) == 0
        out[prec] = {"batch_mode": "batched launches" if cvx.cv_batch_launches(batch)[1] else "graph",
                     "ms_batch": ms_batch, "ms_per_problem_launches": ms_each,
                     "eff_tflops_batch": F / (ms_batch * 1e-3) / 1e12,
                     "eff_tflops_per_problem": F / (ms_each * 1e-3) / 1e12,
                     "speedup_of_batch": ms_each / ms_batch}
        cvx.cv_batch_destroy(batch)
        del plans
    line = {"report": "batched", "workload": f"{len(prs)} problems, N ~ U[500, 20000], K ~ U[16, 512], "
                                           f"M ~ U[1, 8], P in {{5, 10, 20}}, random flags, fp32 storage",
            "algorithmic_flops": F, "results": out}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.p_sweep:
        run_p_sweep(args)
        return
    if args.tune_report:
        run_tune_report(args)
        return
    if args.ridge_report:
        run_ridge_report(args)
        return
    if args.batched_report:
        run_batched_report(args)
        return
    if args.precision_report:
        run_precision_report(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
