"""Benchmark of the blocked FP64 SpMV y = A x on one GB300 (or N independent replicas).

A step is one y = A x over the workload's matrix with the matrix already analysed and
resident in HBM (the preprocessing of the method is amortised over repeated products,
as in the paper's evaluation, and its host time is reported as analyze_ms).

Default workload: the FP64 block-structured FEM-like matrix, 1,048,576 rows of dense 3x3
blocks, ~27 blocks per block row within a 2,000 block-column band (84.8 M nonzeros).
Its packed stream (~0.9 GB) is far larger than the 129 MB L2, so no flush is needed
between timed steps; x (8 MB) stays L2-resident by design of the method.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (no data exchange); the timed
region is bracketed by a barrier and synchronisation, the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMV GFLOP/s & HBM GB/s vs ~8 TB/s roofline; served p50/p99 latency"
WORKLOADS = {
    "fem3x3_band_1m": "FP64 block-structured FEM-like matrix: 1,048,576 rows of dense 3x3 blocks, "
                      "~27 blocks per block row within a 2,000 block-column band, N(0,1) values, "
                      "x U[-1,1], seed 1",
    "fem3x3_band_256k": "FP64 FEM-like 3x3 block band, quarter size (262,144 rows), for profiling",
    "rmat_s21": "FP64 R-MAT scale 21, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05), duplicates summed, "
                "U[-1,1] values, seed 2",
    "rmat_s19": "FP64 R-MAT scale 19 (R-MAT recipe above), for profiling",
    "laplace2d_64": "FP64 2D 5-point Laplacian on a 64x64 grid, x U[-1,1], seed 0",
}
# The FP64 roofline (the run kernel issues one FP64 FMA per stored entry) is measured live
# by cbspmv_measure_fp64_fma: a kernel of independent FMA chains, one CTA per SM. On GB300
# each SM sub-partition retires one warp-wide FP64 FMA per 76 SM cycles (32 lanes / 76 =
# 0.42 lanes per cycle, 1.68 per SM); the derived peak at the maximum clock is printed beside
# the measured one.
SUBPARTITIONS_PER_SM = 4
L2_BYTES = 129 * 2 ** 20

# DRAM bytes (read + write) per launch of the run kernel from one ncu capture of the same
# kernel revision (profiles/): the quarter-size FEM case and R-MAT scale 19, scaled to the
# full workload by its number of stored entries. Used only when the loaded library reports
# the same revision; otherwise the roofline's traffic is null.
KERNEL_TRAFFIC = {
    "run kernel rev 13": {("fem3x3_band_1m", "bf16"): 0.6535e9},
    "run kernel rev 15": {("fem3x3_band_1m", "f64"): 1.0187e9},
    "run kernel rev 16": {("fem3x3_band_1m", "f64"): 1.0192e9},
    "run kernel rev 17": {("fem3x3_band_1m", "f64"): 0.9617e9, ("fem3x3_band_1m", "bf16", "lanes"): 0.4427e9},
    "run kernel rev 20": {("fem3x3_band_1m", "f64"): 0.9603e9, ("fem3x3_band_1m", "bf16", "lanes"): 0.4415e9},
    # revision 21 changed only the FP32 instance's warps per SM: the FP64 and BF16 instances
    # are the code revision 20's captures measured
    "run kernel rev 21": {("fem3x3_band_1m", "f64"): 0.9603e9, ("fem3x3_band_1m", "bf16", "lanes"): 0.4415e9},
}


def measured_traffic(version: str, workload: str, dtype: str, lanes: bool = True):
    """Captured DRAM bytes of the lane kernel (FP64: its default layout; reduced types: the
    lane-stream layout), or None."""
    key = (workload, dtype) if dtype == "f64" else (workload, dtype, "lanes")
    if not lanes:
        return None
    for rev, table in KERNEL_TRAFFIC.items():
        if version.endswith(rev + ")"):
            return table.get(key)
    return None


# The record kernel (reduced value types) is unchanged since revision 13; its capture holds
# for later revisions of the lane kernel.
RECORD_KERNEL_TRAFFIC = KERNEL_TRAFFIC["run kernel rev 13"]


def fp64_peak_gflops(sms: int, sm_mhz: float, cycles_per_warp_fma: float) -> float:
    """FP64 FMA peak from the unit counts: SMs x sub-partitions x 32 lanes per warp-FMA
    interval x 2 flops x clock."""
    return sms * SUBPARTITIONS_PER_SM * 32.0 / cycles_per_warp_fma * 2.0 * sm_mhz / 1e3


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 25 ms in the background."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "25"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        def reader():
            for line in self.proc.stdout:
                self.samples.append((time.time(), [v.strip() for v in line.split(",")]))
        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        inwin = [s for t, s in self.samples if t0 <= t <= t1]
        use = inwin or [s for _, s in self.samples]
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(s[0]) for s in use if num(s[0]) is not None]
        mx = [num(s[1]) for s in use if num(s[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in use for i in range(4) if len(s) > 4 + i and s[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(use), "in_window": len(inwin)}


def timed_repeats(steps, est_ms_per_step, target_s=1.0):
    """Repeats of the `steps`-product block in the timed region: enough for the region to
    last about target_s, so that the clock sampler (one sample per 25 ms) sees it; at least 1."""
    block_s = max(steps, 1) * max(est_ms_per_step, 1e-6) * 1e-3
    return max(1, int(math.ceil(target_s / block_s)))


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of per-rank values over all ranks (a replica job is as slow as
    its slowest rank); the values themselves for a single process."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def job_gflops(world_size: int, flops_per_rank: float, ms_max: float) -> float:
    """Whole-job throughput of independent replicas: every rank's flops over the slowest
    rank's time."""
    return world_size * flops_per_rank / (ms_max * 1e-3) / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample_gflops(A, x, target_s: float = 12.0):
    """Time the CPU oracle (single thread, as it stands) on a bounded sample of the workload:
    whole-matrix products repeated until ~target_s of CPU work. Returns (GFLOP/s, sample)."""
    import oracle
    oracle.spmv(A, x)                       # warm (builds the library, touches memory)
    reps, t_total = 0, 0.0
    while t_total < target_s and reps < 1000:
        t = time.perf_counter()
        oracle.spmv(A, x)
        t_total += time.perf_counter() - t
        reps += 1
    gf = 2.0 * A.nnz * reps / t_total / 1e9
    return gf, f"{reps} full products of the {A.m}x{A.n} matrix ({A.nnz} nonzeros), {t_total:.1f} s"


def row_slices(A, parts: int):
    """The matrix cut into `parts` row ranges of about equal nonzeros, as CSR views sharing
    the column and value arrays (row pointers stay absolute offsets into them)."""
    cuts = np.searchsorted(A.row_ptr, np.linspace(0, A.nnz, parts + 1)[1:-1])
    bounds = [0, *[int(c) for c in cuts], A.m]
    out = []
    for r0, r1 in zip(bounds[:-1], bounds[1:]):
        if r1 > r0:
            out.append(type(A)(r1 - r0, A.n, A.row_ptr[r0:r1 + 1], A.col, A.val))
    return out


def oracle_allcore_gflops(A, x, target_s: float = 8.0):
    """The same oracle (unchanged) on every host core this process may run on: the rows are
    cut into one slice per core and each slice is multiplied by a separate thread (the
    oracle's C routine runs outside Python's lock). Whole-matrix products are repeated until
    ~target_s. Returns (GFLOP/s, threads, sample)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    threads = len(os.sched_getaffinity(0))
    parts = row_slices(A, threads)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda S: oracle.spmv(S, x), parts))      # warm
        reps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < target_s and reps < 5000:
            list(ex.map(lambda S: oracle.spmv(S, x), parts))
            reps += 1
        dt = time.perf_counter() - t0
    gf = 2.0 * A.nnz * reps / dt / 1e9
    return gf, threads, f"{reps} full products on {threads} threads (row slices of equal nonzeros), {dt:.1f} s"


def multi_rhs_bench(M, A, x, vec, stream, ks=(1, 8, 32), reps=20):
    """GFLOP/s of cbspmv_run_multi on k right-hand sides (column-major, ld = n / m)."""
    import torch
    out = []
    for k in ks:
        X = torch.from_numpy(np.tile(x.astype(vec), (k, 1))).cuda()
        Y = torch.empty((k, A.m), dtype=X.dtype, device="cuda")
        for _ in range(3):
            M.run_multi(X, Y, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            M.run_multi(X, Y, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out.append({"k": k, "ms": round(ms, 4), "gflops": round(2.0 * A.nnz * k / (ms * 1e-3) / 1e9, 1)})
        del X, Y
    return out


def spmm_bench(bd, A, x, stream, ks=(1, 8, 32), reps=20):
    """Tensor-core multi-vector product (cbspmv_spmm) on a BF16 copy of the matrix: X (n x k)
    and Y (m x k) row-major FP32. Returns per k the time, GFLOP/s (2 nnz k / t) and the HBM
    fraction of its bytes model (values and coordinates, sub-block metadata, restore_cols,
    X read once, Y written once), beside the BF16 single-vector product of the default
    (lane-stream) handle."""
    import torch
    peak, _ = load_peaks()
    out = {"api": "cbspmv_spmm (mma.sync.m16n8k16 BF16 x BF16 -> FP32, x split into 3 BF16 parts)",
           "values": "bf16", "results": []}
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    yd = torch.empty(A.m, dtype=torch.float32, device="cuda")
    with bd.BlockedMatrix(A, value_dtype="bf16", stream=stream) as M1:
        kt = M1.time_kernels(xd, yd, 200, stream=stream)
        ms1 = kt["ms_main"] + kt["ms_combine"]
    out["spmv_bf16_k1"] = {"ms": round(ms1, 4), "gflops": round(2.0 * A.nnz / (ms1 * 1e-3) / 1e9, 1),
                           "handle": "default BF16 handle (lane kernel)"}
    with bd.BlockedMatrix(A, value_dtype="bf16", plain_records=True, stream=stream) as M:
        st = M.stats()
        mat_bytes = A.nnz * 3 + st["n_tiles"] * 21 + 4 * st["restore_cols_len"]
        for k in ks:
            X = torch.from_numpy(np.tile(x.astype(np.float32)[:, None], (1, k))).cuda()
            Y = torch.empty((A.m, k), dtype=torch.float32, device="cuda")
            for _ in range(3):
                M.spmm(X, Y, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                M.spmm(X, Y, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            byts = mat_bytes + 4 * k * (A.n + A.m)
            out["results"].append({"k": k, "ms": round(ms, 4), "gflops": round(2.0 * A.nnz * k / (ms * 1e-3) / 1e9, 1),
                                   "vs_spmv_bf16_k1": round(ms1 * k / ms, 2),
                                   "hbm_frac": round(byts / (ms * 1e-3) / 1e9 / peak, 4)})
            del X, Y
    return out


def batched_suite(nmat: int = 64, rows_lo: float = 1e4, rows_hi: float = 2e5, seed: int = 4):
    """64 matrices drawn from the three generator families (2D Laplacian, FEM 3x3 band,
    R-MAT), rows log-uniform in [rows_lo, rows_hi], value types FP32 / BF16 / FP16 in turn."""
    from paper_2605_18515_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    fams, dts = ("laplace2d", "fem", "rmat"), ("f32", "bf16", "f16")
    out = []
    for i in range(nmat):
        fam, dt = fams[i % 3], dts[(i // 3) % 3]
        r = int(np.exp(rng.uniform(np.log(rows_lo), np.log(rows_hi))))
        if fam == "laplace2d":
            A = I.laplacian2d(max(8, int(round(np.sqrt(r)))))
        elif fam == "fem":
            nb = (r + 2) // 3
            A = I.fem_block_band(n_rows=r, n_block_rows=nb, half_band=min(1000, max(13, nb // 8)), seed=10 + i)
        else:
            A = I.rmat(max(10, int(round(np.log2(r)))), 16, seed=10 + i)
        out.append((fam, dt, A))
    return out


def batched_bench(bd, stream, ks=(1, 8, 32), reps=10, full=False):
    """64 products in one batched call (cbspmv_run_batched: one launch per value type per
    column round) with options tuned once per (family, value type) on the largest matrix of
    the class; per-result error against the FP64 oracle on sampled rows."""
    import torch
    import oracle
    from paper_2605_18515_gb300 import inputs as I
    t0 = time.perf_counter()
    suite = batched_suite(rows_hi=1e6 if full else 2e5)
    t_gen = time.perf_counter() - t0
    peak, _ = load_peaks()
    best = {}
    for fam in ("laplace2d", "fem", "rmat"):
        for dt in ("f32", "bf16", "f16"):
            cls = [A for f, d, A in suite if f == fam and d == dt]
            if not cls:
                continue
            A = max(cls, key=lambda a: a.nnz)
            M, rep = bd.analyze_tuned(A, reps=5, value_dtype=dt, stream=stream)
            M.close()
            best[(fam, dt)] = {k: rep["best"][k] for k in ("col_agg", "unit_work", "th1", "th2", "record_layout")}
    mats = [bd.BlockedMatrix(A, value_dtype=dt, stream=stream, **best[(fam, dt)]) for fam, dt, A in suite]
    out = {"matrices": len(suite), "families": "2D Laplacian, FEM 3x3 band, R-MAT (one third each)",
           "value_types": "FP32, BF16, FP16 in turn (FP32 x, y, accumulation)",
           "rows": f"log-uniform in [1e4, {'1e6' if full else '2e5'}]",
           "total_nnz": int(sum(A.nnz for _, _, A in suite)), "generate_s": round(t_gen, 1),
           "tuned": {f"{f}/{d}": v for (f, d), v in best.items()},
           "api": "cbspmv_run_batched (one launch per value type per round: passes of four columns, then "
                  "single columns)", "results": []}
    try:
        for k in ks:
            Xs, Ys, X64 = [], [], []
            for i, (fam, dt, A) in enumerate(suite):
                X = np.stack([I.vector_x(A.n, 1000 + 37 * i + j) for j in range(k)]).astype(np.float32)
                X64.append(X)
                Xs.append(torch.from_numpy(X if k > 1 else X[0]).cuda())
                Ys.append(torch.zeros((k, A.m) if k > 1 else (A.m,), dtype=torch.float32, device="cuda"))
            al, be = [1.0] * len(suite), [0.0] * len(suite)
            for _ in range(2):
                bd.run_batched(mats, Xs, Ys, al, be, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                bd.run_batched(mats, Xs, Ys, al, be, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            flops = sum(2.0 * A.nnz * k for _, _, A in suite)
            byts = 0.0     # bytes model of the passes actually run: the matrix once per pass
            passes = k // 4 + k % 4
            for (fam, dt, A), M in zip(suite, mats):
                st = M.stats()
                sv = 4 if dt == "f32" else 2
                byts += passes * (A.nnz * (sv + 1) + st["n_tiles"] * 21 + 4 * st["restore_cols_len"]) + \
                    4 * k * (A.n + A.m)
            errs = []
            for i, (fam, dt, A) in enumerate(suite):
                Y = Ys[i].cpu().numpy().reshape(k, A.m)
                rows = np.unique((I.uniform01(50 + i, 9, 64) * A.m).astype(np.int64))
                for j in range(min(k, 4)):
                    yref, sc = oracle.spmv_rows(A, X64[i][j].astype(np.float64), rows)
                    e = np.abs(Y[j][rows] - yref) / np.where(sc > 0, sc, 1.0)
                    errs.append(float(e.max()))
            out["results"].append({"k": k, "ms": round(ms, 4), "gflops": round(flops / (ms * 1e-3) / 1e9, 1),
                                   "passes": passes,
                                   "hbm_frac_bytes_model": round(byts / (ms * 1e-3) / 1e9 / peak, 4),
                                   "error_vs_fp64_oracle": {"max": max(errs), "median": float(np.median(errs)),
                                                            "results_checked": len(errs),
                                                            "sample": "64 seeded rows per result, up to 4 "
                                                                      "columns per matrix; error / sum |a x|"}})
            del Xs, Ys
    finally:
        for M in mats:
            M.close()
    return out


# The ablation of Sec. 4.4 (Fig. 12) as analysis options: I = intra-block data aggregation
# only (packed records, no column aggregation, one sub-block format: COO below 256 entries),
# II = + column aggregation and format selection (the paper's th0, th1, th2), full = II +
# the load balance of Algorithm 2 (I and II deal units to CTAs round-robin).
ABLATION = [
    ("CB-SpMV-I", dict(col_agg=0, th1=256, th2=256, load_balance=False)),
    ("CB-SpMV-II", dict(col_agg=-1, th1=32, th2=128, load_balance=False)),
    ("CB-SpMV (full)", dict(col_agg=-1, th1=32, th2=128, load_balance=True)),
]


def ablation_bench(bd, A, x, vec, dtype, stream, reps=200):
    import torch
    out = []
    xd = torch.from_numpy(x.astype(vec)).cuda()
    yd = torch.empty(A.m, dtype=xd.dtype, device="cuda")
    for name, opts in ABLATION:
        with bd.BlockedMatrix(A, value_dtype=dtype, stream=stream, **opts) as M:
            kt = M.time_kernels(xd, yd, reps, stream=stream)
            ms = kt["ms_main"] + kt["ms_combine"]
            st = M.stats()
            out.append({"config": name, "ms": round(ms, 4), "gflops": round(2.0 * A.nnz / (ms * 1e-3) / 1e9, 1),
                        "aggregated": bool(st["aggregated"]), "formats_coo_csr_dense": st["n_fmt"],
                        "worker_load_max_over_mean": round(st["worker_load_max"] / max(st["worker_load_mean"], 1), 3)})
    for i in range(1, len(out)):
        out[i]["speedup_vs_previous"] = round(out[i - 1]["ms"] / out[i]["ms"], 3)
    return out


def value_types_bench(bd, A, x, stream, reps=200):
    """The reduced value types (FP32 / BF16 / FP16 storage, FP32 x, y and accumulation) in
    both layouts on this workload: kernel time, the bytes model of the type over it, and
    that bandwidth as a fraction of the measured HBM copy bandwidth."""
    import torch
    peak, kind = load_peaks()
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    yd = torch.empty(A.m, dtype=torch.float32, device="cuda")
    out = {"hbm_peak_gbs": peak, "peak_kind": kind, "results": []}
    for dt in ("bf16", "f16", "f32"):
        for lay, name in ((1, "records"), (2, "lanes")):
            with bd.BlockedMatrix(A, value_dtype=dt, record_layout=lay, stream=stream) as M:
                kt = M.time_kernels(xd, yd, reps, stream=stream)
                ms = kt["ms_main"] + kt["ms_combine"]
                st = M.stats()
            gbs = st["algo_bytes_per_run"] / (ms * 1e-3) / 1e9
            out["results"].append({"dtype": dt, "layout": name, "ms": round(ms, 4),
                                   "gflops": round(2.0 * A.nnz / (ms * 1e-3) / 1e9, 1),
                                   "model_bytes": st["algo_bytes_per_run"], "model_gbs": round(gbs, 1),
                                   "frac_of_hbm": round(gbs / peak, 3),
                                   "stored_bytes": st["stream_bytes"] + st["metadata_bytes"]})
    return out


def step_distribution(run, stream, n: int, flush_buf=None):
    """Device time of n single steps, each between its own pair of events on the run's
    stream; with flush_buf, a buffer larger than L2 is overwritten before every step."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for i in range(n):
        if flush_buf is not None:
            flush_buf.fill_(float(i))
        evs[i][0].record(stream)
        run()
        evs[i][1].record(stream)
    stream.synchronize()
    t = sorted(a.elapsed_time(b) for a, b in evs)
    return {"mean_ms": round(sum(t) / n, 5), "median_ms": round(t[n // 2], 5), "min_ms": round(t[0], 5),
            "n": n}


def cusparse_reference(A, x, stream, steps: int, vec=np.float64):
    """cuSPARSE CSR SpMV (FP64, or FP32 for the reduced value types) through
    torch.sparse_csr_tensor on the same matrix and x: a library reference point, not part of
    this library's path."""
    import torch
    with torch.cuda.stream(stream):
        Acsr = torch.sparse_csr_tensor(torch.from_numpy(A.row_ptr.astype(np.int32)).cuda(),
                                       torch.from_numpy(A.col.astype(np.int32)).cuda(),
                                       torch.from_numpy(A.val.astype(vec)).cuda(), size=(A.m, A.n))
        xd = torch.from_numpy(x.astype(vec)).cuda()
        y = None
        for _ in range(5):
            y = torch.mv(Acsr, xd)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            y = torch.mv(Acsr, xd)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        yc = y.cpu().numpy()
        # sum_k |a_ik x_k| per row, the scale of both results' rounding errors
        Aabs = torch.sparse_csr_tensor(Acsr.crow_indices(), Acsr.col_indices(), Acsr.values().abs(),
                                       size=(A.m, A.n))
        sabs = torch.mv(Aabs, xd.abs()).double().cpu().numpy()
        del Aabs
    del Acsr
    return ms, yc, sabs


def error_vs_fp64_oracle(A, x, y, n_rows: int = 20000):
    """Normalised error |y_i - y_oracle_i| / sum_k |a_ik x_k| of the bench's result on a
    seeded sample of rows against the FP64 CPU oracle (original values and x)."""
    import oracle
    from paper_2605_18515_gb300 import inputs as I
    rows = np.unique((I.uniform01(11, 9, n_rows) * A.m).astype(np.int64))
    yref, s = oracle.spmv_rows(A, x, rows)
    err = np.abs(y[rows] - yref)
    norm = np.where(s > 0, err / np.where(s > 0, s, 1.0), np.where(err > 0, np.inf, 0.0))
    return {"max": float(norm.max()), "median": float(np.median(norm)), "rows": int(rows.size),
            "sample": f"{rows.size} seeded rows, error / sum_k |a_ik x_k|"}


# ---- preprocessing cost (Sec. 4.5): host analysis of a host CSR vs device analysis ------------
def device_analysis_bench(bd, torch, A, st_host, host_call_ms, ms_per_product, device, stream):
    """Wall time of cbspmv_analyze for the same matrix given as host arrays (analysis on the
    host cores, then upload) and as device arrays (analysis on the GPU); the second device
    call is reported (the first one also loads the analysis kernels)."""
    import types
    Ad = types.SimpleNamespace(m=A.m, n=A.n, row_ptr=torch.from_numpy(A.row_ptr).cuda(),
                               col=torch.from_numpy(A.col).cuda(), val=torch.from_numpy(A.val).cuda())
    torch.cuda.synchronize()
    calls = []
    for _ in range(2):
        t0 = time.perf_counter()
        Md = bd.BlockedMatrix(Ad, device=device, stream=stream)
        stream.synchronize()
        calls.append((time.perf_counter() - t0) * 1e3)
        sd = Md.stats()
        Md.close()
    del Ad
    torch.cuda.empty_cache()
    same = all(sd[k] == st_host[k] for k in st_host if k not in ("analyze_ms", "analyzed_on_device"))
    return {"host_analyze_ms": round(st_host["analyze_ms"], 2), "host_call_ms": round(host_call_ms, 2),
            "device_analyze_ms": round(sd["analyze_ms"], 2), "device_call_ms": round(calls[-1], 2),
            "device_first_call_ms": round(calls[0], 2), "analyzed_on_device": int(sd["analyzed_on_device"]),
            "same_plan_as_host": bool(same),
            "products_to_amortize_host": round(st_host["analyze_ms"] / ms_per_product, 1),
            "products_to_amortize_device": round(sd["analyze_ms"] / ms_per_product, 1),
            "note": "analyze_ms: the analysis itself; call_ms: the whole cbspmv_analyze call "
                    "(host path: analysis + upload of the lane arrays)"}


# ---- serving: Poisson mix of y = Ax and CG solves over a resident pool ------------------------
SERVE_POOLS = {
    # SPD 3D 7-point Laplacians (CG and y = Ax) and R-MAT matrices (y = Ax only)
    "small": {"lap": [32, 38, 44, 50, 56, 62], "rmat": [(14, 3), (15, 4), (16, 5)], "requests": 2000,
              "baseline_requests": 300},
    # the 32-matrix pool of the serving workload; "config5" serves 3,000 requests per served
    # run (the default, minutes on the box), "full" the workload's 10,000
    "config5": {"lap": list(range(32, 129, 6)), "rmat": [(s, 3 + k) for s in range(16, 21) for k in range(3)],
                "requests": 3000, "baseline_requests": 1500},
    "full": {"lap": list(range(32, 129, 6)), "rmat": [(s, 3 + k) for s in range(16, 21) for k in range(3)],
             "requests": 10000, "baseline_requests": 1500},
}


def serve_pool(name):
    from paper_2605_18515_gb300 import inputs as I
    spec = SERVE_POOLS[name]
    mats = [("lap%d" % g, I.laplacian3d(g), True) for g in spec["lap"]]
    mats += [("rmat%d_%d" % (sc, sd), I.rmat(sc, 16, seed=sd), False) for sc, sd in spec["rmat"]]
    return mats, spec


def serve_run(S, ids, mats, n_req, rate, seed):
    """Submits n_req requests to server S (70% y = Ax on any pool matrix, 30% CG to 1e-8
    on the SPD ones) at Poisson arrival times of the given rate (req/s; inf = all at once)
    and returns latency percentiles and throughput."""
    import threading
    rng = np.random.default_rng(seed)
    spd = [i for i, m in enumerate(mats) if m[2]]
    kinds = rng.random(n_req) < 0.3
    picks = [int(rng.choice(spd)) if k else int(rng.integers(len(mats))) for k in kinds]
    gaps = rng.exponential(1.0 / rate, n_req) if np.isfinite(rate) else np.zeros(n_req)
    arrivals = np.cumsum(gaps)
    inputs = {i: [np.random.default_rng(100 + 7 * i + j).uniform(-1, 1, A.n) for j in range(2)]
              for i, (_, A, _) in enumerate(mats)}
    st0 = S.stats()
    tickets = [None] * n_req
    t0 = time.perf_counter()

    def client():
        for r in range(n_req):
            dt = t0 + arrivals[r] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            i = picks[r]
            v = inputs[i][r & 1]
            if kinds[r]:
                tickets[r] = (S.submit_cg(ids[i], v, 1e-8)[0], True)
            else:
                tickets[r] = (S.submit_spmv(ids[i], v)[0], False)

    th = threading.Thread(target=client)
    th.start()
    lat, worst_res, fails = [], 0.0, 0
    for r in range(n_req):
        while tickets[r] is None:
            time.sleep(0.0005)
        tk, is_cg = tickets[r]
        res = S.wait(tk, 600000)
        if res["status"] != 0:
            fails += 1
        lat.append(res["t_done"] - res["t_submit"])
        if is_cg:
            worst_res = max(worst_res, res["rel_residual"])
    th.join()
    t_end = time.perf_counter()
    st = S.stats()
    lat = np.sort(np.array(lat)) * 1e3
    return {"requests": n_req, "req_per_s": round(n_req / (t_end - t0), 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3), "failed": fails, "cg_max_rel_residual": worst_res,
            "max_inflight_seen": st["max_inflight_seen"], "ticks": st["ticks"] - st0["ticks"],
            "launches": st["launches"] - st0["launches"]}


def serve_bench(pool_name, seed=5, inner_steps=16, max_cg=0, inner_tol=1e-6):
    """Both modes' burst capacity; then Poisson arrivals at one common rate (70% of the
    one-at-a-time capacity, a load both modes sustain) for both, and the served mode also at
    70% of its own capacity."""
    from paper_2605_18515_gb300 import binding as bd
    mats, spec = serve_pool(pool_name)
    served_opts = dict(max_inflight=64, cg_inner_dtype="bf16", inner_tol=inner_tol, memory_budget=8 << 30,
                       inner_steps=inner_steps, max_inflight_cg=max_cg)
    base_opts = dict(max_inflight=1, cg_inner_dtype="f64", inner_tol=1e-9, memory_budget=8 << 30)
    with bd.Server(**base_opts) as S:
        ids = [S.register(A) for _, A, _ in mats]
        bcap = serve_run(S, ids, mats, spec["baseline_requests"], float("inf"), seed)
        common = 0.7 * bcap["req_per_s"]
        bload = serve_run(S, ids, mats, spec["baseline_requests"], common, seed + 1)
    with bd.Server(**served_opts) as S:
        ids = [S.register(A) for _, A, _ in mats]
        cap = serve_run(S, ids, mats, spec["requests"], float("inf"), seed)
        same = serve_run(S, ids, mats, spec["requests"], common, seed + 1)
        load = serve_run(S, ids, mats, spec["requests"], 0.7 * cap["req_per_s"], seed + 2)
    out = {"pool": f"{len(spec['lap'])} SPD 3D Laplacians {spec['lap'][0]}^3..{spec['lap'][-1]}^3 + "
                   f"{len(spec['rmat'])} R-MAT (scales {spec['rmat'][0][0]}-{spec['rmat'][-1][0]})",
           "mix": "70% y=Ax (FP64), 30% CG to 1e-8 relative residual",
           "served": {"mode": "continuous batching, 64 in flight, BF16-value CG with FP64 refinement, "
                              f"{inner_steps} inner CG iterations per tick, inner tolerance {inner_tol:g} "
                              "(later corrections stop at the gap to the outer tolerance), "
                              f"{max_cg or 64} CG solves in flight at most",
                      "capacity": cap, "poisson_same_load": same, "poisson_at_70pct": load},
           "one_at_a_time_fp64": {"mode": "one request at a time, FP64 products and FP64 CG",
                                  "capacity": bcap, "poisson_same_load": bload},
           "same_load_req_per_s": round(common, 1),
           "capacity_ratio": round(cap["req_per_s"] / max(bcap["req_per_s"], 1e-9), 2),
           "p99_ratio_same_load": round(same["p99_ms"] / max(bload["p99_ms"], 1e-9), 3)}
    out["requests_per_served_run"] = spec["requests"]
    if pool_name == "config5":
        out["note"] = ("default run: the 32-matrix pool with 3,000 requests per served run and 1,500 per "
                       "one-at-a-time run, to keep the bench within minutes; --serve-full serves 10,000")
    elif pool_name == "small":
        out["note"] = "9-matrix pool (--serve-pool small)"
    return out


def run_reference(args, A, x, ws, rank):
    """The reference arm: the CPU oracle as it stands, on the host cores of this machine."""
    if rank != 0:
        return
    import oracle
    # each step is a bounded sample of the workload: the first rows holding ~1/8 of the
    # nonzeros (the full product takes the single-threaded oracle 0.06-0.16 s, too long for
    # thousands of steps); the rate, GFLOP/s, is the same quantity as the GPU arm's
    cut = int(np.searchsorted(A.row_ptr, A.nnz // 8))
    sub = type(A)(cut, A.n, A.row_ptr[:cut + 1].copy(), A.col[:A.row_ptr[cut]], A.val[:A.row_ptr[cut]])
    for _ in range(args.warmup):
        oracle.spmv(sub, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.spmv(sub, x)
    dt = time.perf_counter() - t0
    gf = 2.0 * sub.nnz * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(gf, 4), "unit": "GFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                       "sample": f"each step multiplies rows 0..{cut} of the workload's matrix "
                                 f"({sub.nnz} of {A.nnz} nonzeros), single-threaded oracle"},
            "cpu_baseline": {"value": round(gf, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": f"rows 0..{cut} ({sub.nnz} nonzeros, 1/8 of the matrix) per step"},
            "e2e": {"value": round(gf, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="fem3x3_band_1m")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dtype", choices=["f64", "f32", "bf16", "f16"], default="f64",
                    help="storage type of the matrix values (reduced types: FP32 x, y and accumulation)")
    ap.add_argument("--dist-steps", type=int, default=200, help="single steps timed one by one")
    ap.add_argument("--no-cusparse", action="store_true")
    ap.add_argument("--cusparse-steps", type=int, default=200)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-multi", action="store_true", help="skip the k right-hand-side measurement")
    ap.add_argument("--no-ablation", action="store_true", help="skip the ablation (Sec. 4.4) measurement")
    ap.add_argument("--no-spmm", action="store_true", help="skip the tensor-core multi-vector measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-matrix batched measurement")
    ap.add_argument("--no-value-types", action="store_true", help="skip the reduced value types measurement")
    ap.add_argument("--no-device-analysis", action="store_true",
                    help="skip the device-side analysis measurement (analysis block)")
    ap.add_argument("--layout", choices=["default", "records", "lanes"], default="default",
                    help="layout of the timed handle: default (lane streams for every value type), "
                         "records, or lane streams")
    ap.add_argument("--batched-full", action="store_true", help="batched matrices up to 1e6 rows (default 2e5)")
    ap.add_argument("--serve-full", action="store_true",
                    help="serving measurement with 10,000 requests per served run (the 32-matrix pool)")
    ap.add_argument("--serve-pool", choices=["small", "config5", "full"], default="config5",
                    help="serving pool: 9 small matrices, or the 32-matrix pool with 3,000 (config5) or "
                         "10,000 (full) requests per served run")
    ap.add_argument("--serve-max-cg", type=int, default=0,
                    help="CG solves in flight at most in the served mode (0: no separate limit)")
    ap.add_argument("--serve-inner-steps", type=int, default=16,
                    help="inner CG iterations per tick of the served mode (1..64)")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="ncu DRAM bytes per launch of the timed kernel, if captured for this build")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_env()

    from paper_2605_18515_gb300 import inputs as I
    A, x = I.config_matrix(args.workload)

    if args.impl == "reference":
        run_reference(args, A, x, ws, rank)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2605_18515_gb300 import build
    build.build()
    from paper_2605_18515_gb300 import binding as bd

    lp = args.dtype != "f64"
    vec = np.float32 if lp else np.float64
    tvec = torch.float32 if lp else torch.float64
    esz = 4 if lp else 8
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        t_an = time.perf_counter()
        M = bd.BlockedMatrix(A, device=local, stream=stream, value_dtype=args.dtype,
                             record_layout={"default": 0, "records": 1, "lanes": 2}[args.layout])
        stream.synchronize()
        host_call_ms = (time.perf_counter() - t_an) * 1e3
        st = M.stats()
        xd = torch.from_numpy(x.astype(vec)).cuda()
        yd = torch.empty(A.m, dtype=tvec, device="cuda")
        for _ in range(args.warmup):
            M.run(xd, yd, 1.0, 0.0, stream=stream)
        stream.synchronize()
        M.check_device(stream)
        # the timed region repeats the block of `steps` products until it lasts ~1 s, so that
        # the clock samples fall inside it (ms_per_step is the average over all repeats); the
        # time per product is estimated after the warm-up from a short untimed batch, the
        # slowest rank's estimate giving every rank the same count
        n_cal = max(3, min(args.steps, 50))
        wa, wb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        wa.record(stream)
        for _ in range(n_cal):
            M.run(xd, yd, 1.0, 0.0, stream=stream)
        wb.record(stream)
        stream.synchronize()
        est_ms = wa.elapsed_time(wb) / n_cal
        repeats = timed_repeats(args.steps, max_over_ranks([est_ms], dist, "cuda")[0])
        # the FP64 FMA roofline, measured on this device now (before the timed region)
        fma = bd.measure_fp64_fma(local, stream) if not lp else None

        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        w0 = time.time()
        ev0.record(stream)
        for _ in range(args.steps * repeats):
            M.run(xd, yd, 1.0, 0.0, stream=stream)
        ev1.record(stream)
        ev1.synchronize()
        torch.cuda.synchronize()
        w1 = time.time()
        if dist:
            dist.barrier()
        time.sleep(0.25)
        sampler.stop()
        ms = ev0.elapsed_time(ev1) / (args.steps * repeats)
        M.check_device(stream)

        # end to end through the C ABI from pinned host memory
        xh = torch.from_numpy(x.astype(vec)).pin_memory().numpy()
        yh = torch.empty(A.m, dtype=tvec).pin_memory().numpy()
        for _ in range(3):
            M.run_host(xh, yh, 1.0, 0.0, stream=stream)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            M.run_host(xh, yh, 1.0, 0.0, stream=stream)
        e2e_ms = 1e3 * (time.perf_counter() - t0) / args.e2e_steps

        # device time of each kernel of a step (events around every launch, same stream)
        kt = M.time_kernels(xd, yd, min(args.steps, 1000), stream=stream)
        # per-step distribution, without and with an L2 flush before every step
        run1 = lambda: M.run(xd, yd, 1.0, 0.0, stream=stream)
        per_step = step_distribution(run1, stream, args.dist_steps)
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
        per_step_flushed = step_distribution(run1, stream, args.dist_steps, flush)
        del flush
        y_ours = yd.cpu().numpy().astype(np.float64)
        multi = multi_rhs_bench(M, A, x, vec, stream) if not args.no_multi else None
        spmm = spmm_bench(bd, A, x, stream) if not args.no_spmm else None
        batched = batched_bench(bd, stream, full=args.batched_full) if not args.no_batched else None
        abl = ablation_bench(bd, A, x, vec, args.dtype, stream) if not args.no_ablation else None
        M.check_device(stream)
        sms = torch.cuda.get_device_properties(local).multi_processor_count

    cus = None
    if rank == 0 and not args.no_cusparse:
        cus_ms, y_cus, sabs = cusparse_reference(A, x, stream, args.cusparse_steps, vec)
        # Both results lie within (storage roundoff + gamma_{k+10} of their arithmetic) of
        # sum_k a_ik x_k, relative to sum_k |a_ik x_k|: cuSPARSE rounds the values to FP32
        # (or keeps FP64), this library to the --dtype format; both add in FP32 (FP64).
        u_store = {"f64": 0.0, "f32": 2.0 ** -24, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}[args.dtype]
        u_cus = 2.0 ** -24 if lp else 0.0
        u_ar = 2.0 ** -24 if lp else 2.0 ** -53
        kk = np.diff(A.row_ptr).astype(np.float64) + 10.0
        gam = kk * u_ar / (1.0 - kk * u_ar)
        bound = (u_store + u_cus + 2.0 * gam) * sabs * 1.01
        agree = bool(np.all(np.abs(y_cus.astype(np.float64) - y_ours) <= bound))
        cus = {"gflops": round(2.0 * A.nnz / (cus_ms * 1e-3) / 1e9, 3), "ms_per_step": round(cus_ms, 5),
               "csr_model_bytes": int((A.m + 1) * 8 + A.nnz * (4 + esz) + A.n * esz + A.m * esz),
               "api": "torch.mv on torch.sparse_csr_tensor (cuSPARSE SpMV, CSR, %s)" % ("FP32" if lp else "FP64"),
               "agrees_with_ours": agree,
               "agreement_bound": "per row (u_storage + u_cusparse_values + 2 gamma_{k+10}) sum_k |a_ik x_k|"}

    ms_max, e2e_max = max_over_ranks([ms, e2e_ms], dist, "cuda")

    flops = float(st["flops_per_run"])
    gflops_total = job_gflops(ws, flops, ms_max)
    algo_bytes = float(st["algo_bytes_per_run"])
    gbs = algo_bytes / (ms * 1e-3) / 1e9
    peak, peak_kind = load_peaks()

    if rank == 0:
        cpu = None
        err = None
        if not args.no_cpu_baseline and ws == 1:
            gf, sample = oracle_sample_gflops(A, x)
            gfa, threads, sample_a = oracle_allcore_gflops(A, x)
            cpu = {"value": round(gf, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample,
                   "all_cores": {"value": round(gfa, 4), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                                 "sample": sample_a}}
            err = error_vs_fp64_oracle(A, x, y_ours)
        clocks = sampler.summary(w0, w1)
        fmax = clocks.get("sm_max_mhz") or 2070.0
        if fma:
            peak_alu = round(fma["gflops"], 1)
            peak_derived = round(fp64_peak_gflops(sms, fmax, fma["cycles_per_warp_fma"]), 1)
        k_ms = kt["ms_main"]
        traffic = args.traffic_bytes if args.traffic_bytes is not None else \
            (RECORD_KERNEL_TRAFFIC.get((args.workload, args.dtype)) if lp and not st["lane_layout"] else
             measured_traffic(bd.version(), args.workload, args.dtype, bool(st["lane_layout"])))
        k_gf = flops / (k_ms * 1e-3) / 1e9
        k_gbs = algo_bytes / (k_ms * 1e-3) / 1e9
        if lp:
            kname = ("spmv_lanes_kernel<%s>" if st["lane_layout"] else "spmv_kernel<%s>") % args.dtype
            roof = {"bound": "hbm", "kernel": kname, "achieved": round(k_gbs, 2),
                    "peak": peak, "unit": "GB/s", "frac": round(k_gbs / peak, 4), "peak_kind": peak_kind,
                    "traffic": traffic, "kernel_ms": round(k_ms, 5),
                    "combine_ms": round(kt["ms_combine"], 5), "bytes_per_launch": int(algo_bytes),
                    "gflops": round(k_gf, 2),
                    "note": "FP32 FMA is far from binding; the bytes model (values + coordinates + "
                            "metadata + x + y + restore_cols) over the kernel's time vs measured copy bandwidth"}
        else:
            roof = {"bound": "alu", "kernel": "spmv_lanes_kernel<f64>", "achieved": round(k_gf, 2),
                    "peak": peak_alu, "unit": "GFLOP/s", "frac": round(k_gf / peak_alu, 4),
                    "peak_kind": "measured: FP64 FMA chain kernel on this GPU in this run "
                                 "(cbspmv_measure_fp64_fma)",
                    "peak_derived_at_max_clock": peak_derived,
                    "cycles_per_warp_fp64_fma": round(fma["cycles_per_warp_fma"], 2),
                    "traffic": traffic,
                    "kernel_ms": round(k_ms, 5), "combine_ms": round(kt["ms_combine"], 5),
                    "flops_per_launch": int(flops),
                    "note": "one FP64 FMA per stored entry: bound by the FP64 FMA pipe; derived peak = "
                            "SMs x 4 sub-partitions x 32 lanes / (cycles per warp FMA) x 2 flops x max SM "
                            "clock; HBM view below",
                    "hbm": {"achieved": round(k_gbs, 2), "peak": peak, "unit": "GB/s",
                            "frac": round(k_gbs / peak, 4), "peak_kind": peak_kind,
                            "bytes_per_launch": int(algo_bytes)}}
        line = {
            "metric": METRIC, "value": round(gflops_total, 3), "unit": "GFLOP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.dtype if not lp else f"{args.dtype} values, f32 x/y/accumulate",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                       "m": A.m, "n": A.n, "nnz": A.nnz, "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (packed stream %.2f GB vs 129 MB L2); no flush"
                             % (st["stream_bytes"] / 1e9),
                       "aggregated": bool(st["aggregated"]), "tiles": st["n_tiles"],
                       "formats_coo_csr_dense": st["n_fmt"], "units": st["n_units"],
                       "split_units": st["n_split_units"], "entry_mode_units": st["n_entry_mode_units"],
                       "xseq_units": st["n_xseq_units"]},
            "hbm_gbs": round(gbs, 2),
            "roofline": roof,
            "per_step": per_step,
            "per_step_l2_flushed": per_step_flushed,
            "e2e": {"value": round(job_gflops(ws, flops, e2e_max), 3), "unit": "GFLOP/s",
                    "ms_per_step": round(e2e_max, 4), "h2d_bytes_per_step": esz * A.n,
                    "d2h_bytes_per_step": esz * A.m, "api": "cbspmv_run_host"},
            "gpu_launches": args.steps * repeats * kt["launches_per_run"],
            "timed_region": {"repeats": repeats, "products": args.steps * repeats,
                             "seconds": round(args.steps * repeats * ms * 1e-3, 3),
                             "note": "the block of `steps` products repeated until the region lasts "
                                     "~1 s; ms_per_step is the average over all of them"},
            "clocks": clocks,
            "analyze_ms": round(st["analyze_ms"], 1),
        }
        if cpu:
            line["cpu_baseline"] = cpu
        if cus:
            line["cusparse_csr"] = cus
        if multi:
            line["multi_rhs"] = {"api": "cbspmv_run_multi (FP64: one column per pass; reduced types: passes "
                                        "of 4 vectors)", "results": multi}
            if not lp and ws == 1:
                with bd.BlockedMatrix(A, value_dtype="bf16", stream=stream) as Mb:
                    line["multi_rhs"]["bf16_lane_streams"] = multi_rhs_bench(Mb, A, x, np.float32, stream)
        if spmm:
            line["multi_rhs_tensor"] = spmm
        if batched:
            line["batched"] = batched
        if abl:
            line["ablation"] = abl
        if not lp and ws == 1 and not args.no_device_analysis:
            line["analysis"] = device_analysis_bench(bd, torch, A, st, host_call_ms, ms_max, local, stream)
        if not lp and ws == 1 and not args.no_value_types:
            line["value_types"] = value_types_bench(bd, A, x, stream)
        if not args.no_serve and ws == 1:
            line["serving"] = serve_bench("full" if args.serve_full else args.serve_pool, inner_steps=args.serve_inner_steps,
                                          max_cg=args.serve_max_cg)
        if err:
            line["error_vs_fp64_oracle"] = err
        print(json.dumps(line), flush=True)
    M.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
