#!/usr/bin/env python
"""Benchmark of direct TSQR on GB300 (Benson, Gleich, Demmel, arXiv:1301.1071).

Default workload: the stability-sweep matrix, m = 8,000,000 x n = 25, FP64,
A = G diag(sigma) V^T with sigma log-spaced from 1 to 1e-15 (synthetic,
seeded).  One step = one direct-TSQR forward pass (Step 1 local Householder of
every row block, the Step-2 tree of Alg. 2 with the top QR and sign fix, and
Step 3 Q formation) on inputs already resident in HBM.  Inputs (1.6 GB) are
larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload sweep|small] [--no-extras]

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle (the
plain FP64 Householder QR) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import tsqr_inputs as ti  # noqa: E402

METRIC = "direct-TSQR rows/s and HBM GB/s (fwd; fwd+bwd) at stated ||Q^TQ-I||, 1 GB300"
HBM_PEAK_FALLBACK = 6800.0  # GB/s, used only when MEASURED_PEAKS.json is absent
FP64_PEAK_GFLOPS = 1250.0   # nominal GB300 FP64 rate (152 SMs x ~2 DFMA/clk x 2 flop x 2.07 GHz)
FP32_PEAK_GFLOPS = 80540.0  # nominal GB300 FP32 CUDA-core rate (152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz)

# Algorithmic passes over the tall matrix (m n s bytes each) per call: read A
# and write Y (Step 1), read Y and write Q (Step 3); Cholesky QR and indirect
# TSQR read A twice and write Q once; refinement repeats the method; the
# adjoint reads Q and dQ for the Gram, then Q and dQ again and writes dA.
# The R-only and singular-value-only paths read A once.
ALG_PASSES = {"direct": 4, "direct_native": 4, "cholqr": 3, "cholqr_ir": 6, "indirect": 3, "indirect_ir": 6, "backward": 5,
              "r_only": 1, "svd_values": 1}

# The paper's own direct-TSQR job times (Sec. V-B, Table VI), reported
# beside the GPU figures as context only: another method implementation,
# machine and matrix size.  The cluster (Sec. V): Hadoop MapReduce on 10
# nodes / 40 cores, one Intel Core i7-960 at 3.2 GHz, 24 GB of RAM and six
# 2-TB disks per node, Gigabit Ethernet; Python (Dumbo) over Hadoop
# streaming, every pass reading or writing HDFS.
_PAPER_JOBS = [(4_000_000_000, 4, 6128), (2_500_000_000, 10, 4035), (600_000_000, 25, 1910),
               (500_000_000, 50, 3090), (150_000_000, 100, 2154)]
PAPER_CONTEXT = {
    "source": "Sec. V-B, Table VI (job times, direct TSQR)",
    "machine": "Hadoop MapReduce, 10 nodes / 40 cores (Intel Core i7-960 3.2 GHz, 24 GB RAM, 6 x 2 TB disks "
               "per node, Gigabit Ethernet), Python/Dumbo over Hadoop streaming, data on HDFS",
    "direct_tsqr": [{"m": m_, "n": n_, "job_s": t_, "rows_s": m_ / t_} for m_, n_, t_ in _PAPER_JOBS],
    "note": "context only: not the target and not this workload",
}

WORKLOADS = {
    "sweep": dict(m=8_000_000, n=25, dtype="f64", kappa=1e15, block_rows=0, seed=ti.SEED_SWEEP,
                  name="stability-sweep matrix 8,000,000x25 FP64, A=G diag(sigma) V^T, "
                       "sigma log-spaced 1..1e-15 (kappa 1e15)"),
    "small": dict(m=100_000, n=10, dtype="f64", kappa=None, block_rows=1000, seed=ti.SEED_SMALL,
                  name="100,000x10 FP64 i.i.d. N(0,1), row blocks of 1,000"),
    "mixed": dict(m=50_000_000, n=50, dtype="f32", kappa=None, colscale=1e-4, block_rows=0, seed=ti.SEED_MIXED,
                  name="50,000,000x50 FP32 N(0,1) x column factors 1..1e-4"),
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, device=None) -> float:
    """Max of a scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(rows_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job rows/s of `world` replicas, each factoring `rows_per_rank`
    rows per step, timed by the slowest rank."""
    return rows_per_rank * world * steps / (max_ms * 1e-3)


def make_input(w, rows=None):
    """The workload matrix, or only its first `rows` rows."""
    if w.get("colscale"):
        return ti.column_scaled(w["m"] if rows is None else rows, w["n"], w["colscale"], w["seed"],
                                dtype=np.float32 if w["dtype"] == "f32" else np.float64)
    elif w["kappa"] is None:
        A = ti.gaussian(w["m"], w["n"], w["seed"], rows=rows)
    else:
        A = ti.conditioned(w["m"], w["n"], w["kappa"], w["seed"], rows=rows)
    return A.astype(np.float32) if w["dtype"] == "f32" else A


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", HBM_PEAK_FALLBACK)), "measured"
    return HBM_PEAK_FALLBACK, "fallback"


# Sources that define (and plan the launch of) the two kernels whose DRAM
# traffic bench.py reports from a committed ncu capture.
KERNEL_SOURCES = ["qr_kernels.cuh", "device.cuh", "df64.cuh", "layout.cuh", "kern_inst.cuh", "kern_f64.cu",
                  "kern_df64.cu", "kern_f32.cu", "kern_r_f64.cu", "tiles_f64.h", "tiles_f32.h", "plan.cu", "plan.h",
                  "oz_kernels.cuh", "kern_oz.cu", "tcgen05.cuh", "chunks.cuh"]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1301_1071_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{kernel}@{workload}")
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return float(e["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"tsqr_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_rate(A_host: np.ndarray, threads: int, target_s: float, max_rows: int):
    """rows/s of the oracle's thin QR (Q and R) on the first rows of A_host,
    the sample grown until it takes about target_s seconds."""
    import oracle
    oracle.set_num_threads(threads)
    rows = min(100_000, A_host.shape[0])
    while True:
        sample = np.asarray(A_host[:rows], dtype=np.float64)
        t0 = time.perf_counter()
        oracle.householder_qr(sample)
        t = time.perf_counter() - t0
        if t >= target_s / 3 or rows >= min(max_rows, A_host.shape[0]):
            return rows, t
        rows = int(min(max_rows, A_host.shape[0], rows * target_s / max(t, 1e-3)))


def cpu_baseline(A_host: np.ndarray, target_s: float = 10.0, max_rows: int = 8_000_000):
    """The oracle (plain FP64 Householder QR with explicit Q) on a bounded row
    sample of the same matrix: on all host cores (its loops over independent
    columns in parallel, bit-identical to the serial oracle), and serial."""
    n = A_host.shape[1]
    cores = os.cpu_count() or 1
    rows_p, t_p = _oracle_rate(A_host, cores, target_s, max_rows)
    rows_s, t_s = _oracle_rate(A_host, 1, target_s, max_rows)
    return {"value": rows_p / t_p, "unit": "rows/s", "cores": cores, "kind": "oracle",
            "sample": f"first {rows_p:,} rows x {n} of the workload matrix, one thin QR (Q and R) on "
                      f"{cores} threads, {t_p:.1f} s",
            "serial": {"value": rows_s / t_s, "unit": "rows/s", "cores": 1,
                       "sample": f"first {rows_s:,} rows x {n}, one thread, {t_s:.1f} s"},
            "host_cores": cores}


def _timed_rows(fn, make, target_s: float, rows0: int, max_rows: int):
    """rows/s of fn(sample) on make(rows) rows, the sample grown until one
    call takes about target_s / 3 seconds (at most max_rows rows)."""
    rows = min(rows0, max_rows)
    while True:
        X = make(rows)
        t0 = time.perf_counter()
        fn(X)
        t = time.perf_counter() - t0
        if t >= target_s / 3 or rows >= max_rows:
            return rows, t
        rows = int(min(max_rows, rows * target_s / max(t, 1e-3)))


def cpu_config_baselines(target_s: float = 3.0):
    """The oracle on all host cores at each of the other configurations (a
    bounded row sample of each, drawn with the configuration's recipe on the
    host; the device runs draw theirs on the device), the serial oracle at
    the 100,000 x 10 configuration, numpy's LAPACK QR (a library CPU
    baseline, comparison only) and the peak resident memory.  Each entry
    reports an error instead of raising."""
    import resource

    import oracle
    cores = os.cpu_count() or 1
    out = {}

    def gram_pair(A):
        Q, R = oracle.householder_qr(A)
        g = np.random.default_rng(ti.SEED_GRAD)
        oracle.qr_backward(Q, R, g.standard_normal(A.shape), np.triu(g.standard_normal((A.shape[1], A.shape[1]))))

    entries = [
        ("small_100kx10", 100_000, lambda r: ti.gaussian(100_000, 10, ti.SEED_SMALL, rows=r), oracle.householder_qr,
         "thin QR (Q and R)"),
        ("mixed_50Mx50_upcast", 50_000_000,
         lambda r: ti.column_scaled(r, 50, 1e-4, ti.SEED_MIXED).astype(np.float32).astype(np.float64),
         oracle.householder_qr, "thin QR (Q and R) of the FP32 matrix upcast"),
        ("svd_20Mx100", 20_000_000, lambda r: ti.power_spectrum(20_000_000, 100, ti.SEED_SVD, rows=r), oracle.svd,
         "SVD via thin QR and the SVD of R"),
        ("grad_4Mx64", 4_000_000, lambda r: ti.gaussian(4_000_000, 64, ti.SEED_GRAD, rows=r), gram_pair,
         "thin QR + adjoint"),
    ]
    for name, m_full, make, fn, what in entries:
        try:
            oracle.set_num_threads(cores)
            rows, t = _timed_rows(fn, make, target_s, 20_000, m_full)
            e = {"value": rows / t, "unit": "rows/s", "cores": cores, "kind": "oracle", "op": what,
                 "sample": f"first {rows:,} rows of the {m_full:,}-row configuration, {t:.2f} s"}
            if name == "small_100kx10":
                oracle.set_num_threads(1)
                rows1, t1 = _timed_rows(fn, make, target_s, 20_000, m_full)
                e["serial"] = {"value": rows1 / t1, "unit": "rows/s", "cores": 1,
                               "sample": f"first {rows1:,} rows, one thread, {t1:.2f} s"}
            out[name] = e
        except Exception as ex:  # reported, not fatal
            out[name] = {"error": f"{type(ex).__name__}: {ex}"}
        finally:
            oracle.set_num_threads(cores)
    try:
        make = lambda r: ti.conditioned(8_000_000, 25, 1e15, ti.SEED_SWEEP, rows=r)
        rows, t = _timed_rows(lambda X: np.linalg.qr(X, mode="reduced"), make, target_s, 100_000, 8_000_000)
        out["numpy_lapack_qr_8Mx25"] = {"value": rows / t, "unit": "rows/s", "kind": "library (comparison only)",
                                        "sample": f"first {rows:,} rows x 25 of the sweep matrix, {t:.2f} s"}
    except Exception as ex:  # reported, not fatal
        out["numpy_lapack_qr_8Mx25"] = {"error": f"{type(ex).__name__}: {ex}"}
    out["memory_peak_mb"] = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss / 1024.0
    return out


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_num_threads(cores)
    rows = min(w["m"], 2_000_000)
    sample = np.asarray(make_input(w, rows=rows), dtype=np.float64)
    for _ in range(args.warmup):
        oracle.householder_qr(sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.householder_qr(sample)
    dt = time.perf_counter() - t0
    value = rows * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["name"], "m": w["m"], "n": w["n"]},
        "cpu_baseline": {"value": value, "unit": "rows/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {rows:,} rows x {w['n']} of the workload matrix per step, "
                                   f"{cores} threads"},
        "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep", choices=sorted(WORKLOADS))
    ap.add_argument("--no-extras", action="store_true", help="skip comparators / fwd+bwd / cpu baseline")
    ap.add_argument("--m", type=int, default=0, help="override the row count (profiling a smaller case)")
    ap.add_argument("--prec", default="auto", choices=["native", "df64", "tf32x3", "ozaki", "auto"],
                    help="arithmetic of Steps 1 and 3 (df64, ozaki: FP64 data; tf32x3: FP32 data; auto: the "
                         "library's choice, the Ozaki form for FP64 data at n <= 32)")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.m:
        w["m"] = args.m
        w["name"] = w["name"].replace(f"{WORKLOADS[args.workload]['m']:,}", f"{args.m:,}")
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import torch.distributed as dist
    import paper_1301_1071_gb300 as T

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl")

    def barrier():
        if ws > 1:
            dist.barrier()

    m, n = w["m"], w["n"]
    A_host = make_input(w)
    gb = A_host.nbytes / 1e9
    A = torch.from_numpy(A_host).to(dev)
    Q = torch.empty_like(A)
    R = torch.empty(n, n, dtype=torch.float64, device=dev)
    work = torch.empty(T.workspace_size(T.OP_DIRECT, m, n, A.dtype, w["block_rows"], prec=args.prec),
                       dtype=torch.uint8, device=dev)
    bench_kw = dict(block_rows=w["block_rows"], work=work, out=(Q, R), check=False, prec=args.prec)

    for _ in range(args.warmup):
        T.direct(A, **bench_kw)
    torch.cuda.synchronize()
    T.direct(A, block_rows=w["block_rows"], work=work, out=(Q, R), check=True, prec=args.prec)  # raises on error

    # ---- device-resident timed region
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    for e in (x for step in evs for x in step):
        e.record()  # torch creates the CUDA event on first record; the library then re-records it
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.3)
    start.record()
    for k in range(args.steps):
        T.direct(A, stage_events=evs[k], **bench_kw)
    end.record()
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    total_ms = reduce_max(start.elapsed_time(end), dev)
    ms_step = total_ms / args.steps
    st1 = [e[0].elapsed_time(e[1]) for e in evs]
    st2 = [e[1].elapsed_time(e[2]) for e in evs]
    st3 = [e[2].elapsed_time(e[3]) for e in evs]
    s1, s2, s3 = statistics.mean(st1), statistics.mean(st2), statistics.mean(st3)
    rows_s = replica_throughput(m, args.steps, ws, total_ms)
    elem = 8 if A.dtype == torch.float64 else 4
    alg_bytes = ALG_PASSES["direct"] * m * n * elem
    gbs = alg_bytes / (ms_step * 1e-3) / 1e9
    hbm_peak, peak_src = load_peaks()

    resolved = T.plan_info(T.OP_DIRECT, m, n, A.dtype, w["block_rows"], prec=args.prec)["prec"]
    # dominant kernel: Step 1 (k_local_qr) or Step 3 (k_form_q); both are
    # FMA-bound (binary64 unit for FP64 data, binary32 for FP32 and for
    # double-float compute): 2 m n^2 algorithmic flops per launch
    dom, dom_ms = ("k_local_qr", s1) if s1 >= s3 else ("k_form_q", s3)
    flops = 2.0 * m * n * n
    achieved = flops / (dom_ms * 1e-3) / 1e9
    if elem == 8 and args.prec in ("native", "ozaki", "auto"):
        peak, alu_src = FP64_PEAK_GFLOPS, "nominal FP64 rate (recipe table); probe measured 1196 GFLOP/s"
    else:
        peak, alu_src = FP32_PEAK_GFLOPS, "nominal FP32 CUDA-core rate; probe measured 74.8 TFLOP/s"
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                "frac": achieved / peak, "traffic": load_traffic(dom, args.workload),
                "kernel": dom, "peak_source": alu_src,
                "hbm_view": {"achieved_gbs": 2 * m * n * elem / (dom_ms * 1e-3) / 1e9, "peak_gbs": hbm_peak,
                             "frac": 2 * m * n * elem / (dom_ms * 1e-3) / 1e9 / hbm_peak,
                             "peak_source": peak_src}}

    # ---- accuracy at the stated kappa: the library's compensated (Dot2)
    #      device sums, accurate at the 1e-15 level for any m
    acc = T.accuracy(Q, R, A)
    orth2, resF = acc["orth_2"], acc["res_F"]

    # ---- end to end through the host-buffer entry point (tsqr_direct_host):
    #      pinned host A in, Q and R back to pinned host buffers, the copies
    #      overlapped with the kernels chunk by chunk (a second stream)
    Ah = torch.from_numpy(A_host).pin_memory()
    Qh = torch.empty_like(Ah).pin_memory()
    Rh = torch.empty(n, n, dtype=torch.float64).pin_memory()
    dbuf = Q  # the device-resident run's Q buffer serves as the device copy of A / Y / Q
    work_h = torch.empty(T.workspace_size(T.OP_DIRECT_HOST, m, n, A.dtype, w["block_rows"], prec=args.prec),
                         dtype=torch.uint8, device=dev)
    copy_stream = torch.cuda.Stream(device=dev)
    host_kw = dict(block_rows=w["block_rows"], out=(Qh, Rh), dbuf=dbuf, work=work_h, copy_stream=copy_stream,
                   check=False, prec=args.prec)
    T.direct_host(Ah, **dict(host_kw, check=True))  # raises on error
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k_e2e = max(3, args.steps // 2)
    barrier()
    e0.record()
    for _ in range(k_e2e):
        T.direct_host(Ah, **host_kw)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    e2e_ms = reduce_max(e0.elapsed_time(e1), dev)
    e2e = {"value": replica_throughput(m, k_e2e, ws, e2e_ms), "unit": "rows/s",
           "h2d_bytes_per_step": m * n * elem, "d2h_bytes_per_step": m * n * elem + n * n * 8,
           "api": "tsqr_direct_host (pinned host A, Q, R; copies overlapped with the kernels)"}

    launches = T.launch_count(T.OP_DIRECT, m, n, A.dtype, w["block_rows"], prec=args.prec) * args.steps
    line = {
        "metric": METRIC, "value": rows_s, "unit": "rows/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("df64 (binary64 data, pairs of binary32 in Steps 1 and 3, binary64 tree)" if resolved == "df64"
                  else "f64 (binary64 Householder and tree; the Step-3 product and the T factors' Gram as "
                       "error-free Ozaki splits on tcgen05: 56/64-bit fixed point, exact binary32 accumulation, "
                       "one rounding to binary64)" if resolved == "ozaki"
                  else "f32 (Step 3 product as 3xTF32 on the tensor cores)" if resolved == "tf32x3"
                  else ("f64" if elem == 8 else "f32")),
        "data": "synthetic",
        "config": {"workload": w["name"], "m": m, "n": n, "block_rows": w["block_rows"] or "auto",
                   "prec": args.prec,
                   "plan": T.plan_info(T.OP_DIRECT, m, n, A.dtype, w["block_rows"], prec=args.prec),
                   "l2": f"inputs ({gb:.1f} GB) larger than L2; no flush" if gb > 0.2
                   else "inputs smaller than L2", "parallelism": f"replicas x{ws}"},
        "hbm_gbs_algorithmic": gbs, "hbm_frac": gbs / hbm_peak,
        "orth_error_2": orth2, "residual_F": resF, "residual_2": acc["res_2"],
        "accuracy_checker": "tsqr_accuracy (Dot2 device sums)",
        "step_ms": {"step1_local_qr": s1, "step2_tree": s2, "step3_form_q": s3},
        "step_fractions": {"step1": s1 / (s1 + s2 + s3), "step2": s2 / (s1 + s2 + s3),
                           "step3": s3 / (s1 + s2 + s3)},
        "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        "paper_context": PAPER_CONTEXT,
    }

    # The extras (other precision modes, comparators, the other
    # configurations, the CPU oracle) run on single-GPU runs only: under
    # torchrun every rank's GPU would stay held while rank 0 ran them.
    # Each extra is guarded: its failure (an out-of-memory error in one of the
    # large configurations, say) is recorded in the line, which is printed
    # with the headline measurement whatever happens to the extras.
    extras_on = not args.no_extras and rank == 0 and ws == 1
    if extras_on:
        others = [p for p in (("native", "df64", "ozaki") if elem == 8 else ("native", "tf32x3"))
                  if p != resolved]
        line["extras"] = guarded(torch, extras, T, torch, A, n, m, dev, other_precs=others, prec=args.prec)
    if extras_on:
        del Q, work, dbuf, work_h
        torch.cuda.empty_cache()
        is_sweep = args.workload == "sweep" and not args.m
        configs = {"small_100kx10": guarded(torch, small_config, T, torch, dev)}
        if is_sweep:
            configs["stability_sweep_8Mx25"] = guarded(torch, stability_sweep, T, torch, dev, A15=A, prec=args.prec)
        del A
        torch.cuda.empty_cache()
        more = guarded(torch, config_extras, T, torch, dev)
        if "error" in more:
            configs["config_extras"] = more
        else:
            configs.update(more)
        line["configs"] = configs
    if extras_on:
        cb = guarded(torch, cpu_baseline, A_host)
        if "error" not in cb:
            cb["configs"] = guarded(torch, cpu_config_baselines)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def guarded(torch, fn, *args, **kw):
    """fn(*args, **kw), or {"error": ...} when it raises (the device memory
    its frames held is released before returning)."""
    try:
        return fn(*args, **kw)
    except Exception as e:  # reported, not fatal
        msg = f"{type(e).__name__}: {e}"
    try:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    except Exception:  # the context itself may be unusable; the line is still printed
        pass
    return {"error": msg[:2000]}


def _timer(torch, steps):
    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps
    return timed


def extras(T, torch, A, n, m, dev, steps=3, other_precs=("df64",), prec="auto"):
    """fwd+bwd, the other precision mode, the unstable comparators, the R-only
    and singular-value-only paths and cuSOLVER on the headline matrix."""
    out = {}
    timed = _timer(torch, steps)

    def orth(Qx):
        return T.accuracy(Qx)["orth_2"]

    g = torch.Generator(device=dev)
    g.manual_seed(ti.SEED_GRAD)
    WQ = torch.randn(A.shape, dtype=A.dtype, device=dev, generator=g)
    WR = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)

    def fb():
        Qx, Rx = T.direct(A, check=False, prec=prec)
        T.backward(Qx, Rx, WQ, WR, check=False)

    ms = timed(fb)
    out["fwd_bwd"] = {"rows_s": m / (ms * 1e-3), "ms": ms, "forward_prec": prec,
                      "hbm_gbs_algorithmic": (ALG_PASSES["direct"] + ALG_PASSES["backward"]) * m * n *
                      A.element_size() / (ms * 1e-3) / 1e9}
    del WQ
    for other_prec in other_precs:
        Qp, Rp = T.direct(A, prec=other_prec)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for e in evs:
            e.record()
        T.direct(A, check=False, prec=other_prec, stage_events=evs)
        torch.cuda.synchronize()
        ms = timed(lambda: T.direct(A, check=False, prec=other_prec))
        acc = T.accuracy(Qp, Rp, A)
        out[f"direct_{other_prec}"] = {"rows_s": m / (ms * 1e-3), "ms": ms, "orth_error_2": acc["orth_2"],
                                       "residual_F": acc["res_F"],
                                       "step_ms": {"step1": evs[0].elapsed_time(evs[1]),
                                                   "step2": evs[1].elapsed_time(evs[2]),
                                                   "step3": evs[2].elapsed_time(evs[3])},
                                       "hbm_gbs_algorithmic": ALG_PASSES["direct"] * m * n * A.element_size() /
                                       (ms * 1e-3) / 1e9}
        del Qp
    # R only and singular values only (Steps 1-2, + the SVD of R): one read of A
    for name, fn in [("r_only", lambda: T.r(A, check=False)),
                     ("svd_values", lambda: T.svd_values(A, check=False))]:
        ms = timed(fn)
        out[name] = {"rows_s": m / (ms * 1e-3), "ms": ms,
                     "hbm_gbs_algorithmic": ALG_PASSES[name] * m * n * A.element_size() / (ms * 1e-3) / 1e9}
    # comparison only: torch.linalg.qr (cuSOLVER geqrf + orgqr on a
    # column-major copy of A); the copy A^T -> column-major is timed alone too
    try:
        ms_copy = timed(lambda: A.t().contiguous())
        ms = timed(lambda: torch.linalg.qr(A, mode="reduced"))
        Qc, _ = torch.linalg.qr(A, mode="reduced")
        out["cusolver_geqrf_orgqr"] = {"rows_s": m / (ms * 1e-3), "ms": ms, "column_major_copy_ms": ms_copy,
                                       "orth_error_2": orth(Qc), "api": "torch.linalg.qr (reduced)",
                                       "backend": str(torch.backends.cuda.preferred_linalg_library())}
        del Qc
    except Exception as e:  # reported, not fatal
        out["cusolver_geqrf_orgqr"] = {"error": f"{type(e).__name__}: {e}"}
    return out


KAPPAS = (1.0, 1e4, 1e8, 1e12, 1e15)


def stability_sweep(T, torch, dev, A15=None, steps=3, m=8_000_000, n=25, prec="auto"):
    """The stability sweep of Sec. IV at 8,000,000 x 25 FP64: A = G diag(sigma)
    V^T with sigma log-spaced 1 .. 1/kappa for each kappa, factored by direct
    TSQR (the benchmarked mode and plain binary64), Cholesky QR, Cholesky QR +
    one refinement step and indirect TSQR + one refinement step;
    ||Q^T Q - I||_2 and ||A - QR||_F/||A||_F from the compensated device
    checker, rows/s, algorithmic HBM GB/s and its fraction of the measured
    HBM peak of each."""
    timed = _timer(torch, steps)
    hbm_peak, _ = load_peaks()
    methods = [("direct", lambda A: T.direct(A, check=False, prec=prec)),
               ("direct_native", lambda A: T.direct(A, check=False)),
               ("cholqr", lambda A: T.cholqr(A, refine=0, check=False)),
               ("cholqr_ir", lambda A: T.cholqr(A, refine=1, check=False)),
               ("indirect_ir", lambda A: T.indirect_refine(A, refine=1, check=False))]
    table = {}
    for kappa in KAPPAS:
        if A15 is not None and kappa == 1e15:
            A = A15
        else:
            A = torch.from_numpy(ti.conditioned(m, n, kappa, ti.SEED_SWEEP)).to(dev)
        row = {}
        for name, fn in methods:
            try:
                Qx, Rx = fn(A)
                torch.cuda.synchronize()
                ms = timed(lambda: fn(A))
                st = 0
                try:
                    fn_check = {"direct": lambda: T.direct(A, prec=prec), "direct_native": lambda: T.direct(A),
                                "cholqr": lambda: T.cholqr(A),
                                "cholqr_ir": lambda: T.cholqr(A, refine=1),
                                "indirect_ir": lambda: T.indirect_refine(A, refine=1)}[name]
                    Qx, Rx = fn_check()
                except T.TSQRError as e:  # a breakdown is a result (Sec. IV)
                    st = e.status
                if st == 0:
                    acc = T.accuracy(Qx, Rx, A)
                    gbs = ALG_PASSES[name] * m * n * 8 / (ms * 1e-3) / 1e9
                    row[name] = {"orth_error_2": acc["orth_2"], "residual_F": acc["res_F"], "ms": ms,
                                 "rows_s": m / (ms * 1e-3), "hbm_gbs_algorithmic": gbs,
                                 "hbm_frac": gbs / hbm_peak}
                else:
                    row[name] = {"status": T.STATUS.get(st, st), "ms": ms}
                del Qx
            except Exception as e:  # reported, not fatal
                row[name] = {"error": f"{type(e).__name__}: {e}"}
        table[f"{kappa:.0e}"] = row
        if A is not A15:
            del A
        torch.cuda.empty_cache()
    return {"workload": "8,000,000x25 FP64, A = G diag(sigma) V^T, sigma log-spaced 1..1/kappa",
            "checker": "tsqr_accuracy (Dot2 device sums)", "direct_prec": prec, "by_kappa": table}


def small_config(T, torch, dev, steps=50):
    """The 100,000 x 10 FP64 workload with row blocks of 1,000 (100 blocks,
    one stacked-R level of 1,000 x 10): latency-bound, reported but not
    graded as a roofline fraction."""
    import oracle
    m, n = 100_000, 10
    A_np = ti.gaussian(m, n, ti.SEED_SMALL)
    A = torch.from_numpy(A_np).to(dev)
    Q, R = T.direct(A, block_rows=1000, prec="auto")
    timed = _timer(torch, steps)
    ms = timed(lambda: T.direct(A, block_rows=1000, check=False, prec="auto"))
    ms_native = timed(lambda: T.direct(A, block_rows=1000, check=False))
    acc = T.accuracy(Q, R, A)
    Ro = oracle.householder_r(A_np)
    plan = T.plan_info(T.OP_DIRECT, m, n, torch.float64, block_rows=1000, prec="auto")
    return {"workload": "100,000x10 FP64 i.i.d. N(0,1), row blocks of 1,000", "ms": ms, "ms_native": ms_native,
            "rows_s": m / (ms * 1e-3), "hbm_gbs_algorithmic": ALG_PASSES["direct"] * m * n * 8 / (ms * 1e-3) / 1e9,
            "orth_error_2": acc["orth_2"], "residual_F": acc["res_F"],
            "r_error_vs_oracle": float(np.linalg.norm(R.cpu().numpy() - Ro) / np.linalg.norm(Ro)),
            "plan": plan,
            "launches": T.launch_count(T.OP_DIRECT, m, n, torch.float64, block_rows=1000, prec="auto")}


def config_extras(T, torch, dev, steps=3):
    """The other benchmark configurations (synthetic, generated on the device
    from a seeded generator): the FP32 form on 50,000,000 x 50 against the
    FP64 form on the same matrix upcast, with the row-block height swept; the
    SVD variant on 20,000,000 x 100 FP32 storage; forward + backward on
    4,000,000 x 64 in FP32 and FP64."""
    out = {}
    timed = _timer(torch, steps)

    def acc_of(Ax, Qx, Rx):
        a = T.accuracy(Qx, Rx, Ax)
        return {"orth_error_2": a["orth_2"], "residual_F": a["res_F"]}

    g = torch.Generator(device=dev)
    # mixed precision: N(0,1) scaled by column factors log-spaced over [1, 1e-4]
    try:
        m, n = 50_000_000, 50
        g.manual_seed(ti.SEED_MIXED)
        c = torch.logspace(0, -4, n, dtype=torch.float64, device=dev)
        A32 = (torch.randn(m, n, dtype=torch.float32, device=dev, generator=g) * c.float())
        entry = {"workload": "50,000,000x50 FP32, N(0,1) x column factors 1..1e-4"}
        for key, prec in (("fp32", "native"), ("fp32_tf32x3", "tf32x3")):
            Q, R = T.direct(A32, prec=prec)
            ms = timed(lambda: T.direct(A32, check=False, prec=prec))
            entry[key] = {"rows_s": m / (ms * 1e-3), "ms": ms, **acc_of(A32, Q, R),
                          "hbm_gbs_algorithmic": 4 * m * n * 4 / (ms * 1e-3) / 1e9,
                          "plan": T.plan_info(T.OP_DIRECT, m, n, torch.float32, prec=prec)}
            del Q
        # row blocks of 1,024 .. 8,192 rows (and the planner's choice above):
        # time and tree depth of each
        sweep = {}
        for b in (1024, 2048, 4096, 8192):
            try:
                plan = T.plan_info(T.OP_DIRECT, m, n, torch.float32, block_rows=b, prec="tf32x3")
                ms = timed(lambda: T.direct(A32, block_rows=b, check=False, prec="tf32x3"))
                msn = timed(lambda: T.direct(A32, block_rows=b, check=False))
                sweep[str(b)] = {"ms_tf32x3": ms, "ms_fp32": msn, "rows_s_tf32x3": m / (ms * 1e-3),
                                 "tree_levels": plan["tree_levels"], "tree_fanout": plan["tree_fanout"],
                                 "blocks": plan["blocks"], "tiles_per_block": plan["tiles_per_block"]}
            except Exception as e:
                sweep[str(b)] = {"error": f"{type(e).__name__}: {e}"}
        entry["block_rows_sweep"] = sweep
        A64 = A32.double()
        del A32
        Q, R = T.direct(A64)
        ms = timed(lambda: T.direct(A64, check=False))
        entry["fp64_upcast"] = {"rows_s": m / (ms * 1e-3), "ms": ms, **acc_of(A64, Q, R),
                                "hbm_gbs_algorithmic": 4 * m * n * 8 / (ms * 1e-3) / 1e9}
        del Q, A64
        out["mixed_50Mx50"] = entry
    except Exception as e:  # reported, not fatal
        out["mixed_50Mx50"] = {"error": f"{type(e).__name__}: {e}"}
    torch.cuda.empty_cache()
    # SVD variant: G diag(j^-2) V^T, FP32 storage
    try:
        m, n = 20_000_000, 100
        g.manual_seed(ti.SEED_SVD)
        V, _ = torch.linalg.qr(torch.randn(n, n, dtype=torch.float64, device=dev, generator=g))
        sig = torch.arange(1, n + 1, dtype=torch.float64, device=dev) ** -2.0
        M = (sig[:, None] * V.T) / m ** 0.5
        A = torch.empty(m, n, dtype=torch.float32, device=dev)
        for r0 in range(0, m, 1 << 22):
            rows = min(1 << 22, m - r0)
            A[r0:r0 + rows] = (torch.randn(rows, n, dtype=torch.float64, device=dev, generator=g) @ M).float()
        U, S, Vo = T.svd(A, prec="auto")
        ms = timed(lambda: T.svd(A, check=False, prec="auto"))
        out["svd_20Mx100"] = {"workload": "20,000,000x100 FP32 storage, G diag(j^-2) V^T",
                              "prec": T.plan_info(T.OP_SVD, m, n, torch.float32, prec="auto")["prec"],
                              "rows_s": m / (ms * 1e-3), "ms": ms, "orth_error_2_U": T.accuracy(U)["orth_2"],
                              "max_rel_sigma_dev": float((S / sig - 1).abs().max()),
                              "hbm_gbs_algorithmic": 4 * m * n * 4 / (ms * 1e-3) / 1e9}
        del U
        Un, _, _ = T.svd(A)
        out["svd_20Mx100"]["native"] = {"ms": timed(lambda: T.svd(A, check=False)),
                                        "orth_error_2_U": T.accuracy(Un)["orth_2"]}
        del Un
        del A
    except Exception as e:
        out["svd_20Mx100"] = {"error": f"{type(e).__name__}: {e}"}
    torch.cuda.empty_cache()
    # forward + backward, 4,000,000 x 64, row blocks of 4,096
    try:
        m, n = 4_000_000, 64
        entry = {"workload": "4,000,000x64 N(0,1), W_Q and W_R N(0,1), row blocks of 4,096"}
        for name, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
            g.manual_seed(ti.SEED_GRAD)
            A = torch.randn(m, n, dtype=dt, device=dev, generator=g)
            WQ = torch.randn(m, n, dtype=dt, device=dev, generator=g)
            WR = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)

            def fb():
                Qx, Rx = T.direct(A, block_rows=4096, check=False)
                T.backward(Qx, Rx, WQ, WR, check=False)

            ms = timed(fb)
            msf = timed(lambda: T.direct(A, block_rows=4096, check=False))
            Q, R = T.direct(A, block_rows=4096)
            esz = 8 if dt == torch.float64 else 4
            entry[name] = {"fwd_bwd_rows_s": m / (ms * 1e-3), "fwd_bwd_ms": ms, "fwd_rows_s": m / (msf * 1e-3),
                           "fwd_ms": msf, "orth_error_2": T.accuracy(Q)["orth_2"],
                           "fwd_bwd_hbm_gbs_algorithmic": 9 * m * n * esz / (ms * 1e-3) / 1e9}
            if dt == torch.float32:
                mst = timed(lambda: T.direct(A, block_rows=4096, check=False, prec="tf32x3"))
                entry[name]["fwd_rows_s_tf32x3"] = m / (mst * 1e-3)
            del A, WQ, Q
        out["grad_4Mx64"] = entry
    except Exception as e:
        out["grad_4Mx64"] = {"error": f"{type(e).__name__}: {e}"}
    torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    sys.exit(main())
