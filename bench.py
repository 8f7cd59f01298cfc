#!/usr/bin/env python
"""Exact k-NN throughput of the GB300 iSAX engine (MESSI, arXiv 2110.07519).

Workload (default): 100,000,000 seeded random walks of length 256, z-normalised
(the paper's 100 GB synthetic collection, Sec. 5.1), iSAX with 16 segments and
8-bit symbols; queries half fresh random walks, half dataset members plus
N(0, sigma) noise, sigma in {0.1, 0.5, 1.0} (Sec. 5.3); exact 1-NN under ED.
A step answers one batch of queries against the resident index.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(brute force) on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact 1-NN queries/sec and p50/p99 ms on 100M x 256 fp32 ED at 1 GB300; % HBM roofline"
PAPER_QPS = 20.0          # ~50 ms per exact 1-NN ED query on 100M x 256 (paper, 2x Xeon E5-2650 v4)
DATA_DESC = ("synthetic: seeded random walks (x0~N(0,1), x_t=x_{t-1}+N(0,1)), z-normalised; queries half "
             "fresh walks (separate seed), half dataset members + N(0,sigma) noise, sigma 0.1/0.5/1.0")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="messi", choices=["messi", "reference"])
    ap.add_argument("--n", type=int, default=100_000_000)
    ap.add_argument("--len", type=int, default=256)
    ap.add_argument("--batch", type=int, default=1024, help="queries per step")
    ap.add_argument("--k", type=int, default=1)
    ap.add_argument("--dist", default="ed", choices=["ed", "dtw"])
    ap.add_argument("--window", type=int, default=-1, help="DTW reach in points (default 10%% of len)")
    ap.add_argument("--cpu-sample", type=int, default=4, help="queries in the CPU-oracle sample")
    ap.add_argument("--class-queries", type=int, default=64,
                    help="queries per class in the plain form's per-class breakdown (0: none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--form", default="both", choices=["both", "plain", "batched"])
    ap.add_argument("--serve", action="store_true", help="serving-loop measurement instead of the step bench")
    ap.add_argument("--serve-n", type=int, default=50_000_000)
    ap.add_argument("--serve-len", type=int, default=128)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[1000, 10000, 100000])
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--serve-max", type=int, default=60000)
    ap.add_argument("--serve-streams", type=int, default=4, help="server worker streams")
    ap.add_argument("--batch-mode", default="tc", choices=["tc", "lb"],
                    help="batched kernels: tensor-core screen (tc) or fused lower bound + refine (lb)")
    ap.add_argument("--autotune", action="store_true",
                    help="lower-bound batch form: time its shapes on the warm-up queries first")
    ap.add_argument("--mix", default="mixed", choices=["mixed", "fresh", "s0.1", "s0.5", "s1.0"],
                    help="query class (default: the paper-shaped mix)")
    ap.add_argument("--windows", action="store_true",
                    help="subsequence collection: the n z-normalised sliding windows (length --len, stride 1) "
                         "of one random walk of n + len - 1 points")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_tensor():
    """Dense f16/bf16 tensor peak in TFLOP/s: the sustained cuBLAS bf16 figure
    (the screen runs for hundreds of ms at a time); f16 and bf16 share a rate."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "measured (bf16 sustained; f16 same rate)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback"


def derived_peak_fp32():
    """Plain FP32 arithmetic rate (no measured figure exists): 152 SMs x 128
    FP32 lanes x 2 operations per fused multiply-add x the maximum SM clock."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        mhz = 2070.0
    return 152 * 128 * 2 * mhz * 1e6 / 1e12, f"derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x {mhz:.0f} MHz"


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def scan_source_sha(kernel: str = "k_lb_scan"):
    """Hash of the source a traffic figure was measured on: for the screen,
    the part of screen.cu from its argument block to the end of the screen
    kernel, and the tensor-core and shared device helpers; for the scan, the
    part of query.cu from its code table to the end of the scan kernel, and
    the shared device helpers."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2110_07519_gb300", "csrc")
    if kernel == "k_tc_screen":
        with open(os.path.join(csrc, "screen.cu"), "rb") as f:
            text = f.read()
        a = text.find(b"struct ScreenArgs {")
        b = text.find(b"// ----------------------------------------------------------- recheck")
        h.update(text[a:b] if 0 <= a < b else text)
        for name in ("tc.cuh", "device_common.cuh"):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(f.read())
    else:
        with open(os.path.join(csrc, "query.cu"), "rb") as f:
            text = f.read()
        a = text.find(b"struct ScanCodes {")
        b = text.find(b"// ------------------------------------------------------------ ED refine")
        h.update(text[a:b] if 0 <= a < b else text)
        with open(os.path.join(csrc, "device_common.cuh"), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(units: float, kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled
    to the units one launch processes (series for the screen, scanned words
    for the lower-bound scan), or None when its source changed since it was
    captured."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    try:
        text = open(path).read()
    except OSError:
        return None
    sha = re.search(r"source_sha:\s*(\w+)", text)
    per = re.search(r"dram_bytes_per_(?:series|word):\s*([0-9.eE+-]+)", text)
    if not sha or not per or sha.group(1) != scan_source_sha(kernel):
        return None
    return float(per.group(1)) * units


def replica_elapsed_ms(pg, elapsed_ms, device="cpu"):
    """Replicas only: every rank answers its own queries on its own copy of the
    index; the job's time is the slowest rank's (max over ranks)."""
    if not pg:
        return elapsed_ms
    import torch

    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world_size, units_per_rank, elapsed_ms):
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return world_size * units_per_rank / (elapsed_ms * 1e-3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(data_t, queries_np, k, chunk=1 << 20, dist=0, r=0):
    """FP64 brute force of `queries_np` over the device collection `data_t`,
    copied to the host chunk by chunk; returns (ids, d2, cpu_seconds, threads)."""
    import torch

    import oracle

    best = None
    cpu_s = 0.0
    N = data_t.shape[0]
    host = torch.empty((min(chunk, N), data_t.shape[1]), dtype=torch.float32, pin_memory=True)
    for lo in range(0, N, chunk):
        hi = min(N, lo + chunk)
        host[: hi - lo].copy_(data_t[lo:hi])
        rows = host[: hi - lo].numpy()
        t0 = time.perf_counter()
        part = oracle.knn(rows, queries_np, k, dist, r, id_base=lo)
        best = part if best is None else oracle.merge_topk([best, part], k)
        cpu_s += time.perf_counter() - t0
    return best[0], best[1], cpu_s, oracle.max_threads()


# ------------------------------------------------------------ reference arm
def mixed_order(qpool, rank):
    """The query mix comes grouped by class (fresh, then each noise level); a
    fixed permutation spreads the classes evenly over the steps."""
    import torch

    g = torch.Generator()
    g.manual_seed(4242 + rank)
    perm = torch.randperm(qpool.shape[0], generator=g).to(qpool.device)
    return qpool.index_select(0, perm).contiguous()


def workload_name(args, window=0):
    """The workload both arms name in `config`: collection, distance, k, index shape."""
    coll = (f"{args.n} z-normalised sliding windows (length {args.len}, stride 1) of one "
            f"{args.n + args.len - 1}-point random walk" if args.windows else
            f"{args.n} x {args.len} fp32 random walks")
    dist = "ED" if args.dist == "ed" else f"DTW window {window}"
    return f"{coll}, {dist}, k={args.k}, 16 segments, 8-bit SAX"


def run_reference(args, ws, rank, local):
    if rank != 0:
        return
    if args.windows or args.dist != "ed":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the ED random-walk "
                                                             "workload only (no --windows, no --dist dtw)"}))
        return
    import torch

    import oracle
    import synth

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    oracle.build()
    data = synth.random_walks_torch(args.n, args.len, device=dev)
    qpool = mixed_order(synth.query_mix_torch(data, args.warmup + args.steps, seed=synth.QUERY_SEED), 0).cpu().numpy()
    times = []
    threads = oracle.max_threads()
    for step in range(args.warmup + args.steps):
        _, _, cpu_s, threads = oracle_sample(data, qpool[step:step + 1], args.k)
        if step >= args.warmup:
            times.append(cpu_s)
    total = sum(times)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_QPS, "dtype": "f64",
        "data": DATA_DESC,
        "config": {"workload": workload_name(args), "form": "oracle: FP64 brute force on the host cores",
                   "queries": "mixed", "queries_per_step": 1, "l2": "inputs larger than L2 (host memory)"},
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} timed queries (1 per step), FP64 brute force over all "
                                   f"{args.n} series; device-to-host chunk copies excluded"},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- GPU arm
def time_form(m, ix, qpool, form, B, K, W, k, stream, pg, dev, ids, dists, dist=0, window=0, batch_arg=None):
    """W warm-up and K timed steps of one query form (B queries a step); per-step stats.
    batch_arg: queries per batched launch (None: B; 0: the index's tuned batch)."""
    import torch

    launch_batch = B if batch_arg is None else batch_arg

    def step(qs):
        if form == "plain":
            m.messi_query(ix, qs, k=k, dist=dist, window=window, ids=ids, dists=dists)
        else:
            m.messi_query_batched(ix, qs, k=k, dist=dist, window=window, batch=launch_batch, ids=ids, dists=dists)

    # timed steps carry only the events around the dominant kernel's launches
    # (level 1); per-query latencies come from a separate pass (level 2)
    m.messi_set_profiling(ix, 1)
    for s in range(W):
        step(qpool[s * B:(s + 1) * B])
    m.messi_check(ix)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = ClockSampler(dev.index or 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    agg = {"kern_ms": 0.0, "kern_launches": 0, "launches": 0, "survivors": 0, "rows": 0, "words": 0, "lat": [],
           "screened": 0, "row_bytes": 0, "bsf_updates": 0, "refine_ms": 0.0, "refine_launches": 0,
           "dtw_cells": 0}
    torch.cuda.synchronize()
    e0.record(stream)
    for s in range(W, W + K):
        step(qpool[s * B:(s + 1) * B])
        st = m.messi_query_stats(ix)
        agg["kern_ms"] += st["scan_ms"]
        agg["kern_launches"] += st["scan_launches"]
        agg["screened"] += st["screened_queries"]
        agg["launches"] += st["kernel_launches"]
        agg["survivors"] += st["lb_survivors"]
        agg["rows"] += st["refined"] + st["abandoned"]
        agg["words"] += st["lb_evaluated"]
        agg["row_bytes"] += st["row_bytes"]
        agg["bsf_updates"] += st["bsf_updates"]
        agg["refine_ms"] += st["refine_ms"]
        agg["refine_launches"] += st["refine_launches"]
        agg["dtw_cells"] += st["dtw_cells"]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed_ms = e0.elapsed_time(e1)
    m.messi_check(ix)
    elapsed_ms = replica_elapsed_ms(pg, elapsed_ms, dev)
    # per-query latency percentiles over every timed query in one call
    m.messi_set_profiling(ix, 2)
    if form == "plain":
        m.messi_query(ix, qpool[W * B:(W + K) * B], k=k, dist=dist, window=window)
    else:
        m.messi_query_batched(ix, qpool[W * B:(W + K) * B], k=k, dist=dist, window=window, batch=launch_batch)
    st_all = m.messi_query_stats(ix)
    m.messi_set_profiling(ix, 0)
    agg.update(elapsed_ms=elapsed_ms, clocks=clk, p50=st_all["query_ms_p50"], p99=st_all["query_ms_p99"])
    return agg


def run_messi(args, ws, rank, local):
    import torch

    import paper_2110_07519_gb300 as m
    import synth

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    B, K, W = args.batch, args.steps, args.warmup

    windows = None
    if args.windows:
        walk = synth.random_walks_torch(1, args.n + args.len - 1, seed=synth.DATASET_SEED + rank, device=dev)[0]
        torch.cuda.synchronize()
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0.record()
        data = m.messi_windows(walk, args.len, 1, True)
        w1.record()
        torch.cuda.synchronize()
        wms = w0.elapsed_time(w1)
        del walk
        windows = {"ms": wms, "written_gbps": args.n * args.len * 4 / (wms * 1e-3) / 1e9}
    else:
        data = synth.random_walks_torch(args.n, args.len, seed=synth.DATASET_SEED + rank, device=dev)
    torch.cuda.synchronize()
    ix = m.messi_build(data, 16, 256)
    info = m.messi_index_get_info(ix)
    build_gbps = args.n * args.len * 4 / (info["build_ms"] * 1e-3) / 1e9
    if args.mix == "mixed":
        qpool = mixed_order(synth.query_mix_torch(data, (W + K) * B, seed=synth.QUERY_SEED + rank), rank)
    elif args.mix == "fresh":
        qpool = synth.random_walks_torch((W + K) * B, args.len, seed=synth.QUERY_SEED + rank, device=dev)
    else:
        qpool = synth.noisy_members_torch(data, (W + K) * B, float(args.mix[1:]), seed=synth.NOISE_SEED + rank)[0]
    ids = torch.empty((B, args.k), dtype=torch.int64, device=dev)
    dists = torch.empty((B, args.k), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = measured_peak_hbm()

    # CPU baseline: the FP64 oracle on a bounded sample of the timed queries,
    # over the generated collection (which is then released: the index holds
    # its own copy)
    cpu, oracle_q, r_ids, r_d2 = None, None, None, None
    if rank == 0 and not args.no_cpu_baseline and args.cpu_sample > 0:
        oracle_q = qpool[W * B:W * B + args.cpu_sample].cpu().numpy()
        r_ids, r_d2, cpu_s, threads = oracle_sample(data, oracle_q, args.k,
                                                    dist=1 if args.dist == "dtw" else 0,
                                                    r=(args.window if args.window >= 0 else int(0.10 * args.len))
                                                    if args.dist == "dtw" else 0)
        cpu = {"value": args.cpu_sample / cpu_s, "unit": "queries/s", "cores": threads, "kind": "oracle",
               "sample": f"{args.cpu_sample} queries of the timed mix, FP64 brute force over all {args.n} "
                         f"series (1M-row chunks copied to the host; copy time excluded)"}
    # per-class queries for the plain form's breakdown (fresh walks; members
    # with sigma 0.1 / 0.5 / 1.0 noise), drawn while the collection exists
    class_pools = {}
    if not args.windows and args.form in ("both", "plain") and args.class_queries > 0:
        cq = args.class_queries
        class_pools["fresh"] = synth.random_walks_torch(cq, args.len, seed=synth.QUERY_SEED + 100 + rank, device=dev)
        for i, sg in enumerate((0.1, 0.5, 1.0)):
            class_pools[f"sigma{sg}"] = synth.noisy_members_torch(data, cq, sg,
                                                                  seed=synth.NOISE_SEED + 100 + i + rank)[0]
    qpool = qpool.clone()
    del data
    torch.cuda.empty_cache()

    dist_code = 1 if args.dist == "dtw" else 0
    window = (args.window if args.window >= 0 else int(0.10 * args.len)) if dist_code else 0
    # the screen takes lengths that are multiples of 16 up to 2048 (ED only); other
    # batches run the lower-bound kernels whatever the requested mode
    screen_ok = args.len % 16 == 0 and args.len <= 2048 and args.dist == "ed"
    batch_mode = "tc_screen" if args.batch_mode == "tc" and screen_ok else "lb_refine"
    m.messi_set_batch_mode(ix, m.MESSI_BATCH_TC_SCREEN if args.batch_mode == "tc" else m.MESSI_BATCH_LB_REFINE)
    tuning = None
    if args.autotune and args.batch_mode == "lb" and B >= 32:
        tuning = m.messi_autotune(ix, qpool[:max(256, B)].contiguous(), k=args.k)
    forms = {}
    for form in (["plain", "batched"] if args.form == "both" else [args.form]):
        r = time_form(m, ix, qpool, form, B, K, W, args.k, stream, pg, dev, ids, dists, dist_code, window,
                      batch_arg=0 if tuning else None)
        nqt = B * K
        kern_avg_s = r["kern_ms"] * 1e-3 / max(r["kern_launches"], 1)
        n_leaves = m.messi_index_get_info(ix)["n_leaves"]
        ntiles = (args.n + 1023) // 1024
        refine = None
        if r["refine_launches"]:
            rs = r["refine_ms"] * 1e-3
            if dist_code == 1:
                # banded DTW: 5 FP32 operations per band cell (difference, square,
                # add, two minima) over the cells the recurrence evaluated
                fpk, fkind = derived_peak_fp32()
                refine = {"kernel": "k_dtw_thread", "bound": "alu", "cells": r["dtw_cells"],
                          "achieved": 5.0 * r["dtw_cells"] / rs / 1e12, "peak": fpk, "unit": "TFLOP/s",
                          "frac": 5.0 * r["dtw_cells"] / rs / 1e12 / fpk, "peak_kind": fkind,
                          "avg_launch_ms": r["refine_ms"] / r["refine_launches"], "launches": r["refine_launches"]}
            else:
                # ED refinement: raw-row bytes read plus the survivor lists (8 B each)
                rb = r["row_bytes"] + 8.0 * r["survivors"]
                refine = {"kernel": "k_refine_ed", "bound": "hbm", "achieved": rb / rs / 1e9, "peak": peak,
                          "unit": "GB/s", "frac": rb / rs / 1e9 / peak, "peak_kind": peak_kind,
                          "avg_launch_ms": r["refine_ms"] / r["refine_launches"], "launches": r["refine_launches"]}
        if form == "plain" and dist_code == 1 and refine:
            # DTW per query: the banded DTW kernel (FP32 arithmetic bound)
            kernel = "k_dtw_thread"
            algo = 5.0 * r["dtw_cells"] / r["refine_launches"]
            kern_avg_s = r["refine_ms"] * 1e-3 / r["refine_launches"]
            roof = {k_: v for k_, v in refine.items() if k_ not in ("kernel", "cells", "avg_launch_ms", "launches")}
        elif form == "plain":
            # the timed scan group: leaf boxes + leaf offsets (40 B per leaf), the
            # tile stamps (4 B per tile), and 16 B per word of the live tiles
            kernel = "k_lb_scan"
            algo = 40.0 * n_leaves + 4.0 * ntiles + 16.0 * r["words"] / max(r["kern_launches"], 1)
            roof = {"bound": "hbm", "achieved": algo / kern_avg_s / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": algo / kern_avg_s / 1e9 / peak, "peak_kind": peak_kind,
                    "timed": "k_leaf_prune + k_live_tiles + k_lb_scan per query"}
        elif dist_code == 1 and refine:
            # batched DTW: the banded DTW kernel of the overlapped per-query sequences
            kernel = "k_dtw_thread"
            algo = 5.0 * r["dtw_cells"] / r["refine_launches"]
            kern_avg_s = r["refine_ms"] * 1e-3 / r["refine_launches"]
            roof = {k_: v for k_, v in refine.items() if k_ not in ("kernel", "cells", "avg_launch_ms", "launches")}
        elif batch_mode == "tc_screen":
            # the screen's dense work: 2 * len flops per (series, query) pair, for every
            # query of every launch (a first pass screens the batch, a later one only
            # the queries whose candidate lists overflowed)
            kernel = "k_tc_screen"
            algo = 2.0 * args.len * args.n * r["screened"] / max(r["kern_launches"], 1)
            tpk, tkind = measured_peak_tensor()
            roof = {"bound": "tensor", "achieved": algo / kern_avg_s / 1e12, "peak": tpk, "unit": "TFLOP/s",
                    "frac": algo / kern_avg_s / 1e12 / tpk, "peak_kind": tkind}
        else:
            kernel = "k_fused_ed"
            algo = 16.0 * args.n + 4.0 * args.len * r["rows"] / max(r["kern_launches"], 1)
            roof = {"bound": "hbm", "achieved": algo / kern_avg_s / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": algo / kern_avg_s / 1e9 / peak, "peak_kind": peak_kind}
        if form == "plain" or dist_code == 1:
            # bytes one query moves: leaf boxes and offsets, tile stamps, the
            # words of its live tiles, its survivor list (written once, read by
            # the refinement) and the raw-row bytes its refinement read
            q_bytes = (40.0 * n_leaves + 4.0 * ntiles + 16.0 * r["words"] / nqt + 16.0 * r["survivors"] / nqt
                       + r["row_bytes"] / nqt)
        elif batch_mode == "tc_screen":
            # per query: its share of the f16 rows and norms each screen launch
            # streams, plus the rows its exact recheck read
            q_bytes = ((2.0 * args.len + 8.0) * args.n * r["kern_launches"] + r["row_bytes"]) / nqt
        else:
            q_bytes = (16.0 * args.n * r["kern_launches"] + r["row_bytes"]) / nqt
        forms[form] = {
            "value": replica_throughput(ws, nqt, r["elapsed_ms"]), "ms_per_step": r["elapsed_ms"] / K,
            "p50_ms": r["p50"], "p99_ms": r["p99"], "gpu_launches": r["launches"], "clocks": r["clocks"],
            "roofline": dict(roof, kernel=kernel, algorithmic_per_launch=algo, avg_launch_ms=kern_avg_s * 1e3,
                             launches=r["kern_launches"]),
            **({"refine": refine} if refine else {}),
            "counters": {"lb_survivors_per_query": r["survivors"] / nqt, "rows_read_per_query": r["rows"] / nqt,
                         "row_bytes_per_query": r["row_bytes"] / nqt,
                         "words_scanned_per_query": r["words"] / nqt,
                         "bsf_updates_per_query": r["bsf_updates"] / nqt,
                         **({"dtw_cells_per_query": r["dtw_cells"] / nqt} if dist_code == 1 else {})},
            "query_roofline_frac": q_bytes / (r["elapsed_ms"] * 1e-3 / nqt) / 1e9 / peak,
            **({"tuning": tuning} if tuning and form == "batched" else {}),
        }
    # plain form, query class by class (untimed against the bench clock; CUDA
    # events around each class's call): throughput and the work counters
    if class_pools and "plain" in forms:
        per_class = {}
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for name, cq in class_pools.items():
            m.messi_query(ix, cq[:8], k=args.k, dist=dist_code, window=window)   # warm-up
            torch.cuda.synchronize()
            c0.record(stream)
            m.messi_query(ix, cq, k=args.k, dist=dist_code, window=window)
            c1.record(stream)
            torch.cuda.synchronize()
            st = m.messi_query_stats(ix)
            nq_c = cq.shape[0]
            per_class[name] = {
                "queries": nq_c, "queries_per_s": nq_c / (c0.elapsed_time(c1) * 1e-3),
                "words_scanned_per_query": st["lb_evaluated"] / nq_c,
                "lb_survivors_per_query": st["lb_survivors"] / nq_c,
                "rows_read_per_query": (st["refined"] + st["abandoned"]) / nq_c,
                "row_bytes_per_query": st["row_bytes"] / nq_c,
                "seeded_per_query": st["seeded"] / nq_c,
                "bsf_updates_per_query": st["bsf_updates"] / nq_c,
                "leaves_live_per_query": st["leaves_live"] / nq_c}
        forms["plain"]["per_class"] = per_class
    head_form = max(forms, key=lambda f: forms[f]["value"])
    head = forms[head_form]
    for fm in forms.values():   # every form's dominant kernel, from its committed ncu summary
        fk = fm["roofline"]["kernel"]
        fm["roofline"]["traffic"] = profiled_traffic(
            fm["counters"]["words_scanned_per_query"] if fk == "k_lb_scan" else args.n, fk)

    # end to end through the C ABI with host buffers (pinned), copies inside
    e2e = None
    if not args.no_e2e:
        hq = qpool[W * B:(W + K) * B].cpu().pin_memory().numpy()
        hids = torch.empty((B, args.k), dtype=torch.int64).pin_memory().numpy()
        hd = torch.empty((B, args.k), dtype=torch.float32).pin_memory().numpy()
        call = (lambda q: m.messi_query(ix, q, k=args.k, ids=hids, dists=hd)) if head_form == "plain" else \
            (lambda q: m.messi_query_batched(ix, q, k=args.k, batch=B, ids=hids, dists=hd))
        call(hq[:B])
        t0 = time.perf_counter()
        for s in range(K):
            call(hq[s * B:(s + 1) * B])
        e2e_s = time.perf_counter() - t0
        e2e = {"value": ws * B * K / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": B * args.len * 4,
               "d2h_bytes_per_step": B * args.k * 12, "form": head_form}

    # FP64 oracle on the bounded sample, answered by each form after timing
    parity = {"queries": int(oracle_q.shape[0])} if oracle_q is not None else None
    if oracle_q is not None:
        for form in forms:
            fn = m.messi_query if form == "plain" else m.messi_query_batched
            g_ids, g_d = fn(ix, oracle_q, k=args.k, dist=dist_code, window=window)
            rel = np.abs(g_d.astype(np.float64) - np.sqrt(r_d2)) / np.maximum(np.sqrt(r_d2), 1e-30)
            parity[form] = {"ids_equal": bool(np.array_equal(g_ids, r_ids)), "max_rel_err": float(rel.max())}

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": "queries/s", "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": head["value"] / PAPER_QPS, "dtype": "f32", "data": DATA_DESC,
            "config": {"workload": workload_name(args, window), "form": head_form, "queries": args.mix,
                       "queries_per_step": B, "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": "inputs larger than L2 (16 B iSAX word per series streamed per query)"},
            "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
            "build_gbps": build_gbps, "build_ms": info["build_ms"],
            **({"windows": windows} if windows else {}),
            "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": head["gpu_launches"],
            "clocks": head["clocks"], "parity_sample": parity, "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def run_serve(args, ws, rank, local):
    """Serving loop: Poisson arrivals at several rates, 80% ED / 20% DTW
    (window 10%), k in {1, 10}; submit-to-result latency and completed
    queries/s, for the tensor-core screened and the lower-bound batch kernels."""
    import threading

    import torch

    import paper_2110_07519_gb300 as m
    import synth

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    n, length = args.serve_n, args.serve_len
    data = synth.random_walks_torch(n, length, seed=synth.DATASET_SEED + rank, device=dev)
    ix = m.messi_build(data, 16, 256)
    pool = mixed_order(synth.query_mix_torch(data, 4096, seed=synth.QUERY_SEED), rank).cpu().numpy()
    del data
    torch.cuda.empty_cache()
    r_dtw = int(0.10 * length)
    out = {}
    for mode_name, mode in (("tc_screen", m.MESSI_BATCH_TC_SCREEN), ("lb_refine", m.MESSI_BATCH_LB_REFINE)):
        m.messi_set_batch_mode(ix, mode)
        res_mode = {}
        for rate in args.serve_rates:
            srv = m.messi_server_create(ix, max_batch=1024, max_k=16, streams=args.serve_streams)
            rng = np.random.default_rng(int(rate))
            total = int(min(args.serve_seconds * rate, args.serve_max))
            kinds = rng.random(total) < 0.2
            ks = rng.choice([1, 10], size=total)
            tickets = [None] * total
            t0 = time.perf_counter()

            def producer():
                nxt = time.perf_counter()
                for i in range(total):
                    nxt += rng.exponential(1.0 / rate)
                    while time.perf_counter() < nxt:
                        pass
                    dtw = bool(kinds[i])
                    tickets[i] = m.messi_server_submit(srv, pool[i % len(pool)], int(ks[i]), 1 if dtw else 0,
                                                       r_dtw if dtw else 0)

            th = threading.Thread(target=producer)
            th.start()
            th.join()
            lat = []
            for i in range(total):
                r = None
                while r is None:
                    r = m.messi_server_poll(srv, tickets[i], int(ks[i]), wait_us=500_000)
                lat.append(r[2])
            wall = time.perf_counter() - t0
            st = m.messi_server_get_stats(srv)
            m.messi_server_destroy(srv)
            lat = np.array(lat)
            res_mode[str(rate)] = {"offered_qps": rate, "completed": total, "served_qps": total / wall,
                                   "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                                   "ed": {"requests": int((~kinds).sum()),
                                          "p50_ms": float(np.percentile(lat[~kinds], 50)) if (~kinds).any() else None,
                                          "p99_ms": float(np.percentile(lat[~kinds], 99)) if (~kinds).any() else None},
                                   "dtw": {"requests": int(kinds.sum()),
                                           "p50_ms": float(np.percentile(lat[kinds], 50)) if kinds.any() else None,
                                           "p99_ms": float(np.percentile(lat[kinds], 99)) if kinds.any() else None},
                                   "batches": st["batches"], "inflight_peak": st["inflight_peak"],
                                   "budget_waits": st["budget_waits"], "wall_s": wall}
            print(json.dumps({"mode": "serve-partial", "batch_kernels": mode_name, "rate": rate,
                              **res_mode[str(rate)]}), file=sys.stderr, flush=True)
        out[mode_name] = res_mode
    print(json.dumps({"mode": "serve", "config": {"workload": f"{n} x {length} fp32 random walks, 80% ED / 20% DTW "
                                                              f"(window {r_dtw}), k in {{1,10}}, Poisson arrivals",
                                                  "streams": args.serve_streams,
                                                  "data": DATA_DESC},
                      "results": out}), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.serve:
        if rank == 0:
            run_serve(args, ws, rank, local)
        return
    if args.impl == "reference":
        run_reference(args, ws, rank, local)
    else:
        run_messi(args, ws, rank, local)


if __name__ == "__main__":
    main()
