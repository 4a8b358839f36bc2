#!/usr/bin/env python3
"""Benchmark of exact banded-DTW best-match search on one GB300.

Workload (default ``rw100m``): a 1e8-sample FP32 random walk with seeded sine
bursts and N(0, 0.5) noise; one m=512 query that is a noisy (0.1) copy of a
seeded window; Sakoe-Chiba half-width r = floor(0.1 m) = 51; top-1.  A step is
one dtws_query (query prep, proxy scan and Euclidean seeds, fused lower-bound
scan, survivor ordering, DTW, extended-precision re-score) with the series and
its per-series data (anchored prefix sums, window statistics for m, series
envelope for r) resident in HBM; their one-time cost is reported as
``precompute_ms``.

At N = 1 the same JSON line also carries (unless ``--no-extras``):
``learned`` -- mean ms per query on the learned-proposal workload (n = 2e8,
64 queries m = 1024, r = 102) with the learned ordering, the proxy ordering
and the paper's random seeding, the speedups and whether the answers agree;
``batch`` -- the batched workload (n = 5e7, 256 queries of mixed m and r,
top-10) through dtws_query_batch with a replayed CUDA graph; ``drift`` -- the
precision-stress workload (n = 1e9 with drift and variance regimes, 32
queries m = 1024): ms per query and, against the FP64 oracle at each answer,
the error of the FP32 DTW and of the returned distance; ``wide`` -- bands of
0.9 m (m = 1024 and 2048 on 2e7 samples): ms per query and phase times.
``dtw_roofline`` times the DTW kernel's walk alone (dtws_dtw_at over 1e5
windows of the workload, no pruning) against its ALU ceiling.

Metric: subsequences/s per query (N windows / step time).  Also reported:
brute-force-equivalent DTW cells/s (N * cells(m, r) / step time), the
roofline of the dominant kernel (the lower-bound scan: HBM bytes per launch /
CUDA-event time), the FP64 oracle's throughput on a bounded sample of the
same workload on the host cores, and an end-to-end number through the C ABI
with host buffers (query in, result out, copies inside the timed region).

``--impl reference`` times the FP64 CPU oracle (the reference arm of this
build) on a bounded sample of the same workload.  Under torchrun (N > 1)
each rank searches its own fragment (Sec. 3.1, Eq. 11 overlap partition of an
N-times longer series) and the ranks' k best (distance, offset) pairs are
merged by one all-gather (``shard.allgather_merge``), the analogue of the
paper's Algorithm 1 exchange.
"""
from __future__ import annotations

import argparse
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

from paper_1812_10302_gb300 import synth  # noqa: E402

SPECS = {
    "rw100m": dict(n=100_000_000, m=512, w=0.10, k=1),
    "rw30m": dict(n=30_000_000, m=512, w=0.10, k=1),
    "rw1m": dict(n=1_000_000, m=128, w=0.05, k=1),
    # the learned-proposal workload's kind (walk + bursts, seeds 4/4/6), shortened to 2e7 samples
    "learn20m": dict(n=20_000_000, m=1024, w=0.10, k=1),
    # the learned-proposal workload's series itself (2e8 samples), its first query
    "learn200m": dict(n=200_000_000, m=1024, w=0.10, k=1),
    # wide bands (r = 0.9 m, the regime of the paper's experiments) on 2e7 samples of the
    # same kind: the one-warp walk (r <= 511) and the four-warp walk (511 < r <= 2047)
    "wide512": dict(n=20_000_000, m=512, w=0.90, k=1),
    "wide1024": dict(n=20_000_000, m=1024, w=0.90, k=1),
    "wide2048": dict(n=20_000_000, m=2048, w=0.90, k=1),
}


def cells(m: int, r: int) -> int:
    r = min(r, m - 1)
    return m * (2 * r + 1) - r * (r + 1)


# DRAM bytes (read + write) per window of k_lb_scan, from one ncu --set full capture of the
# current kernel on the n=3e7, m=512, r=51 case (360.05 + 3.35 MB over 29,999,489 windows);
# the bytes are dominated by the 12 B read per window, so they scale with the window count.
LB_SCAN_DRAM_BYTES_PER_WINDOW = 363.40e6 / 29_999_489


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [ln.strip().split(",") for ln in self.f.read().splitlines() if ln.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ workload
def make_workload(name: str, rank: int = 0, world: int = 1):
    """Series fragment of this rank and the query.  For world > 1 the series is
    `world` independent walks back to back (fragment k from seed k); rank k
    holds fragment k plus the first m-1 samples of fragment k+1 (Eq. 11)."""
    spec = SPECS[name]
    n, m = spec["n"], spec["m"]
    r = synth.band(spec["w"], m)

    def frag(k):
        if name in ("rw100m", "rw30m"):
            return synth.walk_with_bursts(n, 0 + 101 * k, 3 + 101 * k, 5 + 101 * k)
        if name in ("learn20m", "learn200m", "wide512", "wide1024", "wide2048"):
            return synth.walk_with_bursts(n, 4 + 101 * k, 4 + 101 * k, 6 + 101 * k)
        return synth.random_walk(n, 101 * k)

    x = frag(rank)
    if name in ("learn20m", "learn200m", "wide512", "wide1024", "wide2048"):
        qs, offs = synth.fixed_queries(frag(0) if rank != 0 else x, 1, m, 9)
        q, o = qs[0], offs[0]
    else:
        q, o = synth.noisy_copy(frag(0) if rank != 0 else x, m, 1, 2)
    if world > 1 and rank < world - 1:
        x = np.concatenate([x, frag(rank + 1)[: m - 1]])
    return x, q, r, spec["k"], o


# ------------------------------------------------------------------ CPU oracle
def cpu_oracle_sample(x, q, r, k, first: int, count: int):
    """Oracle cascade (FP64, anchored window statistics) over the windows
    [first, first + count), fragment-parallel over the host cores (Eq. 11)."""
    import oracle  # test infrastructure: the CPU baseline legs only
    from oracle import fragments
    m = q.size
    N = x.size - m + 1
    cnt = max(1, min(count, N - first))
    cores = fragments.host_threads()
    t0 = time.perf_counter()
    idx, dist = fragments.search_fragments(x, q, r, k, threads=cores, F=cores * 4, first=first,
                                           count=cnt, stats="anchored")
    dt = time.perf_counter() - t0
    _ = oracle
    whole = first == 0 and cnt == N
    what = "all windows" if whole else f"windows [{first}, {first + cnt})"
    return dict(value=cnt / dt, unit="subsequences/s", cores=cores, kind="oracle",
                sample=f"{what} of the same series and query (FP64 UCR-style cascade, anchored stats, "
                       f"Eq. 11 fragments over {cores} threads)", seconds=dt, windows=cnt,
                idx=[int(v) for v in idx], dist=[float(v) for v in dist])


def cpu_oracle_fp64_at(x, qs, r, answers):
    """The FP64 oracle's DTW at the windows the GPU returned (CPU oracle leg:
    the reference values of the FP32 error the drift workload reports)."""
    import oracle  # test infrastructure: the CPU baseline legs only
    return [float(oracle.dtw_at(x, q, r, [int(i)])[0]) for q, i in zip(qs, answers)]


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    x, q, r, k, o = make_workload(args.workload)
    # each step searches the first `budget` windows of the series (a slice
    # that starts at window 0, not one centred on the answer); sized so that
    # the whole warm-up + timed run takes about 150 s of host time
    probe = cpu_oracle_sample(x, q, r, k, 0, 1_000_000)
    rate = probe["windows"] / probe["seconds"]
    budget = int(max(1_000_000, rate * 150.0 / (args.warmup + args.steps)))
    if args.cpu_windows:
        budget = min(budget, args.cpu_windows)
    times = []
    res = None
    for s in range(args.warmup + args.steps):
        res = cpu_oracle_sample(x, q, r, k, 0, budget)
        if s >= args.warmup:
            times.append(res["seconds"])
    ms = 1e3 * statistics.mean(times)
    val = budget / (ms / 1e3)
    line = {
        "impl": "reference", "metric": "subsequences/s per query", "value": val,
        "unit": "subsequences/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: n={x.size}, m={q.size}, r={r}, k={k}; "
                               f"bounded sample of {budget} windows per step",
                   "parallelism": f"host threads x{res['cores']}"},
        "cpu_baseline": {"value": val, "unit": "subsequences/s", "cores": res["cores"],
                         "kind": "oracle", "sample": res["sample"]},
        "e2e": {"value": val, "unit": "subsequences/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
def gpu_arm(args):
    import torch

    from paper_1812_10302_gb300 import dtws

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    x, q, r, k, true_off = make_workload(args.workload, rank, world)
    m = q.size
    N = x.size - m + 1
    dtws.load(build_if_missing=False)
    xs = torch.from_numpy(x).to(dev)
    t0 = time.perf_counter()
    ix = dtws.Index(xs)
    torch.cuda.synchronize(dev)
    create_ms = 1e3 * (time.perf_counter() - t0)
    del xs
    if args.ordering == "learned":
        from paper_1812_10302_gb300 import train
        ix.set_encoder(train.load_weights())
        ix.set_options(ordering=dtws.DTWS_ORDER_LEARNED, seed_proposals=64)
    elif args.ordering == "random":
        ix.set_options(seed_proposals=0)
    qd = torch.from_numpy(q).to(dev)
    idx_d = torch.empty(k, dtype=torch.int64, device=dev)
    dist_d = torch.empty(k, dtype=torch.float32, device=dev)

    # per-series data for this (m, r): timed once, then resident
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ix.query(qd, r, k, out=(idx_d, dist_d))
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    first_ms = ev0.elapsed_time(ev1)

    def step():
        ix.query(qd, r, k, out=(idx_d, dist_d))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    first_query_ms = first_ms

    # -------- timed region (device): K steps, inputs resident, > L2
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    status = ix.sync_status()
    if status != dtws.DTWS_OK:
        raise RuntimeError(f"device-side error during the timed steps: {dtws.strerror(status)}")
    ms = e0.elapsed_time(e1) / args.steps
    st = ix.last_stats()
    launches = int(st["kernel_launches"]) * args.steps

    # -------- per-phase events (a second loop with phase timing on)
    ix.set_options(timing=1)
    phases = np.zeros(8)
    for _ in range(max(3, min(args.steps, 20))):
        step()
        s2 = ix.last_stats()
        phases += np.array(s2["phase_ms"])
    phases /= max(3, min(args.steps, 20))
    ix.set_options(timing=0)

    # -------- end to end through the C ABI with host buffers
    q_host = torch.from_numpy(q).pin_memory()
    idx_h = np.empty(k, np.int64)
    dist_h = np.empty(k, np.float32)
    for _ in range(args.warmup):
        ix.query(q_host, r, k)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        idx_h, dist_h = ix.query(q_host, r, k)   # H2D of Q, D2H of the result, synchronising
    e2e_ms = 1e3 * (time.perf_counter() - t0) / args.steps

    # -------- merge across ranks (Algorithm 1's exchange of {bsf, index}):
    # every rank's k best (distance, offset) pairs, offsets made global by
    # the rank's first window, all-gathered and merged into the global top-k
    merged = None
    if world > 1:
        import torch.distributed as dist

        from paper_1812_10302_gb300 import shard
        tms = torch.tensor([ms, e2e_ms], device=dev)
        dist.all_reduce(tms, op=dist.ReduceOp.MAX)
        ms, e2e_ms = float(tms[0]), float(tms[1])
        first_window = rank * SPECS[args.workload]["n"]  # rank k's fragment starts at sample k*n
        gi, gd = shard.allgather_merge(idx_h, dist_h, k, offset=first_window, device=dev)
        merged = {"offsets": [int(v) for v in gi], "dist": [float(v) for v in gd]}
        total_windows = N * world
    else:
        total_windows = N

    if rank != 0:
        ix.close()
        return 0

    hbm, peak_kind = load_peaks()
    lb_ms = float(phases[2])
    # 12 B read per window (sample, mean's high part, 1/sigma); the scan writes
    # (bound, offset) per survivor
    lb_bytes = N * 12 + st["pass_keogh_q"] * 8
    achieved = lb_bytes / (lb_ms * 1e-3) / 1e9 if lb_ms > 0 else None
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        # the oracle over every window of the same series and query (or the
        # first --cpu-windows of them when that is smaller), and whether it
        # returns the GPU's answer
        cpu = cpu_oracle_sample(x, q, r, k, 0, args.cpu_windows or N)
        cpu["agrees_with_gpu"] = (cpu["windows"] == N and cpu["idx"] == [int(v) for v in idx_h] and
                                  all(abs(a - b) <= 1e-4 * max(abs(b), 1e-6 * m) for a, b in
                                      zip(map(float, dist_h), cpu["dist"])))
    value = total_windows / (ms * 1e-3)
    # The DTW kernel against its ALU ceiling: every SM's 128 FP32/ALU lanes at
    # the maximum SM clock, 5 operations per band cell (subtract, multiply-add,
    # two minimums, the band select).  Measured on the kernel's walk itself:
    # dtws_dtw_at (no pruning) of the workload's query at 1e5 random windows,
    # cells(m, r) per window, CUDA events on the query stream; beside it the
    # survivor stage of the timed query (evaluated cells over the stage's
    # event time), which on this workload is a few hundred mostly abandoned
    # walks and measures latency, not throughput.
    dtw_roof = None
    try:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        peak_cells = sms * 128 * mhz * 1e6 / 5.0
        n_off = 100_000
        offs = torch.from_numpy(np.random.default_rng(7).integers(0, N, n_off).astype(np.int64)).to(dev)
        wout = torch.empty(n_off, dtype=torch.float32, device=dev)
        import ctypes
        sptr = ctypes.c_void_p(stream.cuda_stream)

        def walk():
            rc = ix._lib.dtws_dtw_at(ix.h, qd.data_ptr(), m, r, offs.data_ptr(), n_off, wout.data_ptr(), sptr)
            if rc != dtws.DTWS_OK:
                raise RuntimeError(f"dtws_dtw_at: {dtws.strerror(rc)}")
        walk()
        torch.cuda.synchronize(dev)
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0.record(stream)
        for _ in range(5):
            walk()
        w1.record(stream)
        torch.cuda.synchronize(dev)
        walk_ms = w0.elapsed_time(w1) / 5
        got = n_off * cells(m, r) / (walk_ms * 1e-3)
        dtw_ms = float(phases[4])
        surv = st["dtw_cells"] / (dtw_ms * 1e-3) if dtw_ms > 0 else None
        # the library's shape for DTW at offsets: four cells per lane on 8 or
        # 16 lanes for bands of 9..64 cells, else the survivor pass's shape
        need = r + 1
        shape = (f"{8 if need <= 32 else 16} lanes x 4 cells per window" if 8 < need <= 64
                 else "the survivor pass's shape")
        dtw_roof = {"kernel": "k_dtw (the walk: dtws_dtw_at, no pruning)", "shape": shape,
                    "bound": "alu", "achieved": got,
                    "peak": peak_cells, "unit": "cells/s", "frac": got / peak_cells, "ops_per_cell": 5,
                    "peak_source": f"{sms} SMs x 128 lanes x {mhz:.0f} MHz / 5",
                    "windows": n_off, "cells_per_window": cells(m, r), "ms_per_launch": walk_ms,
                    "survivor_stage": {"cells_per_s": surv, "frac": (surv / peak_cells) if surv else None,
                                       "dtw_started": st["dtw_started"], "dtw_ms": dtw_ms}}
    except (KeyError, IndexError, TypeError, RuntimeError):
        dtw_roof = None
    line = {
        "metric": "subsequences/s per query",
        "value": value,
        "unit": "subsequences/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": f"{args.workload}: random walk + sine bursts + N(0,0.5), n={x.size}, "
                        f"one m={m} noisy copy, r={r}, top-{k}",
            "global_batch": 1, "seq_len": m, "parallelism": f"fragments x{world}", "ordering": args.ordering,
            "l2": "inputs larger than L2 (series 0.4 GB + stats 1.2 GB + envelope 0.8 GB)",
        },
        "cells_per_s_bruteforce_equiv": total_windows * cells(m, r) / (ms * 1e-3),
        "cells_per_s_evaluated": st["dtw_cells"] / (ms * 1e-3),
        "precompute_ms": {"create_prefix": create_ms, "first_query_incl_stats_envelope": first_query_ms},
        "phase_ms": dict(zip(dtws.PHASES, [round(float(v), 4) for v in phases])),
        "survivors": {"kim": st["pass_kim"], "keogh_q": st["pass_keogh_q"], "keogh_s": st["pass_keogh_s"],
                      "dtw_started": st["dtw_started"], "dtw_abandoned": st["dtw_abandoned"]},
        "result": {"offset": int(idx_h[0]), "dist": float(dist_h[0]), "planted_offset": int(true_off),
                   "merged": merged},
        "roofline": {"kernel": "k_lb_scan", "bound": "hbm", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": (achieved / hbm) if achieved else None,
                     "traffic": LB_SCAN_DRAM_BYTES_PER_WINDOW * N, "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": lb_bytes},
        "dtw_roofline": dtw_roof,
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": {"value": total_windows / (e2e_ms * 1e-3), "unit": "subsequences/s",
                "h2d_bytes_per_step": int(m * 4), "d2h_bytes_per_step": int(k * 12),
                "ms_per_step": e2e_ms},
        "cpu_baseline": None if cpu is None else {k_: cpu[k_] for k_ in
                                                  ("value", "unit", "cores", "kind", "sample")},
    }
    if cpu is not None:
        line["cpu_baseline"]["seconds"] = cpu["seconds"]
        line["cpu_baseline"]["answer"] = {"offsets": cpu["idx"], "dist": cpu["dist"],
                                          "agrees_with_gpu": cpu["agrees_with_gpu"]}
    ix.close()
    if world == 1 and not args.no_extras:
        del qd, idx_d, dist_d
        torch.cuda.empty_cache()
        line["learned"] = learned_leg(dev)
        torch.cuda.empty_cache()
        line["batch"] = batch_leg(dev)
        torch.cuda.empty_cache()
        line["drift"] = drift_leg(dev, fp64_oracle=not args.no_cpu_baseline)
        torch.cuda.empty_cache()
        line["wide"] = wide_leg(dev)
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ other workloads (N = 1)
def _mean_query_ms(ix, qds, r, k, dev, reps=1):
    """Mean device time per query over the given device queries (events on
    the query stream), after one untimed query."""
    import torch
    stream = torch.cuda.current_stream(dev)
    idx = torch.empty(k, dtype=torch.int64, device=dev)
    dist = torch.empty(k, dtype=torch.float32, device=dev)
    ix.query(qds[0], r, k, out=(idx, dist))
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        for q in qds:
            ix.query(q, r, k, out=(idx, dist))
    e1.record(stream)
    torch.cuda.synchronize(dev)
    from paper_1812_10302_gb300 import dtws
    if ix.sync_status() != dtws.DTWS_OK:
        raise RuntimeError("device-side error in a timed query")
    return e0.elapsed_time(e1) / (len(qds) * reps)


def _phase_sample(ix, qs, rs, k, count):
    """Per-phase device times (events between the phases) and the cascade's
    survivor counters of `count` single queries (query i with band rs[i]),
    timing option on."""
    from paper_1812_10302_gb300 import dtws
    out = []
    ix.set_options(timing=1)
    for q, r in list(zip(qs, rs))[:count]:
        ix.query(q, int(r), k)
        st = ix.last_stats()
        out.append({"m": int(len(q)), "r": int(r),
                    "phase_ms": dict(zip(dtws.PHASES, [round(float(v), 4) for v in st["phase_ms"]])),
                    "survivors": {c: int(st[s]) for c, s in (("kim", "pass_kim"), ("keogh_q", "pass_keogh_q"),
                                                                ("keogh_s", "pass_keogh_s"),
                                                                ("dtw_started", "dtw_started"))}})
    ix.set_options(timing=0)
    return out


def learned_leg(dev):
    """Learned proposals on the learned-proposal workload (n = 2e8 walk with
    sine bursts, 64 noisy queries m = 1024, r = 102, top-1): mean ms per query
    with the learned ordering, the proxy ordering and the paper's random
    seeding (Algorithm 1; a bounded subset of queries: it is slow), and
    whether all three return the same answers."""
    import torch

    from paper_1812_10302_gb300 import dtws, synth, train
    w = synth.workload("learn")
    x, qs, r = w["series"], w["queries"], w["rs"][0]
    ix = dtws.Index(torch.from_numpy(x).to(dev))
    del x
    qds = [torch.from_numpy(q).to(dev) for q in qs]
    ix.set_encoder(train.load_weights())
    out = {"workload": "learn: walk + sine bursts + N(0,0.5), n=200000000, 64 noisy copies m=1024, r=102, top-1",
           "encoder": "trained on oracle-labelled pairs of a disjoint training series", "ms_per_query": {}}
    modes = {"learned": dict(ordering=dtws.DTWS_ORDER_LEARNED, seed_proposals=64),
             "proxy": dict(ordering=dtws.DTWS_ORDER_PLAIN, seed_proposals=16),
             "random_seeds": dict(ordering=dtws.DTWS_ORDER_PLAIN, seed_proposals=0)}
    answers = {}
    n_random = 4
    out["phase_ms"] = {}
    for name, opts in modes.items():
        ix.set_options(**opts)
        sub = qds if name != "random_seeds" else qds[:n_random]
        out["ms_per_query"][name] = _mean_query_ms(ix, sub, r, 1, dev)
        answers[name] = [tuple(np.concatenate([a.astype(np.float64) for a in ix.query(q, r, 1)])) for q in sub]
        # per-phase device times (events between the phases) over a few queries
        ix.set_options(timing=1)
        ph = np.zeros(len(dtws.PHASES))
        for q in sub[:4]:
            ix.query(q, r, 1)
            ph += np.array(ix.last_stats()["phase_ms"])
        ix.set_options(timing=0)
        out["phase_ms"][name] = dict(zip(dtws.PHASES[:6], [round(float(v) / min(4, len(sub)), 4) for v in ph[:6]]))
    out["random_seeds_queries"] = n_random
    t = out["ms_per_query"]
    out["speedup_vs_random_seeds"] = t["random_seeds"] / t["learned"]
    out["speedup_vs_proxy"] = t["proxy"] / t["learned"]
    out["identical_answers"] = (answers["learned"] == answers["proxy"] and
                                answers["learned"][:n_random] == answers["random_seeds"])
    # the same three orderings through one dtws_query_batch call (4 lanes)
    # over the first 16 queries: host queries and outputs, host wall clock
    # around the synchronising call, the best of the timed calls after one
    # untimed call
    nb = 16
    qb, rb = [np.asarray(q) for q in qs[:nb]], [r] * nb
    bt, bans = {}, {}
    for name, opts in modes.items():
        ix.set_options(batch_lanes=4, batch_graph=1, **opts)
        bans[name] = ix.query_batch(qb, rb, k=1)
        ts = []
        for _ in range(3 if name != "random_seeds" else 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            ix.query_batch(qb, rb, k=1)
            ts.append(time.perf_counter() - t0)
        bt[name] = min(ts)
    if ix.sync_status() != dtws.DTWS_OK:
        raise RuntimeError("device-side error in a batched query")
    out["batch"] = {"queries": nb, "lanes": 4, "seconds_per_batch": bt,
                    "speedup_vs_random_seeds": bt["random_seeds"] / bt["learned"],
                    "speedup_vs_proxy": bt["proxy"] / bt["learned"],
                    "identical_answers": all(np.array_equal(bans["learned"][j], bans[o][j])
                                             for o in ("proxy", "random_seeds") for j in (0, 1))}
    ix.close()
    return out


def batch_leg(dev):
    """The batched workload (n = 5e7 walk, 256 noisy queries with m in
    [128, 2048], r in [5%, 20%] of m, top-10) through dtws_query_batch: the
    first call captures the graph, later calls replay it."""
    import torch

    from paper_1812_10302_gb300 import dtws, synth
    w = synth.workload("batch")
    x, qs, rs, k = w["series"], w["queries"], w["rs"], w["k"]
    ix = dtws.Index(torch.from_numpy(x).to(dev))
    n = x.size
    del x
    ix.set_options(batch_lanes=4, batch_graph=1, exact_envelope=0)
    t0 = time.perf_counter()
    ix.query_batch(qs, rs, k=k)
    first = time.perf_counter() - t0
    ts = []
    for _ in range(3):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ix.query_batch(qs, rs, k=k)
        ts.append(time.perf_counter() - t0)
    if ix.sync_status() != dtws.DTWS_OK:
        raise RuntimeError("device-side error in the batch")
    sec = float(np.median(ts))
    windows = sum(n - len(q) + 1 for q in qs)
    # where a query's time goes: eight queries across the length range, alone
    order = np.argsort([len(q) for q in qs])
    pick = [int(order[j]) for j in np.linspace(0, len(qs) - 1, 8).round().astype(int)]
    sample = _phase_sample(ix, [qs[j] for j in pick], [rs[j] for j in pick], k, 8)
    ix.close()
    return {"workload": "batch: random walk n=50000000, 256 noisy copies m~U{128..2048}, r=floor(w m), "
                        "w~U[0.05,0.2], top-10",
            "seconds_per_batch": sec, "queries_per_s": len(qs) / sec, "subsequences_per_s": windows / sec,
            "first_call_seconds": first, "lanes": 4, "graph": "captured on the first call, replayed",
            "timing": "host wall clock around dtws_query_batch (synchronising; host queries and outputs)",
            "single_query_sample": sample}


def drift_leg(dev, fp64_oracle: bool = True):
    """The precision-stress workload (n = 1e9 walk with drift 1e-3 and
    variance regimes, 32 noisy queries m = 1024, r = 102, top-1): mean ms per
    query and, per query, the relative error against the FP64 oracle's DTW at
    the returned window of (a) the FP32 DTW the search prunes with and (b) the
    returned (extended-precision re-scored) distance."""
    import torch

    from paper_1812_10302_gb300 import dtws, synth
    w = synth.workload("drift")
    x, qs, r = w["series"], w["queries"], w["rs"][0]
    t0 = time.perf_counter()
    ix = dtws.Index(torch.from_numpy(x).to(dev))
    torch.cuda.synchronize(dev)
    create_s = time.perf_counter() - t0
    qds = [torch.from_numpy(q).to(dev) for q in qs]
    ms = _mean_query_ms(ix, qds, r, 1, dev)
    sample = _phase_sample(ix, qds, [r] * len(qds), 1, 4)
    ans, f32, ret = [], [], []
    for q in qs:
        i, d = ix.query(q, r, 1)
        ans.append(int(i[0]))
        ret.append(float(d[0]))
        f32.append(float(ix.dtw_at(q, r, i)[0]))
    ix.close()
    out = {"workload": "drift: walk with drift 1e-3 and variance regimes, n=1000000000, 32 noisy copies "
                       "m=1024, r=102, top-1",
           "ms_per_query": ms, "subsequences_per_s": (1_000_000_000 - 1023) / (ms * 1e-3),
           "create_seconds": create_s, "single_query_sample": sample}
    if fp64_oracle:
        ref = cpu_oracle_fp64_at(x, qs, r, ans)
        e32 = [abs(a - b) / max(b, 1e-30) for a, b in zip(f32, ref)]
        eret = [abs(a - b) / max(b, 1e-30) for a, b in zip(ret, ref)]
        out["fp32_dtw_rel_error_vs_fp64_oracle"] = {"max": max(e32), "median": float(np.median(e32))}
        out["returned_dist_rel_error_vs_fp64_oracle"] = {"max": max(eret), "median": float(np.median(eret))}
    return out


def wide_leg(dev):
    """Wide bands, the regime of the paper's experiments (r = 0.9 m): the
    wide1024 (m = 1024, r = 921) and wide2048 (m = 2048, r = 1843) workloads
    on 2e7 samples, one noisy query each: mean ms per query after the
    per-series data is built, phase times, and the survivor DTW stage's
    evaluated cells per second."""
    import torch

    from paper_1812_10302_gb300 import dtws
    out = {}
    for name in ("wide1024", "wide2048"):
        x, q, r, k, o = make_workload(name)
        ix = dtws.Index(torch.from_numpy(x).to(dev))
        qd = torch.from_numpy(q).to(dev)
        ms = _mean_query_ms(ix, [qd], r, k, dev, reps=5)
        idx, dist = ix.query(q, r, k)
        sample = _phase_sample(ix, [qd], [r], k, 1)[0]
        st = ix.last_stats()
        ix.close()
        dtw_ms = sample["phase_ms"]["dtw"]
        out[name] = {"n": int(x.size), "m": int(q.size), "r": int(r), "ms_per_query": ms,
                     "subsequences_per_s": (x.size - q.size + 1) / (ms * 1e-3),
                     "dtw_cells_evaluated": int(st["dtw_cells"]),
                     "dtw_cells_per_s": (st["dtw_cells"] / (dtw_ms * 1e-3)) if dtw_ms > 0 else None,
                     "phase_ms": sample["phase_ms"], "survivors": sample["survivors"],
                     "result": {"offset": int(idx[0]), "dist": float(dist[0]), "planted_offset": int(o)}}
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="dtws", choices=["dtws", "reference"])
    ap.add_argument("--workload", default="rw100m", choices=sorted(SPECS))
    ap.add_argument("--cpu-windows", type=int, default=0,
                    help="windows in the CPU oracle's sample (0: every window for the GPU arm's "
                         "cpu_baseline; the reference arm sizes its steps itself, at most this many "
                         "when given)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ordering", default="proxy", choices=["proxy", "learned", "random"],
                    help="seeding of the timed queries: proxy scan (default), learned proposals, or "
                         "random windows only (the paper's Algorithm 1)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the learned-proposal and batched workloads (N = 1 only)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
