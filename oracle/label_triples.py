"""Labels of encoder training triples by the FP64 oracle.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``): this script only calls the
oracle and the seeded input generators.  For each query length m it draws
(query, candidate) offset pairs on the training series
(``synth.training_pairs``; queries cut from the noisy copy, candidates from
the series itself) and labels each pair with y = DTW(Q^, C^)/m, the banded
DTW of Eq. 1 with r = floor(0.1 m) over z-normalised windows (Eq. 5), in
FP64 over the host's threads.  Writes an .npz with, per m, the arrays
q_off, c_off (int64) and y (float32).

    python -m oracle.label_triples --out triples.npz --n 20000000 \\
        --m 512 1024 --count 500000
"""
from __future__ import annotations

import argparse
import threading
import time

import numpy as np

from paper_1812_10302_gb300 import synth

from . import dtw_at
from .fragments import host_threads


def label(x, xq, q_off, c_off, m: int, r: int, threads: int) -> np.ndarray:
    """y[i] = DTW(xq[q_off[i]:+m], x[c_off[i]:+m]) / m (pairs grouped by query)."""
    y = np.empty(q_off.size, np.float64)
    starts = np.flatnonzero(np.r_[True, q_off[1:] != q_off[:-1]])
    bounds = np.r_[starts, q_off.size]
    cursor = [0]
    lock = threading.Lock()
    errors = []

    def work():
        while True:
            with lock:
                g = cursor[0]
                cursor[0] += 1
            if g >= bounds.size - 1:
                return
            a, b = bounds[g], bounds[g + 1]
            try:
                q = xq[q_off[a]:q_off[a] + m]
                y[a:b] = dtw_at(x, q, r, c_off[a:b]) / m
            except Exception as e:  # pragma: no cover - surfaced below
                errors.append(e)
                return

    ts = [threading.Thread(target=work) for _ in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errors:
        raise errors[0]
    return y


def make(n: int, ms, count: int, seed: int = 100, threads: int | None = None) -> dict:
    x, xq = synth.training_series(n, seed)
    threads = threads or host_threads()
    out = {}
    for j, m in enumerate(ms):
        q_off, c_off = synth.training_pairs(n, m, count, seed + 10 + j)
        y = label(x, xq, q_off, c_off, m, synth.band(0.1, m), threads)
        out[f"m{m}_q_off"] = q_off
        out[f"m{m}_c_off"] = c_off
        out[f"m{m}_y"] = y.astype(np.float32)
    out["ms"] = np.asarray(ms, np.int64)
    out["n"] = np.int64(n)
    out["seed"] = np.int64(seed)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--n", type=int, default=20_000_000)
    ap.add_argument("--m", type=int, nargs="+", default=[512, 1024])
    ap.add_argument("--count", type=int, default=500_000, help="pairs per query length")
    ap.add_argument("--seed", type=int, default=100)
    args = ap.parse_args(argv)
    t0 = time.perf_counter()
    d = make(args.n, args.m, args.count, args.seed)
    np.savez(args.out, **d)
    print(f"labelled {args.count} pairs for m={args.m} on n={args.n} in {time.perf_counter() - t0:.1f} s "
          f"({host_threads()} threads)")


if __name__ == "__main__":
    main()
