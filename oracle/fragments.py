"""Overlap fragmentation (Sec. 3.1, Eq. 11) over host threads.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  The paper cuts the series
into F fragments of about equal length, each extended by m-1 samples of the
next, so that no window is lost at a seam.  In window units (0-based), with
N windows, fragment k covers windows [k*floor(N/F), k*floor(N/F) + len_k)
with len_k = floor(N/F), plus N mod F for the last fragment.

Each fragment runs the oracle's cascade on its own host thread (ctypes drops
the GIL during the C call); the per-fragment top-k lists are merged by
(distance, index), which is the global top-k because every window belongs to
exactly one fragment.
"""
from __future__ import annotations

import os
import threading

import numpy as np

from . import search_cascade


def partition(N: int, F: int) -> list[tuple[int, int]]:
    """Eq. 11 in window units: list of (first window, number of windows)."""
    if F < 1 or N < 1:
        raise ValueError("need N >= 1 and F >= 1")
    F = min(F, N)
    base = N // F
    out = []
    for k in range(F):
        length = base + (N % F if k == F - 1 else 0)
        out.append((k * base, length))
    return out


def merge_topk(parts, k: int):
    """Merge per-fragment (idx, dist) lists into the k smallest (dist, idx)."""
    idx = np.concatenate([p[0] for p in parts])
    dist = np.concatenate([p[1] for p in parts])
    keep = idx >= 0
    idx, dist = idx[keep], dist[keep]
    order = np.lexsort((idx, dist))[:k]
    out_i = np.full(k, -1, np.int64)
    out_d = np.full(k, np.inf)
    out_i[: order.size] = idx[order]
    out_d[: order.size] = dist[order]
    return out_i, out_d


def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def search_fragments(x, Q, r: int, k: int, F: int | None = None, threads: int | None = None,
                     first: int = 0, count: int | None = None, stats: str = "twopass"):
    """Cascade over windows [first, first+count), cut into F fragments by
    Eq. 11 and run on ``threads`` host threads; returns the merged top-k."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    m = Q.size
    N = x.size - m + 1
    count = N - first if count is None else count
    threads = threads or host_threads()
    F = F or threads
    frags = [(first + s, c) for s, c in partition(count, F)]
    results: list = [None] * len(frags)
    errors: list = []
    cursor = [0]
    lock = threading.Lock()

    def worker():
        while True:
            with lock:
                j = cursor[0]
                cursor[0] += 1
            if j >= len(frags):
                return
            s, c = frags[j]
            try:
                results[j] = search_cascade(x, Q, r, k, first=s, count=c, stats=stats)
            except Exception as e:  # propagate to the caller
                errors.append(e)
                return

    ts = [threading.Thread(target=worker) for _ in range(min(threads, len(frags)))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errors:
        raise errors[0]
    return merge_topk(results, k)
