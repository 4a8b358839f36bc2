"""Sharding one search across processes (one per GPU).

The paper distributes the series over cluster nodes by overlapping fragments
(Sec. 3.1, Eq. 11): with N windows and F fragments, fragment k holds windows
[k*floor(N/F), k*floor(N/F) + len_k), len_k = floor(N/F) (+ N mod F for the
last), i.e. samples [start, start + len_k + m - 1), so no window is lost at a
seam.  Each process searches its fragment; the only exchange is the merge of
the per-fragment best (distance, offset) pairs, the analogue of Algorithm 1's
MIN all-reduce of {bsf, bestmatch}.  Here it is one all-gather of the k best
pairs per rank at the end of a query.

Host logic only (no kernels); torch.distributed carries the exchange.
"""
from __future__ import annotations

import numpy as np


def fragment(N: int, F: int, k: int) -> tuple[int, int]:
    """Eq. 11 in window units: (first window, number of windows) of fragment k."""
    if not (0 <= k < F) or N < F:
        raise ValueError("need 0 <= k < F <= N")
    base = N // F
    length = base + (N % F if k == F - 1 else 0)
    return k * base, length


def fragment_samples(n: int, m: int, F: int, k: int) -> tuple[int, int]:
    """Sample range [start, stop) that fragment k needs (its windows plus the
    m - 1 samples of overlap)."""
    first, length = fragment(n - m + 1, F, k)
    return first, first + length + m - 1


def merge_topk(idx_lists, dist_lists, k: int):
    """The k smallest (distance, offset) pairs over all fragments (offsets
    already global); -1 / inf fill missing entries."""
    idx = np.concatenate([np.asarray(i, np.int64) for i in idx_lists])
    dist = np.concatenate([np.asarray(d, np.float64) for d in dist_lists])
    keep = idx >= 0
    idx, dist = idx[keep], dist[keep]
    order = np.lexsort((idx, dist))[:k]
    out_i = np.full(k, -1, np.int64)
    out_d = np.full(k, np.inf)
    out_i[: order.size] = idx[order]
    out_d[: order.size] = dist[order]
    return out_i, out_d


def allgather_merge(idx, dist, k: int, offset: int, group=None, device=None):
    """Exchange every rank's k best pairs (local offsets + `offset` = global)
    and return the merged global top-k on every rank."""
    import torch
    import torch.distributed as dist_mod
    dev = device or "cpu"
    mine = torch.zeros((k, 2), dtype=torch.float64, device=dev)
    ii = np.asarray(idx, np.int64)
    dd = np.asarray(dist, np.float64)
    glob = np.where(ii >= 0, ii + offset, -1)
    mine[:, 0] = torch.from_numpy(dd)
    mine[:, 1] = torch.from_numpy(glob.astype(np.float64))
    world = dist_mod.get_world_size(group)
    parts = [torch.zeros_like(mine) for _ in range(world)]
    dist_mod.all_gather(parts, mine, group=group)
    parts = [p.cpu().numpy() for p in parts]
    return merge_topk([p[:, 1].astype(np.int64) for p in parts], [p[:, 0] for p in parts], k)
