"""FP64 CPU oracle for banded-DTW best-match subsequence search.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  It shares no code
with the GPU library (``paper_1812_10302_gb300``) and never imports it; the
library never imports this package.

The arithmetic lives in ``dtw_oracle.c`` (plain C, FP64), which cites the
paper's equations function by function:

* z-normalisation, Sec. 2.2, Eq. 5 (population sigma, two-pass evaluation);
* banded DTW, Sec. 2.1, Eq. 1 plus the Sakoe-Chiba band;
* LB_KimFL (Eq. 7), envelope (Eq. 9), LB_Keogh (Eqs. 8 and 10);
* the UCR-DTW-style cascade scan of Sec. 2.2 and the brute-force problem
  statement (Eq. 3);
* anchored block prefix sums for window statistics of long series.

``fragments.py`` adds the overlap partition of Sec. 3.1, Eq. 11, run over
host threads, for the timed CPU baseline.

This module is argument marshalling only (numpy <-> ctypes).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dtw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

INF = float("inf")


def build(force: bool = False) -> str:
    """Compile dtw_oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-Wall", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int64
        D = ctypes.c_double
        sig = {
            "orc_sigma_is_zero": (ctypes.c_int, [D, D]),
            "orc_stats_twopass": (None, [P, I, P, P]),
            "orc_normalize": (None, [P, I, D, D, P]),
            "orc_znorm": (None, [P, I, P]),
            "orc_window_stats_twopass": (None, [P, I, I, P, P]),
            "orc_window_stats_anchored": (ctypes.c_int, [P, I, I, I, P, P]),
            "orc_dtw": (D, [P, P, I, I, D, P]),
            "orc_dtw_full": (D, [P, P, I, I]),
            "orc_lb_kim_fl": (D, [P, P, I]),
            "orc_envelope": (None, [P, I, I, P, P]),
            "orc_lb_keogh": (D, [P, P, P, I, D]),
            "orc_search_brute": (ctypes.c_int, [P, I, P, I, I, I, I, I, P, P]),
            "orc_search_cascade": (ctypes.c_int, [P, I, P, I, I, I, I, I, ctypes.c_int, I, P, P, P]),
            "orc_dtw_at": (ctypes.c_int, [P, I, P, I, I, P, I, P]),
            "orc_series_envelope": (None, [P, I, I, P, P]),
            "orc_lbs_at": (ctypes.c_int, [P, I, P, I, I, P, I, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- z-norm, Eq. 5
def stats_twopass(x) -> tuple[float, float]:
    """(mu, sigma) of x, population sigma, two-pass; sigma=0 by the zero rule."""
    x = _f32(x)
    mu, sg = ctypes.c_double(), ctypes.c_double()
    _load().orc_stats_twopass(_p(x), x.size, ctypes.byref(mu), ctypes.byref(sg))
    return mu.value, sg.value


def sigma_is_zero(mu: float, var: float) -> bool:
    return bool(_load().orc_sigma_is_zero(mu, var))


def znorm(x) -> np.ndarray:
    x = _f32(x)
    out = np.empty(x.size, np.float64)
    _load().orc_znorm(_p(x), x.size, _p(out))
    return out


def window_stats(x, m: int, mode: str = "twopass", B: int | None = None):
    """Per-window (mu, sigma) for every window of length m.  ``B`` is the
    anchored method's block length (default max(8192, m))."""
    x = _f32(x)
    B = max(8192, m) if B is None else B
    N = x.size - m + 1
    mu = np.empty(N, np.float64)
    sg = np.empty(N, np.float64)
    lib = _load()
    if mode == "twopass":
        lib.orc_window_stats_twopass(_p(x), x.size, m, _p(mu), _p(sg))
    elif mode == "anchored":
        if lib.orc_window_stats_anchored(_p(x), x.size, m, B, _p(mu), _p(sg)) != 0:
            raise ValueError("anchored stats need B >= m")
    else:
        raise ValueError(mode)
    return mu, sg


# ---------------------------------------------------------------- DTW, Eq. 1
def dtw(q, c, r: int, bsf: float = INF) -> float:
    """Banded DTW of two equal-length FP64 sequences (already normalised)."""
    q = _f64(q)
    c = _f64(c)
    assert q.size == c.size
    m = q.size
    work = np.empty((m + 1) * (m + 1), np.float64)
    return _load().orc_dtw(_p(q), _p(c), m, r, bsf, _p(work))


# ---------------------------------------------------------------- LBs, Eqs. 7-10
def lb_kim_fl(qh, ch) -> float:
    qh = _f64(qh)
    ch = _f64(ch)
    return _load().orc_lb_kim_fl(_p(qh), _p(ch), qh.size)


def envelope(v, r: int):
    v = _f64(v)
    U = np.empty(v.size, np.float64)
    L = np.empty(v.size, np.float64)
    _load().orc_envelope(_p(v), v.size, r, _p(U), _p(L))
    return U, L


def lb_keogh(v, U, L, bsf: float = INF) -> float:
    v, U, L = _f64(v), _f64(U), _f64(L)
    return _load().orc_lb_keogh(_p(v), _p(U), _p(L), v.size, bsf)


def series_envelope(x, r: int):
    x = _f32(x)
    U = np.empty(x.size, np.float32)
    L = np.empty(x.size, np.float32)
    _load().orc_series_envelope(_p(x), x.size, r, _p(U), _p(L))
    return U, L


# ---------------------------------------------------------------- search
def search_brute(x, Q, r: int, k: int, first: int = 0, count: int | None = None):
    """Eq. 3 by definition: DTW against every window; k smallest (dist, idx)."""
    x, Q = _f32(x), _f32(Q)
    m = Q.size
    N = x.size - m + 1
    count = N - first if count is None else count
    idx = np.empty(k, np.int64)
    dist = np.empty(k, np.float64)
    rc = _load().orc_search_brute(_p(x), x.size, _p(Q), m, r, k, first, count, _p(idx), _p(dist))
    if rc != 0:
        raise ValueError("bad arguments")
    return idx, dist


def search_cascade(x, Q, r: int, k: int, first: int = 0, count: int | None = None,
                   stats: str = "twopass", B: int | None = None, counters: bool = False):
    """UCR-DTW-style cascade (Sec. 2.2) over windows [first, first+count)."""
    x, Q = _f32(x), _f32(Q)
    m = Q.size
    B = max(8192, m) if B is None else B
    N = x.size - m + 1
    count = N - first if count is None else count
    idx = np.empty(k, np.int64)
    dist = np.empty(k, np.float64)
    ctr = np.zeros(5, np.int64)
    mode = {"twopass": 0, "anchored": 1}[stats]
    rc = _load().orc_search_cascade(_p(x), x.size, _p(Q), m, r, k, first, count, mode, B,
                                    _p(idx), _p(dist), _p(ctr))
    if rc != 0:
        raise ValueError("bad arguments")
    if counters:
        return idx, dist, dict(zip(["kim", "keogh_q", "keogh_c", "dtw", "abandoned"], ctr.tolist()))
    return idx, dist


def dtw_at(x, Q, r: int, offsets) -> np.ndarray:
    """FP64 DTW of the normalised query against the normalised windows at offsets."""
    x, Q = _f32(x), _f32(Q)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    out = np.empty(off.size, np.float64)
    _load().orc_dtw_at(_p(x), x.size, _p(Q), Q.size, r, _p(off), off.size, _p(out))
    return out


def lbs_at(x, Q, r: int, offsets):
    """(kim, keogh vs query envelope, keogh vs clipped window envelope,
    keogh vs series-wide envelope) at each offset, FP64."""
    x, Q = _f32(x), _f32(Q)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    outs = [np.empty(off.size, np.float64) for _ in range(4)]
    _load().orc_lbs_at(_p(x), x.size, _p(Q), Q.size, r, _p(off), off.size, *[_p(o) for o in outs])
    return tuple(outs)


# ---------------------------------------------------------------- variants
# (the paper is silent on both; they are defined here for the GPU path's
# next steps and pinned in tests/test_oracle_variants.py)
def search_brute_raw(x, Q, r: int, k: int):
    """Eq. 3 without the z-normalisation of Eq. 5: banded DTW (Eq. 1) of the
    raw query against every raw window, in FP64; the k smallest
    (distance, offset) pairs, ties to the lower offset."""
    x64, q64 = _f64(_f32(x)), _f64(_f32(Q))
    m = q64.size
    N = x64.size - m + 1
    if m < 1 or N < 1 or k < 1:
        raise ValueError("bad arguments")
    d = np.array([dtw(q64, x64[i:i + m], r) for i in range(N)])
    order = np.lexsort((np.arange(N), d))[:k]
    return order.astype(np.int64), d[order]


def exclusion_topk(dists, k: int, z: int):
    """Top-k with an exclusion zone: take windows in (distance, offset) order,
    skipping any window within z samples of one already taken, until k are
    taken (fewer if the windows run out).  dists: the distance of every
    window, by offset."""
    d = np.asarray(dists, np.float64)
    taken: list[int] = []
    for i in np.lexsort((np.arange(d.size), d)):
        if all(abs(int(i) - t) > z for t in taken):
            taken.append(int(i))
            if len(taken) == k:
                break
    idx = np.array(taken, np.int64)
    return idx, d[idx]


def separated_kth(dists, k: int, sep: int, order=None) -> float:
    """A pruning threshold for top-k with an exclusion zone z (``exclusion_topk``),
    taken from windows found so far: insert the windows ``order`` (offsets,
    default every window by offset) one at a time into a set that keeps, of
    any two windows within ``sep`` samples of each other, the one with the
    smaller (distance, offset); return the k-th smallest distance in the set
    (inf if it holds fewer than k).  The kept windows are pairwise more than
    ``sep`` apart.  With sep = 2z the result is an upper bound of the k-th
    distance of the exclusion-zone answer: each window that the greedy
    selection takes, or that it skips because of a taken window, accounts for
    at most one kept window (two kept windows within z of one taken window
    would be at most 2z apart), so the selection has taken k windows before
    its distances pass the k-th kept one.  With sep = z it is not a bound
    (one taken window can shut out two kept ones)."""
    d = np.asarray(dists, np.float64)
    kept: dict[int, float] = {}
    for w in (range(d.size) if order is None else order):
        w = int(w)
        near = [v for v in kept if abs(v - w) <= sep]
        if any((kept[v], v) < (d[w], w) for v in near):
            continue
        for v in near:
            del kept[v]
        kept[w] = float(d[w])
    vals = sorted(kept.values())
    return vals[k - 1] if len(vals) >= k else INF
