"""Seeded synthetic inputs (series and queries) shared by the GPU tests, the
oracle tests and the benchmark.

This module holds no arithmetic of the search method: it only draws numbers.
All generators use NumPy's PCG64 (``numpy.random.default_rng(seed)``); walks
are accumulated in FP64 and stored as FP32, and the first sample is the first
step.  The recipes stand in for the paper's Random Walk series (Sec. 4.2) and
for its real EPG/ECG recordings (Secs. 4.2-4.3), which are not available here.

Workloads (n = series length, m = query length, r = band half-width):

=====  ==============================================================  ======
name   series / queries                                                r, k
=====  ==============================================================  ======
rw1m   n=1e6 random walk (seed 0); one m=128 query, a noisy copy        6, 1
rw100m n=1e8 random walk + sine bursts + N(0,0.5); one m=512 query      51, 1
batch  n=5e7 random walk; 256 queries m~U{128..2048}, w~U[.05,.20]     w*m, 10
drift  n=1e9 walk with drift 1e-3 and variance regimes; 32 x m=1024    102, 1
learn  n=2e8 random walk + sine bursts (seed 4); 64 x m=1024            102, 1
=====  ==============================================================  ======

A noisy copy is ``x[o:o+m] + N(0, 0.1)`` (0.1 is the standard deviation) at a
uniformly drawn offset o.  The band half-width from a fraction w of the query
length is ``floor(w*m)``.
"""
from __future__ import annotations

import math

import numpy as np

_CHUNK = 1 << 22


def _normals(rng: np.random.Generator, n: int, scale=1.0) -> np.ndarray:
    """n standard normals (FP64) drawn in fixed-size chunks, times scale."""
    out = np.empty(n, np.float64)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        out[s:e] = rng.standard_normal(e - s)
    if not (np.isscalar(scale) and scale == 1.0):
        out *= scale
    return out


def random_walk(n: int, seed: int = 0, step_scale=1.0, drift: float = 0.0) -> np.ndarray:
    """x[t] = x[t-1] + drift + N(0,1)*step_scale, x[0] = the first step; FP32.

    Accumulates chunk by chunk in FP64 so memory stays O(chunk) beyond the
    FP32 output."""
    rng = np.random.default_rng(seed)
    out = np.empty(n, np.float32)
    carry = 0.0
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        steps = rng.standard_normal(e - s)
        if not np.isscalar(step_scale):
            steps *= step_scale[s:e]
        elif step_scale != 1.0:
            steps *= step_scale
        if drift:
            steps += drift
        np.cumsum(steps, out=steps)
        steps += carry
        carry = float(steps[-1])
        out[s:e] = steps
    return out


def sine_bursts(n: int, seed: int, mean_gap: float = 1e5, length=(1e3, 1e4),
                period=(50.0, 500.0), amplitude=(1.0, 5.0)) -> np.ndarray:
    """Sum of sine bursts (FP64): Poisson starts with the given mean gap,
    length ~ U[length], period ~ U[period], amplitude ~ U[amplitude],
    phase ~ U[0, 2 pi]."""
    rng = np.random.default_rng(seed)
    out = np.zeros(n, np.float64)
    t = 0.0
    while True:
        t += rng.exponential(mean_gap)
        start = int(t)
        if start >= n:
            break
        ln = int(rng.uniform(*length))
        per = rng.uniform(*period)
        amp = rng.uniform(*amplitude)
        ph = rng.uniform(0.0, 2 * math.pi)
        e = min(n, start + ln)
        tt = np.arange(e - start, dtype=np.float64)
        out[start:e] += amp * np.sin(2 * math.pi * tt / per + ph)
    return out


def walk_with_bursts(n: int, walk_seed: int, burst_seed: int, noise_seed: int,
                     noise: float = 0.5) -> np.ndarray:
    """Random walk + sine bursts + N(0, noise) per point, FP32."""
    x = random_walk(n, walk_seed).astype(np.float64)
    x += sine_bursts(n, burst_seed)
    x += _normals(np.random.default_rng(noise_seed), n, noise)
    return x.astype(np.float32)


def drifting_regimes(n: int, seed: int = 0, drift: float = 1e-3,
                     regime=(5e6, 1.5e7)) -> np.ndarray:
    """Walk with drift whose step variance is scaled by 10^U(-1,1) on regimes
    of length ~ U[regime]; FP32."""
    rng = np.random.default_rng(seed + 1000)
    scale = np.empty(n, np.float64)
    s = 0
    while s < n:
        ln = int(rng.uniform(*regime))
        scale[s:s + ln] = math.sqrt(10.0 ** rng.uniform(-1.0, 1.0))
        s += ln
    return random_walk(n, seed, step_scale=scale, drift=drift)


def noisy_copy(x: np.ndarray, m: int, offset_seed: int, noise_seed: int,
               noise: float = 0.1) -> tuple[np.ndarray, int]:
    """(x[o:o+m] + N(0, noise), o) with o ~ U{0..n-m}."""
    o = int(np.random.default_rng(offset_seed).integers(0, x.size - m + 1))
    q = x[o:o + m].astype(np.float64) + _normals(np.random.default_rng(noise_seed), m, noise)
    return q.astype(np.float32), o


def band(w: float, m: int) -> int:
    """Integer band half-width from a fraction of the query length."""
    return int(math.floor(w * m))


def batch_queries(x: np.ndarray, count: int, seed: int, m_range=(128, 2048),
                  w_range=(0.05, 0.20), noise: float = 0.1):
    """``count`` noisy copies with m ~ U{m_range}, w ~ U[w_range].
    Returns (list of FP32 queries, list of r, list of true offsets)."""
    rng = np.random.default_rng(seed)
    qs, rs, offs = [], [], []
    for _ in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        w = float(rng.uniform(*w_range))
        o = int(rng.integers(0, x.size - m + 1))
        q = x[o:o + m].astype(np.float64) + rng.standard_normal(m) * noise
        qs.append(q.astype(np.float32))
        rs.append(band(w, m))
        offs.append(o)
    return qs, rs, offs


def fixed_queries(x: np.ndarray, count: int, m: int, seed: int, noise: float = 0.1):
    """``count`` noisy copies of length m at uniform offsets."""
    rng = np.random.default_rng(seed)
    qs, offs = [], []
    for _ in range(count):
        o = int(rng.integers(0, x.size - m + 1))
        q = x[o:o + m].astype(np.float64) + rng.standard_normal(m) * noise
        qs.append(q.astype(np.float32))
        offs.append(o)
    return qs, offs


# ------------------------------------------------------------------ workloads
def training_series(n: int, seed: int = 100, noise: float = 0.1):
    """Encoder training data, disjoint from every evaluation series (its own
    seeds): a walk with sine bursts (as the learned-proposal workload) and a
    noisy copy of it (+ N(0, noise)), from which training queries are cut."""
    x = walk_with_bursts(n, seed, seed + 1, seed + 2)
    xq = (x.astype(np.float64) + _normals(np.random.default_rng(seed + 3), n, noise)).astype(np.float32)
    return x, xq


def training_pairs(n: int, m: int, count: int, seed: int, per_query: int = 16):
    """Offsets of (query, candidate) pairs: ``count`` pairs, ``per_query``
    candidates per query offset q: the copy itself (q), 4 near offsets
    (q + U{-b..b}, b = m // 64), 4 at q + U{-m..m}, the rest uniform.
    Returns (q_off, c_off) int64 arrays, grouped by query."""
    if per_query < 10:
        raise ValueError("per_query must be at least 10")
    rng = np.random.default_rng(seed)
    nq = (count + per_query - 1) // per_query
    hi = n - m
    b = max(1, m // 64)
    q = rng.integers(0, hi + 1, nq)
    c = np.empty((nq, per_query), np.int64)
    c[:, 0] = q
    c[:, 1:5] = q[:, None] + rng.integers(-b, b + 1, (nq, 4))
    c[:, 5:9] = q[:, None] + rng.integers(-m, m + 1, (nq, 4))
    c[:, 9:] = rng.integers(0, hi + 1, (nq, per_query - 9))
    c = np.clip(c, 0, hi)
    qq = np.repeat(q, per_query)
    return qq[:count].astype(np.int64), c.reshape(-1)[:count].astype(np.int64)


WORKLOADS = {
    "rw1m": dict(n=1_000_000, m=128, w=0.05, k=1, queries=1),
    "rw100m": dict(n=100_000_000, m=512, w=0.10, k=1, queries=1),
    "batch": dict(n=50_000_000, m=(128, 2048), w=(0.05, 0.20), k=10, queries=256),
    "drift": dict(n=1_000_000_000, m=1024, w=0.10, k=1, queries=32),
    "learn": dict(n=200_000_000, m=1024, w=0.10, k=1, queries=64),
}


def workload(name: str, n: int | None = None):
    """Series and queries of a named workload (``n`` overrides the length for
    scaled-down test cases).  Returns a dict with series, queries, rs, k and
    true_offsets."""
    spec = WORKLOADS[name]
    n = n or spec["n"]
    if name == "rw1m":
        x = random_walk(n, 0)
        q, o = noisy_copy(x, spec["m"], 1, 2)
        return dict(series=x, queries=[q], rs=[band(spec["w"], spec["m"])], k=1, true_offsets=[o])
    if name == "rw100m":
        x = walk_with_bursts(n, 0, 3, 5)
        q, o = noisy_copy(x, spec["m"], 1, 2)
        return dict(series=x, queries=[q], rs=[band(spec["w"], spec["m"])], k=1, true_offsets=[o])
    if name == "batch":
        x = random_walk(n, 0)
        qs, rs, offs = batch_queries(x, spec["queries"], 7)
        return dict(series=x, queries=qs, rs=rs, k=spec["k"], true_offsets=offs)
    if name == "drift":
        x = drifting_regimes(n, 0)
        qs, offs = fixed_queries(x, spec["queries"], spec["m"], 8)
        return dict(series=x, queries=qs, rs=[band(spec["w"], spec["m"])] * len(qs), k=1,
                    true_offsets=offs)
    if name == "learn":
        x = walk_with_bursts(n, 4, 4, 6)
        qs, offs = fixed_queries(x, spec["queries"], spec["m"], 9)
        return dict(series=x, queries=qs, rs=[band(spec["w"], spec["m"])] * len(qs), k=1,
                    true_offsets=offs)
    raise KeyError(name)
