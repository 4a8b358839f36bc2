"""Pins of the oracle's variants (unnormalised DTW search, top-k with an
exclusion zone) against closed forms, invariances and independent paths."""
import numpy as np
import pytest

import oracle
from paper_1812_10302_gb300 import synth


def _sq_ed(x, q):
    """Squared Euclidean distance of q to every window of x (NumPy)."""
    x = x.astype(np.float64)
    q = q.astype(np.float64)
    w = np.lib.stride_tricks.sliding_window_view(x, q.size)
    return ((w - q) ** 2).sum(axis=1)


def test_raw_search_with_r0_is_squared_euclidean():
    x = synth.random_walk(600, 1)
    q = synth.random_walk(24, 2)
    idx, dist = oracle.search_brute_raw(x, q, 0, 5)
    ed = _sq_ed(x, q)
    want = np.lexsort((np.arange(ed.size), ed))[:5]
    np.testing.assert_array_equal(idx, want)
    np.testing.assert_allclose(dist, ed[want], rtol=1e-12)


def test_raw_dtw_is_at_most_euclidean_and_finds_a_planted_copy():
    x = synth.random_walk(500, 3)
    o = 217
    q = x[o:o + 32].copy()
    idx, dist = oracle.search_brute_raw(x, q, 3, 1)
    assert idx[0] == o and dist[0] == 0.0
    ed = _sq_ed(x, q)
    for i in np.random.default_rng(4).integers(0, ed.size, 40):
        assert oracle.dtw(q.astype(np.float64), x[i:i + 32].astype(np.float64), 3) <= ed[i] * (1 + 1e-12)


def test_raw_search_translation_and_scale():
    # values on a 2^-6 grid: the shifted and doubled inputs are exact in FP32
    rng = np.random.default_rng(5)
    x = (np.round(np.cumsum(rng.normal(0, 1, 400)) * 64) / 64).astype(np.float32)
    q = (np.round(np.cumsum(rng.normal(0, 1, 20)) * 64) / 64).astype(np.float32)
    i0, d0 = oracle.search_brute_raw(x, q, 4, 6)
    i1, d1 = oracle.search_brute_raw(x + np.float32(8.0), q + np.float32(8.0), 4, 6)
    i2, d2 = oracle.search_brute_raw(x * np.float32(2.0), q * np.float32(2.0), 4, 6)
    np.testing.assert_array_equal(i1, i0)
    np.testing.assert_allclose(d1, d0, rtol=1e-12)
    np.testing.assert_array_equal(i2, i0)
    np.testing.assert_allclose(d2, 4.0 * d0, rtol=1e-12)


def test_exclusion_zone_zero_is_plain_topk_and_offsets_are_apart():
    rng = np.random.default_rng(6)
    d = rng.random(300)
    d[50] = d[51]  # a tie: lower offset first
    i0, _ = oracle.exclusion_topk(d, 10, 0)
    np.testing.assert_array_equal(i0, np.lexsort((np.arange(d.size), d))[:10])
    for z in (1, 5, 20):
        idx, dist = oracle.exclusion_topk(d, 8, z)
        assert np.all(np.abs(idx[:, None] - idx[None, :])[~np.eye(idx.size, dtype=bool)] > z)
        assert np.all(np.diff(dist) >= 0)


def test_exclusion_zone_returns_separate_planted_copies():
    x = synth.random_walk(3000, 7)
    ql = synth.random_walk(50, 8)
    q = ql[5:45].copy()
    # three planted copies far apart (with 5 samples of the pattern's own
    # context on each side), one nearly exact: its shifted neighbours (the
    # band absorbs a shift of one) beat the noisier copies
    for o, s in ((300, 0.001), (1400, 0.5), (2500, 0.5)):
        x[o - 5:o + 45] = ql + np.random.default_rng(o).normal(0, s, 50).astype(np.float32)
    d = np.array([oracle.dtw(q.astype(np.float64), x[i:i + 40].astype(np.float64), 4)
                  for i in range(x.size - 39)])
    plain = np.lexsort((np.arange(d.size), d))[:3]
    idx, _ = oracle.exclusion_topk(d, 3, 20)
    # one answer at each copy (a noisy copy's best alignment may sit a sample off)
    got = sorted(idx.tolist())
    assert [abs(g - o) <= 2 for g, o in zip(got, (300, 1400, 2500))] == [True] * 3, got
    assert np.ptp(plain) <= 3  # the plain top-3 are neighbours of one copy


@pytest.mark.parametrize("seed", range(5))
def test_exclusion_answer_lies_in_the_plain_top_k_2z_plus_1(seed):
    rng = np.random.default_rng(seed)
    d = np.cumsum(rng.normal(0, 1, 2000)) ** 2  # smooth: near windows have near distances
    for k, z in ((3, 10), (5, 4), (2, 50)):
        idx, _ = oracle.exclusion_topk(d, k, z)
        K = k * (2 * z + 1)
        top = np.lexsort((np.arange(d.size), d))[:K]
        sub = np.full(d.size, np.inf)
        sub[top] = d[top]
        idx2, _ = oracle.exclusion_topk(sub, k, z)
        np.testing.assert_array_equal(idx2, idx)


@pytest.mark.parametrize("seed", range(6))
def test_two_z_separated_set_bounds_the_exclusion_answer(seed):
    """Any windows found so far, kept pairwise more than 2z apart, give a
    threshold no smaller than the exclusion-zone answer's k-th distance,
    whatever the order and subset in which they are found."""
    rng = np.random.default_rng(100 + seed)
    n = 600
    d = np.cumsum(rng.normal(0, 1, n)) ** 2 if seed % 2 else rng.random(n)
    for k, z in ((1, 3), (3, 10), (5, 4), (2, 40), (4, 25)):
        _, dist = oracle.exclusion_topk(d, k, z)
        if dist.size < k:
            continue
        for trial in range(4):
            found = rng.permutation(n)[: int(n * (0.3 + 0.2 * trial))]
            t = oracle.separated_kth(d, k, 2 * z, order=found)
            assert t >= dist[k - 1]
        # all windows found, in offset order: the same holds
        assert oracle.separated_kth(d, k, 2 * z) >= dist[k - 1]


def test_z_separated_set_is_not_a_bound():
    """The threshold needs 2z: with windows kept only z apart, one taken
    window can shut out two kept ones."""
    z = 5
    d = np.full(200, 100.0) + np.arange(200) * 1e-3
    d[50], d[50 - z], d[50 + z] = 1.0, 2.0, 2.0
    _, dist = oracle.exclusion_topk(d, 2, z)
    assert dist[1] >= 100.0  # 45 and 55 lie within z of the first pick, 50
    found = [50 - z, 50 + z]  # found before 50
    assert oracle.separated_kth(d, 2, z, order=found) == 2.0 < dist[1]
    assert oracle.separated_kth(d, 2, 2 * z, order=found) == np.inf
    assert oracle.separated_kth(d, 2, 2 * z, order=found + [50]) >= dist[1]


def test_separated_set_keeps_the_better_neighbour():
    d = np.array([5.0, 3.0, 4.0, 1.0, 9.0, 9.0, 9.0, 2.0])
    # sep 1: kept {3 (1.0), 7 (2.0), 1 (3.0), 5 (9.0)} -> sorted 1, 2, 3, 9
    assert oracle.separated_kth(d, 1, 1) == 1.0
    assert oracle.separated_kth(d, 3, 1) == 3.0
    assert oracle.separated_kth(d, 4, 1) == 9.0
    assert oracle.separated_kth(d, 5, 1) == np.inf
    # insertion order does not matter for sep 1 here: the kept set is the same
    assert oracle.separated_kth(d, 3, 1, order=[7, 6, 5, 4, 3, 2, 1, 0]) == 3.0


def _bucket_kth(d, k, z, found):
    """The bucket form of the threshold that the GPU path keeps: offsets cut
    into buckets of 2z + 1; windows in different buckets of the same parity
    are at least 2z + 2 apart.  Per parity, a list of the best window found
    in each bucket; the k-th smallest of either list bounds the answer (each
    entry is a real window's distance, the entries pairwise more than 2z
    apart)."""
    W = 2 * z + 1
    best_in = {}
    for w in found:
        b = w // W
        best_in[b] = min(best_in.get(b, np.inf), float(d[w]))
    best = np.inf
    for parity in (0, 1):
        vals = sorted(v for b, v in best_in.items() if b % 2 == parity)
        if len(vals) >= k:
            best = min(best, vals[k - 1])
    return best


def _exclusion_search(d, lb, k, z, sep, buckets=False):
    """The search procedure for wide exclusion zones, simulated on the host:
    windows come in lower-bound order (admissible bounds), each one whose
    bound is within the threshold is scored, scored windows within the
    threshold go to a buffer and to the list kept ``sep`` apart (or to the
    bucket lists), the threshold is the smallest k-th distance that list has
    had; at the end the buffer, filtered by the final threshold, is taken
    greedily.  Returns (offsets, distances, final threshold, windows scored)."""
    n = d.size
    thr, found, buf, scored = np.inf, [], [], 0
    for w in np.lexsort((np.arange(n), lb)):
        if lb[w] > thr:
            continue  # pruned
        scored += 1
        if d[w] <= thr:
            buf.append(int(w))
            found.append(int(w))
            t = _bucket_kth(d, k, z, found) if buckets else oracle.separated_kth(d, k, sep, order=found)
            thr = min(thr, t)
    keep = np.array([w for w in buf if d[w] <= thr], np.int64)
    sub = np.full(n, np.inf)
    sub[keep] = d[keep]
    idx, dist = oracle.exclusion_topk(sub, k, z)
    return idx, dist, thr, scored


@pytest.mark.parametrize("seed", range(4))
def test_exclusion_search_with_the_2z_threshold_is_exact(seed):
    """The simulated search with the list kept 2z apart, and with its
    lock-free bucket form, returns the exclusion-zone answer over every
    window, and prunes."""
    rng = np.random.default_rng(200 + seed)
    n = 500
    d = np.cumsum(rng.normal(0, 1, n)) ** 2 + rng.random(n) if seed % 2 else rng.random(n) * 10
    lb = d * rng.uniform(0.3, 1.0, n)
    for k, z in ((2, 30), (4, 12), (3, 60)):
        want_i, want_d = oracle.exclusion_topk(d, k, z)
        for buckets in (False, True):
            got_i, got_d, thr, scored = _exclusion_search(d, lb, k, z, 2 * z, buckets)
            np.testing.assert_array_equal(got_i, want_i)
            np.testing.assert_array_equal(got_d, want_d)
            assert thr >= want_d[-1]
            assert scored < n  # the threshold pruned something


def test_exclusion_search_with_a_z_threshold_loses_a_match():
    """The same search with the list kept only z apart prunes the second
    match: the two windows beside the best one are found first and set a
    threshold that the best one then invalidates."""
    z = 5
    d = np.full(200, 100.0) + np.arange(200) * 1e-3
    d[50], d[50 - z], d[50 + z] = 1.0, 2.0, 2.0
    lb = d * 0.9
    lb[50] = 1.95  # scored after its neighbours
    want_i, want_d = oracle.exclusion_topk(d, 2, z)
    for buckets in (False, True):
        got_i, got_d, _, _ = _exclusion_search(d, lb, 2, z, 2 * z, buckets)
        np.testing.assert_array_equal(got_i, want_i)
        np.testing.assert_array_equal(got_d, want_d)
    _, bad_d, _, _ = _exclusion_search(d, lb, 2, z, z)
    assert want_d[1] < np.inf and bad_d[1] == np.inf  # the second match was pruned
