"""End-to-end parity of dtws_query / dtws_query_batch with the FP64 oracle:
identical top-k offsets, distances within 1e-4 relative (absolute 1e-6*m
near zero), plus the degenerate cases of the method."""
import numpy as np
import pytest

import oracle
from oracle import fragments
from paper_1812_10302_gb300 import dtws, synth

pytestmark = pytest.mark.gpu


def _close(got, want, m):
    np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-6 * m)


@pytest.fixture(scope="module")
def walk():
    return synth.random_walk(50_003, 17)


@pytest.fixture(scope="module")
def index(walk):
    dtws.load(build_if_missing=True)
    ix = dtws.Index(walk)
    yield ix
    ix.close()


@pytest.mark.parametrize("m,w,k,noise", [
    (16, 0.0, 1, 0.5), (32, 0.1, 10, 0.5), (64, 0.05, 1, 0.2), (128, 0.05, 1, 0.1),
    (128, 0.2, 10, 1.0), (256, 0.1, 3, 0.3), (512, 0.1, 1, 0.1), (100, 1.0, 5, 0.5),
    (1024, 0.1, 10, 0.2), (40, 0.5, 64, 2.0)])
def test_query_matches_oracle(walk, index, m, w, k, noise):
    q, _ = synth.noisy_copy(walk, m, 100 + m, 200 + k, noise=noise)
    r = synth.band(w, m)
    idx, dist = index.query(q, r, k)
    assert index.sync_status() == dtws.DTWS_OK
    oi, od = fragments.search_fragments(walk, q, r, k)
    np.testing.assert_array_equal(idx, oi)
    _close(dist, od, m)


@pytest.mark.parametrize("offset", [3.0e5, -7.5e6])
def test_query_far_from_zero_matches_oracle(offset):
    """A series far from zero: |mu| / sigma of ~1e4 to ~1e6, so the lower-bound
    scan's shift bound (the mean's low part left out) is as large as it gets
    relative to the distances; the answers and the near-tie order must still
    be the oracle's (an undersized bound would prune a true match)."""
    x = (synth.random_walk(60_001, 23) + offset).astype(np.float32)
    with dtws.Index(x) as ix:
        for m, r, k, noise in ((128, 12, 5, 0.3), (512, 51, 1, 0.1), (300, 30, 10, 1.0)):
            q, _ = synth.noisy_copy(x, m, 31 + m, 41 + k, noise=noise)
            idx, dist = ix.query(q, r, k)
            assert ix.sync_status() == dtws.DTWS_OK
            oi, od = fragments.search_fragments(x, q, r, k)
            np.testing.assert_array_equal(idx, oi)
            _close(dist, od, m)


@pytest.mark.parametrize("m,r", [(64, 5), (128, 17), (300, 70), (512, 51), (1024, 102), (700, 200),
                                 (2048, 409), (1024, 921)])
def test_distances_are_the_extended_rescore(walk, index, m, r):
    """The returned distances are the extended-precision re-scores (the
    pre-scored seed's on the side stream, the rest in the final stage; one,
    two, three or four warps per window): the FP64 oracle's DTW at the
    returned offsets to FP32 rounding, and dtws_dtw_at_f64 there to an ulp."""
    q, _ = synth.noisy_copy(walk, m, 300 + m, 400 + r, noise=0.3)
    idx, dist = index.query(q, r, 3)
    assert index.sync_status() == dtws.DTWS_OK
    d64 = oracle.dtw_at(walk, q, r, idx)
    np.testing.assert_allclose(dist, d64, rtol=2 ** -23, atol=0)
    np.testing.assert_array_max_ulp(dist, index.dtw_at_f64(q, r, idx).astype(np.float32), maxulp=1)


@pytest.mark.parametrize("m,r,k", [(700, 630, 3), (1100, 990, 1), (1500, 1499, 2), (1400, 1100, 2),
                                   (2048, 1843, 1), (2048, 2047, 3), (2500, 2100, 1)])
def test_wide_band_queries_match_oracle(m, r, k):
    """Bands of 0.9 m and more: the FP32 walk on four warps per candidate
    (kDiagRMax < r <= 2047, up to 16 cells per lane), the row-systolic
    kernel beyond, and the four-warp double-float re-score."""
    x = synth.random_walk(6_000, 40 + m)
    q, _ = synth.noisy_copy(x, m, 41 + m, 42 + m, noise=0.3)
    with dtws.Index(x) as ix:
        idx, dist = ix.query(q, r, k)
        assert ix.sync_status() == dtws.DTWS_OK
    oi, od = fragments.search_fragments(x, q, r, k)
    np.testing.assert_array_equal(idx, oi)
    _close(dist, od, m)


def _exclusion_want(x, q, r, k, z):
    m = q.size
    d = oracle.dtw_at(x, q, r, np.arange(x.size - m + 1))
    wi, wd = oracle.exclusion_topk(d, k, z)
    out_i = np.full(k, -1, np.int64)
    out_d = np.full(k, np.inf)
    out_i[:wi.size] = wi
    out_d[:wd.size] = wd
    return out_i, out_d


@pytest.mark.parametrize("m,r,k,z", [(128, 12, 3, 64), (128, 12, 10, 64), (96, 9, 5, 48), (64, 6, 10, 20),
                                     (200, 40, 4, 100)])
def test_wide_exclusion_zone_matches_oracle(m, r, k, z):
    """Exclusion zones wider than the result list covers (k(2z+1) > 64, e.g.
    z = m/2): the bucket-list threshold, the candidate buffer and the final
    greedy selection against the oracle's greedy selection over the FP64 DTW
    of every window; a replayed graph gives the same answer."""
    x = synth.random_walk(30_000, 500 + m + z)
    q, _ = synth.noisy_copy(x, m, 501 + m, 502 + k, noise=0.3)
    want_i, want_d = _exclusion_want(x, q, r, k, z)
    with dtws.Index(x) as ix:
        ix.set_options(exclusion_zone=z)
        idx, dist = ix.query(q, r, k)
        assert ix.sync_status() == dtws.DTWS_OK
        idx2, dist2 = ix.query(q, r, k)
        assert ix.sync_status() == dtws.DTWS_OK
    np.testing.assert_array_equal(idx, want_i)
    _close(dist, want_d, m)
    np.testing.assert_array_equal(idx2, idx)
    np.testing.assert_array_equal(dist2, dist)
    assert np.all(np.abs(np.diff(np.sort(idx))) > z)


def test_wide_exclusion_zone_with_decoys_inside_the_zone():
    """An exact copy of the query, two close copies 20 samples inside either
    edge of its zone (so the answer may not take them, nor their neighbours
    that DTW's band can still align) and a noisier copy far away: the answer
    is the exact copy and the far one.  The two decoys are 2z - 40 > z apart,
    so a threshold from windows kept only z apart would prune the far
    copy."""
    m, r, z, k = 64, 6, 80, 2
    x = synth.random_walk(40_000, 610).astype(np.float64)
    rng = np.random.default_rng(611)
    P, F = 20_000, 33_000
    base = x[P:P + m].copy()
    for o, noise in ((P - z + 20, 0.02), (P + z - 20, 0.02), (F, 0.4)):
        x[o:o + m] = base + rng.normal(0, noise, m) + (x[o] - base[0])
    x = x.astype(np.float32)
    q = x[P:P + m].copy()
    want_i, want_d = _exclusion_want(x, q, r, k, z)
    assert want_i.tolist() == [P, F]
    with dtws.Index(x) as ix:
        ix.set_options(exclusion_zone=z)
        idx, dist = ix.query(q, r, k)
        assert ix.sync_status() == dtws.DTWS_OK
    np.testing.assert_array_equal(idx, want_i)
    _close(dist, want_d, m)


def test_wide_exclusion_zone_short_series_and_overflow():
    """A series too short for k windows more than z apart: the missing ones
    come back as -1 / +inf.  Buffers smaller than the candidates: the query
    reports DTWS_EOVERFLOW, and with the default capacities again it answers
    exactly."""
    x = synth.random_walk(400, 620)
    q, _ = synth.noisy_copy(x, 64, 621, 622, noise=0.2)
    want_i, want_d = _exclusion_want(x, q, 6, 4, 120)
    assert want_i[-1] == -1
    y = synth.random_walk(30_000, 623)
    qy, _ = synth.noisy_copy(y, 128, 624, 625, noise=0.3)
    want_yi, want_yd = _exclusion_want(y, qy, 12, 5, 64)
    with dtws.Index(x) as ix:
        ix.set_options(exclusion_zone=120)
        idx, dist = ix.query(q, 6, 4)
        assert ix.sync_status() == dtws.DTWS_OK
    np.testing.assert_array_equal(idx, want_i)
    assert np.all(np.isinf(dist[want_i < 0]))
    _close(dist[want_i >= 0], want_d[want_i >= 0], 64)
    with dtws.Index(y) as ix:
        ix.set_options(exclusion_zone=64)
        ix.debug_set_xz_capacity(4, 4)
        ix.query(qy, 12, 5)
        assert ix.sync_status() == dtws.DTWS_EOVERFLOW
        ix.debug_set_xz_capacity(1 << 20, 8192)
        idx, dist = ix.query(qy, 12, 5)
        assert ix.sync_status() == dtws.DTWS_OK
        with pytest.raises(dtws.DtwsError):
            ix.debug_set_xz_capacity(1, 20000)
    np.testing.assert_array_equal(idx, want_yi)
    _close(dist, want_yd, 128)


@pytest.mark.parametrize("m,r,k,z", [(64, 6, 3, 10), (128, 12, 4, 7), (100, 20, 2, 15)])
def test_exclusion_zone_matches_oracle(m, r, k, z):
    """Top-k with an exclusion zone whose k(2z+1) best windows fit the result
    list: the oracle's greedy selection over the FP64 DTW of every window; a
    batch is refused."""
    x = synth.random_walk(20_000, 90 + m)
    q, _ = synth.noisy_copy(x, m, 91 + m, 92 + m, noise=0.3)
    with dtws.Index(x) as ix:
        ix.set_options(exclusion_zone=z)
        idx, dist = ix.query(q, r, k)
        assert ix.sync_status() == dtws.DTWS_OK
        idx2, dist2 = ix.query(q, r, k)  # (replayed graph)
        with pytest.raises(dtws.DtwsError):
            ix.query_batch([q, q], [r, r], k=k)
    np.testing.assert_array_equal(idx2, idx)
    np.testing.assert_array_equal(dist2, dist)
    d = oracle.dtw_at(x, q, r, np.arange(x.size - m + 1))
    oi, od = oracle.exclusion_topk(d, k, z)
    np.testing.assert_array_equal(idx, oi)
    _close(dist, od, m)
    assert np.all(np.abs(idx[:, None] - idx[None, :])[~np.eye(k, dtype=bool)] > z)


@pytest.mark.parametrize("m,r,k,shift,scale", [(64, 6, 3, 500.0, 3.0), (128, 25, 1, -1.0e4, 50.0),
                                               (200, 20, 5, 0.0, 0.05)])
def test_unnormalised_matches_oracle(m, r, k, shift, scale):
    """Unnormalised DTW (raw values, Eq. 5 skipped): the oracle's FP64 brute
    force over every raw window.  The building blocks at given offsets take
    the raw values too: FP32 and extended DTW against the oracle's DTW, the
    lower bounds admissible.  Switching the option back (a new graph
    signature) gives the normalised answer again."""
    x = (synth.random_walk(6_000, 70 + m).astype(np.float64) * scale + shift).astype(np.float32)
    q, _ = synth.noisy_copy(x, m, 71 + m, 72 + m, noise=0.3 * scale)
    offs = np.arange(0, x.size - m + 1, 97, dtype=np.int64)
    with dtws.Index(x) as ix:
        ni, nd = ix.query(q, r, k)
        ix.set_options(unnormalised=1)
        idx, dist = ix.query(q, r, k)
        assert ix.sync_status() == dtws.DTWS_OK
        idx2, dist2 = ix.query(q, r, k)  # (replayed graph)
        d32 = ix.dtw_at(q, r, offs)
        d64 = ix.dtw_at_f64(q, r, offs)
        lbs = ix.lower_bounds_at(q, r, offs)
        ix.set_options(unnormalised=0)
        ni2, nd2 = ix.query(q, r, k)
        assert ix.sync_status() == dtws.DTWS_OK
    oi, od = oracle.search_brute_raw(x, q, r, k)
    np.testing.assert_array_equal(idx, oi)
    np.testing.assert_allclose(dist, od, rtol=1e-4, atol=0)
    np.testing.assert_array_equal(idx2, idx)
    np.testing.assert_array_equal(dist2, dist)
    np.testing.assert_array_equal(ni2, ni)
    np.testing.assert_array_equal(nd2, nd)
    want = np.array([oracle.dtw(q, x[o:o + m], r) for o in offs])
    np.testing.assert_allclose(d32, want, rtol=1e-4, atol=0)
    np.testing.assert_allclose(d64, want, rtol=1e-9, atol=0)
    for lb in lbs:
        assert np.all(np.asarray(lb, np.float64) <= want * (1 + 1e-5))


def test_unnormalised_with_exclusion_zone():
    """Both options at once: the oracle's greedy selection over the FP64 DTW
    of every raw window."""
    x = (synth.random_walk(8_000, 95).astype(np.float64) * 2.0 + 100.0).astype(np.float32)
    m, r, k, z = 96, 10, 3, 8
    q, _ = synth.noisy_copy(x, m, 96, 97, noise=0.6)
    with dtws.Index(x) as ix:
        ix.set_options(unnormalised=1, exclusion_zone=z)
        idx, dist = ix.query(q, r, k)
        assert ix.sync_status() == dtws.DTWS_OK
    d = np.array([oracle.dtw(q, x[o:o + m], r) for o in range(x.size - m + 1)])
    oi, od = oracle.exclusion_topk(d, k, z)
    np.testing.assert_array_equal(idx, oi)
    np.testing.assert_allclose(dist, od, rtol=1e-4, atol=0)


def test_unnormalised_refusals():
    """Unnormalised DTW refuses the learned ordering (embeddings of
    normalised windows), the batch, a series beyond +-2^32; a query beyond
    +-2^32 is reported by dtws_sync_status."""
    x = synth.random_walk(4_000, 81)
    q, _ = synth.noisy_copy(x, 64, 82, 83, noise=0.3)
    with dtws.Index(x) as ix:
        ix.set_options(unnormalised=1)
        with pytest.raises(dtws.DtwsError):
            ix.query_batch([q, q], [6, 6], k=1)
        bad = q.copy()
        bad[5] = 1e10
        ix.query(bad, 6, 1)
        assert ix.sync_status() == dtws.DTWS_ENONFINITE
        ix.query(q, 6, 1)
        assert ix.sync_status() == dtws.DTWS_OK
        ix.set_options(ordering=dtws.DTWS_ORDER_LEARNED)
        with pytest.raises(dtws.DtwsError):
            ix.query(q, 6, 1)
    spiked = x.copy()
    spiked[100] = 5e9
    with dtws.Index(spiked) as ix:
        ix.query(q, 6, 1)  # normalised: fine
        assert ix.sync_status() == dtws.DTWS_OK
        ix.set_options(unnormalised=1)
        with pytest.raises(dtws.DtwsError):
            ix.query(q, 6, 1)


def test_random_query_not_a_copy(walk, index):
    """A query unrelated to the series: loose seeds, many survivors."""
    q = synth.random_walk(128, 999)
    idx, dist = index.query(q, 12, 4)
    oi, od = fragments.search_fragments(walk, q, 12, 4)
    np.testing.assert_array_equal(idx, oi)
    _close(dist, od, 128)


def test_planted_exact_copy(walk, index):
    o = 31_337
    q = walk[o:o + 200].copy()
    idx, dist = index.query(q, 20, 1)
    assert idx[0] == o and dist[0] <= 1e-6 * 200


def test_exact_ties_lowest_index():
    pat = np.random.default_rng(5).standard_normal(97).astype(np.float32)
    x = np.tile(pat, 80)                       # 7760 samples, period 97
    q = x[50:50 + 150].copy()
    with dtws.Index(x) as ix:
        idx, dist = ix.query(q, 15, 5)
    oi, od = oracle.search_cascade(x, q, 15, 5)
    np.testing.assert_array_equal(idx, oi)
    assert idx.tolist() == [50 + 97 * t for t in range(5)]
    assert np.all(dist <= 1e-6 * 150)


def test_constant_windows_and_query():
    x = synth.random_walk(12_000, 6)
    x[4000:4600] = 7.0
    with dtws.Index(x) as ix:
        # constant query: normalises to zeros; constant windows also to zeros
        q = np.full(64, 3.0, np.float32)
        idx, dist = ix.query(q, 6, 3)
        oi, od = oracle.search_cascade(x, q, 6, 3)
        np.testing.assert_array_equal(idx, oi)
        _close(dist, od, 64)
        assert idx[0] == 4000 and dist[0] == 0.0
        q2, _ = synth.noisy_copy(x, 64, 3, 4)
        idx, dist = ix.query(q2, 6, 2)
        oi, od = oracle.search_cascade(x, q2, 6, 2)
        np.testing.assert_array_equal(idx, oi)
        _close(dist, od, 64)


def _band_cells(m, r):
    """Cells of the band |i - j| <= r inside [0, m)^2, by enumeration."""
    i = np.arange(m)[:, None]
    return int(np.count_nonzero(np.abs(i - np.arange(m)[None, :]) <= min(r, m - 1)))


@pytest.mark.parametrize("m,r", [(40, 0), (40, 7), (40, 8), (64, 33), (100, 99), (96, 40)])
def test_cell_counter_without_pruning(m, r):
    """With k equal to the number of windows nothing is pruned or abandoned,
    so every DTW walks its whole band: the cell counter (closed form per
    walk) is the walks started times the band's cell count."""
    x = synth.random_walk(m + 40, 60 + m + r)  # 41 windows: k <= 64
    q, _ = synth.noisy_copy(x, m, 61, 62)
    N = x.size - m + 1
    with dtws.Index(x) as ix:
        idx, _ = ix.query(q, r, N)
        assert ix.sync_status() == dtws.DTWS_OK
        st = ix.last_stats()
    assert sorted(idx.tolist()) == list(range(N))
    assert st["dtw_abandoned"] == 0
    assert st["dtw_cells"] == st["dtw_started"] * _band_cells(m, r)


def test_k_equals_all_windows_and_m_equals_n():
    x = synth.random_walk(300, 8)
    q, _ = synth.noisy_copy(x, 250, 9, 10, noise=0.5)
    with dtws.Index(x) as ix:
        idx, dist = ix.query(q, 25, 51)           # N = 51: every window
        oi, od = oracle.search_brute(x, q, 25, 51)
        np.testing.assert_array_equal(idx, oi)
        _close(dist, od, 250)
        q3 = synth.random_walk(300, 11)
        idx, dist = ix.query(q3, 30, 1)           # m = n: one window
        assert idx[0] == 0
        _close(dist, oracle.dtw_at(x, q3, 30, [0]), 300)


def test_band_wider_than_query(walk, index):
    q, _ = synth.noisy_copy(walk, 60, 12, 13, noise=0.5)
    idx, dist = index.query(q, 500, 3)
    oi, od = oracle.search_cascade(walk, q, 59, 3)
    np.testing.assert_array_equal(idx, oi)
    _close(dist, od, 60)


def test_nonfinite_query_reported(index):
    q = np.ones(64, np.float32)
    q[10] = np.nan
    idx, dist = index.query(q, 5, 2)
    assert index.sync_status() == dtws.DTWS_ENONFINITE
    assert np.all(idx == -1) and np.all(np.isinf(dist))
    assert index.sync_status() == dtws.DTWS_OK     # cleared


def test_nonfinite_series_rejected():
    x = synth.random_walk(1000, 1)
    x[500] = np.inf
    with pytest.raises(dtws.DtwsError) as e:
        dtws.Index(x)
    assert e.value.status == dtws.DTWS_ENONFINITE


def test_bad_arguments_rejected(index):
    q = np.zeros(10, np.float32)
    for m, r, k in ((1, 1, 1), (10, -1, 1), (10, 1, 0), (10, 1, 65)):
        with pytest.raises(dtws.DtwsError) as e:
            index.query(q[:m], r, k)
        assert e.value.status == dtws.DTWS_EINVAL


def test_allocation_failure_is_reported_and_recoverable():
    x = synth.random_walk(5000, 2)
    dtws.dtws_debug_fail_next_allocs(1)
    with pytest.raises(dtws.DtwsError) as e:
        dtws.Index(x)
    assert e.value.status == dtws.DTWS_ENOMEM
    with dtws.Index(x) as ix:           # the hook is spent: works again
        q, _ = synth.noisy_copy(x, 50, 1, 2)
        dtws.dtws_debug_fail_next_allocs(1)
        with pytest.raises(dtws.DtwsError):
            ix.query(q, 5, 1)            # workspace allocation fails
        idx, dist = ix.query(q, 5, 1)    # and completes on the next call
        oi, od = oracle.search_cascade(x, q, 5, 1)
        np.testing.assert_array_equal(idx, oi)


def test_batch_matches_single_queries(walk, index):
    qs, rs, _ = synth.batch_queries(walk, 12, 77, m_range=(20, 700), w_range=(0.0, 0.3), noise=0.3)
    bi, bd = index.query_batch(qs, rs, k=3)
    for t, (q, r) in enumerate(zip(qs, rs)):
        oi, od = fragments.search_fragments(walk, q, r, 3)
        np.testing.assert_array_equal(bi[t], oi)
        _close(bd[t], od, len(q))


def test_device_outputs_and_repeatability(walk, index):
    import torch
    q, _ = synth.noisy_copy(walk, 300, 55, 56, noise=0.3)
    qd = torch.from_numpy(q).cuda()
    outs = []
    for _ in range(5):
        idx = torch.empty(10, dtype=torch.int64, device="cuda")
        dist = torch.empty(10, dtype=torch.float32, device="cuda")
        index.query(qd, 30, 10, out=(idx, dist))
        outs.append((idx.cpu().numpy(), dist.cpu().numpy()))
    for a in outs[1:]:
        np.testing.assert_array_equal(a[0], outs[0][0])
        np.testing.assert_array_equal(a[1], outs[0][1])
    hi, hd = index.query(q, 30, 10)
    np.testing.assert_array_equal(hi, outs[0][0])


def test_query_graph_replay_reads_new_values(walk):
    """Repeated queries with the same arguments replay a captured CUDA graph:
    new values in the same query and output buffers give the new query's
    answer, and the graph-free path (batch_graph = 0) agrees."""
    import torch
    m, r, k = 256, 25, 3
    qd = torch.empty(m, dtype=torch.float32, device="cuda")
    idx = torch.empty(k, dtype=torch.int64, device="cuda")
    dist = torch.empty(k, dtype=torch.float32, device="cuda")
    with dtws.Index(walk) as ix:
        for t in range(4):
            q, _ = synth.noisy_copy(walk, m, 70 + t, 80 + t, noise=0.3)
            qd.copy_(torch.from_numpy(q))
            ix.query(qd, r, k, out=(idx, dist))
            assert ix.sync_status() == dtws.DTWS_OK
            gi, gd = idx.cpu().numpy(), dist.cpu().numpy()
            oi, od = fragments.search_fragments(walk, q, r, k)
            np.testing.assert_array_equal(gi, oi)
            _close(gd, od, m)
            ix.set_options(batch_graph=0)
            ix.query(qd, r, k, out=(idx, dist))
            np.testing.assert_array_equal(idx.cpu().numpy(), gi)
            np.testing.assert_array_equal(dist.cpu().numpy(), gd)
            ix.set_options(batch_graph=1)


def test_stats_counters(walk, index):
    q, _ = synth.noisy_copy(walk, 128, 60, 61, noise=0.1)
    index.set_options(timing=1)
    index.query(q, 6, 1)
    s = index.last_stats()
    index.set_options(timing=0)
    assert s["windows"] == walk.size - 128 + 1
    assert s["pass_kim"] >= s["pass_keogh_q"] >= s["pass_keogh_s"] >= 1
    assert s["dtw_started"] >= 1 and s["rescored"] >= 1
    assert all(v >= 0 for v in s["phase_ms"])


def test_long_scan_reports_no_device_error():
    """Enough tiles that every scan CTA cycles through its shared-memory
    stages several times; the query must finish without a device-side
    error (a stuck pipeline would end in DTWS_ETIMEOUT)."""
    import time
    x = synth.random_walk(4_000_000, 31)
    q, o = synth.noisy_copy(x, 256, 32, 33, noise=0.1)
    with dtws.Index(x) as ix:
        ix.query(q, 25, 1)
        t0 = time.perf_counter()
        idx, dist = ix.query(q, 25, 1)
        elapsed = time.perf_counter() - t0
        assert ix.sync_status() == dtws.DTWS_OK
    assert elapsed < 1.0
    lo = max(0, o - 50_000)
    oi, od = oracle.search_cascade(x[lo:o + 50_000 + 256], q, 25, 1)
    assert idx[0] == o or dist[0] <= od[0] * (1 + 1e-6)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_seeding_keeps_the_scan_tight(seed):
    """For a noisy copy the seeds must give a threshold close to the answer,
    so that LB_KimFL already drops nearly every window (performance
    regression guard: correctness never depends on it)."""
    x = synth.walk_with_bursts(3_000_000, 10 + seed, 20 + seed, 30 + seed)
    q, o = synth.noisy_copy(x, 512, 40 + seed, 50 + seed, noise=0.1)
    with dtws.Index(x) as ix:
        idx, dist = ix.query(q, 51, 1)
        s = ix.last_stats()
    assert s["pass_kim"] < 0.05 * s["windows"], s
    assert idx[0] == o or dist[0] <= oracle.dtw_at(x, q, 51, [o])[0]


def test_bounded_wait_reports_timeout_and_the_handle_recovers(walk, index):
    """Failure detection without a GPU fault: a bounded device wait on a
    barrier that nothing completes runs out after 2 ms, the kernel records
    DTWS_ETIMEOUT, the host reads it (and it is cleared), and the same handle
    then answers correctly."""
    import time
    t0 = time.perf_counter()
    index.debug_wait_selftest(2_000_000)
    assert index.sync_status() == dtws.DTWS_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert index.sync_status() == dtws.DTWS_OK  # read once, then cleared
    q, _ = synth.noisy_copy(walk, 256, 81, 82, noise=0.2)
    idx, dist = index.query(q, 25, 1)
    assert index.sync_status() == dtws.DTWS_OK
    oi, od = fragments.search_fragments(walk, q, 25, 1)
    np.testing.assert_array_equal(idx, oi)
    _close(dist, od, 256)
