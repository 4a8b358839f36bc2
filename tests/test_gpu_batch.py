"""Batched queries (lanes of concurrent queries, the persistent survivor-DTW
stage over the whole batch, CUDA-graph capture and replay), the per-series
block envelope and the learned ordering inside a batch: every variant returns
the oracle's answers."""
import numpy as np
import pytest

from oracle import fragments
from paper_1812_10302_gb300 import dtws, synth, train

pytestmark = pytest.mark.gpu


def _close(got, want, m):
    np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-6 * m)


@pytest.fixture(scope="module")
def walk():
    return synth.walk_with_bursts(400_000, 31, 32, 33)


def _queries(x, count, seed, m_range=(64, 900)):
    return synth.batch_queries(x, count, seed, m_range=m_range, w_range=(0.0, 0.25), noise=0.3)


def test_lanes_and_graph_replay_match_the_oracle(walk):
    qs, rs, _ = _queries(walk, 24, 5)
    k = 5
    want = [fragments.search_fragments(walk, q, r, k) for q, r in zip(qs, rs)]
    with dtws.Index(walk) as ix:
        got = {}
        for lanes, graph in ((1, 0), (4, 0), (4, 1), (3, 1)):
            ix.set_options(batch_lanes=lanes, batch_graph=graph)
            got[(lanes, graph)] = ix.query_batch(qs, rs, k=k)
            assert ix.sync_status() == dtws.DTWS_OK
        ix.set_options(batch_lanes=3, batch_graph=1)
        again = ix.query_batch(qs, rs, k=k)  # replay of the captured graph
        for bi, bd in list(got.values()) + [again]:
            for t, (q, r) in enumerate(zip(qs, rs)):
                np.testing.assert_array_equal(bi[t], want[t][0])
                _close(bd[t], want[t][1], len(q))
        # same shapes, new query values: the replayed graph reads the new queries
        qs2 = [synth.noisy_copy(walk, len(q), 900 + t, 950 + t, noise=0.3)[0] for t, q in enumerate(qs)]
        bi, bd = ix.query_batch(qs2, rs, k=k)
        for t, (q, r) in enumerate(zip(qs2, rs)):
            oi, od = fragments.search_fragments(walk, q, r, k)
            np.testing.assert_array_equal(bi[t], oi)
            _close(bd[t], od, len(q))


def test_persistent_stage_pool_sizes_give_the_same_answers(walk):
    """The batch's survivor DTW in the persistent per-shape launches (default
    pool), on the lanes (no pool), and split between the two (a pool too small
    for some queries' survivors, so those run on their lanes): the oracle's
    answers every time, with and without a captured graph."""
    qs, rs, _ = _queries(walk, 20, 8, m_range=(32, 700))
    k = 4
    want = [fragments.search_fragments(walk, q, r, k) for q, r in zip(qs, rs)]
    with dtws.Index(walk) as ix:
        for cap in (-1, 0, 3000, 1):
            ix.debug_set_pool_capacity(cap)
            for graph in (0, 1):
                ix.set_options(batch_lanes=3, batch_graph=graph)
                bi, bd = ix.query_batch(qs, rs, k=k)
                assert ix.sync_status() == dtws.DTWS_OK
                for t, (q, r) in enumerate(zip(qs, rs)):
                    np.testing.assert_array_equal(bi[t], want[t][0], err_msg=f"cap {cap} graph {graph} query {t}")
                    _close(bd[t], want[t][1], len(q))
                st = ix.last_stats()
                assert st["dtw_started"] >= st["dtw_abandoned"] >= 0
        ix.debug_set_pool_capacity(-1)
        with pytest.raises(dtws.DtwsError):
            ix.debug_set_pool_capacity(-2)


def test_exclusion_lock_wait_is_bounded(walk):
    """The one lock of the library (the wide exclusion zone's bucket lists)
    gives up after the handle's wait limit: held by one device thread while
    another offers, the offer times out, DTWS_ETIMEOUT is reported, and the
    handle answers correctly afterwards."""
    import time
    q, _ = synth.noisy_copy(walk, 128, 70, 71, noise=0.3)
    with dtws.Index(walk) as ix:
        t0 = time.perf_counter()
        ix.debug_lock_selftest(2_000_000)  # 2 ms
        assert ix.sync_status() == dtws.DTWS_ETIMEOUT
        assert time.perf_counter() - t0 < 5.0
        assert ix.sync_status() == dtws.DTWS_OK  # cleared
        ix.set_options(exclusion_zone=64)
        idx, dist = ix.query(q, 12, 3)
        assert ix.sync_status() == dtws.DTWS_OK
    import oracle
    d = oracle.dtw_at(walk, q, 12, np.arange(walk.size - 127))
    oi, od = oracle.exclusion_topk(d, 3, 64)
    np.testing.assert_array_equal(idx, oi)
    _close(dist, od, 128)


def test_batch_with_device_queries_and_outputs(walk):
    import torch
    qs, rs, _ = _queries(walk, 8, 6)
    ms = np.array([len(q) for q in qs], np.int32)
    off = np.zeros(len(qs) + 1, np.int64)
    off[1:] = np.cumsum(ms)
    cat = torch.from_numpy(np.concatenate(qs)).cuda()
    idx = torch.empty((len(qs), 2), dtype=torch.int64, device="cuda")
    dist = torch.empty((len(qs), 2), dtype=torch.float32, device="cuda")
    with dtws.Index(walk) as ix:
        lib = dtws.load()
        rr = np.asarray(rs, np.int32)
        st = lib.dtws_query_batch(ix.h, cat.data_ptr(), off.ctypes.data, ms.ctypes.data, rr.ctypes.data, len(qs), 2,
                                  idx.data_ptr(), dist.data_ptr(), dtws._stream_ptr(None))
        assert st == dtws.DTWS_OK
        assert ix.sync_status() == dtws.DTWS_OK
        hi, hd = ix.query_batch(qs, rs, k=2)
    np.testing.assert_array_equal(idx.cpu().numpy(), hi)
    np.testing.assert_array_equal(dist.cpu().numpy(), hd)


def test_block_envelope_gives_the_same_answers(walk):
    with dtws.Index(walk) as ix:
        for t, m in enumerate((64, 333, 1024, 2048)):
            q, _ = synth.noisy_copy(walk, m, 70 + t, 80 + t, noise=0.3)
            for r in (0, 5, m // 10, m // 3):
                res = {}
                for exact in (1, 0):
                    ix.clear_cache()  # no cached exact envelope to fall back on
                    ix.set_options(exact_envelope=exact)
                    i, d = ix.query(q, r, 3)
                    assert ix.sync_status() == dtws.DTWS_OK
                    res[exact] = (i, d, ix.last_stats())
                # (the survivor counters are not compared: they depend on how
                # the concurrently shrinking threshold interleaves)
                np.testing.assert_array_equal(res[0][0], res[1][0])
                np.testing.assert_array_equal(res[0][1], res[1][1])


def test_batch_with_learned_ordering(walk):
    qs, rs, _ = _queries(walk, 10, 7, m_range=(64, 700))
    with dtws.Index(walk) as ix:
        plain = ix.query_batch(qs, rs, k=3)
        ix.set_encoder(train.load_weights())
        ix.set_options(ordering=dtws.DTWS_ORDER_LEARNED)
        learned = ix.query_batch(qs, rs, k=3)
        assert ix.sync_status() == dtws.DTWS_OK
    np.testing.assert_array_equal(learned[0], plain[0])
    np.testing.assert_array_equal(learned[1], plain[1])


def test_autotune_keeps_the_answers(walk):
    pairs = [(64, 0), (128, 12), (300, 60), (512, 51), (1024, 300), (700, 600)]
    qs = [synth.noisy_copy(walk, m, 400 + m, 500 + m, noise=0.3)[0] for m, _ in pairs]
    with dtws.Index(walk) as ix:
        before = [ix.query(q, r, 4) for q, (_, r) in zip(qs, pairs)]
        offs = np.random.default_rng(9).integers(0, walk.size - 1024, 300)
        dtw_before = [ix.dtw_at(q, r, np.minimum(offs, walk.size - len(q))) for q, (_, r) in zip(qs, pairs)]
        ix.autotune([m for m, _ in pairs], [r for _, r in pairs], samples=512)
        for (m, r), q, (bi, bd), db in zip(pairs, qs, before, dtw_before):
            L, K, W, t_def, t_best = ix.tune_entry(m, r)
            assert t_best <= t_def
            if L:
                assert (K == 0) or L * K >= r + 1
                assert W in (2, 4, 8)
            i, d = ix.query(q, r, 4)
            assert ix.sync_status() == dtws.DTWS_OK
            np.testing.assert_array_equal(i, bi)
            np.testing.assert_array_equal(d, bd)
            np.testing.assert_array_equal(ix.dtw_at(q, r, np.minimum(offs, walk.size - m)), db)
        with pytest.raises(dtws.DtwsError):
            ix.tune_entry(99, 3)
