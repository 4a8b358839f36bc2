"""Parity at the full workload sizes, in the launch configuration bench.py
times (default options, series and query on the device).

The 1e6- and 1e8-sample workloads (the latter is the one bench.py times)
are checked exactly against the oracle's search of every window (the Eq. 11
fragment cascade over the host cores).  For the batch and the 1e9-sample
series the oracle cannot search everything in a test, so each answer is
checked through facts it can compute one by one:
* the returned distances equal the oracle's FP64 DTW at the returned offsets;
* an exact oracle search of a fragment around the planted match, merged with
  the returned list, leaves the returned list unchanged (no window of the
  fragment beats it);
* sampled windows never beat the k-th returned distance."""
import numpy as np
import pytest

import oracle
from oracle import fragments
from paper_1812_10302_gb300 import dtws, synth

pytestmark = pytest.mark.gpu

RTOL = 1e-4


def _close(got, want, m):
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=1e-6 * m)


def _check_fragment_merge(x, q, r, k, idx, dist, center, half):
    """Exact oracle top-k of the windows [center-half, center+half) merged
    with the returned list (re-scored by the oracle) must be the returned
    list itself."""
    m = q.size
    N = x.size - m + 1
    lo, hi = max(0, center - half), min(N, center + half)
    fi, fd = fragments.search_fragments(x, q, r, k, first=lo, count=hi - lo)
    od = oracle.dtw_at(x, q, r, idx)
    _close(dist, od, m)
    extra = ~np.isin(fi, idx)
    mi, _ = fragments.merge_topk([(idx, od), (fi[extra], fd[extra])], k)
    np.testing.assert_array_equal(mi, idx)


def _check_samples(x, q, r, kth, count, seed):
    m = q.size
    offs = np.random.default_rng(seed).integers(0, x.size - m + 1, count)
    d = oracle.dtw_at(x, q, r, offs)
    assert np.all(d >= kth * (1 - 1e-6)), (d.min(), kth)


def test_rw1m_exact():
    w = synth.workload("rw1m")
    x, r = w["series"], w["rs"][0]
    queries = [w["queries"][0]] + [synth.noisy_copy(x, 128, 100 + s, 200 + s)[0] for s in range(3)]
    with dtws.Index(x) as ix:
        for q in queries:
            for k in (1, 10):
                idx, dist = ix.query(q, r, k)
                assert ix.sync_status() == dtws.DTWS_OK
                oi, od = fragments.search_fragments(x, q, r, k)
                np.testing.assert_array_equal(idx, oi)
                _close(dist, od, 128)


@pytest.fixture(scope="module")
def rw100m():
    return synth.workload("rw100m")


def test_rw100m_bench_configuration(rw100m):
    import torch
    x, q, r, o = rw100m["series"], rw100m["queries"][0], rw100m["rs"][0], rw100m["true_offsets"][0]
    ix = dtws.Index(torch.from_numpy(x).cuda())
    idx_d = torch.empty(1, dtype=torch.int64, device="cuda")
    dist_d = torch.empty(1, dtype=torch.float32, device="cuda")
    ix.query(torch.from_numpy(q).cuda(), r, 1, out=(idx_d, dist_d))
    assert ix.sync_status() == dtws.DTWS_OK
    idx, dist = idx_d.cpu().numpy(), dist_d.cpu().numpy()
    ix.close()
    # the oracle's exact search over all 99,999,489 windows (FP64 cascade,
    # anchored window statistics, Eq. 11 fragments over the host cores)
    oi, od = fragments.search_fragments(x, q, r, 1, stats="anchored")
    np.testing.assert_array_equal(idx, oi)
    _close(dist, od, q.size)
    _close(dist, oracle.dtw_at(x, q, r, idx), q.size)


def test_batch_workload():
    w = synth.workload("batch")
    x, qs, rs, k, offs = w["series"], w["queries"], w["rs"], w["k"], w["true_offsets"]
    with dtws.Index(x) as ix:
        bi, bd = ix.query_batch(qs, rs, k=k)
        assert ix.sync_status() == dtws.DTWS_OK
    rng = np.random.default_rng(5)
    checked = rng.choice(len(qs), 24, replace=False)
    for t in checked:
        q, r = qs[t], rs[t]
        assert np.all(np.diff(bd[t]) >= 0)
        _check_fragment_merge(x, q, r, k, bi[t], bd[t], offs[t], 2_000)
        _check_samples(x, q, r, float(bd[t][-1]), 8, 100 + int(t))


def test_drift_1e9_precision():
    """n = 1e9 walk with drift 1e-3 and variance regimes: FP64 window
    statistics, FP32 search, extended-precision re-score; reports the FP32
    DTW's relative error against the FP64 oracle at the answers."""
    w = synth.workload("drift")
    x, qs, r, offs = w["series"], w["queries"], w["rs"][0], w["true_offsets"]
    errs = []
    with dtws.Index(x) as ix:
        for t in range(6):
            q = qs[t]
            idx, dist = ix.query(q, r, 1)
            assert ix.sync_status() == dtws.DTWS_OK
            # an exact oracle search of the 4e6 windows around the planted copy
            _check_fragment_merge(x, q, r, 1, idx, dist, offs[t], 2_000_000)
            od = oracle.dtw_at(x, q, r, idx)
            f32 = ix.dtw_at(q, r, idx)
            errs.append(abs(float(f32[0]) - od[0]) / od[0])
        _check_samples(x, qs[0], r, float(dist[0]), 64, 7)
    print(f"FP32 DTW relative error vs FP64 oracle at the answers: max {max(errs):.2e}")
    assert max(errs) < RTOL
