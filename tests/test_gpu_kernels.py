"""Element-wise parity of each CUDA kernel with the FP64 oracle, called
through the C ABI, on inputs that span several tiles (2048 windows) and
prefix blocks (8192 samples) with a ragged tail."""
import numpy as np
import pytest

import oracle
from paper_1812_10302_gb300 import dtws, synth

pytestmark = pytest.mark.gpu

DELTA = 2.0 ** -10


@pytest.fixture(scope="module")
def series():
    x = synth.random_walk(21_011, 5)
    x[3000:3300] = 42.5          # constant stretch: sigma = 0 windows
    x[9000:9005] += 1e3          # a spike inside a prefix block
    return x


@pytest.fixture(scope="module")
def index(series):
    dtws.load(build_if_missing=True)
    ix = dtws.Index(series)
    yield ix
    ix.close()


@pytest.mark.parametrize("m", [2, 7, 64, 128, 513, 2048])
def test_window_stats_match_oracle(series, index, m):
    mh, ml, inv = index.window_stats(m)
    mu, sg = oracle.window_stats(series, m, "twopass")
    mu_gpu = mh.astype(np.float64) + ml.astype(np.float64)
    zero = sg == 0.0
    # the zero-variance rule agrees exactly
    np.testing.assert_array_equal(inv == 0.0, zero)
    nz = ~zero
    # the mean (split in two floats) to 1e-7 of sigma; 1/sigma to FP32 rounding
    assert np.all(np.abs(mu_gpu[nz] - mu[nz]) <= 1e-7 * sg[nz] + 1e-12 * np.abs(mu[nz]))
    rel = np.abs(inv[nz].astype(np.float64) * sg[nz] - 1.0)
    assert rel.max() <= 2.0 ** -22, rel.max()


def test_window_stats_drifting_series():
    x = synth.drifting_regimes(300_000, 3, drift=1e-2, regime=(2e4, 6e4))
    with dtws.Index(x) as ix:
        for m in (128, 1024):
            mh, ml, inv = ix.window_stats(m)
            sel = np.random.default_rng(m).integers(0, x.size - m + 1, 5000)
            for i in sel:
                mu, sg = oracle.stats_twopass(x[i:i + m])
                assert abs(float(mh[i]) + float(ml[i]) - mu) <= 1e-7 * sg
                assert abs(float(inv[i]) * sg - 1.0) <= 2.0 ** -22


def test_mean_low_part_within_the_scan_shift_bound(series):
    """The lower-bound scan normalises with the mean's high part alone and
    takes each bound on distances reduced by (|mu_hi| 2^-24 + 2^-149) / sigma:
    that holds only if every window's mean is stored as a normalised pair,
    |mu_lo| <= |mu_hi| 2^-24 (+ the subnormal step), on the walk with its
    constant stretch and spike, on a drifting series far from zero and on a
    series with a large offset."""
    walks = [series, synth.drifting_regimes(200_000, 4, drift=1e-2, regime=(2e4, 6e4)),
             (synth.random_walk(50_000, 6) + 3.0e5).astype(np.float32)]
    for x in walks:
        with dtws.Index(x) as ix:
            for m in (2, 64, 512, 2048):
                if m > x.size:
                    continue
                mh, ml, _ = ix.window_stats(m)
                bound = np.abs(mh.astype(np.float64)) * 2.0 ** -24 + 2.0 ** -149
                assert np.all(np.abs(ml.astype(np.float64)) <= bound), m


@pytest.mark.parametrize("r", [0, 1, 6, 51, 409, 2047])
def test_series_envelope_exact(series, index, r):
    U, L = index.series_envelope(r)
    Uo, Lo = oracle.series_envelope(series, r)
    np.testing.assert_array_equal(U, Uo)
    np.testing.assert_array_equal(L, Lo)


@pytest.mark.parametrize("m,r", [(16, 0), (64, 6), (128, 12), (512, 51), (300, 299)])
def test_lower_bounds_match_oracle_and_are_admissible(series, index, m, r):
    q, _ = synth.noisy_copy(series, m, 7 + m, 8 + m, noise=0.4)
    offs = np.random.default_rng(m + r).integers(0, series.size - m + 1, 700)
    offs[:5] = [0, series.size - m, 3000, 2990, 8190]  # ends, constant, block seam
    kim, kq, ks = index.lower_bounds_at(q, r, offs)
    okim, okq, _, oks = oracle.lbs_at(series, q, r, offs)
    d = oracle.dtw_at(series, q, r, offs)
    for g, o in ((kim, okim), (kq, okq), (ks, oks)):
        np.testing.assert_allclose(g, o, rtol=1e-4, atol=1e-5 * m)
        # the FP32 bounds stay admissible within the pruning margin
        assert np.all(g <= d * (1 + DELTA) + 1e-6 * m)


@pytest.mark.parametrize("m,r", [(32, 0), (32, 1), (48, 2), (64, 3), (64, 5), (100, 8), (128, 17), (70, 31),
                                 (256, 40), (512, 51), (700, 127), (64, 63), (1024, 102), (900, 511),
                                 (700, 650), (1024, 921), (2048, 1000), (2048, 1500), (2048, 1100),
                                 (2048, 2047), (3000, 2047), (2048, 600), (1600, 1535), (3000, 2100)])
def test_dtw_fp32_matches_oracle(series, index, m, r):
    q, _ = synth.noisy_copy(series, m, 20 + m, 21 + r, noise=0.3)
    offs = np.random.default_rng(m * 7 + r).integers(0, series.size - m + 1, 300)
    offs[:3] = [0, series.size - m, 3000]
    got = index.dtw_at(q, r, offs)
    want = oracle.dtw_at(series, q, r, offs)
    np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-6 * m)


# shapes of the double-float walk: one warp (r < 32), and 2, 3 or 4 warps with
# 1 to 4 cells per lane (the widest band, the longest query); bands past 511
# on four warps with 6 to 16 cells per lane; and FP64 where those copies do
# not fit in shared memory (m = 8192, r = 2000)
@pytest.mark.parametrize("m,r", [(32, 0), (64, 5), (128, 17), (512, 51), (333, 400), (300, 70), (1024, 102),
                                 (700, 200), (2048, 409), (8192, 511), (700, 650), (1024, 921), (2048, 1400),
                                 (4096, 2000), (8192, 2000)])
def test_dtw_fp64_matches_oracle(series, index, m, r):
    q, _ = synth.noisy_copy(series, m, 30 + m, 31 + r, noise=0.3)
    offs = np.random.default_rng(m + 3 * r).integers(0, series.size - m + 1, 100)
    got = index.dtw_at_f64(q, r, offs)
    want = oracle.dtw_at(series, q, min(r, m - 1), offs)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-11)


def test_dtw_host_and_device_pointers_agree(series, index):
    import torch
    q, _ = synth.noisy_copy(series, 100, 40, 41)
    offs = np.arange(0, 5000, 37, dtype=np.int64)
    a = index.dtw_at(q, 9, offs)
    b = index.dtw_at(torch.from_numpy(q).cuda(), 9, torch.from_numpy(offs).cuda())
    np.testing.assert_array_equal(a, b)
