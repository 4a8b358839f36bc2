"""Pins of the FP64 oracle against values and facts the paper and mathematics
fix, independently of the oracle's own code: hand-computed golden values,
enumeration of every warping path, closed forms (r=0, constant sequences),
NumPy/SciPy routines, invariants, and brute force vs cascade."""
import itertools
import json
import os

import numpy as np
import pytest
from scipy.ndimage import maximum_filter1d, minimum_filter1d

import oracle
from oracle import fragments
from paper_1812_10302_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_values.json")))


# ------------------------------------------------------------------ golden
@pytest.mark.parametrize("case", GOLD["dtw"], ids=lambda c: f"{c['q']}-{c['c']}-r{c['r']}")
def test_dtw_hand_values(case):
    assert oracle.dtw(case["q"], case["c"], case["r"]) == case["dtw"]


@pytest.mark.parametrize("case", GOLD["znorm"], ids=lambda c: str(c["x"]))
def test_znorm_hand_values(case):
    np.testing.assert_allclose(oracle.znorm(case["x"]), case["out"], rtol=0, atol=1e-14)


def test_lb_hand_values():
    for c in GOLD["lb_kim_fl"]:
        assert oracle.lb_kim_fl(c["q"], c["c"]) == c["lb"]
    for c in GOLD["envelope"]:
        U, L = oracle.envelope(c["v"], c["r"])
        assert U.tolist() == c["U"] and L.tolist() == c["L"]
    for c in GOLD["lb_keogh"]:
        assert oracle.lb_keogh(c["v"], c["U"], c["L"]) == c["lb"]


def test_band_reading():
    for c in GOLD["band"]:
        assert synth.band(c["w"], c["m"]) == c["r"]


# ------------------------------------------------------------------ DTW by path enumeration
def _paths_min(q, c, r):
    """min over every monotone, continuous warping path from (0,0) to
    (m-1,m-1) inside |i-j| <= r of the summed squared costs (Sec. 2.1,
    Eq. 2 constraints), by exhaustive enumeration (no dynamic programming)."""
    m = len(q)
    best = [np.inf]

    def walk(i, j, acc):
        acc += (q[i] - c[j]) ** 2
        if acc >= best[0]:
            return
        if i == m - 1 and j == m - 1:
            best[0] = acc
            return
        for di, dj in ((1, 0), (0, 1), (1, 1)):
            a, b = i + di, j + dj
            if a < m and b < m and abs(a - b) <= r:
                walk(a, b, acc)

    walk(0, 0, 0.0)
    return best[0]


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6])
def test_dtw_equals_warping_path_enumeration(m):
    rng = np.random.default_rng(100 + m)
    for _ in range(12):
        q = rng.standard_normal(m)
        c = rng.standard_normal(m)
        for r in range(m):
            want = _paths_min(q, c, r)
            got = oracle.dtw(q, c, r)
            assert abs(got - want) <= 1e-12 * max(1.0, want), (m, r, got, want)


def test_dtw_closed_forms_and_invariants():
    rng = np.random.default_rng(5)
    for m in (8, 31, 64):
        q = rng.standard_normal(m)
        c = rng.standard_normal(m)
        # r = 0 collapses the band to the diagonal: squared Euclidean distance
        assert abs(oracle.dtw(q, c, 0) - np.sum((q - c) ** 2)) <= 1e-12 * m
        # identity and symmetry
        assert oracle.dtw(q, q, m // 3) == 0.0
        for r in (0, 1, m // 4, m - 1):
            assert abs(oracle.dtw(q, c, r) - oracle.dtw(c, q, r)) <= 1e-12 * m
        # a wider band never increases the distance
        vals = [oracle.dtw(q, c, r) for r in range(m)]
        assert all(vals[i + 1] <= vals[i] + 1e-12 for i in range(m - 1))
        # r beyond m-1 is the unconstrained DTW
        assert oracle.dtw(q, c, m + 5) == oracle.dtw(q, c, m - 1)


def test_dtw_early_abandon_is_exact_or_inf():
    rng = np.random.default_rng(9)
    for _ in range(50):
        m = int(rng.integers(4, 40))
        q, c = rng.standard_normal(m), rng.standard_normal(m)
        r = int(rng.integers(0, m))
        full = oracle.dtw(q, c, r)
        bsf = full * rng.uniform(0.3, 1.7)
        got = oracle.dtw(q, c, r, bsf)
        if full <= bsf:
            assert got == full
        else:
            assert got == np.inf or got == full


# ------------------------------------------------------------------ z-normalisation
def test_znorm_matches_numpy_population_std():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(1000) * 7 + 1234.5).astype(np.float32)
    xd = x.astype(np.float64)
    want = (xd - xd.mean()) / xd.std(ddof=0)
    np.testing.assert_allclose(oracle.znorm(x), want, rtol=0, atol=1e-10)
    z = oracle.znorm(x)
    assert abs(z.mean()) < 1e-12 and abs(z.std() - 1.0) < 1e-12


def test_constant_sequence_normalises_to_zero():
    x = np.full(64, 3.25, np.float32)
    assert np.all(oracle.znorm(x) == 0.0)
    mu, sg = oracle.stats_twopass(x)
    assert mu == 3.25 and sg == 0.0
    # DTW of a normalised sequence against zeros: every row is crossed at
    # least once and the diagonal crosses each exactly once, so it is sum(q^2)=m
    q = oracle.znorm(np.random.default_rng(1).standard_normal(64).astype(np.float32))
    assert abs(oracle.dtw(q, np.zeros(64), 6) - 64.0) < 1e-9


def test_dtw_affine_invariance_after_znorm():
    rng = np.random.default_rng(4)
    q = rng.standard_normal(50).astype(np.float32)
    # multiples of 2^-10 so that 4c + 100 is exact in FP32 storage
    c = (np.round(rng.standard_normal(50) * 1024) / 1024).astype(np.float32)
    d0 = oracle.dtw(oracle.znorm(q), oracle.znorm(c), 5)
    d1 = oracle.dtw(oracle.znorm(q), oracle.znorm((c * 4 + 100).astype(np.float32)), 5)
    assert abs(d0 - d1) <= 1e-9 * d0


def test_window_stats_anchored_matches_twopass_and_numpy():
    rng = np.random.default_rng(11)
    x = synth.random_walk(5000, 3)
    x[2000:2100] = 17.0  # a constant stretch: sigma = 0 by the zero rule
    for m, B in ((50, 64), (64, 64), (100, 1024), (7, 7)):
        mu_t, sg_t = oracle.window_stats(x, m, "twopass")
        mu_a, sg_a = oracle.window_stats(x, m, "anchored", B=B)
        np.testing.assert_allclose(mu_a, mu_t, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(sg_a, sg_t, rtol=1e-9, atol=1e-12)
        win = np.lib.stride_tricks.sliding_window_view(x.astype(np.float64), m)
        np.testing.assert_allclose(mu_t, win.mean(axis=1), rtol=1e-12, atol=1e-12)
        sd = win.std(axis=1)
        nz = sg_t > 0
        np.testing.assert_allclose(sg_t[nz], sd[nz], rtol=1e-10)
        assert np.all(sd[~nz] < 1e-6)
    assert rng is not None


def test_window_stats_drifting_series_large_offsets():
    """Values far from zero (drift) with a small local spread: the anchored
    sums keep their digits (error measured relative to the window's sigma,
    which is what the normalisation divides by)."""
    m = 1024
    for drift, step in ((5.0, 0.3), (1e-3, 0.316), (1e-3, 3.16)):
        x = synth.random_walk(400_000, 1, step_scale=step, drift=drift)
        mu_a, sg_a = oracle.window_stats(x, m, "anchored")
        idx = np.random.default_rng(0).integers(0, x.size - m + 1, 300)
        for i in idx:
            mu, sg = oracle.stats_twopass(x[i:i + m])
            assert abs(mu_a[i] - mu) <= 1e-9 * sg
            assert abs(sg_a[i] - sg) <= 1e-9 * sg


# ------------------------------------------------------------------ lower bounds
def test_envelope_matches_scipy_filters():
    rng = np.random.default_rng(12)
    v = rng.standard_normal(300)
    for r in (0, 1, 5, 40, 299, 400):
        U, L = oracle.envelope(v, r)
        np.testing.assert_array_equal(U, maximum_filter1d(v, 2 * r + 1, mode="nearest"))
        np.testing.assert_array_equal(L, minimum_filter1d(v, 2 * r + 1, mode="nearest"))
    x = synth.random_walk(3000, 2)
    U, L = oracle.series_envelope(x, 17)
    np.testing.assert_array_equal(U, maximum_filter1d(x, 35, mode="nearest"))
    np.testing.assert_array_equal(L, minimum_filter1d(x, 35, mode="nearest"))


def test_lower_bounds_are_admissible():
    x = synth.random_walk(20_000, 21)
    rng = np.random.default_rng(22)
    for m, r in ((16, 0), (16, 3), (64, 6), (128, 12), (128, 127)):
        q, _ = synth.noisy_copy(x, m, 31 + m, 32 + m, noise=0.5)
        offs = rng.integers(0, x.size - m + 1, 400)
        kim, kq, kc, ks = oracle.lbs_at(x, q, r, offs)
        d = oracle.dtw_at(x, q, r, offs)
        tol = 1e-9 * np.maximum(1, d)
        assert np.all(kim <= d + tol)
        assert np.all(kq <= d + tol)
        assert np.all(kc <= d + tol)
        assert np.all(ks <= kc + tol)  # the series-wide envelope is looser
        if r == 0:
            qh = oracle.znorm(q)
            for t, o in enumerate(offs[:20]):
                ed = np.sum((qh - oracle.znorm(x[o:o + m])) ** 2)
                assert abs(kq[t] - ed) <= 1e-9 * ed and abs(kc[t] - ed) <= 1e-9 * ed
                # with r = 0 the series-wide envelope at j is the sample
                # itself, so Eq. 10 over it is the squared ED as well
                assert abs(ks[t] - ed) <= 1e-9 * ed


def test_series_envelope_bound_hand_values():
    """Eq. 10 against the series-wide envelope: hand-worked values, one of
    which differs from the window-clipped reading (a slip that clips to the
    window would give 2.5 instead of 0)."""
    for c in GOLD["lb_keogh_series"]:
        _, _, kc, ks = oracle.lbs_at(np.array(c["x"], np.float32), np.array(c["q"], np.float32), c["r"],
                                     [c["offset"]])
        want = c["keogh_series"] if "keogh_series" in c else 3.5 - 2 * np.sqrt(3.0)
        assert abs(ks[0] - want) <= 1e-12, (c, ks[0])
        if "keogh_clipped" in c:
            assert abs(kc[0] - c["keogh_clipped"]) <= 1e-12, (c, kc[0])


def test_series_envelope_bound_matches_scipy_definition():
    """Eq. 10 with the series-wide envelope restated with SciPy filters (max /
    min over [t-r, t+r] clipped to the series = mode 'nearest') and NumPy
    normalisation, at windows near both series ends and in the interior."""
    x = synth.random_walk(5_000, 41)
    rng = np.random.default_rng(42)
    for m, r in ((16, 1), (40, 5), (100, 30), (64, 63)):
        q, _ = synth.noisy_copy(x, m, 43 + m, 44 + m, noise=0.4)
        offs = np.concatenate([[0, 1, 2, x.size - m, x.size - m - 1], rng.integers(0, x.size - m + 1, 40)])
        _, _, _, ks = oracle.lbs_at(x, q, r, offs)
        U = maximum_filter1d(x.astype(np.float64), 2 * r + 1, mode="nearest")
        L = minimum_filter1d(x.astype(np.float64), 2 * r + 1, mode="nearest")
        qd = q.astype(np.float64)
        qh = (qd - qd.mean()) / qd.std()
        for t, o in enumerate(offs):
            w = x[o:o + m].astype(np.float64)
            mu, sg = w.mean(), w.std()
            u, lo = (U[o:o + m] - mu) / sg, (L[o:o + m] - mu) / sg
            want = np.sum(np.maximum(qh - u, 0) ** 2 + np.maximum(lo - qh, 0) ** 2)
            assert abs(ks[t] - want) <= 1e-9 * max(1.0, want), (m, r, o, ks[t], want)


# ------------------------------------------------------------------ search
@pytest.mark.parametrize("m", [8, 16, 32, 128])
def test_cascade_equals_brute_force(m):
    n = 20_000 if m <= 32 else 6_000
    x = synth.random_walk(n, 40 + m)
    q, _ = synth.noisy_copy(x, m, 50 + m, 60 + m, noise=0.3)
    for r in sorted({0, 1, m // 10, m - 1}):
        for k in (1, 10):
            bi, bd = oracle.search_brute(x, q, r, k)
            ci, cd = oracle.search_cascade(x, q, r, k)
            ai, ad = oracle.search_cascade(x, q, r, k, stats="anchored", B=4096)
            np.testing.assert_array_equal(ci, bi)
            np.testing.assert_allclose(cd, bd, rtol=1e-12, atol=1e-12)
            np.testing.assert_array_equal(ai, bi)
            np.testing.assert_allclose(ad, bd, rtol=1e-9, atol=1e-9)


def test_brute_force_is_sorted_definition():
    """Brute force equals a NumPy lexsort over every window's DTW."""
    x = synth.random_walk(600, 70)
    q, _ = synth.noisy_copy(x, 24, 71, 72)
    offs = np.arange(x.size - 24 + 1)
    d = oracle.dtw_at(x, q, 3, offs)
    order = np.lexsort((offs, d))[:10]
    bi, bd = oracle.search_brute(x, q, 3, 10)
    np.testing.assert_array_equal(bi, offs[order])
    np.testing.assert_array_equal(bd, d[order])


def test_planted_exact_copy_has_zero_distance():
    x = synth.random_walk(30_000, 80)
    o = 12_345
    q = x[o:o + 100].copy()
    for fn in (oracle.search_brute, oracle.search_cascade):
        i, d = fn(x, q, 10, 1)
        assert i[0] == o and d[0] == 0.0


def test_exact_ties_go_to_the_lowest_index():
    pat = np.random.default_rng(81).standard_normal(50).astype(np.float32)
    x = np.tile(pat, 40)
    q = x[10:10 + 64].copy()
    for fn in (oracle.search_brute, oracle.search_cascade):
        i, d = fn(x, q, 6, 3)
        assert i.tolist() == [10, 60, 110] and d.tolist() == [0.0, 0.0, 0.0]


def test_k_larger_than_windows():
    x = synth.random_walk(40, 82)
    q = synth.random_walk(30, 83)
    i, d = oracle.search_cascade(x, q, 3, 20)
    assert (i >= 0).sum() == 11 and np.all(i[11:] == -1) and np.all(np.isinf(d[11:]))
    bi, bd = oracle.search_brute(x, q, 3, 20)
    np.testing.assert_array_equal(i, bi)


def test_m_equals_n():
    x = synth.random_walk(64, 84)
    q = synth.random_walk(64, 85)
    i, d = oracle.search_cascade(x, q, 6, 1)
    assert i[0] == 0
    assert abs(d[0] - oracle.dtw(oracle.znorm(q), oracle.znorm(x), 6)) < 1e-12


# ------------------------------------------------------------------ Eq. 11 fragments
def test_partition_covers_each_window_once():
    for N, F in itertools.product((1, 7, 100, 1001), (1, 2, 3, 7, 16)):
        parts = fragments.partition(N, F)
        covered = np.zeros(N, int)
        for s, c in parts:
            covered[s:s + c] += 1
        assert np.all(covered == 1)


@pytest.mark.parametrize("F", [2, 3, 7])
def test_fragment_merge_equals_single_pass(F):
    x = synth.random_walk(15_000, 90)
    q, _ = synth.noisy_copy(x, 64, 91, 92, noise=0.5)
    for k in (1, 10):
        si, sd = oracle.search_cascade(x, q, 6, k)
        fi, fd = fragments.search_fragments(x, q, 6, k, F=F, threads=3)
        np.testing.assert_array_equal(fi, si)
        np.testing.assert_array_equal(fd, sd)


def test_fragment_worker_failure_propagates():
    x = synth.random_walk(1000, 93)
    q = synth.random_walk(10, 94)
    with pytest.raises(ValueError):
        # a fragment whose window range runs past the series is rejected by
        # the oracle; search_fragments must re-raise instead of returning a result
        fragments.search_fragments(x, q, 2, 1, F=2, threads=2, first=500, count=600)
