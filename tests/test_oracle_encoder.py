"""Pins of the FP64 encoder reference (oracle/encoder.py) against facts that
do not come from its own code: finite differences of its loss, SciPy and
NumPy correlations and z-scores, a closed form for an identity-like network,
positive homogeneity, and torch's bfloat16 conversion."""
import numpy as np
import pytest
import scipy.signal
import scipy.stats

from oracle import encoder as enc


def _small_params(seed):
    return enc.init_params(seed).astype(np.float64)


def test_parameter_count_and_segments():
    assert enc.NPARAMS == 224 + 3 * 7168 + 64 * 256 == 38112
    segs = enc.segments()
    assert segs[0][0] == 0 and segs[-1][1] == enc.L4 == 39
    assert all(a[1] == b[0] and a[1] > a[0] for a, b in zip(segs, segs[1:]))


def test_prep_equals_zscore_block_means_differences():
    rng = np.random.default_rng(0)
    for m in (64, 128, 200, 1024, 2047):
        y = np.cumsum(rng.normal(size=m)) * 3 + 50
        z = scipy.stats.zscore(y, ddof=0)
        b = m // 64
        a = np.add.reduceat(z[: 64 * b], np.arange(0, 64 * b, b)) / b
        np.testing.assert_allclose(enc.prep(y), np.diff(a), rtol=1e-10, atol=1e-12)


def test_prep_is_affine_invariant_and_zero_for_constant():
    rng = np.random.default_rng(1)
    y = np.cumsum(rng.normal(size=512))
    np.testing.assert_allclose(enc.prep(2.5 * y - 7.0), enc.prep(y), atol=1e-12)
    assert np.all(enc.prep(np.full(300, 4.0)) == 0)
    with pytest.raises(ValueError):
        enc.prep(np.arange(63.0))


def test_conv1_is_numpy_correlate_and_conv_is_scipy_correlate2d():
    p = _small_params(2)
    W1, W2 = enc.split(p)[:2]
    u = np.random.default_rng(3).normal(size=63)
    _, cache = enc.forward(p, u)
    for c in range(enc.C):
        np.testing.assert_allclose(cache["z1"][:, c], np.correlate(u, W1[c], "valid"), atol=1e-12)
    h1 = cache["h1"]
    for co in (0, 7, 31):
        ref = scipy.signal.correlate2d(h1, W2[co], mode="valid")[:, 0]
        np.testing.assert_allclose(cache["z2"][:, co], ref, atol=1e-10)


def test_identity_network_closed_form():
    """Tap t of conv1 and tap 0 of the rest, channel 0 only, projection
    picking each segment's channel 0: e[s] = mean over segment s of
    max(u[p + t], 0), e[8:] = 0."""
    for t in (0, 3, 6):
        W1 = np.zeros((32, 7)); W1[0, t] = 1
        Wn = np.zeros((32, 7, 32)); Wn[0, 0, 0] = 1
        P = np.zeros((64, 256))
        for s in range(8):
            P[s, s * 32] = 1
        params = np.concatenate([W1.ravel(), Wn.ravel(), Wn.ravel(), Wn.ravel(), P.ravel()])
        u = np.random.default_rng(4 + t).normal(size=63)
        e = enc.forward(params, u)[0]
        want = [np.maximum(u[lo + t:hi + t], 0).mean() for lo, hi in enc.segments()]
        np.testing.assert_allclose(e[:8], want, atol=1e-14)
        assert np.all(e[8:] == 0)


def test_embedding_is_positively_homogeneous():
    p = _small_params(5)
    u = np.random.default_rng(6).normal(size=63)
    e = enc.forward(p, u)[0]
    for c in (0.01, 0.5, 3.0, 1e3):
        np.testing.assert_allclose(enc.forward(p, c * u)[0], c * e, rtol=1e-12, atol=1e-14)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(7)
    p = _small_params(8)
    B = 3
    uq = rng.normal(size=(B, 63))
    uc = uq + 0.5 * rng.normal(size=(B, 63))
    y = np.array([0.05, 0.3, 1.2])
    L, g = enc.loss_and_grad(p, uq, uc, y)
    h = 1e-6
    offs = np.cumsum((0,) + enc.SIZES)
    picks = np.concatenate([rng.integers(offs[i], offs[i + 1], 12) for i in range(5)])
    for j in picks:
        pp, pm = p.copy(), p.copy()
        pp[j] += h
        pm[j] -= h
        fd = (enc.loss_and_grad(pp, uq, uc, y)[0] - enc.loss_and_grad(pm, uq, uc, y)[0]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(g).max()), (j, fd, g[j])


def test_loss_is_zero_when_distance_equals_label():
    p = _small_params(9)
    rng = np.random.default_rng(10)
    uq, uc = rng.normal(size=63), rng.normal(size=63)
    d = np.sum((enc.forward(p, uq)[0] - enc.forward(p, uc)[0]) ** 2)
    L, g = enc.loss_and_grad(p, uq, uc, [d])
    assert L < 1e-20 and np.abs(g).max() < 1e-9


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    v = np.concatenate([np.random.default_rng(11).normal(size=2000) * 10,
                        [1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0, 65504.0]]).astype(np.float32)
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(enc.round_bf16(v), want)


def test_bf16_forward_differs_from_fp64_by_bf16_rounding_only():
    """With the BF16 option the embedding moves by about the bfloat16 unit
    roundoff (2^-9 relative); with weights and inputs that bfloat16 holds
    exactly (the identity-like network on quarter-integer inputs) it does
    not move at all."""
    p = _small_params(12)
    u = np.random.default_rng(13).normal(size=63)
    e64 = enc.forward(p, u)[0]
    e16 = enc.forward(p, u, bf16=True)[0]
    rel = np.linalg.norm(e16 - e64) / np.linalg.norm(e64)
    assert 1e-5 < rel < 3e-2
    W1 = np.zeros((32, 7)); W1[0, 0] = 1
    Wn = np.zeros((32, 7, 32)); Wn[0, 0, 0] = 1
    P = np.zeros((64, 256)); P[0, 0] = 1
    ident = np.concatenate([W1.ravel(), Wn.ravel(), Wn.ravel(), Wn.ravel(), P.ravel()])
    uq = np.round(u * 4) / 4
    np.testing.assert_array_equal(enc.forward(ident, uq, bf16=True)[0], enc.forward(ident, uq)[0])


def test_bf16_gradient_is_exact_where_rounding_is_the_identity():
    """On weights and inputs that bfloat16 holds exactly and whose forward
    intermediates stay exact (identity-like network, quarter-integer
    inputs), the BF16 emulation's loss equals the FP64 one and its gradient
    differs only by the rounded backward terms; on general inputs both agree
    to the BF16 roundoff."""
    W1 = np.zeros((32, 7)); W1[0, 0] = 1
    Wn = np.zeros((32, 7, 32)); Wn[0, 0, 0] = 1
    P = np.zeros((64, 256)); P[0, 0] = 1
    ident = np.concatenate([W1.ravel(), Wn.ravel(), Wn.ravel(), Wn.ravel(), P.ravel()])
    rng = np.random.default_rng(14)
    uq = np.round(rng.normal(size=(2, 63)) * 4) / 4
    uc = np.round(rng.normal(size=(2, 63)) * 4) / 4
    L0, g0 = enc.loss_and_grad(ident, uq, uc, [0.25, 2.0])
    L1, g1 = enc.loss_and_grad(ident, uq, uc, [0.25, 2.0], bf16=True)
    assert L0 == L1
    # the loss factor 2*lr/(dist+eps) is not a short binary fraction, so the
    # rounded gradient terms differ from FP64 by the bfloat16 roundoff; their
    # sums (with cancellation) agree to about 1% in norm
    assert np.linalg.norm(g1 - g0) < 1e-2 * np.linalg.norm(g0)
    p = _small_params(15)
    uq = rng.normal(size=(3, 63)); uc = uq + 0.3 * rng.normal(size=(3, 63))
    La, ga = enc.loss_and_grad(p, uq, uc, [0.1, 0.5, 1.0])
    Lb, gb = enc.loss_and_grad(p, uq, uc, [0.1, 0.5, 1.0], bf16=True)
    assert abs(La - Lb) < 2e-2 * La
    assert np.dot(ga, gb) / (np.linalg.norm(ga) * np.linalg.norm(gb)) > 0.99
