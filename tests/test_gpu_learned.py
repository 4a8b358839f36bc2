"""Learned proposal encoder on the GPU against the FP64 encoder reference,
through the C ABI: input preparation, forward (tensor cores, BF16 operands,
FP32 accumulation), loss and gradient, the series-wide embeddings, the
trainer, and the search with learned ordering (same answers as without it,
less work than the paper's random seeding)."""
import os

import numpy as np
import pytest

import oracle
from oracle import encoder as enc
from oracle import label_triples
from paper_1812_10302_gb300 import dtws, synth, train

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30)


@pytest.fixture(scope="module")
def params():
    return enc.init_params(3)


def _windows(n, ms, count, seed):
    x = synth.walk_with_bursts(n, seed, seed + 1, seed + 2)
    rng = np.random.default_rng(seed)
    return x, {m: rng.integers(0, n - m + 1, count) for m in ms}


def test_prep_matches_oracle():
    x, offs = _windows(300_000, (64, 200, 1024, 8192), 40, 1)
    x[5000:9000] = 3.25  # constant windows: u = 0
    for m, o in offs.items():
        o = np.r_[o, 5000]
        u = dtws.enc_prep(x, o, m)
        assert u.shape == (o.size, 64) and np.all(u[:, 63] == 0)
        want = np.stack([enc.prep(x[i:i + m]) for i in o])
        np.testing.assert_allclose(u[:, :63], want, rtol=2e-5, atol=2e-6)
        if m <= 4000:
            assert np.all(u[-1] == 0)


def test_forward_matches_oracle(params):
    x, offs = _windows(200_000, (1024,), 96, 2)
    u = np.stack([enc.prep(x[i:i + 1024]) for i in offs[1024]])
    u64 = np.zeros((u.shape[0], 64), np.float32)
    u64[:, :63] = u
    e = dtws.enc_forward(params, u64)
    for i in range(u.shape[0]):
        want16 = enc.forward(params, u64[i, :63].astype(np.float64), bf16=True)[0]
        want64 = enc.forward(params, u64[i, :63].astype(np.float64))[0]
        assert _rel(e[i], want16) < 2e-3, i   # same operand rounding, FP32 accumulation
        assert _rel(e[i], want64) < 3e-2, i   # BF16 operands vs FP64
    # homogeneity holds on the GPU too (up to BF16 rounding of scaled activations)
    e2 = dtws.enc_forward(params, 2.0 * u64)
    np.testing.assert_allclose(e2, 2.0 * e, rtol=0, atol=1e-5 * np.abs(e).max() + 1e-6)


def test_loss_and_gradient_match_oracle(params):
    x, xq = synth.training_series(400_000, 7)
    m, B = 512, 24
    q_off, c_off = synth.training_pairs(x.size, m, B, 5, per_query=12)
    y = np.array([oracle.dtw_at(x, xq[q:q + m], 51, [c])[0] / m for q, c in zip(q_off, c_off)])
    uq = dtws.enc_prep(xq, q_off, m)
    uc = dtws.enc_prep(x, c_off, m)
    L, g = dtws.enc_loss_grad(params, uq, uc, y.astype(np.float32))
    Lb, gb = enc.loss_and_grad(params.astype(np.float64), uq[:, :63], uc[:, :63], y, bf16=True)
    Lo, go = enc.loss_and_grad(params.astype(np.float64), uq[:, :63], uc[:, :63], y)
    assert abs(L - Lb) <= 2e-3 * Lb and abs(L - Lo) <= 3e-2 * Lo
    offs = np.cumsum((0,) + enc.SIZES)
    for i in range(5):
        a, b, c = g[offs[i]:offs[i + 1]], gb[offs[i]:offs[i + 1]], go[offs[i]:offs[i + 1]]
        cb = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        co = float(a @ c / (np.linalg.norm(a) * np.linalg.norm(c)))
        # same operand rounding as the GPU: accumulation order only
        assert _rel(a, b) < 2e-2 and cb > 0.9998, (i, _rel(a, b), cb)
        # against exact FP64: the BF16 operands' effect
        assert _rel(a, c) < 0.2 and co > 0.99, (i, _rel(a, c), co)


def test_series_embeddings_match_per_window_oracle(params):
    n, m = 600_000, 1024
    x = synth.walk_with_bursts(n, 11, 12, 13)
    x[300_000:302_000] = -7.0  # constant windows
    with dtws.Index(x) as ix:
        ix.set_encoder(params)
        E = ix.learned_embeddings(m)
        b = m // 64
        assert E.shape == ((n - m) // b + 1, 64)
        rows = np.r_[np.random.default_rng(14).integers(0, E.shape[0], 60), 0, E.shape[0] - 1,
                     300_000 // b + 10]
        for j in rows:
            o = j * b
            want = enc.embed(params, x[o:o + m].astype(np.float64), bf16=True)
            if np.linalg.norm(want) == 0:  # a constant window: zero embedding
                assert np.all(E[j] == 0)
                continue
            assert _rel(E[j], want) < 1.5e-2, (j, _rel(E[j], want))
        # a new encoder replaces the cached embeddings
        ix.set_encoder(2 * params)
        E2 = ix.learned_embeddings(m)
        assert not np.allclose(E2, E)


def test_learned_ordering_gives_the_same_answers(params):
    n = 2_000_000
    x = synth.walk_with_bursts(n, 21, 22, 23)
    queries = [synth.noisy_copy(x, m, 30 + i, 40 + i) for i, m in enumerate((64, 128, 512, 1024, 2048))]
    with dtws.Index(x) as ix:
        for q, _ in queries:
            m = q.size
            r = synth.band(0.1, m)
            for k in (1, 10):
                ix.set_options(ordering=dtws.DTWS_ORDER_PLAIN)
                i0, d0 = ix.query(q, r, k)
                ix.set_encoder(params)
                ix.set_options(ordering=dtws.DTWS_ORDER_LEARNED)
                i1, d1 = ix.query(q, r, k)
                assert ix.sync_status() == dtws.DTWS_OK
                np.testing.assert_array_equal(i1, i0)
                np.testing.assert_array_equal(d1, d0)
        ix.set_options(ordering=dtws.DTWS_ORDER_LEARNED)
        with pytest.raises(dtws.DtwsError):
            ix.query(np.random.default_rng(0).normal(size=32).astype(np.float32), 3, 1)  # m < 64


def test_learned_ordering_needs_an_encoder():
    x = synth.random_walk(100_000, 1)
    with dtws.Index(x) as ix:
        ix.set_options(ordering=dtws.DTWS_ORDER_LEARNED)
        with pytest.raises(dtws.DtwsError):
            ix.query(x[1000:1512], 51, 1)


def test_trainer_reduces_the_loss():
    d = label_triples.make(2_000_000, [512], 8192, seed=200)
    params, hist = train.train(d, epochs=6, batch=512, lr=2e-3, log_every=10, verbose=False)
    losses = [h["loss"] for h in hist if "step" in h]
    val = [h for h in hist if "val_m" in h][0]
    assert losses[-1] < 0.5 * losses[0], losses
    assert val["loss"] < 0.7 * val["loss_init"], val
    assert np.all(np.isfinite(params))


def _work(ix, q, r, k=1):
    idx, dist = ix.query(q, r, k)
    assert ix.sync_status() == dtws.DTWS_OK
    st = ix.last_stats()
    return idx, dist, st


@pytest.mark.skipif(not os.path.exists(train.DEFAULT_WEIGHTS), reason="no trained encoder weights committed")
def test_trained_encoder_gains_over_random_seeding():
    """On a walk-with-bursts series of the learned-proposal workload's kind
    (its own seeds, disjoint from the training series), learned proposals
    give the same answers as the paper's random seeding with far fewer
    windows left after the lower-bound scan; against an untrained encoder
    they find the planted match at least as often."""
    w = synth.workload("learn", n=8_000_000)
    x, qs, offs = w["series"], w["queries"][:12], w["true_offsets"][:12]
    r = w["rs"][0]
    trained = train.load_weights()
    untrained = train.init_params(0)
    res = {}
    with dtws.Index(x) as ix:
        ix.set_options(seed_proposals=0)
        res["random"] = [_work(ix, q, r) for q in qs]
        for name, p in (("trained", trained), ("untrained", untrained)):
            ix.set_encoder(p)
            ix.set_options(ordering=dtws.DTWS_ORDER_LEARNED, seed_proposals=16)
            res[name] = [_work(ix, q, r) for q in qs]
    for name in ("trained", "untrained"):
        for a, b in zip(res[name], res["random"]):
            np.testing.assert_array_equal(a[0], b[0])
            np.testing.assert_array_equal(a[1], b[1])
    surv = {k: np.array([s["pass_keogh_q"] for _, _, s in v]) for k, v in res.items()}
    # the seeding found the answer's neighbourhood when its best seed is no
    # worse than the answer window's own Euclidean distance (r = 0)
    ed = np.array([oracle.dtw_at(x, q, 0, a[0])[0] for q, a in zip(qs, res["random"])])
    seed_hit = {k: float(np.mean([s["seed_bsf"] <= e * (1 + 1e-4) + 1e-6 for (_, _, s), e in zip(v, ed)]))
                for k, v in res.items()}
    print("survivors of the scan (median):", {k: int(np.median(v)) for k, v in surv.items()})
    print("seeding reached the answer's Euclidean distance:", seed_hit)
    assert np.median(surv["trained"]) * 10 < np.median(surv["random"])
    assert seed_hit["trained"] >= seed_hit["untrained"]
    assert seed_hit["trained"] >= 0.9
    del offs


@pytest.mark.skipif(not os.path.exists(train.DEFAULT_WEIGHTS), reason="no trained encoder weights committed")
def test_seeding_by_proposal_count():
    """How well each seeding finds the answer's neighbourhood as the number of
    proposals shrinks: the trained encoder, an untrained (random) one and the
    proxy scan, with 1, 2, 4 and 16 proposals, on 32 queries of the learned
    workload's kind (8e6 samples).  A query counts when its best seed is no
    worse than the answer window's own Euclidean distance.  The answers are
    the same in every case; the counts are printed (they are the record of
    what training buys), and at the default 16 proposals every seeding must
    reach the answer for at least 90% of the queries and the trained encoder
    must be no worse than the untrained one."""
    w = synth.workload("learn", n=8_000_000)
    x, qs = w["series"], w["queries"][:32]
    r = w["rs"][0]
    hits = {}
    with dtws.Index(x) as ix:
        ix.set_options(seed_proposals=0)
        base = [ix.query(q, r, 1) for q in qs]
        ed = np.array([oracle.dtw_at(x, q, 0, a[0])[0] for q, a in zip(qs, base)])
        for P in (1, 2, 4, 16):
            for name in ("proxy", "trained", "untrained"):
                if name == "proxy":
                    ix.set_options(ordering=dtws.DTWS_ORDER_PLAIN, seed_proposals=P)
                else:
                    ix.set_encoder(train.load_weights() if name == "trained" else train.init_params(0))
                    ix.set_options(ordering=dtws.DTWS_ORDER_LEARNED, seed_proposals=P)
                got = 0
                for q, e, a in zip(qs, ed, base):
                    idx, dist = ix.query(q, r, 1)
                    assert ix.sync_status() == dtws.DTWS_OK
                    np.testing.assert_array_equal(idx, a[0])
                    got += ix.last_stats()["seed_bsf"] <= e * (1 + 1e-4) + 1e-6
                hits[(P, name)] = got
    print("queries (of 32) whose best seed reached the answer's Euclidean distance:",
          {f"P={P} {n}": v for (P, n), v in hits.items()})
    for name in ("proxy", "trained", "untrained"):
        assert hits[(16, name)] >= 29
    assert hits[(16, "trained")] >= hits[(16, "untrained")]
