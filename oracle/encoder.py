"""FP64 reference of the learned proposal encoder (forward, loss, backward).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``): imported only by tests,
the smoke check and the benchmark's CPU legs; it shares no code with the
CUDA path.

The paper has no learned component; the encoder's shape is fixed by the
project's goal statement (a 1-D CNN of 4 convolution layers, 32 channels,
kernel 7, a 64-dimensional embedding, BF16 weights with FP32 accumulation on
the GPU), and everything else here is this project's definition:

* Input of a window y of length m (a query or a subsequence): block length
  b = floor(m / 64), block means a_j of y[j*b : (j+1)*b] for j = 0..63 (the
  first 64*b samples), z-normalised with the mean and population deviation
  of all m samples (Eq. 5): v_j = (a_j - mu) / sigma; the network sees the
  63 differences u_j = v_{j+1} - v_j = (a_{j+1} - a_j) / sigma.  A window
  with sigma = 0 gives u = 0 (the same zero-variance rule as the search).
* conv1: 1 -> 32 channels, kernel 7, valid, ReLU        (57 positions)
  conv2, conv3: 32 -> 32, kernel 7, valid, ReLU         (51, 45)
  conv4: 32 -> 32, kernel 7, valid, no activation       (39)
  No layer has a bias.
* Pool: 8 segments, segment s = positions [floor(39 s / 8), floor(39 (s+1) / 8)),
  mean over the segment, per channel -> g[s][c].
* Projection: e[d] = sum_{s,c} P[d][s*32 + c] * g[s][c], 64 outputs, no bias.
* Distance of two embeddings: sum_d (e1[d] - e2[d])^2.
* Training loss of a triple (Q, C, y) with y = DTW(Q^, C^) / m:
  (log(dist + eps) - log(y + eps))^2, eps = 1e-3, averaged over the batch.

Without biases every layer is positively homogeneous, so e(c*u) = c*e(u)
for c > 0: a window's embedding is its raw block-mean differences' embedding
times 1/sigma.

Parameter vector (FP32/FP64, flat, in this order):
  W1 [32][7]            w1[c][t]
  W2, W3, W4 [32][7][32] w[co][t][ci]   (reduction index t*32 + ci)
  P [64][256]           p[d][s*32 + c]
"""
from __future__ import annotations

import numpy as np

C = 32
KW = 7
NB = 64
NU = NB - 1
L1, L2, L3, L4 = NU - 6, NU - 12, NU - 18, NU - 24  # 57, 51, 45, 39
NSEG = 8
DIM = 64
EPS = 1e-3
SIZES = (C * KW, C * KW * C, C * KW * C, C * KW * C, DIM * NSEG * C)
NPARAMS = sum(SIZES)  # 38112


def block_len(m: int) -> int:
    if m < NB:
        raise ValueError("the encoder needs m >= 64")
    return m // NB


def segments():
    """Pooling segment bounds over the 39 conv4 positions."""
    return [(L4 * s // NSEG, L4 * (s + 1) // NSEG) for s in range(NSEG)]


def split(params):
    p = np.asarray(params, np.float64)
    if p.size != NPARAMS:
        raise ValueError(f"expected {NPARAMS} parameters")
    out, o = [], 0
    shapes = ((C, KW), (C, KW, C), (C, KW, C), (C, KW, C), (DIM, NSEG * C))
    for n, sh in zip(SIZES, shapes):
        out.append(p[o:o + n].reshape(sh))
        o += n
    return out


def init_params(seed: int) -> np.ndarray:
    """He-style initial values (the GPU trainer starts from a vector passed in)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2.0 / KW), C * KW)]
    for _ in range(3):
        parts.append(rng.normal(0, np.sqrt(2.0 / (KW * C)), C * KW * C))
    parts.append(rng.normal(0, np.sqrt(1.0 / (NSEG * C)), DIM * NSEG * C))
    return np.concatenate(parts).astype(np.float32)


def prep(y) -> np.ndarray:
    """u (63 values, FP64) of one window, by the definition above."""
    y = np.asarray(y, np.float64)
    m = y.size
    b = block_len(m)
    mu = y.mean()
    var = ((y - mu) ** 2).mean()
    if var <= 1e-24 * max(1.0, mu * mu):
        return np.zeros(NU)
    sigma = np.sqrt(var)
    a = y[: NB * b].reshape(NB, b).mean(axis=1)
    v = (a - mu) / sigma
    return v[1:] - v[:-1]


def _conv(x, w):
    """Valid correlation: out[p][co] = sum_{t, ci} w[co][t][ci] * x[p + t][ci]."""
    P = x.shape[0] - KW + 1
    out = np.zeros((P, w.shape[0]))
    for t in range(KW):
        out += x[t:t + P] @ w[:, t, :].T
    return out


def forward(params, u, bf16: bool = False):
    """Embedding e (64) of one input u (63) and the intermediate values.

    bf16: round the operands the GPU feeds to its BF16 tensor-core products
    (W2..W4, P, the post-ReLU h1..h3 and the pooled g) to bfloat16 first,
    everything else in FP64 -- the storage precision the encoder's GPU
    kernels use (BF16 weights and activations, wide accumulation)."""
    W1, W2, W3, W4, Pm = split(params)
    rb = round_bf16 if bf16 else (lambda a: a)
    if bf16:
        W2, W3, W4, Pm = (rb(w) for w in (W2, W3, W4, Pm))
    u = np.asarray(u, np.float64)
    z1 = _conv(u[:, None], W1[:, :, None])
    h1 = rb(np.maximum(z1, 0))
    z2 = _conv(h1, W2)
    h2 = rb(np.maximum(z2, 0))
    z3 = _conv(h2, W3)
    h3 = rb(np.maximum(z3, 0))
    h4 = _conv(h3, W4)
    g = rb(np.stack([h4[lo:hi].mean(axis=0) for lo, hi in segments()]))  # [8][32]
    e = Pm @ g.reshape(-1)
    return e, dict(u=u, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3, h4=h4, g=g)


def embed(params, y, bf16: bool = False) -> np.ndarray:
    return forward(params, prep(y), bf16)[0]


def _conv_back(x, w, dout):
    """Gradients of the valid correlation w.r.t. its input and weights."""
    P = dout.shape[0]
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t in range(KW):
        dx[t:t + P] += dout @ w[:, t, :]
        dw[:, t, :] += dout.T @ x[t:t + P]
    return dx, dw


def backward(params, cache, de, bf16: bool = False):
    """Gradient of a scalar with d(scalar)/de = de, w.r.t. the flat parameters.

    bf16: the backward pass of the BF16 forward as the GPU runs it -- the
    rounded weights, and the gradients that feed tensor-core products (dh4
    and the masked dz3, dz2, dz1) rounded to bfloat16."""
    W1, W2, W3, W4, Pm = split(params)
    rb = round_bf16 if bf16 else (lambda a: a)
    if bf16:
        W2, W3, W4, Pm = (rb(w) for w in (W2, W3, W4, Pm))
    de = np.asarray(de, np.float64)
    dP = np.outer(de, cache["g"].reshape(-1))
    dg = (Pm.T @ de).reshape(NSEG, C)
    dh4 = np.zeros((L4, C))
    for s, (lo, hi) in enumerate(segments()):
        dh4[lo:hi] = dg[s] / (hi - lo)
    dh4 = rb(dh4)
    dh3, dW4 = _conv_back(cache["h3"], W4, dh4)
    dz3 = rb(dh3 * (cache["z3"] > 0))
    dh2, dW3 = _conv_back(cache["h2"], W3, dz3)
    dz2 = rb(dh2 * (cache["z2"] > 0))
    dh1, dW2 = _conv_back(cache["h1"], W2, dz2)
    dz1 = rb(dh1 * (cache["z1"] > 0))
    _, dW1 = _conv_back(cache["u"][:, None], W1[:, :, None], dz1)
    return np.concatenate([dW1.reshape(-1), dW2.reshape(-1), dW3.reshape(-1), dW4.reshape(-1),
                           dP.reshape(-1)])


def loss_and_grad(params, uq, uc, y, bf16: bool = False):
    """Mean triple loss over a batch and its gradient (FP64; with bf16, the
    GPU's BF16 operand rounding in forward and backward, see forward and
    backward).  uq, uc: [B][63] inputs; y: [B] labels DTW / m."""
    uq = np.atleast_2d(np.asarray(uq, np.float64))
    uc = np.atleast_2d(np.asarray(uc, np.float64))
    y = np.atleast_1d(np.asarray(y, np.float64))
    B = y.size
    total = 0.0
    grad = np.zeros(NPARAMS)
    for i in range(B):
        eq, cq = forward(params, uq[i], bf16)
        ec, cc = forward(params, uc[i], bf16)
        diff = eq - ec
        dist = float(diff @ diff)
        lr = np.log(dist + EPS) - np.log(y[i] + EPS)
        total += lr * lr
        dd = 2.0 * lr / (dist + EPS) / B          # d(mean loss)/d(dist)
        grad += backward(params, cq, 2.0 * diff * dd, bf16)
        grad += backward(params, cc, -2.0 * diff * dd, bf16)
    return total / B, grad


def round_bf16(a) -> np.ndarray:
    """Round-to-nearest-even to bfloat16 (8 significant bits), as FP64 values."""
    f = np.asarray(a, np.float32).copy()
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) >> 16 << 16
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)
