"""Train the learned proposal encoder on the GPU (the library's own forward,
backward and Adam kernels, ``dtws_trainer_*``).

Input: an .npz of labelled (query, candidate) offset pairs on the training
series (per query length m: q_off, c_off, y = DTW/m; the series is rebuilt
from its seed with ``synth.training_series``).  Steps alternate between the
query lengths; each step takes a shuffled batch of one length.  Output: the
FP32 parameter vector (``DTWS_ENC_PARAMS`` values, .npy).

    python -m paper_1812_10302_gb300.train --triples triples.npz \\
        --out paper_1812_10302_gb300/weights/encoder_walk_bursts.npy
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import dtws, synth

WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
DEFAULT_WEIGHTS = os.path.join(WEIGHTS_DIR, "encoder_walk_bursts.npy")


def init_params(seed: int) -> np.ndarray:
    """He-style normal initial values in the parameter layout of dtws.h."""
    rng = np.random.default_rng(seed)
    C, KW = 32, 7
    parts = [rng.normal(0, np.sqrt(2.0 / KW), C * KW)]
    for _ in range(3):
        parts.append(rng.normal(0, np.sqrt(2.0 / (KW * C)), C * KW * C))
    parts.append(rng.normal(0, np.sqrt(1.0 / (8 * C)), 64 * 8 * C))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == dtws.DTWS_ENC_PARAMS
    return p


def load_weights(path: str = DEFAULT_WEIGHTS) -> np.ndarray:
    p = np.load(path).astype(np.float32)
    if p.size != dtws.DTWS_ENC_PARAMS:
        raise ValueError(f"{path}: expected {dtws.DTWS_ENC_PARAMS} parameters")
    return p


def train(data: dict, epochs: float = 2.0, batch: int = 1024, lr: float = 1e-3, init_seed: int = 0,
          log_every: int = 100, params=None, val_frac: float = 0.02, verbose: bool = True):
    """Returns (params, history).  ``data`` as written by the labelling script."""
    import torch

    n, seed = int(data["n"]), int(data["seed"])
    ms = [int(m) for m in data["ms"]]
    x, xq = synth.training_series(n, seed)
    xd = torch.from_numpy(x).cuda()
    xqd = torch.from_numpy(xq).cuda()
    rng = np.random.default_rng(init_seed + 1)
    sets, val = {}, {}
    for m in ms:
        q, c, y = data[f"m{m}_q_off"], data[f"m{m}_c_off"], data[f"m{m}_y"]
        perm = rng.permutation(q.size)
        nv = int(q.size * val_frac)
        val[m] = (q[perm[:nv]], c[perm[:nv]], y[perm[:nv]])
        sets[m] = (q[perm[nv:]], c[perm[nv:]], y[perm[nv:]])
    p0 = init_params(init_seed) if params is None else np.asarray(params, np.float32)
    tr = dtws.Trainer(p0, max_batch=batch, lr=lr)
    total = sum(s[0].size for s in sets.values())
    steps = int(epochs * total / batch)
    hist = []
    order = {m: rng.permutation(sets[m][0].size) for m in ms}
    pos = {m: 0 for m in ms}
    t0 = time.perf_counter()
    for step in range(steps):
        m = ms[step % len(ms)]
        q, c, y = sets[m]
        if pos[m] + batch > q.size:
            order[m] = rng.permutation(q.size)
            pos[m] = 0
        idx = order[m][pos[m]:pos[m] + batch]
        pos[m] += batch
        want = (step % log_every == 0) or step == steps - 1
        loss = tr.step(xqd, xd, q[idx], c[idx], m, y[idx], want_loss=want)
        if want:
            hist.append({"step": step, "m": m, "loss": loss})
            if verbose:
                print(f"step {step}/{steps} m={m} loss {loss:.4f} ({time.perf_counter() - t0:.1f} s)", flush=True)
    params = tr.params()
    tr.close()
    torch.cuda.synchronize()
    # held-out loss per query length
    for m in ms:
        q, c, y = val[m]
        if q.size == 0:
            continue
        uq = dtws.enc_prep(xqd, q, m)
        uc = dtws.enc_prep(xd, c, m)
        vl, _ = dtws.enc_loss_grad(params, uq, uc, y)
        vl0, _ = dtws.enc_loss_grad(p0, uq, uc, y)
        hist.append({"val_m": m, "loss": vl, "loss_init": vl0})
        if verbose:
            print(f"held-out m={m}: loss {vl:.4f} (initial parameters {vl0:.4f})", flush=True)
    return params, hist


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--triples", required=True)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--epochs", type=float, default=2.0)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--log", default=None, help="write the loss history as JSON here")
    args = ap.parse_args(argv)
    data = dict(np.load(args.triples))
    t0 = time.perf_counter()
    params, hist = train(data, args.epochs, args.batch, args.lr, args.init_seed)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.save(args.out, params)
    print(f"trained in {time.perf_counter() - t0:.1f} s -> {args.out}")
    if args.log:
        with open(args.log, "w") as f:
            json.dump(hist, f, indent=1)


if __name__ == "__main__":
    main()
