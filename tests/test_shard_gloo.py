"""Multi-process fragment sharding (Sec. 3.1, Eq. 11) and the merge of the
per-fragment best pairs, on CPU with the gloo backend, world size 2.  The
per-rank search engine here is the FP64 oracle (the host logic under test is
the partition and the exchange); a rank that fails must make the other's
collective end with an error instead of hanging."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1812_10302_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, world, port, timeout_s=60):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=timeout_s))
    return dist


def _worker(rank, world, port, out_q):
    dist = _init(rank, world, port)
    x = synth.random_walk(30_000, 3)
    q, _ = synth.noisy_copy(x, 64, 4, 5, noise=0.4)
    m, r, k = 64, 6, 5
    lo, hi = shard.fragment_samples(x.size, m, world, rank)
    idx, d = oracle.search_cascade(x[lo:hi], q, r, k)
    gi, gd = shard.allgather_merge(idx, d, k, offset=lo)
    out_q.put((rank, gi.tolist(), gd.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_merge_equals_single_pass():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x = synth.random_walk(30_000, 3)
    qq, _ = synth.noisy_copy(x, 64, 4, 5, noise=0.4)
    wi, wd = oracle.search_cascade(x, qq, 6, 5)
    for _, gi, gd in res:
        assert gi == wi.tolist()
        np.testing.assert_array_equal(gd, wd)


def _failing_worker(rank, world, port, out_q):
    dist = _init(rank, world, port, timeout_s=5)
    if rank == 1:
        # this rank fails between steps, before its part of the exchange
        out_q.put((rank, "raised"))
        raise SystemExit(3)
    import torch
    try:
        t = torch.zeros(2)
        parts = [torch.zeros(2) for _ in range(world)]
        dist.all_gather(parts, t)
        out_q.put((rank, "completed"))
    except Exception as e:  # the collective must end with an error
        out_q.put((rank, f"error: {type(e).__name__}"))


def test_failed_rank_surfaces_as_error_not_hang():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert got[1] == "raised"
    assert got[0].startswith("error"), got[0]
    assert procs[1].exitcode == 3


def test_fragments_cover_every_window_once():
    for n, m, F in ((1000, 10, 3), (5000, 128, 7), (64, 64, 1)):
        N = n - m + 1
        seen = np.zeros(N, int)
        for k in range(F):
            first, length = shard.fragment(N, F, k)
            seen[first:first + length] += 1
            lo, hi = shard.fragment_samples(n, m, F, k)
            assert hi - lo == length + m - 1 and hi <= n
        assert np.all(seen == 1)
    with pytest.raises(ValueError):
        shard.fragment(3, 4, 0)
