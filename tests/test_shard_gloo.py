"""Multi-process fragment sharding (Sec. 3.1, Eq. 11) and the merge of the
per-fragment best pairs, with the gloo backend, world size 2.  On CPU the
per-rank search engine is the FP64 oracle (the host logic under test is the
partition and the exchange); the GPU variant runs the library on each rank.
A rank that fails must make the other's collective end with an error instead
of hanging."""
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


def _seam_case(world, k):
    """A series whose best matches straddle the seam between fragments 0 and
    1: the query is a noisy copy of the window that starts one sample before
    the seam, so its neighbours (the rest of the top-k) fall on both sides."""
    x = synth.random_walk(30_000, 3)
    m, r = 64, 6
    seam, _ = shard.fragment(x.size - m + 1, world, 1)
    rng = np.random.default_rng(5)
    q = (x[seam - 1:seam - 1 + m] + rng.normal(0, 0.05, m)).astype(np.float32)
    return x, q, m, r, k


def _worker(rank, world, port, out_q, k, engine):
    dist = _init(rank, world, port)
    x, q, m, r, k = _seam_case(world, k)
    lo, hi = shard.fragment_samples(x.size, m, world, rank)
    if engine == "oracle":
        idx, d = oracle.search_cascade(x[lo:hi], q, r, k)
    else:  # the library on this rank's GPU (both ranks share cuda:0 here)
        from paper_1812_10302_gb300 import dtws
        with dtws.Index(x[lo:hi]) as ix:
            idx, d = ix.query(q, r, k)
            assert ix.sync_status() == dtws.DTWS_OK
    gi, gd = shard.allgather_merge(idx, d, k, offset=lo)
    out_q.put((rank, gi.tolist(), gd.tolist(), [int(v) + lo for v in idx]))
    dist.barrier()
    dist.destroy_process_group()


def _run_two_ranks(k, engine):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, k, engine)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("k", [5, 10])
def test_two_ranks_merge_equals_single_pass(k):
    res = _run_two_ranks(k, "oracle")
    x, qq, m, r, k = _seam_case(2, k)
    wi, wd = oracle.search_cascade(x, qq, r, k)
    seam, _ = shard.fragment(x.size - m + 1, 2, 1)
    assert wi.min() < seam <= wi.max()  # the answer spans both fragments
    for _, gi, gd, _ in res:
        assert gi == wi.tolist()
        np.testing.assert_array_equal(gd, wd)


def test_merge_orders_ties_across_a_seam():
    """Per-rank lists with equal distances on both sides of a seam: the merge
    keeps the k smallest (distance, offset) pairs, ties to the lower global
    offset, and drops missing (-1) entries."""
    # rank 0 holds windows [0, 100), rank 1 [100, 200) (local offsets + 100)
    r0 = ([98, 99, 40, -1], [0.5, 0.25, 0.25, np.inf])
    r1 = ([0, 1, 60, 2], [0.25, 0.5, 0.125, 0.25])
    gi, gd = shard.merge_topk([r0[0], [v + 100 for v in r1[0]]], [r0[1], r1[1]], 6)
    assert gi.tolist() == [160, 40, 99, 100, 102, 98]
    assert gd.tolist() == [0.125, 0.25, 0.25, 0.25, 0.25, 0.5]
    gi, gd = shard.merge_topk([r0[0]], [r0[1]], 5)
    assert gi.tolist() == [40, 99, 98, -1, -1] and gd[-1] == np.inf


@pytest.mark.gpu
def test_two_ranks_with_the_library_as_engine():
    """The same exchange with libdtws as each rank's search engine (two
    processes on one GPU: their kernels never wait on one another, the
    exchange runs on the host over gloo), k = 10 across the seam."""
    res = _run_two_ranks(10, "dtws")
    x, qq, m, r, k = _seam_case(2, 10)
    wi, wd = oracle.search_cascade(x, qq, r, k)
    for _, gi, gd, _ in res:
        assert gi == wi.tolist()
        np.testing.assert_allclose(gd, wd, rtol=1e-4, atol=1e-6 * m)


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
