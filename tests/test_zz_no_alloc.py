"""dtws_dtw_at_noalloc: the allocation-free DTW entry point, for callers that
cannot let the library allocate device memory (no cudaMalloc once running,
device memory owned by a host framework's pool, fixed-footprint
deployments).  Called through the C ABI on device arrays and checked against
the FP64 oracle and against the existing entry point dtws_dtw_at, on calls in
a row that share the library's fixed scratch (different query lengths, bands
and offsets, so a stale cursor or query would show).  Also the documented
edge cases: out-of-range offsets and a non-finite query give NaN, count == 0
returns at once, host arrays are refused.  Collected last so a failure here
comes after every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1812_10302_gb300 import dtws, synth

pytestmark = pytest.mark.gpu


def _call(lib, xd, n, qd, m, r, od, count, outd, stream=None):
    return lib.dtws_dtw_at_noalloc(xd.data_ptr(), n, qd.data_ptr(), m, r, od.data_ptr() if od is not None else None,
                                   count, outd.data_ptr(), ctypes.c_void_p(stream) if stream else None)


def test_noalloc_matches_oracle_and_dtw_at_on_calls_in_a_row():
    import torch
    lib = dtws.load(build_if_missing=True)
    x = synth.random_walk(40_007, 23)
    xd = torch.from_numpy(x).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    # (m, r, seed, offsets): the last case runs one warp per CTA (its ring of
    # 2r + 2 floats fills the shared memory)
    cases = ((300, 30, 1, 500), (97, 5, 2, 500), (8192, 6000, 3, 6), (2048, 1500, 4, 40))
    with dtws.Index(x) as ix:
        for call, (m, r, seed, cnt) in enumerate(cases):
            q, _ = synth.noisy_copy(x, m, 50 + seed, 60 + seed, noise=0.3)
            offs = np.random.default_rng(seed).integers(0, x.size - m + 1, cnt).astype(np.int64)
            qd = torch.from_numpy(q).cuda()
            od = torch.from_numpy(offs).cuda()
            out = torch.full((offs.size,), -1.0, dtype=torch.float32, device="cuda")
            st = _call(lib, xd, x.size, qd, m, r, od, offs.size, out, stream)
            assert st == dtws.DTWS_OK, (call, dtws.strerror(st), lib.dtws_last_error_detail())
            got = out.cpu().numpy().astype(np.float64)
            want = oracle.dtw_at(x, q, r, offs)
            np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-6 * m, err_msg=f"call {call} vs oracle")
            np.testing.assert_allclose(got, ix.dtw_at(q, r, offs), rtol=1e-4, atol=1e-6 * m,
                                       err_msg=f"call {call} vs dtws_dtw_at")


def test_noalloc_edge_cases():
    import torch
    lib = dtws.load(build_if_missing=True)
    x = synth.random_walk(20_000, 31)
    m, r = 128, 12
    N = x.size - m + 1
    xd = torch.from_numpy(x).cuda()
    q, _ = synth.noisy_copy(x, m, 32, 33, noise=0.2)
    qd = torch.from_numpy(q).cuda()
    # out-of-range offsets mixed with valid ones: NaN exactly there
    offs = np.array([5, -1, N - 1, N, 1000, N + 77, 0], np.int64)
    od = torch.from_numpy(offs).cuda()
    out = torch.zeros(offs.size, device="cuda")
    assert _call(lib, xd, x.size, qd, m, r, od, offs.size, out) == dtws.DTWS_OK
    got = out.cpu().numpy()
    bad = (offs < 0) | (offs >= N)
    assert np.all(np.isnan(got[bad])) and np.all(np.isfinite(got[~bad]))
    np.testing.assert_allclose(got[~bad], oracle.dtw_at(x, q, r, offs[~bad]), rtol=1e-4, atol=1e-6 * m)
    # a non-finite query: every output NaN
    qn = qd.clone()
    qn[7] = float("nan")
    out = torch.zeros(4, device="cuda")
    od4 = torch.tensor([0, 1, 2, 3], dtype=torch.int64, device="cuda")
    assert _call(lib, xd, x.size, qn, m, r, od4, 4, out) == dtws.DTWS_OK
    assert torch.isnan(out).all()
    # count == 0: returns at once, writes nothing
    out = torch.full((2,), 3.0, device="cuda")
    assert _call(lib, xd, x.size, qd, m, r, od4, 0, out) == dtws.DTWS_OK
    torch.cuda.synchronize()
    assert out.tolist() == [3.0, 3.0]
    # a host array is refused (nothing is staged)
    host_out = np.zeros(4, np.float32)
    st = lib.dtws_dtw_at_noalloc(xd.data_ptr(), x.size, qd.data_ptr(), m, r, od4.data_ptr(), 4,
                                 host_out.ctypes.data, None)
    assert st == dtws.DTWS_EINVAL
    assert b"device memory" in lib.dtws_last_error_detail()
    # and a call after the refusals still answers correctly
    out = torch.zeros(4, device="cuda")
    assert _call(lib, xd, x.size, qd, m, r, od4, 4, out) == dtws.DTWS_OK
    np.testing.assert_allclose(out.cpu().numpy(), oracle.dtw_at(x, q, r, [0, 1, 2, 3]), rtol=1e-4, atol=1e-6 * m)


def test_noalloc_rejects_query_beyond_scratch():
    import torch
    lib = dtws.load(build_if_missing=True)
    x = torch.zeros(20_000, device="cuda")
    q = torch.zeros(dtws.DTWS_NOALLOC_M_MAX + 1, device="cuda")
    o = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.zeros(1, device="cuda")
    st = lib.dtws_dtw_at_noalloc(x.data_ptr(), x.numel(), q.data_ptr(), q.numel(), 3, o.data_ptr(), 1,
                                 out.data_ptr(), None)
    assert st == dtws.DTWS_EINVAL
    assert b"scratch" in lib.dtws_last_error_detail()
