"""dtws_dtw_at_noalloc: the allocation-free DTW entry point, for callers that
cannot let the library allocate device memory (no cudaMalloc once running,
device memory owned by a host framework's pool, fixed-footprint
deployments).  Called through the C ABI on device arrays and checked against
the existing entry point dtws_dtw_at on two calls in a row (the second with a
different query length, band and offsets, since both calls share the
library's fixed scratch).  Collected last so a failure here comes after
every other test."""
import ctypes

import numpy as np
import pytest

from paper_1812_10302_gb300 import dtws, synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_dtw_at_on_two_calls():
    import torch
    lib = dtws.load(build_if_missing=True)
    x = synth.random_walk(40_007, 23)
    xd = torch.from_numpy(x).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    with dtws.Index(x) as ix:
        for call, (m, r, seed) in enumerate(((300, 30, 1), (97, 5, 2))):
            q, _ = synth.noisy_copy(x, m, 50 + seed, 60 + seed, noise=0.3)
            offs = np.random.default_rng(seed).integers(0, x.size - m + 1, 500).astype(np.int64)
            want = ix.dtw_at(q, r, offs)
            qd = torch.from_numpy(q).cuda()
            od = torch.from_numpy(offs).cuda()
            out = torch.full((offs.size,), -1.0, dtype=torch.float32, device="cuda")
            st = lib.dtws_dtw_at_noalloc(xd.data_ptr(), x.size, qd.data_ptr(), m, r, od.data_ptr(),
                                         offs.size, out.data_ptr(), ctypes.c_void_p(stream))
            assert st == dtws.DTWS_OK, (call, dtws.strerror(st))
            got = out.cpu().numpy()
            np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-6 * m, err_msg=f"call {call}")


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
