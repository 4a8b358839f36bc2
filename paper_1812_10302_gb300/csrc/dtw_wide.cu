// dtw_wide.cu -- the FP32 DTW for bands past the one-warp walks
// (kDiagRMax < r <= kWideRMax): k_dtw_mw, four warps per candidate, in the
// seed, survivor and given-offset modes.
#include "dtw_kernels.cuh"

namespace dtws {

namespace {

template <int K, int MODE>
cudaError_t wide_launch_k(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets, int64_t count, float *out,
                          int64_t count_for_grid, cudaStream_t s) {
    constexpr int W = kWideW;
    const size_t span = wide_span(a.m, a.r, K), tailn = wide_tail(a.m);
    const size_t hard = (size_t)200 * 1024;
    int groups = 8 / W;
    auto bytes = [&](int gr) { return (span + (size_t)gr * (span + tailn)) * 4; };
    while (groups > 1 && bytes(groups) > hard) --groups;
    if (bytes(groups) > hard) return cudaErrorInvalidValue;
    const size_t smem = bytes(groups);
    int64_t want = (count_for_grid + groups - 1) / groups;
    const int64_t cap = (int64_t)b.num_sms * 2;
    if (want < 1) want = 1;
    const int blocks = (int)(want < cap ? want : cap);
    cudaError_t e = cudaFuncSetAttribute(k_dtw_mw<W, K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_dtw_mw<W, K, MODE><<<blocks, groups * W * 32, smem, s>>>(b, a, offsets, count, out);
    return cudaGetLastError();
}

}  // namespace

template <int MODE>
cudaError_t dtw_wide_launch(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets, int64_t count,
                            float *out, int64_t count_for_grid, cudaStream_t s) {
    if (a.r <= kDiagRMax || a.r > kWideRMax) return cudaErrorInvalidValue;
    switch (wide_k(a.r)) {
    case 6: return wide_launch_k<6, MODE>(b, a, offsets, count, out, count_for_grid, s);
    case 8: return wide_launch_k<8, MODE>(b, a, offsets, count, out, count_for_grid, s);
    case 12: return wide_launch_k<12, MODE>(b, a, offsets, count, out, count_for_grid, s);
    default: return wide_launch_k<16, MODE>(b, a, offsets, count, out, count_for_grid, s);
    }
}

template cudaError_t dtw_wide_launch<kModeSeed>(const QueryBufs &, const QueryArgs &, const int64_t *, int64_t,
                                                float *, int64_t, cudaStream_t);
template cudaError_t dtw_wide_launch<kModeSurv>(const QueryBufs &, const QueryArgs &, const int64_t *, int64_t,
                                                float *, int64_t, cudaStream_t);
template cudaError_t dtw_wide_launch<kModeOut>(const QueryBufs &, const QueryArgs &, const int64_t *, int64_t,
                                               float *, int64_t, cudaStream_t);

}  // namespace dtws
