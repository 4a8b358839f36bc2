// dtw_out.cu -- FP32 banded DTW at given offsets (dtws_dtw_at and the
// autotuner's timed shapes): the k_dtw kernel in output mode, no pruning.
#include "dtw_kernels.cuh"

namespace dtws {

namespace {
__global__ void k_reset_cursor(QueryState *st) { st->work = 0; }
}  // namespace

cudaError_t launch_dtw_at(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                          int64_t count, float *out, cudaStream_t s) {
    k_reset_cursor<<<1, 1, 0, s>>>(b.st);
    return dtw_dispatch<kModeOut>(b, a, offsets, count, out, count, s);
}

bool dtw_default_shape(int m, int r, int *L, int *K, int *warps) {
    DtwPlan p;
    if (r > kDiagRMax || !plan_dtw<float>(m, r, false, &p)) return false;
    *L = p.L;
    *K = p.K;
    *warps = p.warps;
    return true;
}

bool dtw_shape_valid(int m, int r, int L, int K, int warps) {
    DtwPlan p;
    return plan_shape<float>(m, r, true, L, K, warps, &p) && plan_shape<float>(m, r, false, L, K, warps, &p);
}

cudaError_t launch_dtw_at_shape(const QueryBufs &b, QueryArgs a, const int64_t *offsets, int64_t count, float *out,
                                int L, int K, int warps, cudaStream_t s) {
    a.tune_l = L;
    a.tune_k = K;
    a.tune_w = warps;
    k_reset_cursor<<<1, 1, 0, s>>>(b.st);
    return dtw_dispatch<kModeOut>(b, a, offsets, count, out, count, s);
}

}  // namespace dtws
