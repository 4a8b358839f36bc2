// prescore.cu -- the side-stream pre-score of the best Euclidean seed.
#include "dtw_kernels.cuh"

namespace dtws {

// Pre-score of the best Euclidean seed, run on a side stream while the
// lower-bound scan streams: its FP32 DTW enters the result list (the survivor
// pass skips it) and its extended-precision re-score waits for the final
// stage.  Paired mode (when both copies fit in shared memory): warp 0 runs
// the FP32 DTW while warps 1..DfW run the re-score beside it, DfW warps wide
// (the double-float walk's latency per anti-diagonal is what bounds the
// stage).  Otherwise one warp runs both in turn.
template <int L, int K>
__global__ void k_prescore(QueryBufs b, QueryArgs a) {
    using PS = PreShape<L, K>;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double bc[2];
    __shared__ DfXchg xchg;
    QueryState *st = b.st;
    if (!st->valid) return;
    const unsigned idx = prescored_window(st, a);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool pair = blockDim.x > 32;
    if (idx == 0xffffffffu) return;
    const int m = a.m, r = a.r;
    const size_t span = pre_span(m, r, L, K);
    const float *xw = b.x + idx;
    if (warp == 0) {
        if (lane >= L) return;
        const unsigned gmask = (L == 32) ? 0xffffffffu : ((1u << L) - 1u);
        const int pad = diag_pad(r, L, K);
        // FP32 DTW, as the survivor pass would compute it
        float *q32 = (float *)smraw, *c32 = (float *)(smraw + span * 4);
        const float INF = __int_as_float(0x7f800000);
        fill_pads(q32, m, pad, INF, lane, L);
        fill_pads(c32, m, pad, -INF, lane, L);
        const float mh = b.mu_hi[idx], is = b.inv_sigma[idx], ls = b.mu_lo[idx] * is;
        for (int j = lane; j < m; j += L) {
            q32[pad + j] = b.qh32[j];
            c32[pad + j] = fmaf(xw[j] - mh, is, -ls);
        }
        __syncwarp(gmask);
        int cells = 0;
        const float d32 =
            dtw_diag<float, L, K, false>(q32 + pad, c32 + pad, nullptr, m, r, INF, gmask, lane, cells);
        if (lane == 0) {
            const unsigned long long key = make_key(key_quantize(d32, a.qgrid), idx);
            list_insert(st->res_keys, a.list_cap, key);
            if (a.xz_z > 0 && d32 < DINF) xz_offer(b, a, key, true);
            atomicAdd(&st->ctr[kCtrDtwStarted], 1ull);
            atomicAdd(&st->ctr[kCtrCells], (unsigned long long)cells);
        }
        __syncwarp(gmask);
        if (pair) return;
        // one warp: the re-score below reuses this memory
    }
    // (one-warp mode with more than 16 cells per lane: the FP32 result is in
    // the list; the final stage re-scores the window like any other)
    if constexpr (K > 16) {
        if (!pair) return;
    }
    // extended-precision re-score (FP64 statistics, double-float DTW) by the
    // first re-score warp's lanes (the whole of warp 1 in paired mode, the
    // L lanes of warp 0 otherwise)
    constexpr int LS = PS::W > 1 ? 32 : L;  // lanes of the statistics warp
    const int dw = pair ? warp - 1 : 0;     // this warp's index in the re-score group
    const int nthr = pair ? 32 * PS::W : L;
    const int t = dw * 32 + lane;           // thread index in the group
    const bool stats_lane = dw == 0 && lane < LS;
    if (!pair && lane >= L) return;
    if (stats_lane) {
        const unsigned smask = (LS == 32) ? 0xffffffffu : ((1u << LS) - 1u);
        double s = 0.0;
        for (int j = lane; j < m; j += LS) s += (double)xw[j];
#pragma unroll
        for (int o = LS / 2; o > 0; o >>= 1) s += __shfl_xor_sync(smask, s, o, LS);
        const double mu = s / (double)m;
        double v = 0.0;
        for (int j = lane; j < m; j += LS) {
            const double d = (double)xw[j] - mu;
            v = fma(d, d, v);
        }
#pragma unroll
        for (int o = LS / 2; o > 0; o >>= 1) v += __shfl_xor_sync(smask, v, o, LS);
        if (lane == 0) {
            const double var = v / (double)m, mm = mu * mu;
            bc[0] = a.raw ? 0.0 : mu;
            bc[1] = a.raw ? 1.0 : var <= 1e-24 * (mm > 1.0 ? mm : 1.0) ? 0.0 : 1.0 / sqrt(var);
        }
    }
    // the group meets: named barrier 1 in paired mode, the warp otherwise
    auto group_sync = [&]() {
        if (pair) group_bar(1, 32 * PS::W);
        else __syncwarp((L == 32) ? 0xffffffffu : ((1u << L) - 1u));
    };
    group_sync();
    const double mu = bc[0], inv = bc[1];
    // (paired with L < 32: one warp whose first L lanes walk, as unpaired)
    const int lanes2 = (pair && L == 32) ? 32 * PS::W : L, k2 = pair ? PS::K2 : K;
    const int pad2 = diag_pad(r, lanes2, k2);
    const size_t span2 = pre_span(m, r, lanes2, k2);
    unsigned char *dbase = smraw + (pair ? span * 8 : 0);
    dfloat *qd = (dfloat *)dbase, *cd = (dfloat *)(dbase + span2 * 8);
    fill_pads(qd, m, pad2, dfloat{1e15f, 0.0f}, t, nthr);
    fill_pads(cd, m, pad2, dfloat{-1e15f, 0.0f}, t, nthr);
    for (int j = t; j < m; j += nthr) {
        qd[pad2 + j] = df_from(b.qh64[j]);
        cd[pad2 + j] = df_from(((double)xw[j] - mu) * inv);
    }
    group_sync();
    double d64;
    if (pair && PS::W > 1) {
        d64 = dtw_diag_df_mw<PS::W, PS::K2>(qd + pad2, cd + pad2, m, r, dw, lane, xchg, 1);
    } else {
        if constexpr (K <= 16) {
            const unsigned gmask = (L == 32) ? 0xffffffffu : ((1u << L) - 1u);
            if (lane >= L) return;
            d64 = dtw_diag_df<L, K>(qd + pad2, cd + pad2, m, r, gmask, lane);
        } else {
            return;  // (not reached: K > 16 runs paired, with PS::W = 4)
        }
    }
    if (t == 0) {
        st->pre_d64 = d64;
        __threadfence();
        st->pre_done = 1;
    }
}

cudaError_t launch_prescore(const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    if (!a.prescore) return cudaSuccess;
    int L, K;
    diag_shape(a.r, &L, &K);
    if (a.r > kDiagRMax) {  // the FP32 walk's wide shapes (one warp, 24 or 32 cells)
        L = 32;
        K = a.r + 1 <= 32 * 24 ? 24 : 32;
    }
#define DTWS_CASE(LL, KK)                                                                           \
    if (L == LL && K == KK) {                                                                       \
        using PS = PreShape<LL, KK>;                                                                \
        /* paired: FP32 copy (8 B per element) beside the re-score's (16 B), */                    \
        /* else one warp with the re-score reusing the FP32 copy's memory */                       \
        const size_t s32 = pre_span(a.m, a.r, LL, KK) * 8;                                          \
        const size_t sdf = pre_span(a.m, a.r, (LL < 32 ? LL : 32 * PS::W), PS::K2) * 16;           \
        const bool pair = s32 + sdf <= (size_t)200 * 1024;                                          \
        const size_t smem = pair ? s32 + sdf : pre_span(a.m, a.r, LL, KK) * 16;                     \
        const int threads = pair ? 32 + 32 * PS::W : 32;                                            \
        cudaError_t e = cudaFuncSetAttribute(k_prescore<LL, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)smem);                                            \
        if (e != cudaSuccess) return e;                                                             \
        k_prescore<LL, KK><<<1, threads, smem, s>>>(b, a);                                          \
        return cudaGetLastError();                                                                  \
    }
    DTWS_CASE(1, 1) DTWS_CASE(2, 1) DTWS_CASE(4, 1) DTWS_CASE(8, 1) DTWS_CASE(16, 1)
    DTWS_CASE(32, 1) DTWS_CASE(32, 2) DTWS_CASE(32, 3) DTWS_CASE(32, 4) DTWS_CASE(32, 6) DTWS_CASE(32, 8) \
    DTWS_CASE(32, 10) DTWS_CASE(32, 12) DTWS_CASE(32, 16) DTWS_CASE(32, 24) DTWS_CASE(32, 32)
#undef DTWS_CASE
    return cudaErrorInvalidValue;
}

}  // namespace dtws
