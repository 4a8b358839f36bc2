// query_kernels.cu -- per-query kernels of the search (arxiv 1812.10302):
//
//   k_query_reset   clear the device query state
//   k_qprep         z-normalise Q (Sec. 2.2, Eq. 5; FP64 two-pass), its
//                   envelope (Eq. 9) and the order of |q_hat| (largest first)
//   k_seed_scan     proxy scan: per tile, the window with the smallest partial
//                   squared distance on the largest-|q_hat| positions
//   k_seed_gather   seed offsets = seeded random windows (the paper's random
//                   first bsf, Algorithm 1) + the proxy proposals
//   k_dtw<SEED>     DTW of the seeds -> k-th seed distance = first bsf
//   k_lb_scan       fused cascade per tile (Sec. 2.2, Eqs. 6-10): LB_KimFL,
//                   LB_Keogh vs the query envelope, LB_Keogh vs the series
//                   envelope, with in-CTA compaction between the stages
//   k_bin_*         order the survivors by lower bound (counting sort)
//   k_dtw<SURV>     banded DTW (Eq. 1 + band) of the survivors in that order,
//                   early abandon, lock-free top-k list
//   k_final_*       FP64 re-score of the top-k and its near-ties, output
//
// Pruning (Eq. 6, strict): a window is dropped when a lower bound exceeds
// thr = bsf*(1+delta) + alpha, bsf being the k-th best distance found so far.
// delta and alpha absorb FP32 rounding so no true top-k window is dropped.
#include <cmath>

#include "dtw_band.cuh"
#include "dtws_internal.h"

namespace dtws {

#define DINF __int_as_float(0x7f800000)

// ------------------------------------------------------------------ reset
__global__ void k_query_reset(QueryState *st) {
    for (int t = threadIdx.x; t < kListMax; t += blockDim.x) st->res_keys[t] = kEmptyKey;
    for (int t = threadIdx.x; t < kKMax; t += blockDim.x) st->seed_keys[t] = kEmptyKey;
    for (int t = threadIdx.x; t < kPropMax; t += blockDim.x) st->prop_keys[t] = kEmptyKey;
    for (int t = threadIdx.x; t < kBins; t += blockDim.x) st->hist[t] = 0;
    for (int t = threadIdx.x; t < kCtrN; t += blockDim.x) st->ctr[t] = 0;
    if (threadIdx.x == 0) {
        st->n_seeds = 0;
        st->n_cand = 0;
        st->work = 0;
        st->work2 = 0;
        st->n_margin = 0;
        st->thr_scan = DINF;
        st->valid = 1;
    }
}

cudaError_t launch_query_reset(const QueryBufs &b, const QueryArgs &, cudaStream_t s) {
    k_query_reset<<<1, 1024, 0, s>>>(b.st);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ block reductions
template <typename T>
__device__ T block_sum(T v, T *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane_id() == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    for (int i = 0; i < nw; ++i) s += red[i];
    return s;
}

// ------------------------------------------------------------------ query prep
// One CTA of 1024 threads.  Dynamic smem: q_hat FP32 [m] + sort keys u64 [P],
// P = next power of two >= m.
__global__ void __launch_bounds__(1024) k_qprep(const float *__restrict__ Q, QueryBufs b, QueryArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[32];
    __shared__ int bad;
    const int m = a.m, r = a.r;
    int P = 1;
    while (P < m) P <<= 1;
    unsigned long long *keys = (unsigned long long *)smraw;
    float *qs = (float *)(keys + P);

    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    bool nf = false;
    for (int j = threadIdx.x; j < m; j += blockDim.x) nf |= !isfinite(Q[j]);
    if (nf) atomicOr(&bad, 1);
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) {
            b.st->valid = 0;
            atomicOr(b.status, kStNonFinite);
        }
        return;
    }
    // Eq. 5, two-pass in FP64: mu, then sum (x - mu)^2 / m (population)
    double s = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) s += (double)Q[j];
    const double mu = block_sum(s, red) / (double)m;
    double v = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double d = (double)Q[j] - mu;
        v = fma(d, d, v);
    }
    const double var = block_sum(v, red) / (double)m;
    const double mm = mu * mu;
    const bool zero = var <= 1e-24 * (mm > 1.0 ? mm : 1.0);
    const double sg = zero ? 0.0 : sqrt(var);
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double qh = zero ? 0.0 : ((double)Q[j] - mu) / sg;
        b.qh64[j] = qh;
        qs[j] = (float)qh;
    }
    __syncthreads();
    // envelope of q_hat, half-width r, clipped (Eq. 9)
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        int lo = j - r > 0 ? j - r : 0, hi = j + r < m - 1 ? j + r : m - 1;
        float u = qs[lo], l = qs[lo];
        for (int t = lo + 1; t <= hi; ++t) {
            u = fmaxf(u, qs[t]);
            l = fminf(l, qs[t]);
        }
        b.Uq[j] = u;
        b.Lq[j] = l;
        b.qh32[j] = qs[j];
    }
    // order by |q_hat| descending, ties by position ascending: bitonic sort of
    // (|q| bits << 32 | ~j) descending; padding keys sort last
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        unsigned kb = j < m ? __float_as_uint(fabsf(qs[j])) : 0u;
        keys[j] = ((unsigned long long)kb << 32) | (unsigned)(0xffffffffu - (unsigned)j);
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                int lo = 2 * t - (t & (stride - 1));
                int hi = lo + stride;
                bool desc = ((lo & size) == 0);
                unsigned long long x0 = keys[lo], x1 = keys[hi];
                if ((x0 < x1) == desc) {
                    keys[lo] = x1;
                    keys[hi] = x0;
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        int j = (int)(0xffffffffu - (unsigned)(keys[t] & 0xffffffffu));
        b.ord[t] = (unsigned short)j;
        b.sq[t] = qs[j];
        b.sU[t] = b.Uq[j];
        b.sL[t] = b.Lq[j];
    }
}

cudaError_t launch_qprep(const float *Q, const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    int P = 1;
    while (P < a.m) P <<= 1;
    size_t smem = (size_t)P * 8 + (size_t)a.m * 4;
    cudaError_t e = cudaFuncSetAttribute(k_qprep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_qprep<<<1, 1024, smem, s>>>(Q, b, a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ tile staging
// A tile is kTile consecutive windows [i0, i0 + kTile).  Its samples
// x[i0, i0 + kTile + m - 1) and its window statistics are staged in shared
// memory by 1-D bulk copies (the TMA engine) on one mbarrier.  The padded
// series and the statistics arrays are allocated so that every full tile is
// in bounds (the library rounds both up to whole tiles plus kMMax).
struct Tile {
    float *xs, *mh, *ml, *is;
    uint64_t *bar;
};

__device__ __forceinline__ unsigned tile_x_floats(int m) { return (unsigned)((kTile + m - 1 + 3) & ~3); }

__device__ __forceinline__ Tile carve_tile(unsigned char *sm, int m) {
    Tile t;
    t.bar = (uint64_t *)sm;
    t.mh = (float *)(sm + 16);
    t.ml = t.mh + kTile;
    t.is = t.ml + kTile;
    t.xs = t.is + kTile;
    return t;
}

// Returns false (and records a timeout) if the copies did not land in time.
__device__ bool stage_tile(const Tile &t, const QueryBufs &b, int64_t i0, int m) {
    const unsigned xb = tile_x_floats(m) * 4u;
    if (threadIdx.x == 0) {
        mbar_init(t.bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(t.bar, xb + 3u * kTile * 4u);
        bulk_g2s(t.xs, b.x + i0, xb, t.bar);
        bulk_g2s(t.mh, b.mu_hi + i0, kTile * 4u, t.bar);
        bulk_g2s(t.ml, b.mu_lo + i0, kTile * 4u, t.bar);
        bulk_g2s(t.is, b.inv_sigma + i0, kTile * 4u, t.bar);
    }
    bool ok = mbar_wait_bounded(t.bar, 0, b.wait_ns);
    if (!ok) {
        atomicOr(b.status, kStTimeout);
        // give the copies in flight one more bounded chance before leaving
        mbar_wait_bounded(t.bar, 0, b.wait_ns);
    }
    return __syncthreads_and(ok) != 0;
}

__host__ __device__ inline size_t tile_smem_bytes(int m) {
    return 16 + (size_t)3 * kTile * 4 + (size_t)(((kTile + m - 1 + 3) & ~3)) * 4;
}

// ------------------------------------------------------------------ proxy scan
// Per window: the squared distance on the `terms` query positions of largest
// |q_hat| (not a lower bound: it only proposes windows whose exact DTW seeds
// the best-so-far).  Each tile proposes its best window.
__global__ void __launch_bounds__(256) k_seed_scan(QueryBufs b, QueryArgs a, int proposals, int terms) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ unsigned long long wbest[8];
    if (!b.st->valid) return;
    const int m = a.m;
    Tile t = carve_tile(smraw, m);
    const int64_t i0 = (int64_t)blockIdx.x * kTile;
    if (!stage_tile(t, b, i0, m)) return;
    int pos[16];
    float qv[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        pos[u] = u < terms ? (int)b.ord[u] : 0;
        qv[u] = u < terms ? b.sq[u] : 0.0f;
    }
    unsigned long long best = kEmptyKey;
    for (int w = threadIdx.x; w < kTile; w += blockDim.x) {
        int64_t i = i0 + w;
        if (i >= a.N) break;
        float mh = t.mh[w], is = t.is[w], ls = t.ml[w] * is;
        float acc = 0.0f;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            if (u < terms) {
                float c = qv[u] - fmaf(t.xs[w + pos[u]] - mh, is, -ls);
                acc = fmaf(c, c, acc);
            }
        }
        unsigned long long key = make_key(acc, (unsigned)i);
        best = key < best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v < best ? v : best;
    }
    if (lane_id() == 0) wbest[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = wbest[w] < best ? wbest[w] : best;
        if (best != kEmptyKey) {
            unsigned long long last = *((volatile unsigned long long *)&b.st->prop_keys[proposals - 1]);
            if (best < last) list_insert(b.st->prop_keys, proposals, best);
        }
    }
}

cudaError_t launch_seed_scan(const QueryBufs &b, const QueryArgs &a, int proposals, int terms,
                             cudaStream_t s) {
    if (proposals <= 0) return cudaSuccess;
    size_t smem = tile_smem_bytes(a.m);
    cudaError_t e = cudaFuncSetAttribute(k_seed_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t tiles = (a.N + kTile - 1) / kTile;
    int t = terms > 16 ? 16 : terms;
    t = t > a.m ? a.m : t;  // positions are taken from the query's order
    k_seed_scan<<<(unsigned)tiles, 256, smem, s>>>(b, a, proposals, t);
    return cudaGetLastError();
}

// splitmix64 (Steele, Lea & Flood, 2014) as the counter-based generator of
// the random seed windows.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_seed_gather(QueryBufs b, QueryArgs a, int n_random, int proposals,
                              unsigned long long rng) {
    if (threadIdx.x != 0 || !b.st->valid) return;
    // distinct offsets only: a repeated seed would fill two of the k seed
    // slots with one window and understate the k-th seed distance
    int n = 0;
    auto add = [&](unsigned o) {
        for (int t = 0; t < n; ++t)
            if (b.st->seed_off[t] == o) return;
        if (n < kSeedMax) b.st->seed_off[n++] = o;
    };
    for (int j = 0; j < n_random; ++j)
        add((unsigned)(splitmix64(rng + (unsigned long long)j) % (unsigned long long)a.N));
    for (int p = 0; p < proposals; ++p) {
        unsigned long long key = b.st->prop_keys[p];
        if (key != kEmptyKey) add(key_idx(key));
    }
    b.st->n_seeds = n;
    b.st->work = 0;
}

cudaError_t launch_seed_gather(const QueryBufs &b, const QueryArgs &a, int n_random, int proposals,
                               unsigned long long rng, cudaStream_t s) {
    k_seed_gather<<<1, 32, 0, s>>>(b, a, n_random, proposals, rng);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ DTW kernels
enum DtwMode { kModeSeed = 0, kModeSurv = 1, kModeOut = 2 };

// FP32 DTW over a candidate list.  Groups of L lanes pull candidates from a
// device cursor.  Shared memory: q_hat [m] + one ring of W+1 per group.
template <int L, int MODE>
__global__ void __launch_bounds__(256) k_dtw(QueryBufs b, QueryArgs a, const int64_t *offsets,
                                             int64_t count_host, float *out) {
    extern __shared__ __align__(16) unsigned char smraw[];
    QueryState *st = b.st;
    if (!st->valid) return;
    const int m = a.m, r = a.r, W = 2 * r + 1;
    float *qs = (float *)smraw;
    for (int t = threadIdx.x; t < m; t += blockDim.x) qs[t] = b.qh32[t];
    __syncthreads();
    const int warp = threadIdx.x >> 5, ln = lane_id();
    const int g = ln / L, lane = ln % L;
    const int gid = warp * (32 / L) + g;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g * L));
    float *ring = qs + ((m + 3) & ~3) + gid * (W + 1);
    int *cursor = MODE == kModeSurv ? &st->work2 : &st->work;
    const int64_t count = MODE == kModeSeed ? (int64_t)st->n_seeds
                        : MODE == kModeSurv ? (int64_t)st->n_cand : count_host;
    long long cells_acc = 0;
    int started = 0, abandoned = 0;
    while (true) {
        int c = 0;
        if (lane == 0) c = atomicAdd(cursor, 1);
        c = __shfl_sync(gmask, c, 0, L);
        if (c >= count) break;
        unsigned idx;
        float lb = 0.0f;
        if (MODE == kModeSeed) idx = st->seed_off[c];
        else if (MODE == kModeSurv) { idx = b.sort_idx[c]; lb = b.sort_lb[c]; }
        else {
            const int64_t o = offsets[c];
            if (o < 0 || o >= a.N) {  // caller's device offsets are checked here
                if (lane == 0) out[c] = __int_as_float(0x7fc00000);
                continue;
            }
            idx = (unsigned)o;
        }
        // the threshold moves while other groups insert: read it once (lane
        // 0) so every lane of the group takes the same branches
        float thr = DINF;
        if (MODE == kModeSeed) {
            float kth = list_kth(st->seed_keys, a.k);
            thr = kth < DINF ? fmaf(kth, 1.0f + a.delta, a.alpha) : DINF;
        } else if (MODE == kModeSurv) {
            thr = current_thr(st, a);
        }
        thr = __shfl_sync(gmask, thr, 0, L);
        if (MODE == kModeSurv && lb > thr) continue;
        const float mh = b.mu_hi[idx], is = b.inv_sigma[idx], ls = b.mu_lo[idx] * is;
        int cells = 0;
        float d;
        if (MODE == kModeOut) {
            d = dtw_band<float, L, false>(qs, b.x + idx, mh, is, ls, nullptr, ring, m, r, thr, gmask,
                                          lane, cells);
        } else {
            TailCtx tc;
            tc.Uw = b.U ? b.U + idx : nullptr;
            tc.Lw = b.L ? b.L + idx : nullptr;
            tc.qs = qs;
            tc.mh = mh;
            tc.is = is;
            tc.ls = ls;
            d = dtw_band<float, L, true>(qs, b.x + idx, mh, is, ls, (b.U && MODE == kModeSurv) ? &tc : nullptr,
                                         ring, m, r, thr, gmask, lane, cells);
        }
        cells_acc += cells;
        if (lane == 0) {
            ++started;
            if (!(d < DINF)) ++abandoned;
            if (MODE == kModeOut) out[c] = d;
            else if (MODE == kModeSeed) {
                if (d < DINF) list_insert(st->seed_keys, a.k, make_key(key_quantize(d, a.qgrid), idx));
            } else if (d <= thr) {
                list_insert(st->res_keys, a.list_cap, make_key(key_quantize(d, a.qgrid), idx));
            }
        }
        __syncwarp(gmask);
    }
    if (MODE != kModeOut) {
        // counters: one atomic per warp
        unsigned long long cs = (unsigned long long)cells_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
        int ns = started, na = abandoned;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ns += __shfl_xor_sync(0xffffffffu, ns, o);
            na += __shfl_xor_sync(0xffffffffu, na, o);
        }
        if (ln == 0) {
            atomicAdd(&st->ctr[kCtrCells], cs);
            atomicAdd(&st->ctr[kCtrDtwStarted], (unsigned long long)ns);
            atomicAdd(&st->ctr[kCtrDtwAbandoned], (unsigned long long)na);
        }
    }
}

// FP64 re-score: per window two-pass FP64 statistics (Eq. 5) and FP64 banded
// DTW, no pruning.  Candidates: the margin list (offsets == null) or offsets.
template <int L>
__global__ void __launch_bounds__(256) k_dtw64(QueryBufs b, QueryArgs a, const int64_t *offsets,
                                               int64_t count_host, double *out) {
    extern __shared__ __align__(16) unsigned char smraw[];
    QueryState *st = b.st;
    if (!st->valid) return;
    const int m = a.m, r = a.r, W = 2 * r + 1;
    double *qs = (double *)smraw;
    for (int t = threadIdx.x; t < m; t += blockDim.x) qs[t] = b.qh64[t];
    __syncthreads();
    const int warp = threadIdx.x >> 5, ln = lane_id();
    const int g = ln / L, lane = ln % L;
    const int gid = warp * (32 / L) + g;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g * L));
    double *ring = qs + ((m + 3) & ~3) + gid * (W + 1);
    const int64_t count = offsets ? count_host : (int64_t)st->n_margin;
    while (true) {
        int c = 0;
        if (lane == 0) c = atomicAdd(&st->work, 1);
        c = __shfl_sync(gmask, c, 0, L);
        if (c >= count) break;
        unsigned idx;
        if (offsets) {
            const int64_t o = offsets[c];
            if (o < 0 || o >= a.N) {
                if (lane == 0) out[c] = __longlong_as_double(0x7ff8000000000000ll);
                continue;
            }
            idx = (unsigned)o;
        } else {
            idx = st->margin_idx[c];
        }
        const float *xw = b.x + idx;
        double s = 0.0;
        for (int j = lane; j < m; j += L) s += (double)xw[j];
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, L);
        const double mu = s / (double)m;
        double v = 0.0;
        for (int j = lane; j < m; j += L) {
            double d = (double)xw[j] - mu;
            v = fma(d, d, v);
        }
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o, L);
        const double var = v / (double)m, mm = mu * mu;
        const bool zero = var <= 1e-24 * (mm > 1.0 ? mm : 1.0);
        const double inv = zero ? 0.0 : 1.0 / sqrt(var);
        int cells = 0;
        double d = dtw_band<double, L, false>(qs, xw, mu, inv, 0.0, nullptr, ring, m, r, tinf<double>(),
                                              gmask, lane, cells);
        if (lane == 0) {
            if (offsets) out[c] = d;
            else st->margin_d64[c] = d;
        }
        __syncwarp(gmask);
    }
}

template <typename T>
static void dtw_launch_shape(int m, int r, int L, int num_sms, int64_t count, int *blocks,
                             int *threads, size_t *smem) {
    const int W = 2 * r + 1;
    const size_t qbytes = (size_t)((m + 3) & ~3) * sizeof(T);
    const size_t per_warp = (size_t)(32 / L) * (W + 1) * sizeof(T);
    int warps = 8;
    while (warps > 1 && qbytes + warps * per_warp > 100 * 1024) --warps;
    *threads = warps * 32;
    *smem = qbytes + warps * per_warp;
    const int groups = warps * (32 / L);
    int64_t want = (count + groups - 1) / groups;
    int64_t cap = (int64_t)num_sms * 4;
    if (want < 1) want = 1;
    *blocks = (int)(want < cap ? want : cap);
}

template <int MODE>
static cudaError_t dtw_dispatch(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                                int64_t count, float *out, int64_t count_for_grid, cudaStream_t s) {
    int L = lanes_for(a.r), blocks, threads;
    size_t smem;
    dtw_launch_shape<float>(a.m, a.r, L, b.num_sms, count_for_grid, &blocks, &threads, &smem);
#define DTWS_LAUNCH(LL)                                                                             \
    {                                                                                                \
        cudaError_t e = cudaFuncSetAttribute(k_dtw<LL, MODE>,                                        \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                              \
        k_dtw<LL, MODE><<<blocks, threads, smem, s>>>(b, a, offsets, count, out);                    \
        return cudaGetLastError();                                                                   \
    }
    switch (L) {
    case 1: DTWS_LAUNCH(1)
    case 2: DTWS_LAUNCH(2)
    case 4: DTWS_LAUNCH(4)
    case 8: DTWS_LAUNCH(8)
    case 16: DTWS_LAUNCH(16)
    default: DTWS_LAUNCH(32)
    }
#undef DTWS_LAUNCH
}

static cudaError_t dtw64_dispatch(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                                  int64_t count, double *out, int64_t count_for_grid, cudaStream_t s) {
    int L = lanes_for(a.r), blocks, threads;
    size_t smem;
    dtw_launch_shape<double>(a.m, a.r, L, b.num_sms, count_for_grid, &blocks, &threads, &smem);
#define DTWS_LAUNCH(LL)                                                                             \
    {                                                                                                \
        cudaError_t e = cudaFuncSetAttribute(k_dtw64<LL>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)smem);                                             \
        if (e != cudaSuccess) return e;                                                              \
        k_dtw64<LL><<<blocks, threads, smem, s>>>(b, a, offsets, count, out);                        \
        return cudaGetLastError();                                                                   \
    }
    switch (L) {
    case 1: DTWS_LAUNCH(1)
    case 2: DTWS_LAUNCH(2)
    case 4: DTWS_LAUNCH(4)
    case 8: DTWS_LAUNCH(8)
    case 16: DTWS_LAUNCH(16)
    default: DTWS_LAUNCH(32)
    }
#undef DTWS_LAUNCH
}

cudaError_t launch_dtw_seeds(const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    return dtw_dispatch<kModeSeed>(b, a, nullptr, 0, nullptr, kSeedMax, s);
}

cudaError_t launch_dtw_survivors(const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    return dtw_dispatch<kModeSurv>(b, a, nullptr, 0, nullptr, (int64_t)b.num_sms * 1024, s);
}

__global__ void k_reset_cursor(QueryState *st) { st->work = 0; }

cudaError_t launch_dtw_at(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                          int64_t count, float *out, cudaStream_t s) {
    k_reset_cursor<<<1, 1, 0, s>>>(b.st);
    return dtw_dispatch<kModeOut>(b, a, offsets, count, out, count, s);
}

cudaError_t launch_dtw_at_f64(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                              int64_t count, double *out, cudaStream_t s) {
    k_reset_cursor<<<1, 1, 0, s>>>(b.st);
    return dtw64_dispatch(b, a, offsets, count, out, count, s);
}

// ------------------------------------------------------------------ LB scan
// Fused cascade over one tile of windows (Sec. 2.2, Eqs. 6-10, prune when a
// bound exceeds thr).  Stage 1: LB_KimFL (Eq. 7, squared) for every window;
// the survivors are compacted into a shared queue so that stage 2 keeps all
// lanes busy: LB_Keogh of the window against the query envelope (Eq. 8),
// terms taken in |q_hat|-descending order with early abandon every 8 terms.
// Stage 3 on stage 2's survivors: LB_Keogh of the query against the
// window's envelope (Eq. 10), the envelope read from the series-wide
// envelope and normalised with the window's statistics (looser than the
// window-clipped envelope, still admissible).  Survivors (lb = max of the
// three bounds, offset) are appended to the global survivor list.
constexpr int kLbThreads = 256;

__device__ __forceinline__ float keogh_term(float v, float u, float l) {
    float d = fmaxf(v - u, 0.0f) + fmaxf(l - v, 0.0f);
    return d * d;
}

__global__ void __launch_bounds__(kLbThreads) k_lb_scan(QueryBufs b, QueryArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int n1, n2;
    __shared__ unsigned short q1[kTile], q2[kTile];
    __shared__ float l1[kTile], l2[kTile];
    QueryState *st = b.st;
    if (!st->valid) return;
    const int m = a.m;
    Tile t = carve_tile(smraw, m);
    const int64_t i0 = (int64_t)blockIdx.x * kTile;
    const float thr = current_thr(st, a);
    if (blockIdx.x == 0 && threadIdx.x == 0) st->thr_scan = thr;
    if (threadIdx.x == 0) { n1 = 0; n2 = 0; }
    if (!stage_tile(t, b, i0, m)) return;
    const float qf = b.qh32[0], ql = b.qh32[m - 1];

    // stage 1: LB_KimFL
    for (int w = threadIdx.x; w < kTile; w += blockDim.x) {
        const int64_t i = i0 + w;
        bool pass = false;
        float kim = 0.0f;
        if (i < a.N) {
            const float mh = t.mh[w], is = t.is[w], ls = t.ml[w] * is;
            const float c0 = fmaf(t.xs[w] - mh, is, -ls);
            const float c1 = fmaf(t.xs[w + m - 1] - mh, is, -ls);
            const float d0 = qf - c0, d1 = ql - c1;
            kim = fmaf(d0, d0, d1 * d1);
            pass = !(kim > thr);
        }
        int pos = warp_append(&n1, pass, 0xffffffffu);
        if (pass) { q1[pos] = (unsigned short)w; l1[pos] = kim; }
    }
    __syncthreads();
    const int c1n = n1;
    // stage 2: LB_Keogh, window vs query envelope
    for (int base = 0; base < c1n; base += blockDim.x) {
        const int e = base + threadIdx.x;
        bool pass = false;
        float lb = 0.0f;
        int w = 0;
        if (e < c1n) {
            w = q1[e];
            const float mh = t.mh[w], is = t.is[w], ls = t.ml[w] * is;
            const float *xw = t.xs + w;
            float s = 0.0f;
            int j = 0;
            for (; j + 8 <= m; j += 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int p = b.ord[j + u];
                    const float c = fmaf(xw[p] - mh, is, -ls);
                    s += keogh_term(c, b.sU[j + u], b.sL[j + u]);
                }
                if (s > thr) break;
            }
            if (!(s > thr)) {
                for (; j < m; ++j) {
                    const int p = b.ord[j];
                    const float c = fmaf(xw[p] - mh, is, -ls);
                    s += keogh_term(c, b.sU[j], b.sL[j]);
                }
            }
            pass = !(s > thr);
            lb = fmaxf(l1[e], s);
        }
        int pos = warp_append(&n2, pass, 0xffffffffu);
        if (pass) { q2[pos] = (unsigned short)w; l2[pos] = lb; }
    }
    __syncthreads();
    const int c2n = n2;
    // stage 3: LB_Keogh, query vs the window's series-wide envelope
    int n3 = 0;
    for (int base = 0; base < c2n; base += blockDim.x) {
        const int e = base + threadIdx.x;
        bool pass = false;
        float lb = 0.0f;
        int64_t i = 0;
        if (e < c2n) {
            const int w = q2[e];
            i = i0 + w;
            const float mh = t.mh[w], is = t.is[w], ls = t.ml[w] * is;
            const float *Uw = b.U + i, *Lw = b.L + i;
            float s = 0.0f;
            int j = 0;
            for (; j + 8 <= m; j += 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int p = b.ord[j + u];
                    const float uu = fmaf(Uw[p] - mh, is, -ls), ll = fmaf(Lw[p] - mh, is, -ls);
                    s += keogh_term(b.sq[j + u], uu, ll);
                }
                if (s > thr) break;
            }
            if (!(s > thr)) {
                for (; j < m; ++j) {
                    const int p = b.ord[j];
                    const float uu = fmaf(Uw[p] - mh, is, -ls), ll = fmaf(Lw[p] - mh, is, -ls);
                    s += keogh_term(b.sq[j], uu, ll);
                }
            }
            pass = !(s > thr);
            lb = fmaxf(l2[e], s);
        }
        int pos = warp_append(&st->n_cand, pass, 0xffffffffu);
        if (pass) {
            b.cand_lb[pos] = lb;
            b.cand_idx[pos] = (unsigned)i;
            ++n3;
        }
    }
    // counters
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n3 += __shfl_xor_sync(0xffffffffu, n3, o);
    if (lane_id() == 0 && n3) atomicAdd(&st->ctr[kCtrKeoghS], (unsigned long long)n3);
    if (threadIdx.x == 0) {
        if (c1n) atomicAdd(&st->ctr[kCtrKim], (unsigned long long)c1n);
        if (c2n) atomicAdd(&st->ctr[kCtrKeoghQ], (unsigned long long)c2n);
    }
}

cudaError_t launch_lb_scan(const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    size_t smem = tile_smem_bytes(a.m);
    cudaError_t e = cudaFuncSetAttribute(k_lb_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t tiles = (a.N + kTile - 1) / kTile;
    k_lb_scan<<<(unsigned)tiles, kLbThreads, smem, s>>>(b, a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ survivor ordering
// Counting sort of the survivors into kBins bins by lower bound, so the DTW
// stage meets the most promising windows first.  With a finite scan
// threshold the bins split [0, thr] evenly; otherwise they follow the
// float's exponent and leading mantissa bits (monotone for lb >= 0).
__device__ __forceinline__ int bin_of(float lb, float thr) {
    if (thr < DINF) {
        int bn = (int)(lb * ((float)kBins / thr));
        return bn < 0 ? 0 : (bn >= kBins ? kBins - 1 : bn);
    }
    return (int)(__float_as_uint(lb) >> 21);
}

__global__ void k_bin_hist(QueryBufs b) {
    __shared__ int h[kBins];
    QueryState *st = b.st;
    for (int t = threadIdx.x; t < kBins; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const int n = st->n_cand;
    const float thr = st->thr_scan;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        atomicAdd(&h[bin_of(b.cand_lb[c], thr)], 1);
    __syncthreads();
    for (int t = threadIdx.x; t < kBins; t += blockDim.x)
        if (h[t]) atomicAdd(&st->hist[t], h[t]);
}

__global__ void __launch_bounds__(kBins) k_bin_scan(QueryState *st) {
    __shared__ int wsum[kBins / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int v = st->hist[t], inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int carry = 0;
    for (int q = 0; q < w; ++q) carry += wsum[q];
    st->bin_off[t] = carry + inc - v;
    if (t == 0) st->work2 = 0;
}

__global__ void k_bin_scatter(QueryBufs b) {
    QueryState *st = b.st;
    const int n = st->n_cand;
    const float thr = st->thr_scan;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        float lb = b.cand_lb[c];
        int pos = atomicAdd(&st->bin_off[bin_of(lb, thr)], 1);
        b.sort_lb[pos] = lb;
        b.sort_idx[pos] = b.cand_idx[c];
    }
}

cudaError_t launch_order(const QueryBufs &b, const QueryArgs &, cudaStream_t s) {
    int blocks = b.num_sms * 2;
    k_bin_hist<<<blocks, 512, 0, s>>>(b);
    k_bin_scan<<<1, kBins, 0, s>>>(b.st);
    k_bin_scatter<<<blocks, 512, 0, s>>>(b);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ finalise
// The result list holds the smallest FP32 distances of the survivors within
// thr.  Every window whose exact distance is among the k smallest has an
// FP32 distance within bsf*(1+delta)+alpha of the k-th, so the entries
// within that margin are re-scored in FP64 and ordered by (FP64 distance,
// offset).  If the list is full and its last entry is still inside the
// margin, more near-ties may exist than it holds: DTWS_EOVERFLOW.
__global__ void k_final_select(QueryBufs b, QueryArgs a) {
    QueryState *st = b.st;
    if (threadIdx.x != 0) return;
    st->work = 0;
    if (!st->valid) { st->n_margin = 0; return; }
    int count = 0;
    while (count < a.list_cap && st->res_keys[count] != kEmptyKey) ++count;
    if (count == 0) { st->n_margin = 0; return; }
    const float dk = key_dist(st->res_keys[(count < a.k ? count : a.k) - 1]);
    const float lim = fmaf(dk, 1.0f + a.delta, a.alpha);
    int nm = 0;
    for (int j = 0; j < count; ++j) {
        if (key_dist(st->res_keys[j]) <= lim) st->margin_idx[nm++] = key_idx(st->res_keys[j]);
    }
    if (count == a.list_cap && key_dist(st->res_keys[count - 1]) <= lim) atomicOr(b.status, kStOverflow);
    st->n_margin = nm;
    st->ctr[kCtrRescored] = (unsigned long long)nm;
}

__global__ void k_final_sort(QueryBufs b, QueryArgs a, int64_t *out_idx, float *out_dist) {
    QueryState *st = b.st;
    const int nm = st->valid ? st->n_margin : 0;
    const int t = threadIdx.x;
    if (t < nm) {
        const double d = st->margin_d64[t];
        const unsigned idx = st->margin_idx[t];
        int rank = 0;
        for (int u = 0; u < nm; ++u) {
            const double du = st->margin_d64[u];
            const unsigned iu = st->margin_idx[u];
            rank += (du < d) || (du == d && iu < idx);
        }
        if (rank < a.k) {
            out_idx[rank] = (int64_t)idx;
            out_dist[rank] = (float)d;
        }
    }
    for (int u = nm + t; u < a.k; u += blockDim.x) {
        out_idx[u] = -1;
        out_dist[u] = DINF;
    }
}

cudaError_t launch_finalize(const QueryBufs &b, const QueryArgs &a, int64_t *out_idx,
                            float *out_dist, cudaStream_t s) {
    k_final_select<<<1, 32, 0, s>>>(b, a);
    cudaError_t e = dtw64_dispatch(b, a, nullptr, 0, nullptr, kListMax, s);
    if (e != cudaSuccess) return e;
    k_final_sort<<<1, kListMax, 0, s>>>(b, a, out_idx, out_dist);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ LBs at offsets
// One warp per offset, full sums (no abandon); same arithmetic as the scan.
__global__ void k_lbs_at(QueryBufs b, QueryArgs a, const int64_t *offsets, int64_t count,
                         float *kim, float *kq, float *ks) {
    if (!b.st->valid) return;
    const int m = a.m;
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (wg >= count) return;
    const int ln = lane_id();
    const int64_t i = offsets[wg];
    if (i < 0 || i >= a.N) {
        if (ln == 0) kim[wg] = kq[wg] = ks[wg] = __int_as_float(0x7fc00000);
        return;
    }
    const float mh = b.mu_hi[i], is = b.inv_sigma[i], ls = b.mu_lo[i] * is;
    const float *xw = b.x + i;
    float sq = 0.0f, ss = 0.0f;
    for (int j = ln; j < m; j += 32) {
        const float c = fmaf(xw[j] - mh, is, -ls);
        sq += keogh_term(c, b.Uq[j], b.Lq[j]);
        const float uu = fmaf(b.U[i + j] - mh, is, -ls), ll = fmaf(b.L[i + j] - mh, is, -ls);
        ss += keogh_term(b.qh32[j], uu, ll);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
    }
    if (ln == 0) {
        const float c0 = fmaf(xw[0] - mh, is, -ls), c1 = fmaf(xw[m - 1] - mh, is, -ls);
        const float d0 = b.qh32[0] - c0, d1 = b.qh32[m - 1] - c1;
        kim[wg] = fmaf(d0, d0, d1 * d1);
        kq[wg] = sq;
        ks[wg] = ss;
    }
}

cudaError_t launch_lbs_at(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                          int64_t count, float *kim, float *kq, float *ks, cudaStream_t s) {
    int64_t blocks = (count * 32 + 255) / 256;
    if (blocks < 1) return cudaSuccess;
    k_lbs_at<<<(unsigned)blocks, 256, 0, s>>>(b, a, offsets, count, kim, kq, ks);
    return cudaGetLastError();
}

}  // namespace dtws
