// query_kernels.cu -- per-query kernels of the search (arxiv 1812.10302):
//
//   k_query_reset   clear the device query state
//   k_qprep         z-normalise Q (Sec. 2.2, Eq. 5; FP64 two-pass; taken as
//                   it is for unnormalised DTW), its envelope (Eq. 9) and the
//                   order of |q_hat| (largest first)
//   k_seed_scan     proxy scan: each CTA's window with the smallest squared
//                   distance on evenly spaced query positions, to its slot
//   k_prop_merge    the P best of the per-CTA slots (rank selection)
//   k_seed_gather   seed offsets = seeded random windows (the paper's random
//                   first bsf, Algorithm 1) + the proposals
//   k_seed_ed       Euclidean distance of each seed (an upper bound of the
//                   banded DTW) -> first bsf
//   k_seed_expand   k > 1: offsets within +-k of the two best Euclidean
//                   seeds join the seeds, distinct
//   k_dtw<SEED>     exact DTW of the seeds when k > 1
//   k_prescore      the best seed's FP32 DTW and its extended re-score, on a
//                   side stream during the scan
//   k_lb_scan       LB_KimFL (Eq. 7) and LB_Keogh vs the query envelope
//                   (Eq. 8) per window of a bulk-copied tile; survivors
//                   appended by warp ballot
//   k_bin_*         order the survivors by lower bound (counting sort)
//   k_dtw<SURV>     LB_Keogh vs the series envelope (Eq. 10) as a pre-check,
//                   then banded DTW (Eq. 1 + band) of the survivors in that
//                   order, early abandon, lock-free top-k list
//   k_final_select  the top-k and every near-tie within the margin
//   k_dtw64*        their extended-precision re-score (FP64 statistics,
//                   double-float DTW)
//   k_final_sort    order by (re-scored distance, offset), output
//   k_exclusion_select  greedy top-k with an exclusion zone over the K best
//
// Pruning (Eq. 6, strict): a window is dropped when a lower bound exceeds
// thr = bsf*(1+delta) + alpha, bsf being the k-th best distance found so far.
// delta and alpha absorb FP32 rounding so no true top-k window is dropped.
#include <cmath>
#include <utility>
#include <type_traits>

#include "dtw_kernels.cuh"

namespace dtws {

// ------------------------------------------------------------------ reset
// Clear a query's device state (by every thread of one block; the caller
// synchronises the block before any of it is read).
__device__ __forceinline__ void reset_state(QueryState *st) {
    for (int t = threadIdx.x; t < kListMax; t += blockDim.x) st->res_keys[t] = kEmptyKey;
    for (int t = threadIdx.x; t < kKMax; t += blockDim.x) st->seed_keys[t] = kEmptyKey;
    for (int t = threadIdx.x; t < kPropMax; t += blockDim.x) st->prop_keys[t] = kEmptyKey;
    for (int t = threadIdx.x; t < kKMax; t += blockDim.x) st->ed_keys[t] = kEmptyKey;
    for (int t = threadIdx.x; t < kBins; t += blockDim.x) st->hist[t] = 0;
    for (int t = threadIdx.x; t < kCtrN; t += blockDim.x) st->ctr[t] = 0;
    for (int t = threadIdx.x; t < 2 * kKMax; t += blockDim.x) st->xz_keys[t / kKMax][t % kKMax] = kEmptyKey;
    if (threadIdx.x == 0) {
        st->xz_count = 0;
        st->xz_nsel = 0;
        st->xz_lock[0] = 0;
        st->xz_lock[1] = 0;
        st->deferred = 0;
        st->pool_off = 0;
        st->prop_done = 0;
        st->bin_done = 0;
        st->final_done = 0;
        st->n_seeds = 0;
        st->n_cand = 0;
        st->work = 0;
        st->work2 = 0;
        st->n_margin = 0;
        st->thr_scan = DINF;
        st->valid = 1;
        st->tile_ctr[0] = 0;
        st->tile_ctr[1] = 0;
        st->n_ed = 0;
        st->pre_done = 0;
        st->margin_skip = 0;
    }
}

__global__ void k_query_reset(QueryState *st) { reset_state(st); }

cudaError_t launch_query_reset(const QueryBufs &b, const QueryArgs &, cudaStream_t s) {
    k_query_reset<<<1, 1024, 0, s>>>(b.st);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ query prep
// One CTA of 128, 256 or 512 threads.  Dynamic smem: one row of kQBins
// 16-bit counters per warp (the ordering's counting sort), then q_hat, its
// upper and its lower envelope, FP32 [m] each.
constexpr int kQBins = 1024;  // |q_hat| quantised to 1/256, up to 4
__global__ void __launch_bounds__(512) k_qprep(const float *__restrict__ Q, QueryBufs b, QueryArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int bad;
    __shared__ unsigned wsum[16];
    const int m = a.m, r = a.r;
    const int nw = (int)(blockDim.x >> 5), wid = (int)(threadIdx.x >> 5), lane = lane_id();
    unsigned short *tab = reinterpret_cast<unsigned short *>(smraw);
    float *qs = reinterpret_cast<float *>(tab + nw * kQBins);
    float *us = qs + m, *ls = us + m;

    // the query's state starts clear (this kernel opens every query)
    reset_state(b.st);
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    bool nf = false;
    for (int j = threadIdx.x; j < m; j += blockDim.x)
        nf |= !isfinite(Q[j]) || (a.raw && fabsf(Q[j]) > kRawAbsMax);
    if (nf) atomicOr(&bad, 1);
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) {
            b.st->valid = 0;
            atomicOr(b.status, kStNonFinite);
        }
        return;
    }
    // Eq. 5, two-pass in FP64: mu, then sum (x - mu)^2 / m (population).
    // One warp does the FP64 work: this part's FP64 units retire about one
    // lane operation per cycle per SM, so FP64 shuffle reductions in every
    // warp of the block would cost far more than the sums themselves.
    // Unnormalised DTW takes the query as it is.
    __shared__ double mu_s, isg_s;
    if (threadIdx.x < 32 && a.raw) {
        for (int j = threadIdx.x; j < m; j += 32) {
            b.qh64[j] = (double)Q[j];
            qs[j] = Q[j];
        }
    } else if (threadIdx.x < 32) {
        double s = 0.0;
        for (int j = threadIdx.x; j < m; j += 32) s += (double)Q[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) mu_s = s / (double)m;  // one division
        __syncwarp();
        const double mu = mu_s;
        double v = 0.0;
        for (int j = threadIdx.x; j < m; j += 32) {
            const double d = (double)Q[j] - mu;
            v = fma(d, d, v);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) {
            const double var = v / (double)m, mm = mu * mu;
            // one square root and reciprocal
            isg_s = var <= 1e-24 * (mm > 1.0 ? mm : 1.0) ? 0.0 : 1.0 / sqrt(var);
        }
        __syncwarp();
        const double isg = isg_s;
        for (int j = threadIdx.x; j < m; j += 32) {
            const double qh = ((double)Q[j] - mu) * isg;
            b.qh64[j] = qh;
            qs[j] = (float)qh;
        }
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
        us[j] = u;
        ls[j] = l;
        b.qh32[j] = qs[j];
    }
    // order by |q_hat| descending, quantised to 1/256 (the order only decides
    // which terms the early-abandoning bounds take first: any order is
    // admissible), ties by position ascending: a stable counting sort over
    // the warps.  Warp w owns positions [w C, (w + 1) C) and a row of
    // counters: (1) each warp counts its keys, 32 positions at a time (equal
    // keys found by a match, counted once by their lowest lane); (2) per key,
    // from the largest |q_hat| down, the rows' counts become each row's first
    // slot (a scan over the keys of the rows' totals, then down the rows);
    // (3) each warp places its positions in order, ranking equal keys within
    // 32 positions by lane.
    for (int t = threadIdx.x; t < nw * kQBins; t += blockDim.x) tab[t] = 0;
    __syncthreads();
    auto qkey = [&](int j) {
        const int v = (int)(fabsf(qs[j]) * 256.0f);
        return (kQBins - 1) - (v < kQBins - 1 ? v : kQBins - 1);  // 0 = the largest |q_hat|
    };
    const int C = ((m + nw - 1) / nw + 31) & ~31;
    const int j0 = wid * C < m ? wid * C : m, j1 = j0 + C < m ? j0 + C : m;
    unsigned short *row = tab + wid * kQBins;
    for (int c0 = j0; c0 < j1; c0 += 32) {
        const int j = c0 + lane;
        const bool in = j < j1;
        const int kk = in ? qkey(j) : -1 - lane;  // (out-of-range lanes match nobody)
        const unsigned peers = __match_any_sync(0xffffffffu, kk);
        if (in && (peers & ((1u << lane) - 1u)) == 0u) row[kk] = (unsigned short)(row[kk] + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
    {
        const int per = kQBins / (int)blockDim.x;  // 8, 4 or 2 keys per thread
        const int k0 = (int)threadIdx.x * per;
        unsigned run = 0;
        for (int u = 0; u < per; ++u)
            for (int w = 0; w < nw; ++w) run += tab[w * kQBins + k0 + u];
        unsigned incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        unsigned start = incl - run;
        for (int w = 0; w < wid; ++w) start += wsum[w];
        for (int u = 0; u < per; ++u)
            for (int w = 0; w < nw; ++w) {
                const unsigned v = tab[w * kQBins + k0 + u];
                tab[w * kQBins + k0 + u] = (unsigned short)start;
                start += v;
            }
    }
    __syncthreads();
    for (int c0 = j0; c0 < j1; c0 += 32) {
        const int j = c0 + lane;
        const bool in = j < j1;
        const int kk = in ? qkey(j) : -1 - lane;
        const unsigned peers = __match_any_sync(0xffffffffu, kk);
        const unsigned rank = __popc(peers & ((1u << lane) - 1u));
        const unsigned slot = in ? row[kk] + rank : 0u;
        __syncwarp();
        if (in && rank == 0) row[kk] = (unsigned short)(row[kk] + __popc(peers));
        if (in) {
            b.ord[slot] = (unsigned short)j;
            b.sq[slot] = qs[j];
            b.sU[slot] = us[j];
            b.sL[slot] = ls[j];
        }
        __syncwarp();
    }
}

cudaError_t launch_qprep(const float *Q, const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    const int threads = a.m < 256 ? 128 : (a.m < 1024 ? 256 : 512);
    const size_t smem = (size_t)(threads / 32) * kQBins * 2 + (size_t)a.m * 12;
    cudaError_t e = cudaFuncSetAttribute(k_qprep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_qprep<<<1, threads, smem, s>>>(Q, b, a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ tile pipeline
// A tile is W consecutive windows [i0, i0 + W).  Its samples
// x[i0, i0 + W + m - 1) and its window statistics are staged in shared
// memory by 1-D bulk copies (the TMA engine) completing on an mbarrier.  The
// padded series and the statistics arrays are allocated so that every full
// tile is in bounds (the library rounds both up to whole tiles plus kMMax).
//
// Scan kernels are persistent and warp-specialised.  The last warp is the
// producer: it takes the next tile from a device-wide cursor (so CTAs that
// meet expensive windows simply take fewer tiles), writes its index into a
// free shared-memory stage and issues the stage's copies; a stage is free
// once its "empty" barrier shows that every consumer warp has released it.
// The other warps are consumers: each waits for the stage's "full" barrier
// (the copies landed), processes its own share of the tile and releases the
// stage with one arrive.  There is no CTA-wide barrier in the loop, so a warp
// held up by a rare expensive window delays only the refill of one stage.
// Use u of a stage waits for phase u & 1 of its barriers.  The end is a stage
// whose tile index is -1, completed without copies.
//
// Two stage layouts, each a tile's mean (high part) and 1/sigma arrays and
// its samples.  LbLayout<TW>: TW windows, every window's statistics and all
// their samples (the lower-bound scan; see shift_bound for the mean's low
// part).  ProxyLayout: kProxyTile windows, the statistics of every
// kProxyStride-th window and only every kProxyStride-th sample (the proxy
// scan scores those windows at term positions that are multiples of
// kProxyStride).
template <int TW>
struct LbLayout {
    static constexpr int W = TW, S = TW, kStride = 1, XDIV = 1;
    __device__ static const float *xs(const QueryBufs &b) { return b.x; }
    __device__ static const float *mh(const QueryBufs &b) { return b.mu_hi; }
    __device__ static const float *is(const QueryBufs &b) { return b.inv_sigma; }
};
struct ProxyLayout {
    static constexpr int W = kProxyTile, S = kProxyTile / kProxyStride, kStride = kProxyStride,
                         XDIV = kProxyStride;
    __device__ static const float *xs(const QueryBufs &b) { return b.x_sub; }
    __device__ static const float *mh(const QueryBufs &b) { return b.smu_hi; }
    __device__ static const float *is(const QueryBufs &b) { return b.sinv_sigma; }
};

struct Tile {
    float *xs, *mh, *is;
    uint64_t *full, *empty;
    long long *tile;
};

constexpr int kStageHeader = 32;  // full, empty barriers and the tile index

// samples staged per tile: W + m - 1, or every XDIV-th of them
template <class LY>
__host__ __device__ __forceinline__ unsigned tile_x_floats(int m) {
    return (unsigned)(((LY::W + m - 1 + LY::XDIV - 1) / LY::XDIV + 3) & ~3);
}
template <class LY>
__host__ __device__ __forceinline__ size_t stage_bytes(int m) {
    return kStageHeader + (size_t)2 * LY::S * 4 + (size_t)tile_x_floats<LY>(m) * 4;
}

template <class LY>
__device__ __forceinline__ Tile carve_stage(unsigned char *sm, int m, int stage) {
    Tile t;
    unsigned char *base = sm + stage * stage_bytes<LY>(m);
    t.full = (uint64_t *)base;
    t.empty = (uint64_t *)(base + 8);
    t.tile = (long long *)(base + 16);
    t.mh = (float *)(base + kStageHeader);
    t.is = t.mh + LY::S;
    t.xs = t.is + LY::S;
    return t;
}

template <class LY>
__device__ __forceinline__ void issue_tile(const Tile &t, const QueryBufs &b, int64_t i0, int m) {
    const unsigned xb = tile_x_floats<LY>(m) * 4u, sb = LY::S * 4u;
    const int64_t s0 = i0 / LY::kStride;
    // the transaction count covers exactly the copies issued below
    mbar_arrive_expect_tx(t.full, xb + 2u * sb);
    bulk_g2s(t.xs, LY::xs(b) + i0 / LY::XDIV, xb, t.full);
    bulk_g2s(t.mh, LY::mh(b) + s0, sb, t.full);
    bulk_g2s(t.is, LY::is(b) + s0, sb, t.full);
}

constexpr int kScanConsumers = 8;                       // consumer warps
constexpr int kLaneEqMin = 20;  // LB_KimFL passers in a row of 32 above which each lane takes its own Eq. 8
constexpr int kScanThreads = (kScanConsumers + 1) * 32;  // + one producer warp

// Runs process(tile, i0) in every consumer warp for each tile this CTA takes
// from *cursor.  A wait that runs past the bound records DTWS_ETIMEOUT and
// ends the loop for that warp (the other warps' waits then run out too);
// the thread's return value is false then.
template <class LY, typename F>
__device__ bool tile_pipeline(unsigned char *sm, const QueryBufs &b, int m, int64_t ntiles,
                              unsigned long long *cursor, int kS, F &&process) {
    const int warp = threadIdx.x >> 5, lane = lane_id();
    if (threadIdx.x == 0) {
        for (int q = 0; q < kS; ++q) {
            const Tile t = carve_stage<LY>(sm, m, q);
            mbar_init(t.full, 1);
            mbar_init(t.empty, kScanConsumers);
        }
        mbar_fence_init();
    }
    __syncthreads();
    bool ok = true;
    if (warp == kScanConsumers) {
        if (lane == 0) {
            int64_t u = 0;
            for (;; ++u) {
                const Tile t = carve_stage<LY>(sm, m, (int)(u % kS));
                if (u >= kS &&
                    !mbar_wait_bounded(t.empty, (unsigned)(((u / kS) - 1) & 1), b.wait_ns)) {
                    ok = false;
                    break;
                }
                const long long tile = (long long)atomicAdd(cursor, 1ull);
                if (tile >= ntiles) {
                    *t.tile = -1;
                    mbar_arrive(t.full);  // completes the phase with no copies
                    break;
                }
                *t.tile = tile;
                issue_tile<LY>(t, b, tile * LY::W, m);
            }
            // Before the producer leaves, every copy it issued has landed, so
            // that no CTA ever leaves with a copy still writing its shared
            // memory -- even when the consumers gave up on a wait: the last
            // use of each other stage, u-S+1 .. u-1 (u: the end marker), and
            // after a timeout also use u-S (the wait that ran out was for its
            // release).  Each of these is its stage's last copy, so its
            // barrier has completed at most that one phase.  On the normal
            // path they have landed already (the consumers wait for them).
            // The drain has its own bound (at least 0.2 s) so that a short
            // wait limit cannot cut it short.
            {
                const long long drain_ns = b.wait_ns > 200000000LL ? b.wait_ns : 200000000LL;
                const int64_t first = ok ? u - kS + 1 : u - kS;
                for (int64_t v = first > 0 ? first : 0; v < u; ++v)
                    mbar_wait_bounded(carve_stage<LY>(sm, m, (int)(v % kS)).full,
                                      (unsigned)((v / kS) & 1), drain_ns);
            }
        }
    } else {
        for (int64_t j = 0;; ++j) {
            const Tile t = carve_stage<LY>(sm, m, (int)(j % kS));
            if (!mbar_wait_bounded(t.full, (unsigned)((j / kS) & 1), b.wait_ns)) {
                ok = false;
                break;
            }
            const long long tile = *(volatile long long *)t.tile;
            if (tile < 0) break;
            process(t, (int64_t)tile * LY::W);
            __syncwarp();
            if (lane == 0) mbar_arrive(t.empty);
        }
    }
    if (!ok) atomicOr(b.status, kStTimeout);
    return ok;
}

static int scan_grid(const void *kernel, int threads, size_t smem, int num_sms, int64_t ntiles) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t g = (int64_t)num_sms * per_sm;
    return (int)(g < ntiles ? g : ntiles);
}

// Pipeline depth of a scan: between min_stages and kStages stages, the one
// with the most resident CTAs per SM (ties: the deeper ring); the shared
// memory goes to more consumer warps when a deeper ring would cost a CTA.
static int scan_stages(const void *kernel, size_t stage_bytes, int min_stages, size_t *smem) {
    int best_s = kStages, best_occ = -1;
    for (int st = kStages; st >= min_stages; --st) {
        int occ = 0;
        const size_t bytes = (size_t)st * stage_bytes;
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kScanThreads, bytes) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (occ > best_occ) {
            best_occ = occ;
            best_s = st;
        }
    }
    *smem = (size_t)best_s * stage_bytes;
    return best_s;
}

// ------------------------------------------------------------------ proxy scan
// For every kProxyStride-th window: the squared distance on TERMS evenly
// spaced query positions (not a lower bound: it only proposes windows whose
// exact distances seed the best-so-far).  Spread-out positions make the terms
// nearly independent, so a random window scores near 2*TERMS while a window
// within a sample or two of a noisy copy scores far lower.  Each thread keeps
// its best window over all the tiles it scans; each CTA proposes its best.
// Scoring one window in four, with the mean's high part and 1/sigma of those
// windows only, and with every term position a multiple of four so that only
// every fourth sample of the series is read, the scan moves 3 bytes per
// window (1 of samples, 2 of statistics) instead of 16; the seed step then
// covers the neighbours of each proposal.  (With one window in eight, a
// window four samples off a match scored no better than lucky random windows
// and matches were lost.)
// Packed FP32 pairs (sm_100 family): one instruction does the operation on
// both halves, each half rounded exactly as the scalar operation would be.
__device__ __forceinline__ unsigned long long x2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float x2_sum(unsigned long long v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo + hi;
}
__device__ __forceinline__ unsigned long long x2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long x2_add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long x2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ void x2_unpack(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// Shared-memory load at a 32-bit shared address plus a constant byte offset
// (volatile: it stays after the barrier wait that made the data visible).
template <int OFF>
__device__ __forceinline__ float lds_at(unsigned addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(OFF));
    return v;
}
template <int OFF>
__device__ __forceinline__ unsigned long long lds64_at(unsigned addr) {
    unsigned long long v;
    asm volatile("ld.shared.b64 %0, [%1+%2];" : "=l"(v) : "r"(addr), "n"(OFF));
    return v;
}

__device__ void prop_rank_select(QueryState *st, const unsigned long long *keys, int n, int first, int stride,
                                 int proposals);
__device__ void seed_lists(const QueryBufs &b, const QueryArgs &a, int n_random, int proposals, int H,
                           unsigned long long rng, unsigned *cand, int *wcnt, int *total);

// The last CTA of the scan to finish (a completion count; nothing waits)
// then merges every CTA's best into the proposals and builds the seed
// lists, the work of k_prop_merge and k_seed_gather without their launches.
template <int TERMS>
__global__ void __launch_bounds__(kScanThreads) k_seed_scan(QueryBufs b, QueryArgs a, int proposals, int stages,
                                                            int n_random, int H, unsigned long long rng) {
    constexpr int kPer = kScanConsumers * 64;           // scored windows per pass of the CTA (two per lane)
    constexpr int kIt = ProxyLayout::S / kPer;          // passes per tile
    static_assert(ProxyLayout::S % kPer == 0 && kIt % 2 == 0, "whole pairs of passes per tile");
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ unsigned long long wbest[kScanConsumers + 1];
    if (!b.st->valid) return;
    const int m = a.m;
    // Term positions, evenly spread, each rounded down to a multiple of
    // 2 * kProxyStride.  Lane l scores the adjacent scored windows 2l and
    // 2l + 1 (+ const; window offsets kProxyStride times those), whose term-p
    // samples are the staged words 2l + p/kProxyStride and the next: one
    // aligned 8-byte load (p/kProxyStride is even), consecutive across the
    // warp (conflict-free), and one packed FP32x2 operation serves both.
    // (the pairs (q_p, q_p) stay in registers: with them in shared memory,
    // 56 registers and four CTAs per SM, the scan was no faster, 89.3 against
    // 87.7 us per 1e8 windows -- its FMA pipe is the busiest unit either way)
    unsigned poff[TERMS];
    unsigned long long qq[TERMS];
#pragma unroll
    for (int u = 0; u < TERMS; ++u) {
        const int pu = (int)(((2 * u + 1) * (long long)m) / (2 * TERMS)) & ~(2 * kProxyStride - 1);
        poff[u] = 4u * (unsigned)(pu / kProxyStride);  // bytes
        const float q = b.qh32[pu];
        qq[u] = x2_pack(q, q);
    }
    unsigned long long best = kEmptyKey;
    const int64_t ntiles = (a.N + ProxyLayout::W - 1) / ProxyLayout::W;
    const bool piped = tile_pipeline<ProxyLayout>(smraw, b, m, ntiles, &b.st->tile_ctr[0], stages, [&](const Tile &t, int64_t i0) {
        // the pair (2v, 2v + 1), v = threadIdx.x + it * kPer / 2: its staged
        // samples from byte offset 8v in xs, its statistics at 8v in mh / is.
        // Two pairs (passes it, it + kIt/2) at a time, each with two partial
        // sums, so four independent FMA chains are in flight.
        const unsigned xa = smem_u32(t.xs) + 8u * threadIdx.x;
        const unsigned sa = smem_u32(t.mh) + 8u * threadIdx.x;
        static_for<kIt / 2>([&](auto itc) {
            constexpr int itA = decltype(itc)::value, itB = itA + kIt / 2;
            constexpr int oA = itA * kPer * 4, oB = itB * kPer * 4;  // bytes, in mh and in xs alike
            // window offsets within the tile, and the windows the tile has
            const int wA = kProxyStride * (2 * (int)threadIdx.x + itA * kPer);
            const int wB = kProxyStride * (2 * (int)threadIdx.x + itB * kPer);
            const int rem = a.N - i0 < ProxyLayout::W ? (int)(a.N - i0) : ProxyLayout::W;
            const bool liveA0 = wA < rem, liveA1 = wA + kProxyStride < rem;
            const bool liveB0 = wB < rem, liveB1 = wB + kProxyStride < rem;
            const unsigned long long mhA = lds64_at<oA>(sa), isA = lds64_at<oA + ProxyLayout::S * 4>(sa);
            const unsigned long long mhB = lds64_at<oB>(sa), isB = lds64_at<oB + ProxyLayout::S * 4>(sa);
            // q_hat - x_hat = (q + mh*is) - x*is, with the mean's high part
            // only (its low part moves every term of a window by the same
            // ~ulp(mu)/sigma: the proxy only ranks proposals)
            const unsigned long long kwA = x2_mul(mhA, isA), kwB = x2_mul(mhB, isB);
            float kA0, kA1, kB0, kB1;
            x2_unpack(kwA, kA0, kA1);
            x2_unpack(kwB, kB0, kB1);
            float accA0, accA1, accB0, accB1;
            if (!__any_sync(0xffffffffu, (liveA0 && !(fabsf(kA0) < 4096.0f)) || (liveA1 && !(fabsf(kA1) < 4096.0f)) ||
                                             (liveB0 && !(fabsf(kB0) < 4096.0f)) || (liveB1 && !(fabsf(kB1) < 4096.0f)))) {
                // one FMA per term; the absolute error stays below ~2^-11
                // when |mu|/sigma < 2^12 (the proxy only ranks proposals)
                const unsigned long long m1 = x2_pack(-1.0f, -1.0f);
                const unsigned long long nisA = x2_mul(isA, m1), nisB = x2_mul(isB, m1);
                unsigned long long sA0 = 0ull, sA1 = 0ull, sB0 = 0ull, sB1 = 0ull;  // (+0, +0)
#pragma unroll
                for (int u = 0; u < TERMS; ++u) {
                    const unsigned long long xA = lds64_at<oA>(xa + poff[u]);
                    const unsigned long long xB = lds64_at<oB>(xa + poff[u]);
                    const unsigned long long cA = x2_fma(xA, nisA, x2_add(qq[u], kwA));
                    const unsigned long long cB = x2_fma(xB, nisB, x2_add(qq[u], kwB));
                    if (u & 1) {
                        sA1 = x2_fma(cA, cA, sA1);
                        sB1 = x2_fma(cB, cB, sB1);
                    } else {
                        sA0 = x2_fma(cA, cA, sA0);
                        sB0 = x2_fma(cB, cB, sB0);
                    }
                }
                x2_unpack(x2_add(sA0, sA1), accA0, accA1);
                x2_unpack(x2_add(sB0, sB1), accB0, accB1);
            } else {
                float mA0, mA1, mB0, mB1, sA0, sA1, sB0, sB1;
                x2_unpack(mhA, mA0, mA1);
                x2_unpack(mhB, mB0, mB1);
                x2_unpack(isA, sA0, sA1);
                x2_unpack(isB, sB0, sB1);
                accA0 = accA1 = accB0 = accB1 = 0.0f;
#pragma unroll
                for (int u = 0; u < TERMS; ++u) {
                    float q, q1, xA0, xA1, xB0, xB1;
                    x2_unpack(qq[u], q, q1);
                    x2_unpack(lds64_at<oA>(xa + poff[u]), xA0, xA1);
                    x2_unpack(lds64_at<oB>(xa + poff[u]), xB0, xB1);
                    const float cA0 = q - (xA0 - mA0) * sA0, cA1 = q - (xA1 - mA1) * sA1;
                    const float cB0 = q - (xB0 - mB0) * sB0, cB1 = q - (xB1 - mB1) * sB1;
                    accA0 = fmaf(cA0, cA0, accA0);
                    accA1 = fmaf(cA1, cA1, accA1);
                    accB0 = fmaf(cB0, cB0, accB0);
                    accB1 = fmaf(cB1, cB1, accB1);
                }
            }
            const unsigned iA = (unsigned)i0 + (unsigned)wA, iB = (unsigned)i0 + (unsigned)wB;
            const unsigned long long kyA0 = make_key(accA0, iA), kyA1 = make_key(accA1, iA + kProxyStride);
            const unsigned long long kyB0 = make_key(accB0, iB), kyB1 = make_key(accB1, iB + kProxyStride);
            best = liveA0 && kyA0 < best ? kyA0 : best;
            best = liveA1 && kyA1 < best ? kyA1 : best;
            best = liveB0 && kyB0 < best ? kyB0 : best;
            best = liveB1 && kyB1 < best ? kyB1 : best;
        });
    });
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v < best ? v : best;
    }
    if (lane_id() == 0) wbest[threadIdx.x >> 5] = best;
    __shared__ int last, wcnt[kScanConsumers + 2], total;
    // (every copy into the stages has landed unless a wait ran out)
    const bool all_ok = __syncthreads_and(piped);
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = wbest[w] < best ? wbest[w] : best;
        b.st->cta_best[blockIdx.x] = best;
        __threadfence();
        last = atomicAdd(&b.st->prop_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || !all_ok) return;  // (a timed-out query ends with an error)
    __threadfence();
    // the stages are idle: the data part of stage 0 (past its barriers,
    // which stay untouched) holds the keys, then the candidates
    unsigned char *spare = smraw + kStageHeader;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(spare);
    const int n = (int)gridDim.x, n8 = (n + 7) & ~7;
    for (int t = threadIdx.x; t < n8; t += blockDim.x) keys[t] = t < n ? __ldcg(&b.st->cta_best[t]) : kEmptyKey;
    __syncthreads();
    prop_rank_select(b.st, keys, n, threadIdx.x, blockDim.x, proposals);
    __syncthreads();
    seed_lists(b, a, n_random, proposals, H, rng, reinterpret_cast<unsigned *>(spare), wcnt, &total);
}

template <int TERMS>
static cudaError_t launch_seed_scan_t(const QueryBufs &b, const QueryArgs &a, int proposals, int n_random, int H,
                                      unsigned long long rng, int *ctas, cudaStream_t s) {
    size_t smem = 0;
    const int stages = scan_stages((const void *)k_seed_scan<TERMS>, stage_bytes<ProxyLayout>(a.m), 2, &smem);
    // the last CTA's keys and candidates fit in the data part of stage 0
    const size_t tail = (size_t)(kCtaSlots + 8) * 8 > (size_t)(n_random + proposals * (2 * H + 1)) * 4
                            ? (size_t)(kCtaSlots + 8) * 8
                            : (size_t)(n_random + proposals * (2 * H + 1)) * 4;
    if (stage_bytes<ProxyLayout>(a.m) < kStageHeader + tail) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_seed_scan<TERMS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (a.N + ProxyLayout::W - 1) / ProxyLayout::W;
    int grid = scan_grid((const void *)k_seed_scan<TERMS>, kScanThreads, smem, b.num_sms, tiles);
    if (grid > kCtaSlots) grid = kCtaSlots;
    k_seed_scan<TERMS><<<grid, kScanThreads, smem, s>>>(b, a, proposals, stages, n_random, H, rng);
    *ctas = grid;
    return cudaGetLastError();
}

cudaError_t launch_seed_scan(const QueryBufs &b, const QueryArgs &a, int proposals, int terms, int n_random, int H,
                             unsigned long long rng, int *ctas, cudaStream_t s) {
    *ctas = 0;
    if (proposals <= 0 || proposals > kPropMax || n_random + proposals * (2 * H + 1) > kEdMax)
        return cudaErrorInvalidValue;
    // evenly spaced positions at multiples of 2 * kProxyStride, so at most
    // m / (2 * kProxyStride) distinct terms
    constexpr int g = 2 * kProxyStride;
    if (terms >= 16 && a.m >= 16 * g) return launch_seed_scan_t<16>(b, a, proposals, n_random, H, rng, ctas, s);
    if (terms >= 8 && a.m >= 8 * g) return launch_seed_scan_t<8>(b, a, proposals, n_random, H, rng, ctas, s);
    if (terms >= 4 && a.m >= 4 * g) return launch_seed_scan_t<4>(b, a, proposals, n_random, H, rng, ctas, s);
    return launch_seed_scan_t<2>(b, a, proposals, n_random, H, rng, ctas, s);
}

// The proposals: the `proposals` smallest of the per-CTA best windows of one
// or two proposal scans (slots 0 .. ctas0-1 and kCtaSlots .. kCtaSlots +
// ctas1-1), ascending.  The CTAs cover disjoint windows, so the keys other
// than the empty key are distinct: each key's rank is the number of keys
// below it, and a key of rank < proposals goes to that slot (the list was
// emptied by the query reset; empty keys are not written).  keys[0 .. n8)
// in shared memory, n8 = n rounded up to 8 (the padding empty); this thread
// ranks keys first, first + stride, ..., eight keys per step in four
// independent 16-byte loads.
__device__ void prop_rank_select(QueryState *st, const unsigned long long *keys, int n, int first, int stride,
                                 int proposals) {
    const int n8 = (n + 7) & ~7;
    const ulonglong2 *k2 = reinterpret_cast<const ulonglong2 *>(keys);
    for (int t = first; t < n; t += stride) {
        const unsigned long long k = keys[t];
        if (k == kEmptyKey) continue;
        int r0 = 0, r1 = 0, r2 = 0, r3 = 0;
        for (int u = 0; u < n8 / 2; u += 4) {
            const ulonglong2 a = k2[u], c = k2[u + 1], d = k2[u + 2], e = k2[u + 3];
            r0 += (a.x < k) + (a.y < k);
            r1 += (c.x < k) + (c.y < k);
            r2 += (d.x < k) + (d.y < k);
            r3 += (e.x < k) + (e.y < k);
        }
        const int rank = r0 + r1 + r2 + r3;
        if (rank < proposals) st->prop_keys[rank] = k;
    }
}

// 128 keys per CTA (one per thread), each CTA with its own copy of all the
// keys in shared memory.
constexpr int kMergeThreads = 128;
__global__ void __launch_bounds__(kMergeThreads) k_prop_merge(QueryBufs b, int n0, int n1, int proposals) {
    __shared__ __align__(16) unsigned long long keys[2 * kCtaSlots + 8];
    QueryState *st = b.st;
    if (!st->valid) return;
    const int n = n0 + n1, n8 = (n + 7) & ~7;
    for (int t = threadIdx.x; t < n8; t += blockDim.x)
        keys[t] = t < n0 ? st->cta_best[t] : (t < n ? st->cta_best[kCtaSlots + (t - n0)] : kEmptyKey);
    __syncthreads();
    const int t = blockIdx.x * kMergeThreads + threadIdx.x;
    if (t < n) prop_rank_select(st, keys, n, t, n, proposals);
}

cudaError_t launch_prop_merge(const QueryBufs &b, int ctas0, int ctas1, int proposals, cudaStream_t s) {
    if (proposals <= 0 || ctas0 + ctas1 <= 0) return cudaSuccess;
    if (ctas0 > kCtaSlots || ctas1 > kCtaSlots || proposals > kPropMax) return cudaErrorInvalidValue;
    const int n = ctas0 + ctas1;
    k_prop_merge<<<(n + kMergeThreads - 1) / kMergeThreads, kMergeThreads, 0, s>>>(b, ctas0, ctas1, proposals);
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

// Seed windows.  seed_off (exact DTW seeds, used when k > 1): the random
// windows (the paper's random first bsf, Algorithm 1) and the proposals.
// ed_off (Euclidean seeds): the random windows and, for each proposal, the
// 2 * kProxyHalf + 1 windows centred on it, since the proxy scan looked at
// every kProxyStride-th window only.  Both lists hold distinct offsets: a repeated seed
// would fill two of the k slots with one window.
// Append the distinct values of src[0..n) (0xffffffff: none) to dst after
// its first `start` entries, in first-occurrence order, up to cap entries in
// all; returns the count.  Every thread of
// the block takes elements t = threadIdx.x + c * blockDim.x and keeps t when
// no earlier element equals it (the earlier elements are read in the same
// order by all lanes: shared-memory broadcasts); the kept flags of a chunk
// are placed by warp ballots and a prefix over the block's warps.
__device__ int distinct_append(unsigned *dst, int cap, const unsigned *src, int n, int start, int *wcnt,
                               int *total) {
    const int lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) *total = start;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int t = c0 + threadIdx.x;
        bool keep = false;
        unsigned v = 0xffffffffu;
        if (t < n && (v = src[t]) != 0xffffffffu) {
            // the earlier elements, four per 16-byte load (src is 16-byte
            // aligned); the last group is checked element by element
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
            const int full = t >> 2;
            bool dup = false;
            for (int g = 0; g < full; ++g) {
                const uint4 q = s4[g];
                dup |= (q.x == v) | (q.y == v) | (q.z == v) | (q.w == v);
            }
            for (int u = full << 2; u < t; ++u) dup |= src[u] == v;
            keep = !dup;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {  // exclusive prefix over the warps, then the chunk's total
            int acc = *total;
            for (int w = 0; w < nwarps; ++w) {
                const int c = wcnt[w];
                wcnt[w] = acc;
                acc += c;
            }
            wcnt[nwarps] = acc;
        }
        __syncthreads();
        const int pos = wcnt[warp] + __popc(bal & ((1u << lane) - 1u));
        if (keep && pos < cap) dst[pos] = v;
        __syncthreads();
        if (threadIdx.x == 0) *total = wcnt[nwarps];
        __syncthreads();
    }
    return *total < cap ? *total : cap;
}

// cand: room for n_random + proposals * (2H + 1) offsets (16-byte aligned);
// wcnt: one int per warp of the block and one more.
__device__ void seed_lists(const QueryBufs &b, const QueryArgs &a, int n_random, int proposals, int H,
                           unsigned long long rng, unsigned *cand, int *wcnt, int *total_p) {
    int &total = *total_p;
    // exact-DTW seeds: random windows + proposals
    for (int j = threadIdx.x; j < n_random; j += blockDim.x)
        cand[j] = (unsigned)(splitmix64(rng + (unsigned long long)j) % (unsigned long long)a.N);
    for (int p = threadIdx.x; p < proposals; p += blockDim.x) {
        const unsigned long long key = b.st->prop_keys[p];
        cand[n_random + p] = key != kEmptyKey ? key_idx(key) : 0xffffffffu;
    }
    __syncthreads();
    const int ns = distinct_append(b.st->seed_off, kSeedMax, cand, n_random + proposals, 0, wcnt, &total);
    // Euclidean seeds: random windows + neighbourhoods of the proposals
    const int span = 2 * H + 1;
    for (int e = threadIdx.x; e < proposals * span; e += blockDim.x) {
        const int p = e / span, d = e - p * span - H;
        const unsigned long long key = b.st->prop_keys[p];
        unsigned o = 0xffffffffu;
        if (key != kEmptyKey) {
            const long long v = (long long)key_idx(key) + d;
            if (v >= 0 && v < a.N) o = (unsigned)v;
        }
        cand[n_random + e] = o;
    }
    __syncthreads();
    const int ne = distinct_append(b.st->ed_off, kEdMax, cand, n_random + proposals * span, 0, wcnt, &total);
    if (threadIdx.x == 0) {
        // exact seeds only pay off for k > 1, and not with a wide exclusion
        // zone (no seed pass runs then, so the survivor pass must not skip them)
        b.st->n_seeds = (a.k > 1 && a.xz_z == 0) ? ns : 0;
        b.st->n_ed = ne;
        b.st->work = 0;
    }
}

__global__ void __launch_bounds__(1024) k_seed_gather(QueryBufs b, QueryArgs a, int n_random, int proposals, int H,
                                                      unsigned long long rng) {
    __shared__ __align__(16) unsigned cand[kEdMax];
    __shared__ int wcnt[33], total;
    if (!b.st->valid) return;
    seed_lists(b, a, n_random, proposals, H, rng, cand, wcnt, &total);
}

// Squared Euclidean distance of the normalised query and window (the
// diagonal warping path, so an upper bound of the banded DTW, Eq. 4) for
// every Euclidean seed, one warp each; the k smallest go to ed_keys.
__global__ void k_seed_ed(QueryBufs b, QueryArgs a) {
    QueryState *st = b.st;
    if (!st->valid) return;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = lane_id();
    if (w >= st->n_ed) return;
    const unsigned idx = st->ed_off[w];
    const float mh = b.mu_hi[idx], is = b.inv_sigma[idx], ls = b.mu_lo[idx] * is;
    const float *xw = b.x + idx;
    float acc = 0.0f;
    for (int j = lane; j < a.m; j += 32) {
        const float d = b.qh32[j] - fmaf(xw[j] - mh, is, -ls);
        acc = fmaf(d, d, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const unsigned long long key = make_key(key_quantize(acc, a.qgrid), idx);
        list_insert(st->ed_keys, a.k, key);
        // the Euclidean distance bounds the window's DTW from above, so it
        // may stand for the window in a bucket list (never in the buffer)
        if (a.xz_z > 0) xz_offer(b, a, key, false);
    }
}

// k > 1: the k-th best distance needs k good windows.  The windows nearest
// in DTW to the best match are its neighbours (warping absorbs small
// shifts), so the offsets within +-k of the two best Euclidean seeds join
// the exact-DTW seeds (one warp).
__global__ void k_seed_expand(QueryBufs b, QueryArgs a) {
    __shared__ __align__(16) unsigned cand[2 * (2 * kKMax + 1)];
    __shared__ int wcnt[33], total;
    QueryState *st = b.st;
    if (!st->valid || a.k < 2) return;
    const int lane = threadIdx.x;
    const int H = a.k < kKMax ? a.k : kKMax, W = 2 * H + 1;
    for (int c = 0; c < 2; ++c) {
        const unsigned long long key = st->ed_keys[c];
        for (int d = lane; d < W; d += 32) {
            unsigned o = 0xffffffffu;
            if (key != kEmptyKey) {
                const long long v = (long long)key_idx(key) + d - H;
                if (v >= 0 && v < a.N) o = (unsigned)v;
            }
            cand[c * W + d] = o;
        }
    }
    __syncwarp();
    const int have = st->n_seeds;
    for (int t = lane; t < 2 * W; t += 32)  // drop offsets that are seeds already
        for (int u = 0; u < have; ++u)
            if (cand[t] == st->seed_off[u]) cand[t] = 0xffffffffu;
    __syncwarp();
    const int ns = distinct_append(st->seed_off, kSeedMax, cand, 2 * W, have, wcnt, &total);
    if (lane == 0) st->n_seeds = ns;
}

cudaError_t launch_seed_expand(const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    k_seed_expand<<<1, 32, 0, s>>>(b, a);
    return cudaGetLastError();
}

cudaError_t launch_seed_ed(const QueryBufs &b, const QueryArgs &a, int max_seeds, cudaStream_t s) {
    // one warp per seed, for at most max_seeds seeds (the lists' bound)
    if (max_seeds < 1) max_seeds = 1;
    if (max_seeds > kEdMax) max_seeds = kEdMax;
    k_seed_ed<<<(max_seeds * 32 + 255) / 256, 256, 0, s>>>(b, a);
    return cudaGetLastError();
}

cudaError_t launch_seed_gather(const QueryBufs &b, const QueryArgs &a, int n_random, int proposals,
                               int half, unsigned long long rng, cudaStream_t s) {
    // one block: the distinctness test is O(n^2) over n <= kEdMax candidates
    const int n = n_random + proposals * (2 * half + 1);
    const int threads = n < 1024 ? (n < 32 ? 32 : (n + 31) / 32 * 32) : 1024;
    k_seed_gather<<<1, threads, 0, s>>>(b, a, n_random, proposals, half, rng);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ wait self-test
// One thread waits, bounded, on a fresh mbarrier that nothing arrives on:
// the wait runs out after wait_ns and records the timeout status the same way
// the scans do -- the failure path of the bounded waits, exercised without a
// fault or a hang.
__global__ void k_wait_selftest(int *status, long long wait_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_fence_init();
    if (!mbar_wait_bounded(&bar, 0u, wait_ns)) atomicOr(status, kStTimeout);
}

// The bounded lock of the wide exclusion zone's bucket lists: one thread
// holds list 0's lock while a second offers a key to that list, so the offer
// waits out wait_ns, records the timeout and drops the key; the holder then
// releases the lock.  Both lists and the lock are left as the query reset
// makes them.  No spin here is unbounded: the holder waits only for the
// offer to return.
__global__ void k_lock_selftest(QueryBufs b, QueryArgs a) {
    QueryState *st = b.st;
    if (threadIdx.x == 0) {
        for (int t = 0; t < 2 * kKMax; ++t) st->xz_keys[t / kKMax][t % kKMax] = kEmptyKey;
        st->xz_lock[0] = 1;  // held by this thread
        st->xz_lock[1] = 0;
        st->xz_count = 0;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 32) xz_offer(b, a, make_key(1.0f, 0u), false);  // another warp: bucket 0 has parity 0
    __syncthreads();
    if (threadIdx.x == 0) atomicExch(&st->xz_lock[0], 0);
}

cudaError_t launch_lock_selftest(const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    k_lock_selftest<<<1, 64, 0, s>>>(b, a);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int *status, long long wait_ns, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(status, wait_ns);
    return cudaGetLastError();
}

// Re-score: per window two-pass FP64 statistics (Eq. 5), the normalised
// values formed in FP64, and the banded DTW in double-float arithmetic
// (about 48 significant bits; FP64 itself, on the row-systolic kernel, where
// the multi-warp walk k_dtw64_mw does not apply or fit).
// No pruning.  Candidates: the margin list (offsets == null) or offsets.
template <int L, int K>
__global__ void __launch_bounds__(256) k_dtw64(QueryBufs b, QueryArgs a, const int64_t *offsets,
                                               int64_t count_host, double *out, int staged) {
    extern __shared__ __align__(16) unsigned char smraw[];
    QueryState *st = b.st;
    if (!st->valid) return;
    const int m = a.m, r = a.r;
    const DtwSmem<double> lay = dtw_smem<double, L, K>(m, r, staged != 0, false);
    // K > 0: double-float arrays (8 B per element, as for a double), padded
    // with finite poison values (+1e15 query, -1e15 window)
    double *qbase = (double *)smraw;
    dfloat *qd = (dfloat *)smraw + lay.pad;
    double *qs = qbase + lay.pad;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        if (K > 0) qd[t] = df_from(b.qh64[t]);
        else qs[t] = b.qh64[t];
    }
    if (K > 0) fill_pads((dfloat *)smraw, m, lay.pad, dfloat{1e15f, 0.0f}, threadIdx.x, blockDim.x);
    const int warp = threadIdx.x >> 5, ln = lane_id();
    const int g = ln / L, lane = ln % L;
    const int gid = warp * (32 / L) + g;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g * L));
    unsigned char *gbase = smraw + lay.q_bytes() + (size_t)gid * lay.group_bytes();
    double *cbuf = lay.staged ? (double *)gbase + lay.pad : nullptr;
    dfloat *cd = (dfloat *)gbase + lay.pad;
    if (K > 0) fill_pads((dfloat *)gbase, m, lay.pad, dfloat{-1e15f, 0.0f}, lane, L);
    double *ring = lay.ring ? (double *)(gbase + (lay.staged ? lay.span() * 8 : 0)) : nullptr;
    __syncthreads();
    const int64_t count = offsets ? count_host
                        : a.xz_z > 0 ? (int64_t)min(st->xz_nsel, b.xz_sel_cap)
                                     : (int64_t)st->n_margin;
    __shared__ double bc[2 * 8 * 32];  // per group: mu, 1/sigma
    // (the margin list's first margin_skip entries were re-scored already)
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
            idx = a.xz_z > 0 ? b.xz_sel[c] : st->margin_idx[c];
        }
        const float *xw = b.x + idx;
        double s = 0.0;
        for (int j = lane; j < m; j += L) s += (double)xw[j];
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, L);
        double v = 0.0;
        const double mu0 = s * (1.0 / (double)m);
        for (int j = lane; j < m; j += L) {
            const double d = (double)xw[j] - mu0;
            v = fma(d, d, v);
        }
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o, L);
        // one division and square root per group (long FP64 sequences)
        if (lane == 0) {
            const double mu = s / (double)m, var = v / (double)m, mm = mu * mu;
            bc[2 * gid] = a.raw ? 0.0 : mu;
            bc[2 * gid + 1] = a.raw ? 1.0 : var <= 1e-24 * (mm > 1.0 ? mm : 1.0) ? 0.0 : 1.0 / sqrt(var);
        }
        __syncwarp(gmask);
        const double mu = bc[2 * gid], inv = bc[2 * gid + 1];
        double d;
        if constexpr (K > 0) {
            for (int j = lane; j < m; j += L) cd[j] = df_from(((double)xw[j] - mu) * inv);
            __syncwarp(gmask);
            d = dtw_diag_df<L, K>(qd, cd, m, r, gmask, lane);
        } else {
            if (cbuf) {
                for (int j = lane; j < m; j += L) cbuf[j] = ((double)xw[j] - mu) * inv;
            }
            __syncwarp(gmask);
            int cells = 0;
            d = dtw_band<double, L, false>(qs, xw, cbuf, mu, inv, 0.0, nullptr, ring, m, r, tinf<double>(), gmask,
                                           lane, cells);
        }
        if (lane == 0) {
            if (offsets) out[c] = d;
            else if (a.xz_z > 0) b.xz_d64[c] = d;
            else st->margin_d64[c] = d;
        }
        __syncwarp(gmask);
    }
}

// Where the final stage writes the answer (the multi-warp re-score kernel
// does the whole stage when idx is set).
struct FinalOut {
    int64_t *idx = nullptr;
    float *dist = nullptr;
};
__device__ __forceinline__ int margin_select(const unsigned long long *keys, const QueryState *st, const QueryArgs &a,
                             unsigned *idx, int *skip, bool *overflow);
__device__ __forceinline__ void final_order(const unsigned *idx, const double *d64, int nm, const QueryArgs &a, int64_t *out_idx,
                            float *out_dist, int tid, int nthreads);

// The re-score with the anti-diagonal walk spread over W warps per window
// (dtw_diag_df_mw): G = blockDim.x / (32 W) groups per CTA, group g owning
// named barrier 1 + g; the query's double-float copy is shared, each group
// stages its window.  Used when a window's r+1 cells need more than one
// cell per lane of one warp: per window it is the latency of the walk that
// counts, and W warps cut the cells each lane steps through per
// anti-diagonal by W.
//
// With fin set (the end of a search, no exclusion zone) the kernel is the
// whole final stage: every CTA makes the margin list itself from the result
// list (margin_select: the same list in every CTA), group gg of the grid
// re-scores entries skip + gg, skip + gg + groups, ..., and the last CTA to
// finish (a completion count; nothing waits) orders the list and writes the
// output (final_order) -- k_final_select and k_final_sort without their
// launches.
template <int W, int K>
__global__ void __launch_bounds__(256, 1) k_dtw64_mw(QueryBufs b, QueryArgs a, const int64_t *offsets,
                                                  int64_t count_host, double *out, FinalOut fin) {
    constexpr int GMAX = 8 / W;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ DfXchg xch[GMAX];
    __shared__ double bc[2 * GMAX];
    __shared__ int cur[GMAX];
    QueryState *st = b.st;
    const bool fused = fin.idx != nullptr;
    if (!fused && !st->valid) return;
    const int m = a.m, r = a.r;
    const int G = (int)(blockDim.x / (32 * W));
    const int pad = diag_pad(r, 32 * W, K);
    const size_t span = (size_t)((m + 2 * pad + 3) & ~3);
    dfloat *qd = (dfloat *)smraw + pad;
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const int g = warp / W, w = warp % W, t = w * 32 + lane;
    const int nthr = 32 * W, bar = 1 + g;
    dfloat *cbase = (dfloat *)(smraw + span * 8 * (size_t)(1 + g));
    dfloat *cd = cbase + pad;
    __shared__ unsigned long long ms_keys[kListMax];
    __shared__ unsigned ms_idx[kListMax];
    __shared__ double ms_d[kListMax];
    __shared__ int ms_n, ms_skip, last;
    if (fused) {
        const bool valid = st->valid != 0;
        for (int j = threadIdx.x; j < a.list_cap; j += blockDim.x) ms_keys[j] = valid ? st->res_keys[j] : kEmptyKey;
        __syncthreads();
        if (threadIdx.x == 0) {
            int skip = 0;
            bool ovf = false;
            ms_n = valid ? margin_select(ms_keys, st, a, ms_idx, &skip, &ovf) : 0;
            ms_skip = skip;
            if (blockIdx.x == 0) {
                st->n_margin = ms_n;
                st->margin_skip = skip;
                st->ctr[kCtrRescored] = (unsigned long long)ms_n;
                if (ovf) atomicOr(b.status, kStOverflow);
            }
        }
    }
    __syncthreads();
    // (a CTA of the fused final stage with no window to re-score skips the
    // copies: usually all but the first, the best window being pre-scored)
    const bool work = !fused || ms_skip + (int)blockIdx.x * G < ms_n;
    if (work) {
        for (int j = threadIdx.x; j < m; j += blockDim.x) qd[j] = df_from(b.qh64[j]);
        fill_pads((dfloat *)smraw, m, pad, dfloat{1e15f, 0.0f}, threadIdx.x, blockDim.x);
        if (g < G) fill_pads(cbase, m, pad, dfloat{-1e15f, 0.0f}, t, nthr);
    }
    __syncthreads();
    if (g >= G || !work) {
        if (!fused) return;
    } else {
    const int64_t count = offsets ? count_host
                        : fused ? (int64_t)ms_n
                        : a.xz_z > 0 ? (int64_t)min(st->xz_nsel, b.xz_sel_cap)
                                     : (int64_t)st->n_margin;
    int c_next = fused ? ms_skip + (int)blockIdx.x * G + g : 0;
    while (true) {
        int c;
        if (fused) {
            c = c_next;
            c_next += (int)gridDim.x * G;
        } else {
            // (the previous window's last barrier lies between every thread's
            // read of cur[g] and this write)
            if (t == 0) cur[g] = atomicAdd(&st->work, 1);
            group_bar(bar, nthr);
            c = cur[g];
        }
        if (c >= count) break;
        unsigned idx = 0;
        bool bad = false;
        if (offsets) {
            const int64_t o = offsets[c];
            bad = o < 0 || o >= a.N;
            idx = bad ? 0u : (unsigned)o;
        } else {
            idx = fused ? ms_idx[c] : a.xz_z > 0 ? b.xz_sel[c] : st->margin_idx[c];
        }
        if (bad) {
            if (t == 0) out[c] = __longlong_as_double(0x7ff8000000000000ll);
            group_bar(bar, nthr);
            continue;
        }
        const float *xw = b.x + idx;
        if (w == 0) {  // two-pass FP64 statistics (Eq. 5) in the group's first warp
            double sum = 0.0;
            for (int j = lane; j < m; j += 32) sum += (double)xw[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            const double mu0 = sum * (1.0 / (double)m);
            double v = 0.0;
            for (int j = lane; j < m; j += 32) {
                const double d = (double)xw[j] - mu0;
                v = fma(d, d, v);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) {
                const double mu = sum / (double)m, var = v / (double)m, mm = mu * mu;
                bc[2 * g] = a.raw ? 0.0 : mu;
                bc[2 * g + 1] = a.raw ? 1.0 : var <= 1e-24 * (mm > 1.0 ? mm : 1.0) ? 0.0 : 1.0 / sqrt(var);
            }
        }
        group_bar(bar, nthr);
        const double mu = bc[2 * g], inv = bc[2 * g + 1];
        for (int j = t; j < m; j += nthr) cd[j] = df_from(((double)xw[j] - mu) * inv);
        group_bar(bar, nthr);
        const double d = dtw_diag_df_mw<W, K>(qd, cd, m, r, w, lane, xch[g], bar);
        if (t == 0) {
            if (offsets) out[c] = d;
            else if (a.xz_z > 0 && !fused) b.xz_d64[c] = d;
            else st->margin_d64[c] = d;
            if (fused) __threadfence();  // (before this CTA counts itself done)
        }
        // (in the fused form the next window's first barrier is this one:
        // no thread of the group reuses cd or bc before all have passed it)
        if (fused) group_bar(bar, nthr);
    }
    }
    if (!fused) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&st->final_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int j = threadIdx.x; j < ms_n; j += blockDim.x) ms_d[j] = j < ms_skip ? st->pre_d64 : __ldcg(&st->margin_d64[j]);
    __syncthreads();
    final_order(ms_idx, ms_d, ms_n, a, fin.idx, fin.dist, threadIdx.x, blockDim.x);
}

template <int W, int K>
static cudaError_t dtw64_mw_launch(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets, int64_t count,
                                   double *out, int64_t count_for_grid, cudaStream_t s, FinalOut fin) {
    // the query's copy plus one window copy per group (double-float: 8 B per element)
    const size_t span = (size_t)((a.m + 2 * diag_pad(a.r, 32 * W, K) + 3) & ~3), bytes = span * sizeof(dfloat);
    const size_t hard = (size_t)200 * 1024;
    int groups = 8 / W;
    while (groups > 1 && bytes * (size_t)(1 + groups) > hard) --groups;
    if (bytes * (size_t)(1 + groups) > hard) return cudaErrorNotSupported;  // the caller falls back
    const size_t smem = bytes * (size_t)(1 + groups);
    int64_t want = (count_for_grid + groups - 1) / groups;
    const int64_t cap = (int64_t)b.num_sms * 4;
    if (want < 1) want = 1;
    const int blocks = (int)(want < cap ? want : cap);
    cudaError_t e = cudaFuncSetAttribute(k_dtw64_mw<W, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_dtw64_mw<W, K><<<blocks, groups * W * 32, smem, s>>>(b, a, offsets, count, out, fin);
    return cudaGetLastError();
}

// fin set: the whole final stage in the multi-warp kernel, or nothing is
// launched and the result is cudaErrorNotSupported.
static cudaError_t dtw64_dispatch(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                                  int64_t count, double *out, int64_t count_for_grid, cudaStream_t s,
                                  FinalOut fin) {
    DtwPlan p;
    if (!plan_dtw<double>(a.m, a.r, false, &p)) return cudaErrorInvalidValue;
    // anti-diagonal with more than one cell per lane of a warp: the
    // multi-warp walk (the same arithmetic, the same result)
    cudaError_t mw = cudaErrorNotSupported;
    if (p.L == 32 && p.K >= 2) {
#define DTWS_MW(KK)                                                                                       \
        if (p.K == KK)                                                                                     \
            mw = dtw64_mw_launch<PreShape<32, KK>::W, PreShape<32, KK>::K2>(b, a, offsets, count, out,    \
                                                                             count_for_grid, s, fin);
        DTWS_MW(2) DTWS_MW(3) DTWS_MW(4) DTWS_MW(6) DTWS_MW(8) DTWS_MW(10) DTWS_MW(12) DTWS_MW(16)
#undef DTWS_MW
    } else if (a.r > kDiagRMax && a.r < 8 * 32 * 8) {
        // bands past the one-warp walks (r > 511, up to 2047): the double-float
        // walk over four warps (r <= 1023) or eight (a window's walk is latency:
        // more warps, fewer cells per lane per anti-diagonal) with up to 8
        // cells per lane, instead of FP64 arithmetic, which this part issues
        // at a small fraction of its FP32 rate
        const int k4 = (a.r + 1 + 127) / 128, k8 = (a.r + 1 + 255) / 256;
        if (k4 <= 6) mw = dtw64_mw_launch<4, 6>(b, a, offsets, count, out, count_for_grid, s, fin);
        else if (k4 <= 8) mw = dtw64_mw_launch<4, 8>(b, a, offsets, count, out, count_for_grid, s, fin);
        else if (k8 <= 6) mw = dtw64_mw_launch<8, 6>(b, a, offsets, count, out, count_for_grid, s, fin);
        else mw = dtw64_mw_launch<8, 8>(b, a, offsets, count, out, count_for_grid, s, fin);
    }
    if (mw != cudaErrorNotSupported || fin.idx) return mw;
    // (the shared-memory copies do not fit: the one-group kernels below)
    const int blocks = dtw_blocks(p, b.num_sms, count_for_grid);
#define DTWS_CASE(LL, KK)                                                                                     \
    if (p.L == LL && p.K == KK) {                                                                             \
        cudaError_t e = cudaFuncSetAttribute(k_dtw64<LL, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                             (int)p.smem);                                                    \
        if (e != cudaSuccess) return e;                                                                       \
        k_dtw64<LL, KK><<<blocks, p.warps * 32, p.smem, s>>>(b, a, offsets, count, out, p.staged);            \
        return cudaGetLastError();                                                                            \
    }
    DTWS_CASE(1, 1) DTWS_CASE(2, 1) DTWS_CASE(4, 1) DTWS_CASE(8, 1) DTWS_CASE(16, 1)
    DTWS_CASE(32, 1) DTWS_CASE(32, 2) DTWS_CASE(32, 3) DTWS_CASE(32, 4) DTWS_CASE(32, 6) DTWS_CASE(32, 8) \
    DTWS_CASE(32, 10) DTWS_CASE(32, 12) DTWS_CASE(32, 16)
    DTWS_CASE(1, 0) DTWS_CASE(2, 0) DTWS_CASE(4, 0) DTWS_CASE(8, 0) DTWS_CASE(16, 0) DTWS_CASE(32, 0)
#undef DTWS_CASE
    return cudaErrorInvalidValue;
}

namespace {
__global__ void k_reset_cursor(QueryState *st) { st->work = 0; }
}  // namespace

cudaError_t launch_dtw_at_f64(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                              int64_t count, double *out, cudaStream_t s) {
    k_reset_cursor<<<1, 1, 0, s>>>(b.st);
    return dtw64_dispatch(b, a, offsets, count, out, count, s, FinalOut{});
}

// ------------------------------------------------------------------ LB scan
// Cascade over tiles of windows (Sec. 2.2, Eqs. 6-8, prune when a bound
// exceeds thr): LB_KimFL (Eq. 7, squared) for every window, then LB_Keogh of
// the window against the query envelope (Eq. 8), terms in |q_hat|-descending
// order with early abandon.  Survivors (lb = max of the two, offset) are
// appended to the global survivor list.  The third bound, LB_Keogh of the
// query against the window's envelope (Eq. 10, from the series-wide envelope
// normalised with the window's statistics: looser than the window-clipped
// envelope, still admissible), is evaluated for each survivor by the DTW
// kernel, whose tail bound consists of exactly its per-row terms.
// LB_Keogh (Eq. 8) chunks of 32 terms the scan takes at most per window; the
// first kEqSmem of them come from shared memory, any further ones through L1
// (the same few values for every window).  Measured: 8 chunks moved work
// from the survivor stage into the scan (whose warp holds all 32 lanes per
// passing window) and slowed the m = 512 workload by 7 %, so the scan stops
// after 2 and the survivor stage's pre-check takes over.
constexpr int kEqChunks = 2, kEqSmem = 2;

// The lower-bound scan normalises with the mean's high part alone: the
// window's values then sit shifted by mu_lo / sigma, and |mu_lo| <= ulp(mu_hi)
// / 2 <= |mu_hi| 2^-24 (the pair is normalised; 2^-149 covers a subnormal
// mu_hi).  A value at most D from the true one is at least |d| - D from a
// point the true one is d from, so each bound is taken on distances reduced
// by D -- (|d| - D)+ for LB_KimFL's end points, the query envelope widened
// by D for LB_Keogh -- and stays a lower bound; D is ~1e-7 of |mu| / sigma.
// The scan then reads 12 bytes per window instead of 16.
__device__ __forceinline__ float shift_bound(float mh, float is) {
    return fmaf(fabsf(mh), 0x1p-24f, 0x1p-149f) * is;
}

__device__ __forceinline__ float keogh_term(float v, float u, float l) {
    const float d = fmaxf(v - u, 0.0f) + fmaxf(l - v, 0.0f);
    return d * d;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Each warp scans 32 windows at a time with LB_KimFL (one window per lane);
// the rare windows that pass are then bounded by the whole warp, one at a
// time: lanes take 32 consecutive terms of the |q_hat|-ordered LB_Keogh sums
// and the warp abandons as soon as a chunk's running total exceeds thr.  No
// thread waits on another warp's survivors.
// The rare part of a row of 32 windows (entered only when some window
// passed LB_KimFL): the windows that passed (bal) are bounded by
// LB_Keogh of the window against the query envelope (Eq. 8) over the
// kEqChunks * 32 largest-|q_hat| terms, and the survivors are appended as
// (bound, offset) by one warp-aggregated atomic.  A dense row (a loose
// bound) gives each passing lane its own window's terms; otherwise the warp
// takes one window at a time, 32 terms per step.  Returns the survivors.
// (Eq. 10's first 32 terms here as well, for each window past Eq. 8, halved
// the survivors on 1e8 windows, m = 512 -- 38,000 to 21,000, the survivor
// pass 55 -> 43 us -- but slowed the scan 278 -> 300 us: the random loads of
// the series envelope stall the warps that feed the ring.)
__device__ __forceinline__ int lb_row_keogh(const Tile &t, const QueryBufs &b, QueryState *st, const int *o_s,
                                         const float *u_s, const float *l_s, int m, float thr, unsigned bal,
                                         int wrow, int lane, float kim, float mh, float is, float sd, int64_t i0) {
    const int w = wrow + lane;
    unsigned keep = 0;   // windows of this row that survive Eq. 8
    float my_lb = 0.0f;  // lane t holds window t's bound when it survives
    if (__popc(bal) >= kLaneEqMin) {
        // the same terms in the same |q_hat| order, each lane abandoning once
        // its sum exceeds thr (checked every 8 terms): 32 windows per step
        // instead of one window and a shuffle reduction per chunk
        const int nt = m < kEqChunks * 32 ? m : kEqChunks * 32;
        float s2 = 0.0f;
        bool alive = (bal >> lane) & 1u;
        for (int j0 = 0; j0 < nt; j0 += 8) {
            if (!__any_sync(0xffffffffu, alive)) break;
            if (alive) {
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const int j = j0 + v;
                    if (j < nt) {
                        const bool sm = j < kEqSmem * 32;
                        const int o = sm ? o_s[j] : (int)__ldg(b.ord + j);
                        const float uq = sm ? u_s[j] : __ldg(b.sU + j), lq = sm ? l_s[j] : __ldg(b.sL + j);
                        s2 += keogh_term((t.xs[w + o] - mh) * is, uq + sd, lq - sd);
                    }
                }
                alive = !(s2 > thr);
            }
        }
        keep = __ballot_sync(0xffffffffu, alive);
        my_lb = fmaxf(kim, s2);
    } else {
        while (bal) {
            const int src = __ffs(bal) - 1;
            bal &= bal - 1;
            const int ws = wrow + src;
            const float smh = t.mh[ws], sis = t.is[ws], ssd = shift_bound(smh, sis);
            const float *xw = t.xs + ws;
            // a window that survives these chunks (the neighbourhood of a
            // match) goes to the DTW stage with the partial sum, itself a
            // lower bound, rather than holding this warp for the full sum
            float s2 = 0.0f;
            for (int base = 0; base < m && base < kEqChunks * 32; base += 32) {
                const int j = base + lane;
                float term = 0.0f;
                if (j < m) {
                    const bool sm = base < kEqSmem * 32;
                    const int o = sm ? o_s[j] : (int)__ldg(b.ord + j);
                    const float uq = sm ? u_s[j] : __ldg(b.sU + j), lq = sm ? l_s[j] : __ldg(b.sL + j);
                    term = keogh_term((xw[o] - smh) * sis, uq + ssd, lq - ssd);
                }
                s2 += warp_sum(term);
                if (s2 > thr) break;
            }
            if (s2 > thr) continue;
            keep |= 1u << src;
            if (lane == src) my_lb = fmaxf(kim, s2);
        }
    }
    // one append per row of 32 windows: a warp-aggregated atomic
    if (keep) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&st->n_cand, __popc(keep));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep & (1u << lane)) {
            const int pos = base + __popc(keep & ((1u << lane) - 1u));
            b.cand_lb[pos] = my_lb;
            b.cand_idx[pos] = (unsigned)(i0 + w);
        }
    }
    return __popc(keep);
}

template <int TW>
__global__ void __launch_bounds__(kScanThreads, 5) k_lb_scan(QueryBufs b, QueryArgs a, int stages) {
    extern __shared__ __align__(16) unsigned char smraw[];
    QueryState *st = b.st;
    if (!st->valid) return;
    const int m = a.m;
    const float thr = current_thr(st, a);
    if (blockIdx.x == 0 && threadIdx.x == 0) st->thr_scan = thr;
    const float qf = b.qh32[0], ql = b.qh32[m - 1];
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    constexpr int kPerWarp = TW / kScanConsumers;
    // the ordered query terms the scan uses, in shared memory
    __shared__ int o_s[kEqSmem * 32];
    __shared__ float u_s[kEqSmem * 32], l_s[kEqSmem * 32];
    for (int j = threadIdx.x; j < kEqSmem * 32; j += blockDim.x) {
        o_s[j] = j < m ? (int)b.ord[j] : 0;
        u_s[j] = j < m ? b.sU[j] : 0.0f;
        l_s[j] = j < m ? b.sL[j] : 0.0f;
    }
    unsigned c1 = 0, c2 = 0;  // (per lane: at most the windows its warp scans)
    const int64_t ntiles = (a.N + TW - 1) / TW;
    tile_pipeline<LbLayout<TW>>(smraw, b, m, ntiles, &st->tile_ctr[1], stages, [&](const Tile &t, int64_t i0) {
        // 32-bit shared addresses of this lane's first window (row 0); the
        // rows follow at constant offsets
        const unsigned w0 = (unsigned)(warp * kPerWarp + lane);
        const unsigned sa = smem_u32(t.mh) + 4u * w0, xa = smem_u32(t.xs) + 4u * w0;
        const unsigned xl = xa + 4u * (unsigned)(m - 1);
        // windows of this tile that exist: w < rem
        const int rem = a.N - i0 < TW ? (int)(a.N - i0) : TW;
        constexpr int kRows = kPerWarp / 32;
        // LB_KimFL for every row first (unrolled, constant offsets), then the
        // rare part for the rows where some window passed (one copy of it)
        unsigned bals[kRows];
        float kims[kRows];
        static_for<kRows>([&](auto uc) {
            constexpr int u = decltype(uc)::value;
            constexpr int RO = u * 32 * 4;
            bool pass = false;
            float kim = 0.0f;
            if ((int)w0 + u * 32 < rem) {
                const float mh = lds_at<RO>(sa), is = lds_at<RO + TW * 4>(sa);
                const float sd = shift_bound(mh, is);
                const float d0 = fmaxf(fabsf(fmaf(mh - lds_at<RO>(xa), is, qf)) - sd, 0.0f);
                const float d1 = fmaxf(fabsf(fmaf(mh - lds_at<RO>(xl), is, ql)) - sd, 0.0f);
                kim = fmaf(d0, d0, d1 * d1);
                pass = !(kim > thr);
            }
            bals[u] = __ballot_sync(0xffffffffu, pass);
            kims[u] = kim;
        });
        unsigned any = 0;
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
            c1 += (unsigned)__popc(bals[u]);
            any |= bals[u];
        }
        if (any) {
#pragma unroll 1
            for (int u = 0; u < kRows; ++u) {
                // (the row's ballot and bound picked by constant indices, so
                // the arrays stay in registers)
                unsigned bu = 0;
                float ku = 0.0f;
                static_for<kRows>([&](auto vc) {
                    constexpr int v = decltype(vc)::value;
                    bu = u == v ? bals[v] : bu;
                    ku = u == v ? kims[v] : ku;
                });
                if (!bu) continue;
                const int w = (int)w0 + u * 32;
                const float mh = t.mh[w], is = t.is[w];
                c2 += lb_row_keogh(t, b, st, o_s, u_s, l_s, m, thr, bu, w - lane, lane, ku, mh, is,
                                   shift_bound(mh, is), i0);
            }
        }
    });
    if (lane == 0) {
        if (c1) atomicAdd(&st->ctr[kCtrKim], (unsigned long long)c1);
        if (c2) atomicAdd(&st->ctr[kCtrKeoghQ], (unsigned long long)c2);
    }
}

template <int TW>
static cudaError_t launch_lb_scan_t(const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    size_t smem = 0;
    const int stages = scan_stages((const void *)k_lb_scan<TW>, stage_bytes<LbLayout<TW>>(a.m), 3, &smem);
    cudaError_t e = cudaFuncSetAttribute(k_lb_scan<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (a.N + TW - 1) / TW;
    int grid = scan_grid((const void *)k_lb_scan<TW>, kScanThreads, smem, b.num_sms, tiles);
    // the scan is persistent and would occupy every CTA slot: leave one free
    // so the side-stream pre-score runs beside it instead of after it
    if (a.prescore && grid > b.num_sms) --grid;
    k_lb_scan<TW><<<grid, kScanThreads, smem, s>>>(b, a, stages);
    return cudaGetLastError();
}

cudaError_t launch_lb_scan(const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    // Tile width by query length: a tile's stage holds its TW windows'
    // statistics and TW + m - 1 samples (the m - 1 halo read from L2).  Up
    // to m = 768 the 1024-window tile keeps 4 CTAs per SM with 3 stages;
    // beyond it the stage grows and residency drops to 3, and the 512-window
    // tile (more CTAs in flight, a larger halo share) is faster (measured:
    // m = 512 0.293 ms vs 0.326 ms per 1e8 windows with 512; m = 1024
    // 1.01 ms vs 1.28 ms per 2e8 with 1024).
    return a.m <= 768 ? launch_lb_scan_t<kTile>(b, a, s) : launch_lb_scan_t<kTile / 2>(b, a, s);
}

// ------------------------------------------------------------------ survivor ordering
// Counting sort of the survivors into kBins bins by lower bound, so the DTW
// stage meets the most promising windows first.  With a finite scan
// threshold the bins split [0, thr] evenly; otherwise they follow the
// float's exponent and leading mantissa bits (monotone for lb >= 0).
// Each CTA takes a contiguous chunk of the survivors.  (A minimum chunk of
// 4096, leaving most CTAs idle when there are few survivors, measured
// slower: 7.9 -> 12.4 us for the scatter of 38,000 survivors.)
__device__ __forceinline__ void bin_chunk(int64_t n, int64_t *c0, int64_t *c1) {
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    *c0 = (int64_t)blockIdx.x * per;
    if (*c0 > n) *c0 = n;
    *c1 = *c0 + per < n ? *c0 + per : n;
}

// The histogram over all CTAs; the last CTA to finish (a completion count,
// nothing waits) turns it into each bin's first position.
constexpr int kBinThreads = 512;
__global__ void __launch_bounds__(kBinThreads) k_bin_hist(QueryBufs b) {
    static_assert(kBins == 2 * kBinThreads, "two bins per thread in the prefix");
    __shared__ int h[kBins];
    __shared__ int wsum[kBinThreads / 32], last;
    QueryState *st = b.st;
    for (int t = threadIdx.x; t < kBins; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const float thr = st->thr_scan;
    int64_t c0, c1;
    bin_chunk(st->n_cand, &c0, &c1);
    for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) atomicAdd(&h[bin_of(b.cand_lb[c], thr)], 1);
    __syncthreads();
    if (c1 > c0)
        for (int t = threadIdx.x; t < kBins; t += blockDim.x)
            if (h[t]) atomicAdd(&st->hist[t], h[t]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->bin_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // exclusive prefix over the bins: thread t holds bins 2t and 2t + 1
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int v0 = __ldcg(&st->hist[2 * t]), v1 = __ldcg(&st->hist[2 * t + 1]);
    const int v = v0 + v1;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int carry = 0;
    for (int q = 0; q < w; ++q) carry += wsum[q];
    const int base = carry + inc - v;
    st->bin_off[2 * t] = base;
    st->bin_off[2 * t + 1] = base + v0;
    if (t == 0) st->work2 = 0;
}

// Each CTA takes a contiguous chunk of the survivors, counts its bins in
// shared memory, reserves each bin's range with one global atomic, and
// scatters with shared-memory atomics (one global atomic per CTA and bin
// instead of one per survivor: with a loose bound tens of millions of
// survivors would otherwise queue on ~1000 addresses).  The order inside a
// bin is arbitrary; the DTW stage takes bins in order.
__global__ void __launch_bounds__(512) k_bin_scatter(QueryBufs b) {
    __shared__ int h[kBins];
    QueryState *st = b.st;
    const float thr = st->thr_scan;
    int64_t c0, c1;
    bin_chunk(st->n_cand, &c0, &c1);
    if (c1 <= c0) return;
    for (int t = threadIdx.x; t < kBins; t += blockDim.x) h[t] = 0;
    __syncthreads();
    for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) atomicAdd(&h[bin_of(b.cand_lb[c], thr)], 1);
    __syncthreads();
    for (int t = threadIdx.x; t < kBins; t += blockDim.x)
        if (h[t]) h[t] = atomicAdd(&st->bin_off[t], h[t]);
    __syncthreads();
    for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        const float lb = b.cand_lb[c];
        const int pos = atomicAdd(&h[bin_of(lb, thr)], 1);
        b.sort_lb[pos] = lb;
        b.sort_idx[pos] = b.cand_idx[c];
    }
}

cudaError_t launch_order(const QueryBufs &b, const QueryArgs &, cudaStream_t s) {
    int blocks = b.num_sms * 2;
    k_bin_hist<<<blocks, kBinThreads, 0, s>>>(b);
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
// keys: the result list (a.list_cap slots, ascending, empty keys last).
// Writes the windows to re-score to idx (the pre-scored window first: *skip
// of them, 0 or 1, are re-scored already), returns their count and sets
// *overflow when the list is full and its last entry is still inside the
// margin.
__device__ __forceinline__ int margin_select(const unsigned long long *keys, const QueryState *st, const QueryArgs &a,
                             unsigned *idx, int *skip, bool *overflow) {
    int count = 0;
    while (count < a.list_cap && keys[count] != kEmptyKey) ++count;
    *skip = 0;
    *overflow = false;
    if (count == 0) return 0;
    const float dk = key_dist(keys[(count < a.k ? count : a.k) - 1]);
    const float lim = fmaf(dk, 1.0f + a.delta, a.alpha);
    // the pre-scored window (side stream) goes first with its re-score
    const unsigned pre = st->pre_done ? prescored_window(st, a) : 0xffffffffu;
    int nm = 0;
    for (int j = 0; j < count; ++j)
        if (key_dist(keys[j]) <= lim && key_idx(keys[j]) == pre) idx[nm++] = pre;
    *skip = nm;
    for (int j = 0; j < count; ++j) {
        const unsigned w = key_idx(keys[j]);
        if (key_dist(keys[j]) <= lim && w != pre) idx[nm++] = w;
    }
    *overflow = count == a.list_cap && key_dist(keys[count - 1]) <= lim;
    return nm;
}

// The output: the k smallest (re-scored distance, offset) pairs of the nm
// entries, ascending; slots past nm get offset -1, distance +inf.
__device__ __forceinline__ void final_order(const unsigned *idx, const double *d64, int nm, const QueryArgs &a, int64_t *out_idx,
                            float *out_dist, int tid, int nthreads) {
    for (int t = tid; t < nm; t += nthreads) {
        const double d = d64[t];
        const unsigned w = idx[t];
        int rank = 0;
        for (int u = 0; u < nm; ++u) {
            const double du = d64[u];
            const unsigned iu = idx[u];
            rank += (du < d) || (du == d && iu < w);
        }
        if (rank < a.k) {
            out_idx[rank] = (int64_t)w;
            out_dist[rank] = (float)d;
        }
    }
    for (int u = nm + tid; u < a.k; u += nthreads) {
        out_idx[u] = -1;
        out_dist[u] = DINF;
    }
}

__global__ void k_final_select(QueryBufs b, QueryArgs a) {
    QueryState *st = b.st;
    if (threadIdx.x != 0) return;
    st->work = 0;
    st->margin_skip = 0;
    if (!st->valid) { st->n_margin = 0; return; }
    int skip = 0;
    bool ovf = false;
    const int nm = margin_select(st->res_keys, st, a, st->margin_idx, &skip, &ovf);
    for (int j = 0; j < skip; ++j) st->margin_d64[j] = st->pre_d64;
    st->margin_skip = skip;
    st->work = skip;
    if (ovf) atomicOr(b.status, kStOverflow);
    st->n_margin = nm;
    st->ctr[kCtrRescored] = (unsigned long long)nm;
}

// Top-k with an exclusion zone: the search's K best windows in (distance,
// offset) order are taken one by one, skipping any window within z samples
// of one already taken, until k are taken; the rest of the output (a series
// too short for k such windows) is offset -1, distance +inf.  K <= 64: one
// thread.
__global__ void k_exclusion_select(const int64_t *idx, const float *dist, int K, int k, int z, int64_t *out_idx,
                                   float *out_dist) {
    if (threadIdx.x != 0) return;
    int64_t taken[kKMax];
    int n = 0;
    for (int j = 0; j < K && n < k; ++j) {
        const int64_t i = idx[j];
        if (i < 0) continue;
        bool ok = true;
        for (int t = 0; t < n; ++t) {
            const int64_t d = taken[t] - i;
            if (d <= z && d >= -z) {
                ok = false;
                break;
            }
        }
        if (!ok) continue;
        taken[n] = i;
        out_idx[n] = i;
        out_dist[n] = dist[j];
        ++n;
    }
    for (; n < k; ++n) {
        out_idx[n] = -1;
        out_dist[n] = __int_as_float(0x7f800000);
    }
}

cudaError_t launch_exclusion_select(const int64_t *idx, const float *dist, int K, int k, int z, int64_t *out_idx,
                                    float *out_dist, cudaStream_t s) {
    if (K > kKMax || k > kKMax) return cudaErrorInvalidValue;
    k_exclusion_select<<<1, 32, 0, s>>>(idx, dist, K, k, z, out_idx, out_dist);
    return cudaGetLastError();
}

__global__ void k_final_sort(QueryBufs b, QueryArgs a, int64_t *out_idx, float *out_dist) {
    QueryState *st = b.st;
    final_order(st->margin_idx, st->margin_d64, st->valid ? st->n_margin : 0, a, out_idx, out_dist, threadIdx.x,
                blockDim.x);
}

// One launch when the re-score takes the multi-warp walk (it then selects
// and orders too); otherwise select, re-score, order.  *launches: how many.
cudaError_t launch_finalize(const QueryBufs &b, const QueryArgs &a, int64_t *out_idx,
                            float *out_dist, cudaStream_t s, int *launches) {
    *launches = 1;
    cudaError_t e = dtw64_dispatch(b, a, nullptr, 0, nullptr, kListMax, s, FinalOut{out_idx, out_dist});
    if (e != cudaErrorNotSupported) return e;
    cudaGetLastError();
    *launches = 3;
    k_final_select<<<1, 32, 0, s>>>(b, a);
    e = dtw64_dispatch(b, a, nullptr, 0, nullptr, kListMax, s, FinalOut{});
    if (e != cudaSuccess) return e;
    k_final_sort<<<1, kListMax, 0, s>>>(b, a, out_idx, out_dist);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ wide exclusion zone
// The end of a search with a wide exclusion zone z.  Every window whose FP32
// DTW was within the threshold when it was computed is in the candidate
// buffer; the final threshold (the smaller k-th of the bucket lists, with
// the margin) bounds the answer's k-th distance, so the windows of the
// answer, and every window that could shut one of them out, are among the
// buffer's windows within it.  Those are re-scored in extended precision,
// ordered by (re-scored distance, offset) and taken greedily, skipping any
// window within z samples of one already taken -- the definition of the
// answer, applied to a superset of its windows.
__global__ void __launch_bounds__(1024) k_xz_compact(QueryBufs b, QueryArgs a) {
    QueryState *st = b.st;
    __shared__ int cnt;
    if (threadIdx.x == 0) {
        cnt = 0;
        st->work = 0;
    }
    __syncthreads();
    if (!st->valid) {
        if (threadIdx.x == 0) st->xz_nsel = 0;
        return;
    }
    const float thr = current_thr(st, a);
    const int n = min(st->xz_count, b.xz_cap);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long key = b.xz_buf[i];
        if (key_dist(key) <= thr) {
            const int j = atomicAdd(&cnt, 1);
            if (j < b.xz_sel_cap) b.xz_sel[j] = key_idx(key);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st->xz_nsel = cnt;
        if (cnt > b.xz_sel_cap) atomicOr(b.status, kStOverflow);  // answers may be inexact
        st->ctr[kCtrRescored] = (unsigned long long)min(cnt, b.xz_sel_cap);
    }
}

// Sort the re-scored candidates by (distance, offset) in shared memory
// (bitonic, padded to a power of two), then one warp takes them greedily.
__global__ void __launch_bounds__(1024) k_xz_select(QueryBufs b, QueryArgs a, int64_t *out_idx, float *out_dist) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ unsigned taken[kKMax];
    __shared__ float takend[kKMax];
    QueryState *st = b.st;
    const int n = st->valid ? min(st->xz_nsel, b.xz_sel_cap) : 0;
    int P = 1;
    while (P < n) P <<= 1;
    int Pmax = 1;
    while (Pmax < b.xz_sel_cap) Pmax <<= 1;
    double *sd = (double *)smraw;
    unsigned *so = (unsigned *)(sd + Pmax);
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        sd[j] = j < n ? b.xz_d64[j] : __longlong_as_double(0x7ff0000000000000ll);
        so[j] = j < n ? b.xz_sel[j] : 0xffffffffu;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const double d0 = sd[lo], d1 = sd[hi];
                const unsigned o0 = so[lo], o1 = so[hi];
                const bool gt = d0 > d1 || (d0 == d1 && o0 > o1);
                if (gt == asc) {
                    sd[lo] = d1;
                    sd[hi] = d0;
                    so[lo] = o1;
                    so[hi] = o0;
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    int nt = 0;
    for (int j = 0; j < n && nt < a.k; ++j) {
        const unsigned o = so[j];
        if (j > 0 && so[j - 1] == o) continue;  // the same window twice
        bool near = false;
        for (int t = lane; t < nt; t += 32) {
            const long long dd = (long long)taken[t] - (long long)o;
            near |= (dd < 0 ? -dd : dd) <= a.xz_z;
        }
        if (__any_sync(0xffffffffu, near)) continue;
        if (lane == 0) {
            taken[nt] = o;
            takend[nt] = (float)sd[j];
        }
        ++nt;
        __syncwarp();
    }
    for (int t = lane; t < a.k; t += 32) {
        out_idx[t] = t < nt ? (int64_t)taken[t] : -1;
        out_dist[t] = t < nt ? takend[t] : DINF;
    }
}

cudaError_t launch_xz_finalize(const QueryBufs &b, const QueryArgs &a, int64_t *out_idx, float *out_dist,
                               cudaStream_t s) {
    k_xz_compact<<<1, 1024, 0, s>>>(b, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = dtw64_dispatch(b, a, nullptr, 0, nullptr, b.xz_sel_cap, s, FinalOut{});
    if (e != cudaSuccess) return e;
    int Pmax = 1;
    while (Pmax < b.xz_sel_cap) Pmax <<= 1;
    const size_t smem = (size_t)Pmax * 12;
    e = cudaFuncSetAttribute(k_xz_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_xz_select<<<1, 1024, smem, s>>>(b, a, out_idx, out_dist);
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
