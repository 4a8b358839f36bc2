// dtw_kernels.cuh -- the FP32 banded-DTW kernel of the search (Sec. 2.1,
// Eq. 1 with the Sakoe-Chiba band) in its three modes, its shared-memory
// layout and the choice of kernel shape.  Each mode is instantiated in its
// own translation unit (dtw_seed.cu, dtw_surv.cu, dtw_out.cu) so that the
// unrolled walks of every shape compile in parallel.
#pragma once

#include <cmath>
#include <type_traits>
#include <utility>

#include "dtw_band.cuh"
#include "dtws_internal.h"

#ifndef DINF
#define DINF __int_as_float(0x7f800000)
#endif

namespace dtws {

// the multi-warp FP32 kernel for bands past one warp (k_dtw_mw below): four
// warps per candidate, up to 16 cells per lane
constexpr int kWideW = 4;
constexpr int kWideRMax = 32 * kWideW * 16 - 1;  // 2047

// Bin of a survivor's lower bound for the counting sort (see launch_order):
// with a finite scan threshold the bins split [0, thr] evenly; otherwise
// they follow the float's exponent and leading mantissa bits (monotone for
// lb >= 0).
__device__ __forceinline__ int bin_of(float lb, float thr) {
    if (thr < DINF) {
        int bn = (int)(lb * ((float)kBins / thr));
        return bn < 0 ? 0 : (bn >= kBins ? kBins - 1 : bn);
    }
    return (int)(__float_as_uint(lb) >> 21);
}

// A value that every bound in bins >= k (bin_of with the same thr) is at
// least: the bin's lower edge, lowered by 2^-20 to cover the rounding of the
// product in bin_of.
__device__ __forceinline__ float bin_floor(int k, float thr) {
    if (thr < DINF) return ((float)k / ((float)kBins / thr)) * (1.0f - 9.5367431640625e-07f);
    return __uint_as_float((unsigned)k << 21);
}

// ------------------------------------------------------------------ DTW kernels
enum DtwMode { kModeSeed = 0, kModeSurv = 1, kModeOut = 2 };

// Shared memory of a DTW CTA: the query [pad + m + pad] then, per group,
// its staged normalised window [pad + m + pad] (when staged), the rows' tail
// bound [m4 + 4] (FP32; anti-diagonal kernel with abandon) and the ring
// [W + 1] (row-systolic kernel, K == 0).  pad = diag_pad(r, L, K) for the
// anti-diagonal kernel, 0 for the row-systolic one.
template <typename T>
struct DtwSmem {
    int m, m4, W, pad;
    bool staged, tail, ring;
    __host__ __device__ size_t span() const { return (size_t)((m + 2 * pad + 3) & ~3); }
    // the coarse tail bound: tail_entries(m) floats, rounded up to 4
    __host__ __device__ size_t tail_bytes() const { return (size_t)((tail_entries(m) + 3) & ~3) * 4; }
    __host__ __device__ size_t group_bytes() const {
        return (staged ? span() * sizeof(T) : 0) + (tail ? tail_bytes() : 0) +
               (ring ? (size_t)(W + 1) * sizeof(T) : 0);
    }
    __host__ __device__ size_t q_bytes() const { return span() * sizeof(T); }
};

template <typename T, int L, int K>
__host__ __device__ inline DtwSmem<T> dtw_smem(int m, int r, bool staged, bool tail) {
    DtwSmem<T> d;
    d.m = m;
    d.m4 = (m + 3) & ~3;
    d.W = 2 * r + 1;
    d.pad = K > 0 ? diag_pad(r, L, K) : 0;
    d.staged = staged;
    d.tail = staged && tail && K > 0;
    d.ring = K == 0;
    return d;
}

// Fill [base, base + pad) and [base + pad + m, base + 2 pad + m) with v.
template <typename T>
__device__ __forceinline__ void fill_pads(T *base, int m, int pad, T v, int tid, int nthreads) {
    for (int t = tid; t < 2 * pad; t += nthreads) base[t < pad ? t : m + t] = v;
}

// FP32 DTW over a candidate list (MODE: seeds, survivors, or given offsets).
// Groups of L lanes pull candidates from a device cursor.  K > 0: the
// anti-diagonal kernel with K cells per lane (window staged in shared
// memory); K == 0: the row-systolic kernel (staged when it fits).
// Resident CTAs of 256 threads per SM that the FP32 DTW kernel is compiled
// for (its register bound): more for the short register windows, one for
// the widest, whose 4K window and cell registers need the whole budget.
__host__ __device__ constexpr int dtw_min_blocks(int K) {
    return (K >= 1 && K <= 2) ? 4 : (K >= 1 && K <= 4) ? 3 : (K >= 16) ? 1 : 2;
}

// The body of k_dtw for one query (the CTA's part of its candidate stream);
// the persistent batch stage (k_dtw_pool) runs it for one query after
// another.  In survivor mode with b.surv_mh set, the survivors' window
// statistics come from per-survivor arrays (indexed like sort_idx) instead
// of the per-window statistics; without it, a query whose survivors were
// handed to the persistent stage (st->deferred) is left to that stage.
template <int L, int K, int MODE>
__device__ __forceinline__ void dtw_body(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                                         int64_t count_host, float *out, int staged) {
    extern __shared__ __align__(16) unsigned char smraw[];
    QueryState *st = b.st;
    if (!st->valid) return;
    if (MODE == kModeSurv && b.surv_mh == nullptr && st->deferred) return;
    const int m = a.m, r = a.r;
    const bool has_env = b.U != nullptr || b.stmax != nullptr;
    const DtwSmem<float> lay = dtw_smem<float, L, K>(m, r, staged != 0, MODE == kModeSurv && has_env);
    const float INF = DINF;
    float *qbase = (float *)smraw, *qs = qbase + lay.pad;
    for (int t = threadIdx.x; t < m; t += blockDim.x) qs[t] = b.qh32[t];
    fill_pads(qbase, m, lay.pad, INF, threadIdx.x, blockDim.x);
    const int warp = threadIdx.x >> 5, ln = lane_id();
    const int g = ln / L, lane = ln % L;
    const int gid = warp * (32 / L) + g;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g * L));
    unsigned char *gbase = smraw + lay.q_bytes() + (size_t)gid * lay.group_bytes();
    float *cbuf = nullptr;
    if (lay.staged) {
        fill_pads((float *)gbase, m, lay.pad, -INF, lane, L);
        cbuf = (float *)gbase + lay.pad;
    }
    float *cbs = lay.tail ? (float *)(gbase + (lay.staged ? lay.span() * 4 : 0)) : nullptr;
    float *ring = lay.ring ? (float *)(gbase + (lay.staged ? lay.span() * 4 : 0) +
                                       (lay.tail ? lay.tail_bytes() : 0))
                           : nullptr;
    // survivor pass: the seeds' offsets (already evaluated by the seed pass)
    // and the first 128 query positions in |q_hat| order with q_hat and the
    // query envelope there (the pre-check reads them for every candidate)
    __shared__ unsigned seeds_s[kSeedMax];
    __shared__ int n_seeds_s;
    __shared__ int ord_s[128];
    __shared__ float sq_s[128], su_s[128], sl_s[128];
    if (MODE == kModeSurv) {
        if (threadIdx.x == 0) n_seeds_s = st->n_seeds;
        for (int t = threadIdx.x; t < st->n_seeds; t += blockDim.x) seeds_s[t] = st->seed_off[t];
        for (int t = threadIdx.x; t < 128; t += blockDim.x) {
            const bool in = t < m;
            ord_s[t] = in ? (int)b.ord[t] : 0;
            sq_s[t] = in ? b.sq[t] : 0.0f;
            su_s[t] = in ? b.sU[t] : 0.0f;
            sl_s[t] = in ? b.sL[t] : 0.0f;
        }
    }
    __syncthreads();
    int *cursor = MODE == kModeSurv ? &st->work2 : &st->work;
    const float thr_scan = MODE == kModeSurv ? st->thr_scan : 0.0f;
    const unsigned pre = MODE == kModeSurv ? prescored_window(st, a) : 0xffffffffu;
    const int64_t count = MODE == kModeSeed ? (int64_t)st->n_seeds
                        : MODE == kModeSurv ? (int64_t)st->n_cand : count_host;
    long long cells_acc = 0;
    int started = 0, abandoned = 0, passed_s = 0;
    // survivor pass, two schedules chosen per launch (the same for every
    // group): with many survivors (more than 64 per group) a group takes L
    // candidates per cursor step and each lane runs the pre-check (bin floor,
    // seeds, Eq. 10 and Eq. 8 with early abandon) for its own candidate, the
    // ones that pass then being scored one at a time by the whole group;
    // with fewer a group takes one candidate at a time and pre-checks it
    // cooperatively, L terms per step (shorter critical path when most of
    // them sit near the best match; measured on 1e8 windows, m = 512,
    // ~38,000 survivors over 4,864 groups: 54 us, against 117 us with each
    // group's 8 survivors pre-checked lane by lane, 61 us with each group
    // taking every groups-th survivor, the next one's offset loaded ahead
    // (the cursor balances the groups), 56 us with the survivors'
    // statistics gathered in order by the ordering kernel, and 59 us with
    // each group taking its next slot one candidate ahead).
    unsigned pend = 0, my_idx = 0;
    float my_mh = 0.0f, my_is = 0.0f, my_ls = 0.0f;
    bool stop = false;
    const unsigned lmask = L == 32 ? 0xffffffffu : ((1u << L) - 1u);
    const bool lanewise = MODE == kModeSurv && count > (int64_t)gridDim.x * (blockDim.x / L) * 64;
    while (true) {
        int c = 0, psrc = 0;
        unsigned idx;
        float lb = 0.0f;
        bool coop = false;  // the one-candidate schedule's cooperative pre-check is still due
        if (MODE == kModeSurv && lanewise) {
            if (!pend) {
                if (stop) break;
                int c0 = 0;
                if (lane == 0) c0 = atomicAdd(cursor, L);
                c0 = __shfl_sync(gmask, c0, 0, L);
                if (c0 >= count) break;
                const int cc = c0 + lane;
                const bool valid = cc < count;
                const unsigned id = valid ? b.sort_idx[cc] : 0u;
                const float lbv = valid ? b.sort_lb[cc] : DINF;
                float th = 0.0f;
                if (lane == 0) th = current_thr(st, a);
                th = __shfl_sync(gmask, th, 0, L);
                bool pass = valid && !(lbv > th);
                // survivors are in ascending bins and thr only shrinks: once a
                // candidate's bin floor is above thr, so is every later one's
                const bool done = valid && lbv > th && bin_floor(bin_of(lbv, thr_scan), thr_scan) > th;
                if (pass) {  // scored already: by the seed pass or on the side stream
                    bool seen = id == pre;
                    for (int t = 0; t < n_seeds_s; ++t) seen |= seeds_s[t] == id;
                    pass = !seen;
                }
                float pmh = 0.0f, pis = 0.0f, pls = 0.0f;
                if (pass && b.surv_mh) {
                    pmh = b.surv_mh[cc];
                    pis = b.surv_is[cc];
                    pls = b.surv_ls[cc];
                } else if (pass) {
                    pmh = b.mu_hi[id];
                    pis = b.inv_sigma[id];
                    pls = b.mu_lo[id] * pis;
                }
                if (pass && has_env) {
                    // Eq. 10 (q_hat against the window's envelope) and Eq. 8
                    // (the window against the query's envelope; the scan took
                    // only its first terms) with early abandon, terms in
                    // |q_hat| descending order until either partial sum passes
                    // thr -- each is a lower bound on its own (rows and
                    // columns of the same warping path).  Past 128 terms the
                    // full Eq. 10 below (row order, with the suffix sums the
                    // DTW needs) takes over.
                    TailCtx pc;
                    pc.Uw = b.U ? b.U + id : nullptr;
                    pc.Lw = b.L ? b.L + id : nullptr;
                    pc.stmax = b.stmax;
                    pc.stmin = b.stmin;
                    pc.nblk = b.nblk;
                    pc.n = b.n;
                    pc.t0 = id;
                    pc.r = r;
                    const float *xp = b.x + id;
                    const int budget = m < 128 ? m : 128;
                    float acc = 0.0f, acc8 = 0.0f;
                    // 8 terms per step: their loads are issued together, the
                    // abandon test runs once per step
                    constexpr int kB = 8;
                    for (int j0 = 0; j0 < budget; j0 += kB) {
                        float xv[kB], uv[kB], lv[kB];
#pragma unroll
                        for (int t = 0; t < kB; ++t) {
                            const int j = j0 + t < budget ? j0 + t : budget - 1;
                            const int pos = ord_s[j];
                            xv[t] = xp[pos];
                            env_at(pc, pos, uv[t], lv[t]);
                        }
#pragma unroll
                        for (int t = 0; t < kB; ++t) {
                            if (j0 + t >= budget) break;
                            const int j = j0 + t;
                            const float u = fmaf(uv[t] - pmh, pis, -pls), l = fmaf(lv[t] - pmh, pis, -pls);
                            const float q = sq_s[j];
                            const float dq = fmaxf(q - u, 0.0f) + fmaxf(l - q, 0.0f);
                            const float cv = fmaf(xv[t] - pmh, pis, -pls);
                            const float e = fmaxf(cv - su_s[j], 0.0f) + fmaxf(sl_s[j] - cv, 0.0f);
                            acc = fmaf(dq, dq, acc);
                            acc8 = fmaf(e, e, acc8);
                        }
                        if (acc > th || acc8 > th) {
                            pass = false;
                            break;
                        }
                    }
                }
                my_idx = id;
                my_mh = pmh;
                my_is = pis;
                my_ls = pls;
                const int gshift = (ln / L) * L;
                pend = (__ballot_sync(gmask, pass) >> gshift) & lmask;
                stop = ((__ballot_sync(gmask, done) >> gshift) & lmask) != 0u;
                continue;
            }
            psrc = __ffs(pend) - 1;
            pend &= pend - 1;
            idx = __shfl_sync(gmask, my_idx, psrc, L);
        } else {
            if (lane == 0) c = atomicAdd(cursor, 1);
            c = __shfl_sync(gmask, c, 0, L);
            if (c >= count) break;
            if (MODE == kModeSurv) {
                idx = b.sort_idx[c];
                lb = b.sort_lb[c];
                coop = true;
            }
        }
        if (MODE == kModeSeed) {
            idx = st->seed_off[c];
        } else if (MODE == kModeOut) {
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
            const float kth = list_kth(st->seed_keys, a.k);
            thr = kth < DINF ? fmaf(kth, 1.0f + a.delta, a.alpha) : DINF;
        } else if (MODE == kModeSurv) {
            thr = current_thr(st, a);
        }
        thr = __shfl_sync(gmask, thr, 0, L);
        if (coop) {
            if (lb > thr) {
                // see the batch schedule: past this bin floor nothing is left
                if (bin_floor(bin_of(lb, thr_scan), thr_scan) > thr) break;
                continue;
            }
            bool seen = idx == pre;  // scored already: by the seed pass or on the side stream
            for (int t = lane; t < n_seeds_s; t += L) seen |= seeds_s[t] == idx;
            if (__any_sync(gmask, seen)) continue;
        }
        float mh, is, ls;
        if (MODE == kModeSurv && !coop) {  // pre-checked by its lane: take its statistics
            mh = __shfl_sync(gmask, my_mh, psrc, L);
            is = __shfl_sync(gmask, my_is, psrc, L);
            ls = __shfl_sync(gmask, my_ls, psrc, L);
        } else if (MODE == kModeSurv && b.surv_mh) {
            mh = b.surv_mh[c];
            is = b.surv_is[c];
            ls = b.surv_ls[c];
        } else {
            mh = b.mu_hi[idx];
            is = b.inv_sigma[idx];
            ls = b.mu_lo[idx] * is;
        }
        const float *xw = b.x + idx;
        TailCtx tc;
        tc.Uw = b.U ? b.U + idx : nullptr;
        tc.Lw = b.L ? b.L + idx : nullptr;
        tc.stmax = b.stmax;
        tc.stmin = b.stmin;
        tc.nblk = b.nblk;
        tc.n = b.n;
        tc.t0 = idx;
        tc.r = r;
        tc.qs = qs;
        tc.mh = mh;
        tc.is = is;
        tc.ls = ls;
        if (coop && has_env) {
            // the same pre-check as the batch schedule's, L terms per step
            // over the group (the sums are reduced, so every lane takes the
            // same exit)
            float acc = 0.0f, acc8 = 0.0f;
            bool pruned = false;
            const int budget = m < 128 ? m : 128;
            for (int c0 = 0; c0 < budget; c0 += L) {
                const int j = c0 + lane;
                float v = 0.0f, v8 = 0.0f;
                if (j < budget) {
                    const int pos = ord_s[j];
                    const float x = xw[pos];
                    float U, Lo;
                    env_at(tc, pos, U, Lo);
                    const float u = fmaf(U - mh, is, -ls), l = fmaf(Lo - mh, is, -ls), q = sq_s[j];
                    const float dq = fmaxf(q - u, 0.0f) + fmaxf(l - q, 0.0f);
                    v = dq * dq;
                    const float cv = fmaf(x - mh, is, -ls);
                    const float e = fmaxf(cv - su_s[j], 0.0f) + fmaxf(sl_s[j] - cv, 0.0f);
                    v8 = e * e;
                }
#pragma unroll
                for (int o = L / 2; o > 0; o >>= 1) {
                    v += __shfl_xor_sync(gmask, v, o, L);
                    v8 += __shfl_xor_sync(gmask, v8, o, L);
                }
                acc += v;
                acc8 += v8;
                if (acc > thr || acc8 > thr) {
                    pruned = true;
                    break;
                }
            }
            if (pruned) continue;
        }
        if (cbuf) {  // the group's normalised copy of the window
            for (int j = lane; j < m; j += L) cbuf[j] = fmaf(xw[j] - mh, is, -ls);
        }
        if (cbs) {
            tail_suffix<L>(tc, cbs, m, gmask, lane);
            // cbs[0] is LB_Keogh of q_hat against the window's envelope
            // (Eq. 10 with the series-wide envelope): the third bound
            if (cbs[0] > thr) continue;
            if (lane == 0) ++passed_s;
        }
        __syncwarp(gmask);
        int cells = 0;
        float d;
        if constexpr (K == 0) {
            if (MODE == kModeOut)
                d = dtw_band<float, L, false>(qs, xw, cbuf, mh, is, ls, nullptr, ring, m, r, thr, gmask, lane,
                                              cells);
            else
                d = dtw_band<float, L, true>(qs, xw, cbuf, mh, is, ls,
                                             (has_env && MODE == kModeSurv) ? &tc : nullptr, ring, m, r, thr,
                                             gmask, lane, cells);
        } else {
            if (MODE == kModeOut)
                d = dtw_diag<float, L, K, false>(qs, cbuf, nullptr, m, r, thr, gmask, lane, cells);
            else
                d = dtw_diag<float, L, K, true>(qs, cbuf, cbs, m, r, thr, gmask, lane, cells);
        }
        cells_acc += cells;
        if (lane == 0) {
            ++started;
            if (!(d < DINF)) ++abandoned;
            if (MODE == kModeOut) out[c] = d;
            else if (MODE == kModeSeed) {
                if (d < DINF) {
                    // a finished seed is also a result candidate; the survivor
                    // pass skips the seeds, so each window enters once
                    const unsigned long long key = make_key(key_quantize(d, a.qgrid), idx);
                    list_insert(st->seed_keys, a.k, key);
                    list_insert(st->res_keys, a.list_cap, key);
                }
            } else if (d <= thr) {
                const unsigned long long key = make_key(key_quantize(d, a.qgrid), idx);
                list_insert(st->res_keys, a.list_cap, key);
                if (a.xz_z > 0) xz_offer(b, a, key, true);
            }
        }
        __syncwarp(gmask);
    }
    if (MODE != kModeOut) {
        // counters: one atomic per warp
        unsigned long long cs = (unsigned long long)cells_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
        int ns = started, na = abandoned, np = passed_s;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ns += __shfl_xor_sync(0xffffffffu, ns, o);
            na += __shfl_xor_sync(0xffffffffu, na, o);
            np += __shfl_xor_sync(0xffffffffu, np, o);
        }
        if (ln == 0) {
            atomicAdd(&st->ctr[kCtrCells], cs);
            atomicAdd(&st->ctr[kCtrDtwStarted], (unsigned long long)ns);
            atomicAdd(&st->ctr[kCtrDtwAbandoned], (unsigned long long)na);
            if (np) atomicAdd(&st->ctr[kCtrKeoghS], (unsigned long long)np);
        }
    }
}

template <int L, int K, int MODE>
__global__ void __launch_bounds__(256, dtw_min_blocks(K)) k_dtw(QueryBufs b, QueryArgs a, const int64_t *offsets,
                                                              int64_t count_host, float *out, int staged) {
    dtw_body<L, K, MODE>(b, a, offsets, count_host, out, staged);
}

// The persistent survivor-DTW stage of a batch (one launch per kernel shape
// in the batch): every CTA walks the list of the shape's deferred queries in
// order and runs the survivor pass of each with the others, pulling that
// query's survivors from its cursor; a CTA whose share of one query is done
// moves on to the next at once, so no launch boundary or tail separates the
// queries.  base: the series, envelopes and status of the handle, with
// sort_idx / sort_lb / surv_* pointing at the survivor pool (each query's
// survivors at st->pool_off).
template <int L, int K>
__global__ void __launch_bounds__(256, dtw_min_blocks(K)) k_dtw_pool(QueryBufs base, const PoolQuery *pq,
                                                                   const int *list, int nlist, int staged) {
    for (int j = 0; j < nlist; ++j) {
        const PoolQuery &p = pq[list[j]];
        QueryState *st = p.st;
        if (!st->deferred) continue;
        const long long off = st->pool_off;
        QueryBufs b = base;
        b.st = st;
        b.qh32 = p.qh32;
        b.ord = p.ord;
        b.sq = p.sq;
        b.sU = p.sU;
        b.sL = p.sL;
        b.U = p.U;
        b.L = p.L;
        b.sort_idx = base.sort_idx + off;
        b.sort_lb = base.sort_lb + off;
        b.surv_mh = base.surv_mh + off;
        b.surv_is = base.surv_is + off;
        b.surv_ls = base.surv_ls + off;
        const QueryArgs a = p.a;
        dtw_body<L, K, kModeSurv>(b, a, nullptr, 0, nullptr, staged);
        __syncthreads();  // shared copies of this query are read before the next query's are written
    }
}

// Shape of the double-float re-score walk.
template <int L, int K>
struct PreShape {
    // the double-float walk for the FP32 walk's shape (L lanes, K cells):
    // one warp with the same cells per lane up to 4 (no exchange between
    // warps at each step), four warps beyond, the r+1 <= L*K cells spread
    // over them
    static constexpr int W = (L < 32 || K <= 4) ? 1 : 4;
    static constexpr int K2 = (L < 32) ? 1 : (K <= 4 ? K : (K * 32 + 127) / 128);
};
__host__ __device__ inline size_t pre_span(int m, int r, int lanes, int k) {
    return (size_t)((m + 2 * diag_pad(r, lanes, k) + 3) & ~3);
}

// Kernel choice and CTA shape.  The anti-diagonal kernel (K > 0) is used
// when r <= kDiagRMax and one warp's groups can stage their windows;
// otherwise the row-systolic kernel (K == 0), staged when it fits.  Warps
// per CTA shrink until the CTA fits in ~100 KB (two CTAs per SM).
struct DtwPlan {
    int L, K, staged, warps;
    size_t smem;
};

template <typename T, int L, int K>
static bool plan_fits(int m, int r, bool tail, DtwPlan *p) {
    // as many resident CTAs per SM as the kernel's register bound allows
    // (dtw_min_blocks), each within its share of the SM's shared memory
    const size_t per_sm = (size_t)(sizeof(T) == 4 ? 224 / dtw_min_blocks(K) : 100);
    const size_t budget = (per_sm < 200 ? per_sm : 200) * 1024, hard = 200 * 1024;
    for (int staged = 1; staged >= (K > 0 ? 1 : 0); --staged) {
        const DtwSmem<T> lay = dtw_smem<T, L, K>(m, r, staged != 0, tail);
        auto total = [&](int w) { return lay.q_bytes() + (size_t)w * (32 / L) * lay.group_bytes(); };
        int warps = 8;
        while (warps > 1 && total(warps) > budget) --warps;
        if (total(warps) <= hard) {
            *p = DtwPlan{L, K, staged, warps, total(warps)};
            return true;
        }
    }
    return false;
}

// A given shape (K > 0: anti-diagonal with L*K >= r+1 lanes' cells; K == 0:
// row-systolic with lanes_for(r) lanes) if it is instantiated and fits;
// warps <= 0 keeps the largest count within the shared-memory budget.
template <typename T>
static bool plan_shape(int m, int r, bool tail, int L, int K, int warps, DtwPlan *p) {
    if (K > 0 && (r > kDiagRMax || L * K < r + 1)) return false;
    if (K == 0 && L != lanes_for(r)) return false;
    bool ok = false;
#define DTWS_TRY(LL, KK) \
    if (!ok && L == LL && K == KK) ok = plan_fits<T, LL, KK>(m, r, tail, p);
    DTWS_TRY(1, 1) DTWS_TRY(2, 1) DTWS_TRY(4, 1) DTWS_TRY(8, 1) DTWS_TRY(16, 1)
    DTWS_TRY(4, 2) DTWS_TRY(8, 2) DTWS_TRY(16, 2) DTWS_TRY(8, 4) DTWS_TRY(16, 4)
    DTWS_TRY(32, 1) DTWS_TRY(32, 2) DTWS_TRY(32, 3) DTWS_TRY(32, 4) DTWS_TRY(32, 6) DTWS_TRY(32, 8) \
        DTWS_TRY(32, 10) DTWS_TRY(32, 12) DTWS_TRY(32, 16)
    DTWS_TRY(1, 0) DTWS_TRY(2, 0) DTWS_TRY(4, 0) DTWS_TRY(8, 0) DTWS_TRY(16, 0) DTWS_TRY(32, 0)
#undef DTWS_TRY
    if (!ok) return false;
    // fewer warps than the budget allows: the allocation for more groups
    // stays valid (each group addresses only its own slice)
    if (warps > 0 && warps < p->warps) p->warps = warps;
    return true;
}

template <typename T>
static bool plan_dtw(int m, int r, bool tail, DtwPlan *p) {
    if (r <= kDiagRMax) {
        int L, K;
        if (std::is_same<T, float>::value) diag_shape_f32(r, &L, &K);
        else diag_shape(r, &L, &K);
#define DTWS_TRY(LL, KK) \
    if (L == LL && K == KK && plan_fits<T, LL, KK>(m, r, tail, p)) return true;
        DTWS_TRY(1, 1) DTWS_TRY(2, 1) DTWS_TRY(4, 1) DTWS_TRY(8, 1) DTWS_TRY(16, 1)
        if (std::is_same<T, float>::value) {
            DTWS_TRY(4, 2) DTWS_TRY(8, 2) DTWS_TRY(16, 2)
        }
        DTWS_TRY(32, 1) DTWS_TRY(32, 2) DTWS_TRY(32, 3) DTWS_TRY(32, 4) DTWS_TRY(32, 6) DTWS_TRY(32, 8) \
        DTWS_TRY(32, 10) DTWS_TRY(32, 12) DTWS_TRY(32, 16)
#undef DTWS_TRY
    }
    // (FP32 bands kDiagRMax < r <= kWideRMax go to the multi-warp kernel,
    // dtw_wide_launch; the row-systolic kernel below takes the rest)
    const int L = lanes_for(r);
#define DTWS_TRY(LL) \
    if (L == LL) return plan_fits<T, LL, 0>(m, r, tail, p);
    DTWS_TRY(1) DTWS_TRY(2) DTWS_TRY(4) DTWS_TRY(8) DTWS_TRY(16) DTWS_TRY(32)
#undef DTWS_TRY
    return false;
}

inline int dtw_blocks(const DtwPlan &p, int num_sms, int64_t count) {
    const int groups = p.warps * (32 / p.L);
    int64_t want = (count + groups - 1) / groups;
    const int64_t cap = (int64_t)num_sms * 4;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

// Launch of the wide-band kernel for one mode (instantiated in dtw_wide.cu).
template <int MODE>
cudaError_t dtw_wide_launch(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets, int64_t count,
                            float *out, int64_t count_for_grid, cudaStream_t s);
template <int MODE>
static cudaError_t dtw_dispatch(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                                int64_t count, float *out, int64_t count_for_grid, cudaStream_t s) {
    DtwPlan p;
    const bool tail = MODE == kModeSurv && (b.U != nullptr || b.stmax != nullptr);
    const bool tuned = a.tune_l > 0 && plan_shape<float>(a.m, a.r, tail, a.tune_l, a.tune_k, a.tune_w, &p);
    if constexpr (MODE == kModeOut) {
        // DTW at given offsets: every walk runs to its end, so the grid's
        // throughput counts, not one walk's latency -- four cells per lane
        // (half as many shuffles, rotations and band checks per cell as two)
        // for bands of 9 to 64 cells; the same cells, the same values
        const int need = a.r + 1;
        if (!tuned && need > 8 && need <= 64) {
            const bool fit = need <= 32 ? plan_fits<float, 8, 4>(a.m, a.r, false, &p)
                                        : plan_fits<float, 16, 4>(a.m, a.r, false, &p);
            if (fit) {
                const int blocks = dtw_blocks(p, b.num_sms, count_for_grid);
                cudaError_t e;
                if (p.L == 8) {
                    e = cudaFuncSetAttribute(k_dtw<8, 4, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)p.smem);
                    if (e == cudaSuccess)
                        k_dtw<8, 4, MODE><<<blocks, p.warps * 32, p.smem, s>>>(b, a, offsets, count, out, p.staged);
                } else {
                    e = cudaFuncSetAttribute(k_dtw<16, 4, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)p.smem);
                    if (e == cudaSuccess)
                        k_dtw<16, 4, MODE><<<blocks, p.warps * 32, p.smem, s>>>(b, a, offsets, count, out, p.staged);
                }
                return e != cudaSuccess ? e : cudaGetLastError();
            }
        }
    }
    if (!tuned && a.r > kDiagRMax && a.r <= kWideRMax)
        return dtw_wide_launch<MODE>(b, a, offsets, count, out, count_for_grid, s);
    if (!tuned && !plan_dtw<float>(a.m, a.r, tail, &p)) return cudaErrorInvalidValue;
    const int blocks = dtw_blocks(p, b.num_sms, count_for_grid);
#define DTWS_CASE(LL, KK)                                                                                     \
    if (p.L == LL && p.K == KK) {                                                                             \
        cudaError_t e = cudaFuncSetAttribute(k_dtw<LL, KK, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)p.smem);                                                    \
        if (e != cudaSuccess) return e;                                                                       \
        k_dtw<LL, KK, MODE><<<blocks, p.warps * 32, p.smem, s>>>(b, a, offsets, count, out, p.staged);        \
        return cudaGetLastError();                                                                            \
    }
    DTWS_CASE(1, 1) DTWS_CASE(2, 1) DTWS_CASE(4, 1) DTWS_CASE(8, 1) DTWS_CASE(16, 1)
    DTWS_CASE(4, 2) DTWS_CASE(8, 2) DTWS_CASE(16, 2) DTWS_CASE(8, 4) DTWS_CASE(16, 4)
    DTWS_CASE(32, 1) DTWS_CASE(32, 2) DTWS_CASE(32, 3) DTWS_CASE(32, 4) DTWS_CASE(32, 6) DTWS_CASE(32, 8) \
    DTWS_CASE(32, 10) DTWS_CASE(32, 12) DTWS_CASE(32, 16)
    DTWS_CASE(1, 0) DTWS_CASE(2, 0) DTWS_CASE(4, 0) DTWS_CASE(8, 0) DTWS_CASE(16, 0) DTWS_CASE(32, 0)
#undef DTWS_CASE
    return cudaErrorInvalidValue;
}


// ------------------------------------------------------------------ wide bands
// The FP32 DTW kernel for bands past the one-warp walks (kDiagRMax < r <=
// 2047): a group of W = 4 warps per candidate (dtw_diag_mw, K cells per
// lane, 128 K >= r + 1), two groups per CTA of 256 threads (one when the
// copies do not fit).  The same three modes and the same per-candidate
// steps as k_dtw (one candidate at a time per group, the pre-check of the
// survivor mode over the group's 128 threads); group decisions come from
// values every thread of the group reads after the group's barrier, so all
// its threads take the same branches.

__host__ __device__ inline int wide_k(int r) {
    const int need = (r + 1 + 32 * kWideW - 1) / (32 * kWideW);
    return need <= 6 ? 6 : need <= 8 ? 8 : need <= 12 ? 12 : 16;
}
__host__ __device__ inline size_t wide_span(int m, int r, int K) {
    return (size_t)((m + 2 * diag_pad(r, 32 * kWideW, K) + 3) & ~3);
}
__host__ __device__ inline size_t wide_tail(int m) { return (size_t)((tail_entries(m) + 3) & ~3); }

template <int W, int K, int MODE>
__global__ void __launch_bounds__(256, 2) k_dtw_mw(QueryBufs b, QueryArgs a, const int64_t *offsets,
                                                   int64_t count_host, float *out) {
    constexpr int GMAX = 8 / W;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ MwXchg xch[GMAX];
    __shared__ int cur_s[GMAX][2];
    __shared__ float thr_s[GMAX][2];
    __shared__ unsigned seeds_s[kSeedMax];
    __shared__ int n_seeds_s;
    __shared__ int ord_s[128];
    __shared__ float sq_s[128], su_s[128], sl_s[128];
    QueryState *st = b.st;
    if (!st->valid) return;
    const int m = a.m, r = a.r;
    const bool has_env = MODE == kModeSurv && (b.U != nullptr || b.stmax != nullptr);
    const int G = (int)(blockDim.x / (32 * W));
    const int pad = diag_pad(r, 32 * W, K);
    const size_t span = wide_span(m, r, K), tailn = wide_tail(m);
    float *qs = (float *)smraw + pad;
    for (int t = threadIdx.x; t < m; t += blockDim.x) qs[t] = b.qh32[t];
    fill_pads((float *)smraw, m, pad, DINF, threadIdx.x, blockDim.x);
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const int g = warp / W, w = warp % W, t = w * 32 + lane;
    const int nthr = 32 * W, bar = 1 + g;
    float *gbase = (float *)smraw + span + (size_t)g * (span + tailn);
    float *cd = gbase + pad;
    float *cbs = gbase + span;
    if (g < G) fill_pads(gbase, m, pad, -DINF, t, nthr);
    if (MODE == kModeSurv) {
        if (threadIdx.x == 0) n_seeds_s = st->n_seeds;
        for (int i = threadIdx.x; i < st->n_seeds; i += blockDim.x) seeds_s[i] = st->seed_off[i];
        for (int i = threadIdx.x; i < 128; i += blockDim.x) {
            const bool in = i < m;
            ord_s[i] = in ? (int)b.ord[i] : 0;
            sq_s[i] = in ? b.sq[i] : 0.0f;
            su_s[i] = in ? b.sU[i] : 0.0f;
            sl_s[i] = in ? b.sL[i] : 0.0f;
        }
    }
    __syncthreads();
    if (g >= G) return;
    int *cursor = MODE == kModeSurv ? &st->work2 : &st->work;
    const float thr_scan = MODE == kModeSurv ? st->thr_scan : 0.0f;
    const unsigned pre = MODE == kModeSurv ? prescored_window(st, a) : 0xffffffffu;
    const int64_t count = MODE == kModeSeed ? (int64_t)st->n_seeds
                        : MODE == kModeSurv ? (int64_t)st->n_cand : count_host;
    long long cells_acc = 0;
    int started = 0, abandoned = 0, passed_s = 0;
    int cells = 0;
    for (int it = 0;; it ^= 1) {
        // cur_s / thr_s alternate between two slots: a slot is written again
        // only after the next iteration's barrier, which every thread of the
        // group reaches after reading it
        if (t == 0) {
            cur_s[g][it] = atomicAdd(cursor, 1);
            float th = DINF;
            if (MODE == kModeSeed) {
                const float kth = list_kth(st->seed_keys, a.k);
                th = kth < DINF ? fmaf(kth, 1.0f + a.delta, a.alpha) : DINF;
            } else if (MODE == kModeSurv) {
                th = current_thr(st, a);
            }
            thr_s[g][it] = th;
        }
        group_bar(bar, nthr);
        const int c = cur_s[g][it];
        if (c >= count) break;
        const float thr = thr_s[g][it];
        unsigned idx = 0;
        if (MODE == kModeSeed) {
            idx = st->seed_off[c];
        } else if (MODE == kModeOut) {
            const int64_t o = offsets[c];
            if (o < 0 || o >= a.N) {
                if (t == 0) out[c] = __int_as_float(0x7fc00000);
                continue;
            }
            idx = (unsigned)o;
        } else {
            idx = b.sort_idx[c];
            const float lb = b.sort_lb[c];
            if (lb > thr) {
                // survivors are in ascending bins and thr only shrinks
                if (bin_floor(bin_of(lb, thr_scan), thr_scan) > thr) break;
                continue;
            }
            bool seen = idx == pre;  // scored already: by the seed pass or on the side stream
            for (int i = 0; i < n_seeds_s; ++i) seen |= seeds_s[i] == idx;
            if (seen) continue;
        }
        const float mh = b.mu_hi[idx], is = b.inv_sigma[idx], ls = b.mu_lo[idx] * is;
        const float *xw = b.x + idx;
        TailCtx tc;
        tc.Uw = b.U ? b.U + idx : nullptr;
        tc.Lw = b.L ? b.L + idx : nullptr;
        tc.stmax = b.stmax;
        tc.stmin = b.stmin;
        tc.nblk = b.nblk;
        tc.n = b.n;
        tc.t0 = idx;
        tc.r = r;
        tc.qs = qs;
        tc.mh = mh;
        tc.is = is;
        tc.ls = ls;
        if (has_env) {
            // Eq. 10 and Eq. 8 over the 128 largest-|q_hat| rows (one pass:
            // 128 threads, one term each), reduced over the group
            const int budget = m < 128 ? m : 128;
            float v = 0.0f, v8 = 0.0f;
            for (int j = t; j < budget; j += nthr) {
                const int pos = ord_s[j];
                float U, Lo;
                env_at(tc, pos, U, Lo);
                const float u = fmaf(U - mh, is, -ls), l = fmaf(Lo - mh, is, -ls), q = sq_s[j];
                const float dq = fmaxf(q - u, 0.0f) + fmaxf(l - q, 0.0f);
                v = fmaf(dq, dq, v);
                const float cv = fmaf(xw[pos] - mh, is, -ls);
                const float e = fmaxf(cv - su_s[j], 0.0f) + fmaxf(sl_s[j] - cv, 0.0f);
                v8 = fmaf(e, e, v8);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v += __shfl_xor_sync(0xffffffffu, v, o);
                v8 += __shfl_xor_sync(0xffffffffu, v8, o);
            }
            if (lane == 0) {
                xch[g].red[0][w] = v;
                xch[g].red[1][w] = v8;
            }
            group_bar(bar, nthr);
            float acc = 0.0f, acc8 = 0.0f;
#pragma unroll
            for (int u = 0; u < W; ++u) {
                acc += xch[g].red[0][u];
                acc8 += xch[g].red[1][u];
            }
            if (acc > thr || acc8 > thr) continue;
        }
        for (int j = t; j < m; j += nthr) cd[j] = fmaf(xw[j] - mh, is, -ls);
        if (has_env) {
            // the coarse tail bound: kTailG-row sums, then a suffix scan by
            // the group's first warp
            const int ne = tail_entries(m);
            for (int gi = t; gi < ne - 1; gi += nthr) {
                float sum = 0.0f;
                const int i1 = (gi + 1) * kTailG < m ? (gi + 1) * kTailG : m;
                for (int i = gi * kTailG; i < i1; ++i) sum += tail_term(tc, i);
                cbs[gi] = sum;
            }
            group_bar(bar, nthr);
            if (w == 0) {
                float carry = 0.0f;
                for (int c0 = ((ne - 1 + 31) / 32 - 1) * 32; c0 >= 0; c0 -= 32) {
                    const int gi = c0 + lane;
                    float v = gi < ne - 1 ? cbs[gi] : 0.0f;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const float u = __shfl_down_sync(0xffffffffu, v, o);
                        if (lane + o < 32) v += u;
                    }
                    if (gi < ne - 1) cbs[gi] = carry + v;
                    carry += __shfl_sync(0xffffffffu, v, 0);
                }
                __syncwarp();
                const float slack = 1e-5f * carry;
                for (int gi = lane; gi < ne - 1; gi += 32) cbs[gi] = fmaxf(0.0f, cbs[gi] - slack);
                if (lane == 0) cbs[ne - 1] = 0.0f;
            }
        }
        group_bar(bar, nthr);
        if (has_env) {
            if (cbs[0] > thr) continue;  // Eq. 10 over every row
            if (t == 0) ++passed_s;
        }
        const float d = dtw_diag_mw<W, K, MODE != kModeOut>(qs, cd, has_env ? cbs : nullptr, m, r, thr, w, lane,
                                                            xch[g], bar, cells);
        if (t == 0) {
            ++started;
            if (!(d < DINF)) ++abandoned;
            if (MODE == kModeOut) {
                out[c] = d;
            } else if (MODE == kModeSeed) {
                if (d < DINF) {
                    const unsigned long long key = make_key(key_quantize(d, a.qgrid), idx);
                    list_insert(st->seed_keys, a.k, key);
                    list_insert(st->res_keys, a.list_cap, key);
                }
            } else if (d <= thr) {
                const unsigned long long key = make_key(key_quantize(d, a.qgrid), idx);
                list_insert(st->res_keys, a.list_cap, key);
                if (a.xz_z > 0) xz_offer(b, a, key, true);
            }
        }
    }
    cells_acc = cells;
    if (MODE != kModeOut && t == 0) {
        atomicAdd(&st->ctr[kCtrCells], (unsigned long long)cells_acc);
        atomicAdd(&st->ctr[kCtrDtwStarted], (unsigned long long)started);
        atomicAdd(&st->ctr[kCtrDtwAbandoned], (unsigned long long)abandoned);
        if (passed_s) atomicAdd(&st->ctr[kCtrKeoghS], (unsigned long long)passed_s);
    }
}


}  // namespace dtws
