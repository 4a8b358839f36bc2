// dtws_internal.h -- host-side launchers shared between the library's
// translation units.  Every launcher enqueues on `s` and returns the launch
// status; none synchronises.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dtws_common.cuh"

namespace dtws {

// Record the text returned by dtws_last_error_detail() (printf format).
void set_error_detail(const char *fmt, ...);

// ---- series level (series_kernels.cu)
cudaError_t launch_check_finite(const float *x, int64_t n, int *flag, unsigned *absmax, cudaStream_t s);
cudaError_t launch_fill(float *p, int64_t count, float v, int num_sms, cudaStream_t s);
// xe[j] = x[2j], j < count
cudaError_t launch_subsample(const float *x, int64_t count, float *xs, int num_sms, cudaStream_t s);
// pf: 4*n floats (P1 hi, P1 lo, P2 hi, P2 lo); bf: 5*nb floats (T1 hi, lo,
// T2 hi, lo, anchors); ok: nb flags; nb = ceil(n / kBlockB); maxabs: one
// word of scratch; scale: one float (the series' power-of-two scale)
cudaError_t launch_prefix(const float *x, int64_t n, float *pf, float *bf, int *ok, unsigned *maxabs,
                          float *scale, cudaStream_t s);
cudaError_t launch_window_stats(const float *x, int64_t n, int m, const float *pf, const float *bf,
                                const int *ok, const float *scale, float *mu_hi, float *mu_lo, float *inv_sigma,
                                float *smu_hi, float *sinv_sigma, int num_sms, cudaStream_t s);
cudaError_t launch_envelope(const float *x, int64_t n, int r, float *U, float *L, cudaStream_t s);
// block envelope: st = [max levels 0..kEnvLevels-1 | min levels], nblk floats each
cudaError_t launch_block_envelope(const float *x, int64_t n, float *st, int64_t nblk, cudaStream_t s);

// ---- query level (query_kernels.cu)
struct QueryBufs {
    QueryState *st;
    const float *x;              // padded series
    const float *x_sub;          // its every kProxyStride-th sample (the proxy scan's copy)
    const float *mu_hi, *mu_lo, *inv_sigma;  // window stats for m
    const float *smu_hi, *sinv_sigma;  // mean (high part) and 1/sigma of every kProxyStride-th window
    const float *U, *L;          // exact series envelope for r, or null:
    const float *stmax, *stmin;  // per-series block envelope (sparse table), used when U is null
    int64_t nblk, n;             // its blocks; series length
    float *qh32;                 // normalised query, FP32 [m]
    double *qh64;                // normalised query, FP64 [m]
    float *Uq, *Lq;              // query envelope [m]
    unsigned short *ord;         // query positions by |q_hat| descending [m]
    float *sq, *sU, *sL;         // q_hat, Uq, Lq in that order [m]
    float *cand_lb, *sort_lb;    // survivors [cap]
    unsigned int *cand_idx, *sort_idx;
    int *status;
    long long wait_ns;
    int num_sms;
    // survivor pass of the persistent batch stage: the survivors' window
    // statistics (mean high part, 1/sigma, mean low part * 1/sigma), indexed
    // like sort_idx; null elsewhere
    const float *surv_mh, *surv_is, *surv_ls;
    // wide exclusion zone (QueryArgs::xz_z > 0): the candidate buffer of
    // windows scored within the threshold, and the re-score list of those
    // within the final threshold (offsets, extended-precision distances)
    unsigned long long *xz_buf;
    unsigned *xz_sel;
    double *xz_d64;
    int xz_cap, xz_sel_cap;
};

// Offer a scored window (key: its quantised distance and offset) to the bucket
// list of its bucket's parity: offsets are cut into buckets of 2z+1, so
// windows in different buckets of one parity are more than 2z apart, and the
// list keeps the k smallest keys with at most one per bucket (a better window
// replaces its bucket's entry).  One thread at a time rewrites a list, under
// a spin lock bounded by wait_ns (on timeout the offer is dropped, which only
// loosens the bound, and DTWS_ETIMEOUT is recorded).  Readers take only the
// k-th entry, which changes by one 64-bit store, from one valid bound to a
// smaller valid one.  With `append` the window also joins the candidate
// buffer (DTWS_EOVERFLOW when full).
static __device__ __noinline__ void xz_offer(const QueryBufs &b, const QueryArgs &a, unsigned long long key, bool append) {
    QueryState *st = b.st;
    if (append) {
        const int i = atomicAdd(&st->xz_count, 1);
        if (i < b.xz_cap) b.xz_buf[i] = key;
        else atomicOr(b.status, kStOverflow);
    }
    const int k = a.k;
    const unsigned W = (unsigned)(2 * a.xz_z + 1);
    const unsigned bk = key_idx(key) / W;
    unsigned long long *Lp = st->xz_keys[bk & 1u];
    if (key >= *((volatile unsigned long long *)&Lp[k - 1])) return;  // changes nothing
    int *lock = &st->xz_lock[bk & 1u];
    const long long t0 = global_ns();
    while (atomicCAS(lock, 0, 1) != 0) {
        if (global_ns() - t0 > b.wait_ns) {
            atomicOr(b.status, kStTimeout);
            return;
        }
        __nanosleep(64);
    }
    __threadfence();
    unsigned long long v[kKMax];
    int n = 0, same = -1;
    for (int j = 0; j < k; ++j) {
        v[j] = *((volatile unsigned long long *)&Lp[j]);
        if (v[j] != kEmptyKey) {
            ++n;
            if (key_idx(v[j]) / W == bk) same = j;
        }
    }
    bool changed = false;
    if (same >= 0) {
        if (key < v[same]) {  // the bucket's entry improves: drop it, insert below
            for (int j = same; j + 1 < k; ++j) v[j] = v[j + 1];
            v[k - 1] = kEmptyKey;
            changed = true;
        }
    } else {
        changed = key < v[k - 1];
    }
    if (changed) {
        int pos = k - 1;
        while (pos > 0 && v[pos - 1] > key) {
            v[pos] = v[pos - 1];
            --pos;
        }
        v[pos] = key;
        for (int j = 0; j < k - 1; ++j) Lp[j] = v[j];
        __threadfence();
        *((volatile unsigned long long *)&Lp[k - 1]) = v[k - 1];
    }
    __threadfence();
    atomicExch(lock, 0);
}

// A query of a batch whose survivor DTW runs in the persistent stage.
struct PoolQuery {
    QueryState *st;
    float *qh32;
    unsigned short *ord;
    float *sq, *sU, *sL;
    const float *U, *L;  // the exact envelope for its r, or null (block envelope)
    QueryArgs a;
};

// The survivor pool of a batch: survivors (offset, bound) and their window
// statistics, each query's run reserved from one cursor.
struct SurvPool {
    unsigned *idx;
    float *lb, *mh, *is, *ls;
    unsigned long long *cursor;
    long long cap;
};

cudaError_t launch_query_reset(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_qprep(const float *Q, const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
// proposal scans: each CTA writes its best window to cta_best[slot * kCtaSlots + cta];
// *ctas receives the grid size; launch_prop_merge then keeps the best `proposals`.
// The proxy scan does that merge itself, and the seed lists (launch_seed_gather
// with n_random, H and rng), in the last of its CTAs to finish.
cudaError_t launch_seed_scan(const QueryBufs &b, const QueryArgs &a, int proposals, int terms, int n_random, int H,
                             unsigned long long rng, int *ctas, cudaStream_t s);
// half: Euclidean seeds cover the proposals' offsets +-half
cudaError_t launch_seed_gather(const QueryBufs &b, const QueryArgs &a, int n_random,
                               int proposals, int half, unsigned long long rng, cudaStream_t s);
// max_seeds: an upper bound on the Euclidean seed list's length (grid size)
cudaError_t launch_seed_ed(const QueryBufs &b, const QueryArgs &a, int max_seeds, cudaStream_t s);
// k > 1: offsets within +-k of the two best Euclidean seeds join the DTW seeds
cudaError_t launch_seed_expand(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_dtw_seeds(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_prescore(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_lb_scan(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_order(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_dtw_survivors(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
// the final stage: one launch, or three (*launches says which)
cudaError_t launch_finalize(const QueryBufs &b, const QueryArgs &a, int64_t *out_idx,
                            float *out_dist, cudaStream_t s, int *launches);
// persistent batch stage (dtw_pool.cu): the default anti-diagonal shape of a
// band (false when the band takes another kernel), and the stage's launch
// over the shape's queries list[0..nlist) of pq (device arrays); m_max,
// r_max size its shared memory
bool pool_shape(int r, int *L, int *K);
cudaError_t launch_dtw_pool(const QueryBufs &base, const SurvPool &pool, const PoolQuery *pq, const int *list,
                            int nlist, int L, int K, int m_max, int r_max, cudaStream_t s);
// hand the ordered survivors of b's query to the pool (st->deferred = 1), or
// leave them to the query's own survivor pass when the pool is full
cudaError_t launch_defer(const QueryBufs &b, const SurvPool &pool, cudaStream_t s);
// wide exclusion zone: the candidates within the final threshold,
// re-scored, sorted, taken greedily (k results; -1 / +inf where missing)
cudaError_t launch_xz_finalize(const QueryBufs &b, const QueryArgs &a, int64_t *out_idx, float *out_dist,
                               cudaStream_t s);

// element-wise building blocks
cudaError_t launch_dtw_at(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                          int64_t count, float *out, cudaStream_t s);
// the autotuner's probes: a shape (see plan_shape) and DTW at offsets with it;
// the survivor pass's default shape for (m, r) (false: the multi-warp or
// row-systolic kernel, not a plan_shape shape)
bool dtw_default_shape(int m, int r, int *L, int *K, int *warps);
bool dtw_shape_valid(int m, int r, int L, int K, int warps);
cudaError_t launch_dtw_at_shape(const QueryBufs &b, QueryArgs a, const int64_t *offsets, int64_t count, float *out,
                                int L, int K, int warps, cudaStream_t s);
cudaError_t launch_dtw_at_f64(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                              int64_t count, double *out, cudaStream_t s);
cudaError_t launch_lbs_at(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                          int64_t count, float *kim, float *kq, float *ks, cudaStream_t s);

// one bounded wait on an mbarrier nothing arrives on (records kStTimeout)
cudaError_t launch_wait_selftest(int *status, long long wait_ns, cudaStream_t s);
// the exclusion zone's list lock held while an offer waits (records kStTimeout)
cudaError_t launch_lock_selftest(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);

// ---- learned proposal encoder (encoder.cu)
// params -> packed blob; with `adam`, one Adam step first (c1, c2: bias corrections)
cudaError_t launch_enc_pack(float *params, const float *grad, float *m1, float *v1, uint8_t *blob, bool adam,
                            float lr, float beta1, float beta2, float eps, float c1, float c2, cudaStream_t s);
cudaError_t launch_enc_prep(const float *X, const int64_t *off, int rows, int m, float *u, cudaStream_t s);
// ws == nullptr: embeddings to e; else the training workspace receives activations
cudaError_t launch_enc_forward(const uint8_t *blob, const float *u, int rows, float *e, uint8_t *ws, int num_sms,
                               cudaStream_t s);
// loss (accumulated into *loss), data and weight gradients of B triples
cudaError_t launch_enc_backward(const uint8_t *blob, const float *y, int B, float *loss, float *grad,
                                uint8_t *ws, int num_sms, cudaStream_t s);
size_t enc_workspace_bytes(int rows);
cudaError_t launch_enc_series(const uint8_t *blob, const float *x, int64_t n, int b, const float *inv_sigma,
                              int64_t Nw, void *E, int num_sms, cudaStream_t s);
cudaError_t launch_enc_query(const uint8_t *blob, const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
// windows at offsets j*stride + phase (j < Nw)
// int8 copy of BF16 embeddings for the scan: Q [rows][64], S [rows] = (scale, squared norm) as float2
cudaError_t launch_enc_quant(const void *E, int64_t rows, void *Q, void *S, cudaStream_t s);
cudaError_t launch_learn_scan(const QueryBufs &b, const void *Q, const void *S, int64_t Nw, int stride,
                              int phase, int slot, int *ctas, cudaStream_t s);
cudaError_t launch_prop_merge(const QueryBufs &b, int ctas0, int ctas1, int proposals, cudaStream_t s);
// greedy exclusion-zone selection of k of the K ordered results (idx, dist)
cudaError_t launch_exclusion_select(const int64_t *idx, const float *dist, int K, int k, int z, int64_t *out_idx,
                                    float *out_dist, cudaStream_t s);
cudaError_t launch_bf16_to_f32(const void *src, int64_t count, float *dst, cudaStream_t s);

}  // namespace dtws
