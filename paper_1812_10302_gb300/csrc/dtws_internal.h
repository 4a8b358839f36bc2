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
    // wide exclusion zone (QueryArgs::xz_z > 0): one key per bucket of 2z+1
    // offsets (EMPTY = none yet), the candidate buffer of windows scored
    // within the threshold, and the re-score list of those within the final
    // threshold (offsets, extended-precision distances)
    unsigned long long *xz_bkey;
    unsigned long long *xz_buf;
    unsigned *xz_sel;
    double *xz_d64;
    int xz_cap, xz_sel_cap;
};

// Offer a scored window (key: its quantised distance and offset) to the wide
// exclusion-zone state: the first window of its bucket enters the bucket
// list of the bucket's parity; with `append` it also joins the candidate
// buffer (DTWS_EOVERFLOW when full).
__device__ __forceinline__ void xz_offer(const QueryBufs &b, const QueryArgs &a, unsigned long long key, bool append) {
    QueryState *st = b.st;
    const unsigned idx = key_idx(key);
    const unsigned bucket = idx / (unsigned)(2 * a.xz_z + 1);
    if (atomicCAS(&b.xz_bkey[bucket], kEmptyKey, key) == kEmptyKey) list_insert(st->xz_keys[bucket & 1u], a.k, key);
    if (append) {
        const int i = atomicAdd(&st->xz_count, 1);
        if (i < b.xz_cap) b.xz_buf[i] = key;
        else atomicOr(b.status, kStOverflow);
    }
}

cudaError_t launch_query_reset(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_qprep(const float *Q, const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
// proposal scans: each CTA writes its best window to cta_best[slot * kCtaSlots + cta];
// *ctas receives the grid size; launch_prop_merge then keeps the best `proposals`
cudaError_t launch_seed_scan(const QueryBufs &b, const QueryArgs &a, int proposals, int terms, int *ctas,
                             cudaStream_t s);
// half: Euclidean seeds cover the proposals' offsets +-half
cudaError_t launch_seed_gather(const QueryBufs &b, const QueryArgs &a, int n_random,
                               int proposals, int half, unsigned long long rng, cudaStream_t s);
cudaError_t launch_seed_ed(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
// k > 1: offsets within +-k of the two best Euclidean seeds join the DTW seeds
cudaError_t launch_seed_expand(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_dtw_seeds(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_prescore(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_lb_scan(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_order(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_dtw_survivors(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_finalize(const QueryBufs &b, const QueryArgs &a, int64_t *out_idx,
                            float *out_dist, cudaStream_t s);
// wide exclusion zone: the candidates within the final threshold,
// re-scored, sorted, taken greedily (k results; -1 / +inf where missing)
cudaError_t launch_xz_finalize(const QueryBufs &b, const QueryArgs &a, int64_t *out_idx, float *out_dist,
                               cudaStream_t s);

// element-wise building blocks
cudaError_t launch_dtw_at(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                          int64_t count, float *out, cudaStream_t s);
// the autotuner's probes: a shape (see plan_shape) and DTW at offsets with it
bool dtw_shape_valid(int m, int r, int L, int K, int warps);
cudaError_t launch_dtw_at_shape(const QueryBufs &b, QueryArgs a, const int64_t *offsets, int64_t count, float *out,
                                int L, int K, int warps, cudaStream_t s);
cudaError_t launch_dtw_at_f64(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                              int64_t count, double *out, cudaStream_t s);
cudaError_t launch_lbs_at(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                          int64_t count, float *kim, float *kq, float *ks, cudaStream_t s);

// one bounded wait on an mbarrier nothing arrives on (records kStTimeout)
cudaError_t launch_wait_selftest(int *status, long long wait_ns, cudaStream_t s);

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
