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
cudaError_t launch_check_finite(const float *x, int64_t n, int *flag, cudaStream_t s);
cudaError_t launch_prefix(const float *x, int64_t n, double *P1, double *P2, double *T1,
                          double *T2, double *A, cudaStream_t s);
cudaError_t launch_window_stats(const float *x, int64_t n, int m, const double *P1,
                                const double *P2, const double *T1, const double *T2,
                                const double *A, float *mu_hi, float *mu_lo, float *inv_sigma,
                                float *smu_hi, float *smu_lo, float *sinv_sigma, cudaStream_t s);
cudaError_t launch_envelope(const float *x, int64_t n, int r, float *U, float *L, cudaStream_t s);

// ---- query level (query_kernels.cu)
struct QueryBufs {
    QueryState *st;
    const float *x;              // padded series
    const float *mu_hi, *mu_lo, *inv_sigma;  // window stats for m
    const float *smu_hi, *smu_lo, *sinv_sigma;  // the same for every kProxyStride-th window
    const float *U, *L;          // series envelope for r (may be null for *_at)
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
};

cudaError_t launch_query_reset(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_qprep(const float *Q, const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_seed_scan(const QueryBufs &b, const QueryArgs &a, int proposals, int terms,
                             cudaStream_t s);
cudaError_t launch_seed_gather(const QueryBufs &b, const QueryArgs &a, int n_random,
                               int proposals, unsigned long long rng, cudaStream_t s);
cudaError_t launch_seed_ed(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_dtw_seeds(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_prescore(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_lb_scan(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_order(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_dtw_survivors(const QueryBufs &b, const QueryArgs &a, cudaStream_t s);
cudaError_t launch_finalize(const QueryBufs &b, const QueryArgs &a, int64_t *out_idx,
                            float *out_dist, cudaStream_t s);

// element-wise building blocks
cudaError_t launch_dtw_at(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                          int64_t count, float *out, cudaStream_t s);
cudaError_t launch_dtw_at_f64(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                              int64_t count, double *out, cudaStream_t s);
cudaError_t launch_lbs_at(const QueryBufs &b, const QueryArgs &a, const int64_t *offsets,
                          int64_t count, float *kim, float *kq, float *ks, cudaStream_t s);

}  // namespace dtws
