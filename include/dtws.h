/*
 * dtws.h -- exact best-match subsequence search under Sakoe-Chiba-banded
 * Dynamic Time Warping over z-normalised windows, on one GB300 (sm_103a).
 *
 * The problem is the one of arxiv 1812.10302 (Kraeva & Zymbler), Sec. 2.1,
 * Eq. 3: given a long series T and a query Q, find the window of T whose
 * z-normalised shape (Sec. 2.2, Eq. 5) is closest to the z-normalised query
 * under DTW (Eq. 1) restricted to a Sakoe-Chiba band of half-width r.
 * Distances are squared (no square root, Sec. 2.2, Eq. 4 remark).  This
 * library returns the k smallest (distance, offset) pairs in lexicographic
 * order, so ties go to the lowest offset; neighbouring offsets of one match
 * may fill the list (no exclusion zone).
 *
 * Notation: n = series length, m = query length, r = band half-width in
 * samples, N = n - m + 1 windows, offsets are 0-based in [0, N).
 *
 * Pointers: every array argument may be a device pointer or a host pointer
 * (pinned or pageable); the library stages host arrays through its own
 * device buffers.  All calls are asynchronous on `stream` (a cudaStream_t
 * passed as void*, NULL = the legacy default stream) unless stated
 * otherwise; outputs are valid once `stream` has completed (host outputs
 * are valid when the call returns, since staging a host output
 * synchronises the stream).  Argument errors are returned synchronously.
 * Device-side errors (a non-finite query, an overflowed near-tie list, a
 * wait that ran out) are recorded in the handle and returned by
 * dtws_sync_status().
 *
 * Threading: a handle may be used from one host thread at a time.
 */
#ifndef DTWS_H
#define DTWS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dtws_ctx *dtws_t;

typedef enum {
    DTWS_OK = 0,
    DTWS_EINVAL = 1,      /* bad argument (null pointer, size out of range) */
    DTWS_ENOMEM = 2,      /* device or host allocation failed */
    DTWS_ECUDA = 3,       /* a CUDA runtime call failed */
    DTWS_ENONFINITE = 4,  /* NaN or +-Inf in the series or the query */
    DTWS_ETIMEOUT = 5,    /* a bounded device-side wait ran out */
    DTWS_ENOTIMPL = 6,    /* not implemented */
    DTWS_EOVERFLOW = 7    /* more near-ties than the re-score list holds; the
                             returned order among near-ties may be inexact */
} dtws_status;

/* Limits of this build. */
#define DTWS_M_MAX 8192      /* longest query (and block length of the
                                anchored prefix sums, see dtws_create) */
#define DTWS_K_MAX 64        /* largest k */
#define DTWS_N_MAX 2000000000LL

/* Candidate ordering used to seed the best-so-far before the lower-bound
   scan.  Neither changes the answer: pruning only ever uses admissible
   lower bounds against the exact k-th distance found so far. */
typedef enum {
    DTWS_ORDER_PLAIN = 0,   /* DTW of a few seeded random windows (the
                               paper's random first bsf, Algorithm 1) plus the
                               best windows of a cheap proxy scan */
    DTWS_ORDER_LEARNED = 1  /* reserved for the learned proposal encoder */
} dtws_ordering;

typedef struct {
    float delta;            /* relative pruning margin: prune when
                               LB > bsf*(1+delta) + alpha_per_m*m.
                               Default 2^-10: it covers the FP32 rounding of
                               the lower bounds and of the DTW with a wide
                               headroom, so rounding never prunes a true
                               top-k window */
    float alpha_per_m;      /* absolute margin per query sample, default 1e-6 */
    int32_t seed_random;    /* random seed windows, default 4 (0..64) */
    int32_t seed_proposals; /* proxy-scan proposals, default 16 (0..64) */
    int32_t proxy_terms;    /* evenly spaced query positions in the proxy
                               distance: 16, 8, 4 (other values round down to
                               one of them, or 2), default 16 */
    int32_t ordering;       /* dtws_ordering, default DTWS_ORDER_PLAIN */
    int32_t timing;         /* 1: record per-phase CUDA events (small cost) */
    int32_t reserved0;
    int64_t wait_limit_ns;  /* bound on every device-side wait, default 2e9 */
    uint64_t rng_seed;      /* seed of the random seed windows, default 0 */
} dtws_options;

/* Per-query counters of the last dtws_query() (reset by each call; read
   after the stream has completed).  Phases: 0 query prep, 1 proxy scan +
   seeds, 2 lower-bound scan, 3 survivor ordering, 4 DTW, 5 finalise
   (extended-precision re-score), 6 window statistics (when computed by this
   call), 7 series envelope (when computed by this call). */
typedef struct {
    int64_t windows;          /* N */
    int64_t pass_kim;         /* windows whose LB_KimFL did not prune */
    int64_t pass_keogh_q;     /* ... whose LB_Keogh vs the query envelope did not */
    int64_t pass_keogh_s;     /* ... whose LB_Keogh vs the series envelope did not
                                 (checked by the DTW stage, so counted among
                                 the windows it examined before its threshold
                                 ended the pass) */
    int64_t dtw_started;      /* DTW computations begun (seeds + survivors) */
    int64_t dtw_abandoned;    /* ... abandoned early */
    int64_t dtw_cells;        /* band cells evaluated by the FP32 DTW */
    int64_t rescored;         /* candidates re-scored in extended precision */
    float seed_bsf;           /* smallest seed distance (inf if no seed) */
    float phase_ms[8];        /* valid when options.timing == 1 */
    int64_t kernel_launches;  /* kernels this library launched for the query */
} dtws_query_stats;

/* Default options (see field comments). */
void dtws_default_options(dtws_options *opt);

/*
 * Create a search handle over series[0..n) (FP32, host or device).  The
 * series is COPIED into library-owned device memory padded to the tile size,
 * so the caller may release its buffer once the call returns; this call
 * synchronises `stream`.  It also builds the anchored FP64 prefix sums of the
 * series (blocks of DTWS_M_MAX samples, each summed relative to its first
 * sample) that every window statistic derives from.
 * Errors: DTWS_EINVAL (n < 2, n > DTWS_N_MAX, null), DTWS_ENONFINITE (a NaN
 * or Inf sample), DTWS_ENOMEM, DTWS_ECUDA.  On error *out is NULL.
 */
dtws_status dtws_create(const float *series, int64_t n, void *stream, dtws_t *out);

/* Free the handle and every device buffer it owns (synchronises the device). */
dtws_status dtws_destroy(dtws_t h);

dtws_status dtws_set_options(dtws_t h, const dtws_options *opt);
dtws_status dtws_get_options(dtws_t h, dtws_options *opt);

/*
 * Best match search, Sec. 2.1 Eq. 3, top-k.
 * Q: FP32 [m], raw (the library z-normalises it, Eq. 5, population sigma).
 * m: 2 <= m <= min(n, DTWS_M_MAX).  r >= 0; r > m-1 is treated as m-1.
 * k: 1 <= k <= min(N, DTWS_K_MAX).
 * out_idx: int64 [k], offsets ascending by (distance, offset).
 * out_dist: FP32 [k], squared banded DTW of the z-normalised query and
 *   window, re-scored in extended precision (FP64 statistics, DTW in
 *   double-float arithmetic, ~48 significant bits) and rounded to FP32.
 *   The offsets are ordered by that re-scored distance, then by offset.
 * A window (or query) whose variance is <= 1e-24*max(1, mean^2) normalises
 * to all zeros.  Per-series data for this m (window statistics) and r
 * (series envelope) are computed on first use and cached in the handle.
 * Errors: DTWS_EINVAL synchronously; DTWS_ENONFINITE via dtws_sync_status.
 */
dtws_status dtws_query(dtws_t h, const float *Q, int32_t m, int32_t r, int32_t k,
                       int64_t *out_idx, float *out_dist, void *stream);

/*
 * Many queries of uneven length and band in one call.  Q_cat holds the
 * queries back to back; q_off (HOST int64 [nq+1]) gives query q as
 * Q_cat[q_off[q] .. q_off[q+1]); m_arr and r_arr are HOST int32 [nq] with
 * m_arr[q] == q_off[q+1]-q_off[q].  out_idx / out_dist are [nq*k]
 * row-major.  Same per-query semantics and limits as dtws_query().
 */
dtws_status dtws_query_batch(dtws_t h, const float *Q_cat, const int64_t *q_off,
                             const int32_t *m_arr, const int32_t *r_arr, int32_t nq,
                             int32_t k, int64_t *out_idx, float *out_dist, void *stream);

/* Synchronise `stream`, return (and clear) the first device-side error
   recorded since the last call, DTWS_OK if none. */
dtws_status dtws_sync_status(dtws_t h, void *stream);

/* Counters of the last query (synchronises the handle's work). */
dtws_status dtws_last_stats(dtws_t h, dtws_query_stats *out);

/* Drop the cached per-m window statistics and per-r series envelopes; the
   next query recomputes what it needs. */
dtws_status dtws_clear_cache(dtws_t h);

const char *dtws_strerror(dtws_status s);

/* Text of the last error the calling host thread met in this library (the
   failing call and the CUDA message); "" if none.  Owned by the library. */
const char *dtws_last_error_detail(void);

/* Test hook for failure handling: the next `count` device allocations made
   by this library fail as if the device were out of memory (the calls that
   need them return DTWS_ENOMEM and release what they allocated). */
void dtws_debug_fail_next_allocs(int count);

/* ---- building blocks, exposed for element-wise checking and reuse ---- */

/*
 * Window statistics for length m (Sec. 2.2, Eq. 5), as the kernels use them:
 * for window i, mu_hi[i] + mu_lo[i] is the FP64 mean split into two floats,
 * inv_sigma[i] = 1/sigma in FP32 (0 under the zero-variance rule).  Arrays
 * are FP32 [N].  Computes and caches them if needed.
 */
dtws_status dtws_window_stats(dtws_t h, int32_t m, float *mu_hi, float *mu_lo,
                              float *inv_sigma, void *stream);

/* Raw series envelope with half-width r (Sec. 2.2, Eq. 9 applied to the
   series, clipped to [0, n)): U[t] = max(x[t-r..t+r]), L[t] = min(...).
   FP32 [n] each.  Computes and caches it if needed. */
dtws_status dtws_series_envelope(dtws_t h, int32_t r, float *U, float *L, void *stream);

/* FP32 banded DTW (Eq. 1 + band) of the z-normalised query against the
   z-normalised windows at offsets[0..count) (int64, each in [0, N)), no
   pruning: the search's DTW kernel.  out: FP32 [count]. */
dtws_status dtws_dtw_at(dtws_t h, const float *Q, int32_t m, int32_t r,
                        const int64_t *offsets, int64_t count, float *out, void *stream);

/* Same, in extended precision: per-window two-pass FP64 statistics (Eq. 5),
   normalised values formed in FP64 and the DTW in double-float arithmetic
   (~48 significant bits; plain FP64 for bands wider than 511): the re-score
   kernel of dtws_query.  out: FP64 [count]. */
dtws_status dtws_dtw_at_f64(dtws_t h, const float *Q, int32_t m, int32_t r,
                            const int64_t *offsets, int64_t count, double *out,
                            void *stream);

/* FP32 lower bounds at offsets, full (no early abandon): LB_KimFL (Eq. 7,
   squared), LB_Keogh of the window against the query envelope (Eq. 8), and
   LB_Keogh of the query against the window's envelope taken from the
   series-wide envelope (Eq. 10; looser than the window-clipped envelope,
   still admissible).  Each output FP32 [count]. */
dtws_status dtws_lower_bounds_at(dtws_t h, const float *Q, int32_t m, int32_t r,
                                 const int64_t *offsets, int64_t count, float *kim,
                                 float *keogh_q, float *keogh_s, void *stream);

/* ---- allocation-free variant (the paper has no counterpart) ---- */

/* Longest query dtws_dtw_at_noalloc accepts: the size of its fixed scratch. */
#define DTWS_NOALLOC_M_MAX 8192

/*
 * dtws_dtw_at without a handle and without any device allocation, for
 * callers that cannot let a library call cudaMalloc (it synchronises the
 * device and stalls other work, a host framework may own all device memory
 * through its own pool, or the deployment fixes its memory at start-up).
 * Inputs and outputs are the caller's DEVICE arrays: series FP32 [n],
 * Q FP32 [m] (raw), offsets int64 [count] (each in [0, n-m]), out FP32
 * [count]; nothing is staged.  Result: the FP32 banded DTW (Eq. 1 + band) of
 * the z-normalised query against each z-normalised window, each window's
 * statistics computed two-pass in FP64; an offset out of range, or a
 * non-finite query, gives NaN.
 * Working memory is one fixed device array inside the library (about 33 KB,
 * held by every GPU that loads the library until the process exits).  Its
 * device address is looked up on the first call made on each device, so
 * that first call should come before any stream capture.  Calls share the
 * array: each call resets what it uses, and calls whose work overlaps on the
 * GPU race, so do not run two at once.
 * Errors (synchronous): DTWS_EINVAL for null or host pointers, n or r out of
 * range, or m beyond DTWS_NOALLOC_M_MAX (the scratch size); DTWS_ECUDA.
 */
dtws_status dtws_dtw_at_noalloc(const float *series, int64_t n, const float *Q, int32_t m,
                                int32_t r, const int64_t *offsets, int64_t count, float *out,
                                void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DTWS_H */
