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
 * may fill the list (no exclusion zone, unless options.exclusion_zone
 * asks for one).  options.unnormalised = 1 drops the z-normalisation and
 * compares raw values (an API variant the paper does not treat).
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
    DTWS_ENONFINITE = 4,  /* NaN or +-Inf in the series or the query (with
                             unnormalised DTW: also a query value beyond
                             +-2^32) */
    DTWS_ETIMEOUT = 5,    /* a bounded device-side wait ran out */
    DTWS_ENOTIMPL = 6,    /* not implemented */
    DTWS_EOVERFLOW = 7    /* more near-ties than the re-score list holds; the
                             returned order among near-ties may be inexact */
} dtws_status;

/* Limits of the library. */
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
    DTWS_ORDER_LEARNED = 1  /* DTW of the random seed windows plus the best
                               windows of a scan of learned embeddings (see
                               dtws_set_encoder; needs an encoder and m >= 64) */
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
    int32_t seed_proposals; /* proposals of the proxy (or learned) scan,
                               default 16 (0..64) */
    int32_t proxy_terms;    /* evenly spaced query positions in the proxy
                               distance: 16, 8, 4 (other values round down to
                               one of them, or 2), default 16 */
    int32_t ordering;       /* dtws_ordering, default DTWS_ORDER_PLAIN */
    int32_t timing;         /* 1: record per-phase CUDA events (small cost) */
    int32_t exact_envelope; /* 1 (default): Eq. 10 uses the exact series
                               envelope for r, computed once per r and
                               cached; 0: a per-series block envelope (max /
                               min over 16-sample blocks covering
                               [t-r, t+r], built at dtws_create) -- slightly
                               looser, so a few more windows reach DTW, but no
                               per-r pass; an exact envelope already cached
                               is still used.  The answer is the same. */
    int32_t batch_lanes;    /* dtws_query_batch: queries in flight at once, each
                               lane with its own buffers and streams (1..16,
                               default 4; fewer when memory is short) */
    int32_t batch_graph;    /* 1 (default): repeated calls replay CUDA graphs.
                               dtws_query_batch captures the batch into a
                               graph once and replays it for later calls with
                               the same arguments (not with the learned
                               ordering); dtws_query does the same for one
                               query (not while timing is on).  The query
                               values may change between replays. */
    int32_t exclusion_zone; /* z >= 0 (default 0): dtws_query returns the k
                               best windows of which no two lie within z
                               samples of each other, taken greedily in
                               (distance, offset) order.  Exact.  When
                               k*(2z+1) <= DTWS_K_MAX the answer lies among
                               the k*(2z+1) best windows, which the search
                               finds first; otherwise (e.g. z ~ m/2 with
                               k > 1) the search prunes against the k-th
                               distance of windows found more than 2z apart
                               (offsets cut into buckets of 2z+1, one window
                               per bucket, two lists by bucket parity), keeps
                               every window scored within its threshold in a
                               candidate buffer, and at the end re-scores
                               those within the final threshold and takes
                               them greedily (DTWS_EOVERFLOW if the buffer of
                               2^20 or the re-score list of 8192 fills).
                               Not for dtws_query_batch.  Missing windows
                               (the series too short) come back as offset
                               -1, distance +inf. */
    int32_t unnormalised;   /* 1: DTW of the raw values (no z-normalisation of
                               the windows or the query, Eq. 5 skipped);
                               default 0.  dtws_query and the building
                               blocks at given offsets only; not with the
                               learned ordering (its embeddings are of
                               normalised windows).  The series and the
                               query must lie within +-2^32 (so that every
                               squared path sum stays far inside FP32's
                               range): dtws_query returns DTWS_EINVAL for
                               such a series, dtws_sync_status
                               DTWS_ENONFINITE for such a query.
                               Distances are then in squared units of the
                               data, and so is alpha_per_m: the raw values
                               enter the differences unscaled, so the FP32
                               errors are relative and delta covers them;
                               keep alpha_per_m*m well below the distances
                               of interest (near-ties within it are
                               re-scored, DTWS_EOVERFLOW beyond k + 64). */
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
    float seed_bsf;           /* smallest seed distance: DTW of a seed window or
                                 the Euclidean distance (an upper bound of the
                                 DTW) of one; inf if no seed */
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
 * With options.exclusion_zone = z > 0 the k results are more than z
 * samples apart (see dtws_options).  With options.batch_graph = 1 a call
 * whose arguments (pointers, m, r, k, options) repeat the previous one's
 * replays the captured search; the query values may differ.
 * With options.unnormalised = 1 neither side is normalised (raw values).
 * Errors: DTWS_EINVAL synchronously (also unnormalised DTW with the learned
 * ordering or with a series beyond +-2^32); DTWS_ENONFINITE and
 * DTWS_EOVERFLOW via dtws_sync_status.
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

/* Test hook for the wide exclusion zone (the paper has no counterpart):
   capacities of its candidate buffer (windows scored within the threshold,
   default 2^20) and re-score list (windows within the final threshold,
   default 8192) from the next query on; a query that fills either reports
   DTWS_EOVERFLOW from dtws_sync_status (its answer may then be inexact).
   Synchronises the device.  Errors: DTWS_EINVAL (buf_cap < 1, sel_cap
   outside [1, 16384]), DTWS_ECUDA. */
dtws_status dtws_debug_set_xz_capacity(dtws_t h, int32_t buf_cap, int32_t sel_cap);

/* Test hook for dtws_query_batch (the paper has no counterpart): capacity of
   the survivor pool of the batch's persistent DTW stage, in survivors, from
   the next batch on; 0 = no pool (every query runs its survivor pass on its
   lane), -1 = the default (the batch's window count, at most 2^27).  A query
   whose survivors do not fit runs its survivor pass on its lane; the answers
   are the same either way.  Synchronises the device.  Errors: DTWS_EINVAL
   (cap < -1), DTWS_ECUDA. */
dtws_status dtws_debug_set_pool_capacity(dtws_t h, int64_t cap);

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
   pruning: the search's DTW kernel.  out: FP32 [count].  With
   options.unnormalised = 1 (here and in the two calls below) the raw query
   and windows. */
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

/* Failure-detection self-test (the paper has no counterpart): one device
   thread waits, with the library's bounded wait, on a barrier that nothing
   completes; after wait_ns (1 .. 1e10) it records a timeout, which the next
   dtws_sync_status(h, stream) returns as DTWS_ETIMEOUT (and clears).  The
   same bounded wait guards every device-side wait of the search, so no
   kernel of the library spins forever; this entry point exercises that path
   without a fault or a hang.  Errors: DTWS_EINVAL, DTWS_ECUDA. */
dtws_status dtws_debug_wait_selftest(dtws_t h, int64_t wait_ns, void *stream);

/* Failure-detection self-test of the one lock in the library (the paper has
   no counterpart): the wide exclusion zone's bucket lists are rewritten under
   a spin lock whose wait is bounded by options.wait_limit_ns.  Here one
   device thread holds the lock while another offers a window to the same
   list; after wait_ns (1 .. 1e10) the offer gives up, drops the window (which
   only loosens the pruning bound) and records a timeout that the next
   dtws_sync_status(h, stream) returns as DTWS_ETIMEOUT; then the lock is
   released.  Overwrites the handle's query state (run it between queries).
   Errors: DTWS_EINVAL, DTWS_ENOMEM, DTWS_ECUDA. */
dtws_status dtws_debug_lock_selftest(dtws_t h, int64_t wait_ns, void *stream);

/* ---- autotuner (the paper has no counterpart) ----
 *
 * For each (m, r) pair (r > m-1 taken as m-1), times the banded-DTW kernel
 * over `samples` evenly spread windows of the handle's series in every
 * admissible shape -- lanes per candidate L (1..32), cells per lane K
 * (anti-diagonal kernel, L*K >= r+1) or the row-systolic kernel (K = 0),
 * warps per CTA (2, 4, 8) -- and keeps the fastest whose results are
 * bit-identical to the default shape's (and at least 3% faster); later
 * queries, batches and dtws_dtw_at with that (m, r) use it.  Synchronises;
 * drops a captured batch graph.  Errors: DTWS_EINVAL (null, count < 1,
 * samples outside [32, 2^20], m or r out of range), DTWS_ENOMEM, DTWS_ECUDA.
 */
dtws_status dtws_autotune(dtws_t h, const int32_t *m, const int32_t *r, int32_t count, int32_t samples,
                          void *stream);
/* The tuned entry of (m, r): shape = {L, K, warps} (L = 0: the default was
   kept), ms = {default time, chosen time} per probe launch.  DTWS_EINVAL if
   the pair was not tuned. */
dtws_status dtws_tune_entry(dtws_t h, int32_t m, int32_t r, int32_t *shape, float *ms);

/* ---- learned proposals (the paper has no learned component) ----
 *
 * An encoder e(.) maps a window of length m to 64 numbers; windows whose
 * embeddings lie close to the query's are proposed as seeds of the
 * best-so-far (as the paper's random first bsf, Algorithm 1).  Pruning never
 * uses it, so the answer of dtws_query is the same with or without it.
 *
 * Encoder input of a window y: b = floor(m/64), the block means a_j of
 * y[j*b, (j+1)*b) for j < 64, and u_j = (a_{j+1} - a_j) / sigma(y) for j < 63,
 * sigma the population deviation of all m samples (Eq. 5); u = 0 when sigma
 * is 0.  Network: conv 1->32, 32->32, 32->32, 32->32 channels, kernel 7,
 * valid, no biases, ReLU after the first three; mean over 8 position segments
 * [floor(39 s/8), floor(39 (s+1)/8)); e = P g, P [64][256].  With no biases
 * e(u/sigma) = e(u)/sigma exactly, so the library embeds every window at
 * offsets that are multiples of b from one series-wide pass.
 * Parameters: FP32 [DTWS_ENC_PARAMS] = W1 [32][7], W2..W4 [32][7][32]
 * ([out][tap][in]), P [64][256] (column s*32 + channel).  The GPU keeps an
 * FP32 master copy and computes with BF16 weights and activations and FP32
 * accumulation (tensor cores).  Training loss of a triple (Q, C, y),
 * y = DTW(Q^, C^)/m: (log(|e(Q) - e(C)|^2 + 1e-3) - log(y + 1e-3))^2, mean
 * over the batch.
 *
 * Arrays marked "host or device" may be either; the others are stated.
 */
#define DTWS_ENC_PARAMS 38112
#define DTWS_ENC_DIM 64
#define DTWS_ENC_U 64   /* a row of u: the 63 inputs and one unused slot */

/* Install encoder parameters (host or device FP32 [count], count must be
   DTWS_ENC_PARAMS; copied) on the handle; enables DTWS_ORDER_LEARNED and
   drops embeddings made with earlier parameters.  Synchronises `stream`.
   Errors: DTWS_EINVAL (count, null), DTWS_ENOMEM, DTWS_ECUDA. */
dtws_status dtws_set_encoder(dtws_t h, const float *params, int32_t count, void *stream);

/* The handle's embeddings for query length m: rows = floor((n-m)/b) + 1
   windows at offsets j*b, each 64 FP32 (out [rows][64], host or device;
   `rows` must equal that count).  Computes and caches them if needed (the
   learned ordering also embeds the windows at offsets j*b + b/2 when b >= 2;
   those are not returned here).
   Errors: DTWS_EINVAL (no encoder, m < 64 or > n, rows mismatch). */
dtws_status dtws_learned_embeddings(dtws_t h, int32_t m, float *out, int64_t rows, void *stream);

/* u of the windows X[offsets[i] .. offsets[i]+m) (X host or device FP32 [n];
   offsets HOST int64 [rows], each in [0, n-m]) -> u [rows][DTWS_ENC_U]
   (host or device).  Synchronises `stream`.  Errors: DTWS_EINVAL. */
dtws_status dtws_enc_prep(const float *X, int64_t n, const int64_t *offsets, int32_t rows, int32_t m,
                          float *u, void *stream);

/* Embeddings e [rows][64] (host or device) of u [rows][DTWS_ENC_U] (host or
   device) under `params` (host or device FP32 [DTWS_ENC_PARAMS]).
   Synchronises `stream`.  Errors: DTWS_EINVAL, DTWS_ENOMEM, DTWS_ECUDA. */
dtws_status dtws_enc_forward(const float *params, const float *u, int32_t rows, float *e, void *stream);

/* Mean training loss of `batch` triples (uq[i], uc[i], y[i]) and its
   gradient w.r.t. the parameters (grad FP32 [DTWS_ENC_PARAMS], host or
   device; loss: one HOST float).  All inputs host or device.  Synchronises
   `stream`.  Errors: DTWS_EINVAL, DTWS_ENOMEM, DTWS_ECUDA. */
dtws_status dtws_enc_loss_grad(const float *params, const float *uq, const float *uc, const float *y,
                               int32_t batch, float *loss, float *grad, void *stream);

/* Training on the GPU: Adam on an FP32 master copy. */
typedef struct dtws_trainer_ctx *dtws_trainer_t;
typedef struct {
    float lr;      /* step size, e.g. 1e-3 */
    float beta1;   /* e.g. 0.9 */
    float beta2;   /* e.g. 0.999 */
    float eps;     /* e.g. 1e-8 */
} dtws_adam;

/* params: initial values (host or device FP32 [count = DTWS_ENC_PARAMS]);
   max_batch: largest batch of triples per step (1..65536). */
dtws_status dtws_trainer_create(const float *params, int32_t count, int32_t max_batch,
                                const dtws_adam *hp, dtws_trainer_t *out);
/* One step on `batch` triples: query i is the window xq[q_off[i] .. +m),
   candidate i the window xc[c_off[i] .. +m), label y[i] = DTW/m.  xq, xc:
   DEVICE FP32 [n] (e.g. a series and a noisy copy of it); q_off, c_off:
   HOST int64 [batch], each in [0, n-m]; y: HOST FP32 [batch]; loss: HOST
   float or null (when given, the step's mean loss before the update, and
   the call synchronises `stream`). */
dtws_status dtws_trainer_step(dtws_trainer_t t, const float *xq, const float *xc, int64_t n,
                              const int64_t *q_off, const int64_t *c_off, int32_t m, const float *y,
                              int32_t batch, float *loss, void *stream);
/* Current parameters -> params (host or device FP32 [DTWS_ENC_PARAMS]);
   synchronises `stream`. */
dtws_status dtws_trainer_params(dtws_trainer_t t, float *params, void *stream);
dtws_status dtws_trainer_destroy(dtws_trainer_t t);

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
 * [count]; nothing is staged.  Result: the FP32 Sakoe-Chiba-banded DTW of
 * the z-normalised query against each z-normalised window, each window's
 * mean and deviation computed two-pass in FP64, the same quantity as
 * dtws_dtw_at; an offset out of range, or a non-finite query, gives NaN.
 * count may be any value >= 0 (the work cursor is 64-bit); count == 0
 * returns at once.
 * Working memory is one fixed device array inside the library (about 33 KB,
 * held by every GPU that loads the library until the process exits).  Its
 * device address is looked up on the first call made on each device, so
 * that first call should come before any stream capture.  Calls share the
 * array: each call resets what it uses, and calls whose work overlaps on the
 * GPU race, so do not run two at once.
 * Errors (synchronous): DTWS_EINVAL for null or host pointers, n or r out of
 * range, m beyond DTWS_NOALLOC_M_MAX (the scratch size), or a query length
 * and band whose one-warp shared memory (4 m + 8 (r + 1) bytes) exceeds the
 * device's per-block limit (not reached on GB300 within DTWS_NOALLOC_M_MAX);
 * DTWS_ECUDA.
 */
dtws_status dtws_dtw_at_noalloc(const float *series, int64_t n, const float *Q, int32_t m,
                                int32_t r, const int64_t *offsets, int64_t count, float *out,
                                void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DTWS_H */
