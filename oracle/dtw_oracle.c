/*
 * dtw_oracle.c -- plain, slow, FP64 CPU oracle for exact best-match subsequence
 * search under Sakoe-Chiba-banded DTW over z-normalised windows
 * (arxiv 1812.10302, Kraeva & Zymbler, "PhiBestMatch").
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  The GPU library shares no code,
 * header, table or constant with this file and never calls it.
 *
 * Notation (the repository's, not the paper's; the paper swaps the letters):
 *   n = series length, m = query length, r = band half-width in samples,
 *   N = n - m + 1 windows, 0-based offsets i in [0, N).
 *
 * Every function states the passage of the paper it follows.  Readings of
 * passages that are silent or garbled:
 *   R1  sigma is the population deviation (Sec. 2.2, Eq. 5: 1/m), evaluated
 *       two-pass as sum((t-mu)^2)/m, which equals Eq. 5's
 *       (1/m)sum(t^2) - mu^2 in exact arithmetic.
 *   R2  sigma = 0 is unspecified.  A window (or query) with
 *       var <= 1e-24 * max(1, mu^2) is normalised to all zeros.
 *   R3  LB_KimFL (Eq. 7) uses squared differences, consistent with dropping
 *       the square root (Eq. 4).
 *   R4  The envelope of Eq. 9 is clipped to the sequence's own index range.
 *   R5  Pruning is strict: prune only when LB > bsf (Eq. 6); Eq. 15's "<"
 *       disagrees at equality and is not followed.
 *   R6  bsf is the k-th best distance found so far (+inf until k results);
 *       results are the k smallest (distance, index) pairs in lexicographic
 *       order, so ties go to the lowest index.
 *   R7  DTW early abandoning (named in Sec. 1, passed as the 4th argument of
 *       DTW in Algorithm 1): every warping path crosses every row, so the row
 *       minimum of the cumulative matrix is a lower bound of the DTW; abandon
 *       when it exceeds bsf (strict).
 *
 * parity pins: see tests/test_oracle.py (hand-computed golden values, warping
 * path enumeration, closed forms, library routines, brute force).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF HUGE_VAL

/* ------------------------------------------------------------------ */
/* z-normalisation, Sec. 2.2, Eq. 5                                    */
/* ------------------------------------------------------------------ */

/* R2: the zero-variance rule. */
int orc_sigma_is_zero(double mu, double var)
{
    double s = mu * mu;
    if (s < 1.0) s = 1.0;
    return var <= 1e-24 * s;
}

/* Mean and population sigma of x[0..m), two-pass (R1).  sigma is 0 under R2. */
void orc_stats_twopass(const float *x, int64_t m, double *mu_out, double *sigma_out)
{
    double s = 0.0;
    for (int64_t j = 0; j < m; ++j) s += (double)x[j];
    double mu = s / (double)m;
    double v = 0.0;
    for (int64_t j = 0; j < m; ++j) {
        double d = (double)x[j] - mu;
        v += d * d;
    }
    v /= (double)m;
    *mu_out = mu;
    *sigma_out = orc_sigma_is_zero(mu, v) ? 0.0 : sqrt(v);
}

/* t_hat_j = (t_j - mu) / sigma (Eq. 5); all zeros when sigma == 0 (R2). */
void orc_normalize(const float *x, int64_t m, double mu, double sigma, double *out)
{
    for (int64_t j = 0; j < m; ++j)
        out[j] = (sigma == 0.0) ? 0.0 : ((double)x[j] - mu) / sigma;
}

void orc_znorm(const float *x, int64_t m, double *out)
{
    double mu, sigma;
    orc_stats_twopass(x, m, &mu, &sigma);
    orc_normalize(x, m, mu, sigma, out);
}

/* Two-pass stats of every window of length m (O(N*m)). */
void orc_window_stats_twopass(const float *x, int64_t n, int64_t m,
                              double *mu, double *sigma)
{
    int64_t N = n - m + 1;
    for (int64_t i = 0; i < N; ++i) orc_stats_twopass(x + i, m, &mu[i], &sigma[i]);
}

/* Compensated summation (Neumaier): s + c carries the sum to about one ulp. */
static void comp_add(double *s, double *c, double v)
{
    double t = *s + v;
    *c += fabs(*s) >= fabs(v) ? (*s - t) + v : (v - t) + *s;
    *s = t;
}

/* Sum over [bB, e) of block b's anchored terms, for bB < e <= end of block b:
   the block total when e is the block's end, else the prefix entry P[e]. */
static double block_upto(const double *P, const double *T, int64_t n, int64_t B,
                         int64_t b, int64_t e)
{
    int64_t end = (b + 1) * B < n ? (b + 1) * B : n;
    return e == end ? T[b] : P[e];
}

/*
 * Anchored block prefix sums (the paper never considers numerics at scale;
 * this is the reading used for long series).  The series is cut into blocks
 * of B >= m samples; inside block b, sums run over (x - a_b) with a_b the
 * block's first sample, so no sum grows with the series.  A window spans at
 * most two blocks; the second block's sums are moved to anchor a_b0 with
 *   sum(x - a0)   = sum(x - a1) + k (a1 - a0)
 *   sum(x - a0)^2 = sum(x - a1)^2 + 2 (a1 - a0) sum(x - a1) + k (a1 - a0)^2.
 * Then mu = a0 + S1/m and var = S2/m - (S1/m)^2, and R2 applies.  The block
 * sums are compensated, and when the subtraction cancels (var <= 1e-6*S2/m)
 * or m*var <= 1e-9 times the block's sum of squares, the window is evaluated
 * two-pass instead.
 * Returns 0, or -1 when B < m or memory is short.
 */
int orc_window_stats_anchored(const float *x, int64_t n, int64_t m, int64_t B,
                              double *mu, double *sigma)
{
    if (B < m) return -1;
    int64_t nb = (n + B - 1) / B;
    /* P1[t], P2[t] = sums over [block start, t) of (x - a) and (x - a)^2,
       for t in [0, n]; one extra slot per block holds the block total. */
    double *P1 = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *P2 = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *T1 = (double *)malloc(sizeof(double) * (size_t)nb);
    double *T2 = (double *)malloc(sizeof(double) * (size_t)nb);
    double *A = (double *)malloc(sizeof(double) * (size_t)nb);
    if (!P1 || !P2 || !T1 || !T2 || !A) {
        free(P1); free(P2); free(T1); free(T2); free(A);
        return -1;
    }
    for (int64_t b = 0; b < nb; ++b) {
        int64_t t0 = b * B, t1 = t0 + B < n ? t0 + B : n;
        double a = (double)x[t0], s1 = 0.0, c1 = 0.0, s2 = 0.0, c2 = 0.0;
        A[b] = a;
        for (int64_t t = t0; t < t1; ++t) {
            P1[t] = s1 + c1;
            P2[t] = s2 + c2;
            double d = (double)x[t] - a;
            comp_add(&s1, &c1, d);
            comp_add(&s2, &c2, d * d);
        }
        T1[b] = s1 + c1;
        T2[b] = s2 + c2;
    }
    int64_t N = n - m + 1;
    for (int64_t i = 0; i < N; ++i) {
        int64_t b0 = i / B, e = i + m; /* window is [i, e) */
        double a0 = A[b0], S1, S2;
        if (e <= (b0 + 1) * B) {
            S1 = block_upto(P1, T1, n, B, b0, e) - P1[i];
            S2 = block_upto(P2, T2, n, B, b0, e) - P2[i];
        } else {
            int64_t b1 = b0 + 1;
            double k = (double)(e - b1 * B), da = A[b1] - a0;
            double e1 = block_upto(P1, T1, n, B, b1, e);
            double e2 = block_upto(P2, T2, n, B, b1, e);
            S1 = (T1[b0] - P1[i]) + (e1 + k * da);
            S2 = (T2[b0] - P2[i]) + (e2 + 2.0 * da * e1 + k * da * da);
        }
        double mr = S1 / (double)m;
        double v = S2 / (double)m - mr * mr;
        double M2 = T2[b0] + (e > (b0 + 1) * B ? T2[b0 + 1] + S2 : 0.0);
        if (v <= 1e-6 * (S2 / (double)m) || v * (double)m <= 1e-9 * M2) {
            /* the shifted sums cancelled, or var is not far above the
               rounding of the block sums: evaluate Eq. 5 two-pass for this
               window instead */
            orc_stats_twopass(x + i, m, &mu[i], &sigma[i]);
            continue;
        }
        double mu_i = a0 + mr;
        mu[i] = mu_i;
        sigma[i] = orc_sigma_is_zero(mu_i, v) ? 0.0 : sqrt(v);
    }
    free(P1); free(P2); free(T1); free(T2); free(A);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Banded DTW, Sec. 2.1, Eq. 1 with the Sakoe-Chiba band               */
/* ------------------------------------------------------------------ */

/*
 * d(i,j) = (q_i - c_j)^2 + min(d(i-1,j), d(i,j-1), d(i-1,j-1)),
 * d(0,0) = 0, d(i,0) = d(0,j) = inf (1-based), and d(i,j) = inf when
 * |i - j| > r (the path may not leave the diagonal by more than r cells).
 * Squared costs, no square root (Eq. 4's remark).  DTW = d(m,m).
 *
 * work holds (m+1)*(m+1) doubles; only band cells are written, and cells
 * outside the band or on row/column 0 are read through cell() as defined
 * above.  Early abandon (R7): returns +inf as soon as a whole row exceeds bsf.
 */
static double cell(const double *D, int64_t m, int64_t r, int64_t i, int64_t j)
{
    if (i == 0 && j == 0) return 0.0;
    if (i == 0 || j == 0) return ORC_INF;
    if (i - j > r || j - i > r) return ORC_INF;
    return D[i * (m + 1) + j];
}

double orc_dtw(const double *q, const double *c, int64_t m, int64_t r, double bsf, double *work)
{
    if (r > m - 1) r = m - 1;
    for (int64_t i = 1; i <= m; ++i) {
        int64_t jlo = i - r > 1 ? i - r : 1;
        int64_t jhi = i + r < m ? i + r : m;
        double rowmin = ORC_INF;
        for (int64_t j = jlo; j <= jhi; ++j) {
            double a = cell(work, m, r, i - 1, j);
            double b = cell(work, m, r, i, j - 1);
            double d = cell(work, m, r, i - 1, j - 1);
            double best = a < b ? a : b;
            best = best < d ? best : d;
            double diff = q[i - 1] - c[j - 1];
            double v = diff * diff + best;
            work[i * (m + 1) + j] = v;
            if (v < rowmin) rowmin = v;
        }
        if (rowmin > bsf) return ORC_INF;
    }
    return work[m * (m + 1) + m];
}

/* Convenience: DTW without abandoning; allocates its own matrix. */
double orc_dtw_full(const double *q, const double *c, int64_t m, int64_t r)
{
    double *work = (double *)malloc(sizeof(double) * (size_t)(m + 1) * (size_t)(m + 1));
    if (!work) return -1.0;
    double v = orc_dtw(q, c, m, r, ORC_INF, work);
    free(work);
    return v;
}

/* ------------------------------------------------------------------ */
/* Lower bounds, Sec. 2.2, Eqs. 7-10                                   */
/* ------------------------------------------------------------------ */

/* LB_KimFL, Eq. 7, squared (R3): first and last pairs. */
double orc_lb_kim_fl(const double *qh, const double *ch, int64_t m)
{
    double a = qh[0] - ch[0], b = qh[m - 1] - ch[m - 1];
    return a * a + b * b;
}

/* Envelope, Eq. 9: u_i = max(v_{i-r..i+r}), l_i = min(...), clipped (R4). */
void orc_envelope(const double *v, int64_t m, int64_t r, double *U, double *L)
{
    for (int64_t i = 0; i < m; ++i) {
        int64_t lo = i - r > 0 ? i - r : 0, hi = i + r < m - 1 ? i + r : m - 1;
        double u = v[lo], l = v[lo];
        for (int64_t t = lo + 1; t <= hi; ++t) {
            if (v[t] > u) u = v[t];
            if (v[t] < l) l = v[t];
        }
        U[i] = u;
        L[i] = l;
    }
}

/*
 * Eq. 8: sum over i of (c_i - u_i)^2 if c_i > u_i, (c_i - l_i)^2 if c_i < l_i,
 * else 0; (U, L) is the envelope of the OTHER sequence.  The paper's
 * LB_Keogh EC(Q,C) is orc_lb_keogh(c_hat, U_q, L_q); Eq. 10's
 * LB_Keogh EQ(Q,C) := EC(C,Q) is orc_lb_keogh(q_hat, U_c, L_c).
 * Early abandon: stops once the partial sum exceeds bsf (the partial sum is
 * itself a lower bound, so the caller prunes either way).
 */
double orc_lb_keogh(const double *v, const double *U, const double *L, int64_t m, double bsf)
{
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double d = 0.0;
        if (v[i] > U[i]) d = v[i] - U[i];
        else if (v[i] < L[i]) d = v[i] - L[i];
        s += d * d;
        if (s > bsf) return s;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* Top-k bookkeeping (R6)                                               */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t k, count;
    double *dist;
    int64_t *idx;
} topk_t;

static int key_less(double d1, int64_t i1, double d2, int64_t i2)
{
    return d1 < d2 || (d1 == d2 && i1 < i2);
}

static double topk_bsf(const topk_t *t)
{
    return t->count < t->k ? ORC_INF : t->dist[t->k - 1];
}

static void topk_offer(topk_t *t, double d, int64_t i)
{
    if (t->count == t->k && !key_less(d, i, t->dist[t->k - 1], t->idx[t->k - 1])) return;
    int64_t pos = t->count < t->k ? t->count++ : t->k - 1;
    while (pos > 0 && key_less(d, i, t->dist[pos - 1], t->idx[pos - 1])) {
        t->dist[pos] = t->dist[pos - 1];
        t->idx[pos] = t->idx[pos - 1];
        --pos;
    }
    t->dist[pos] = d;
    t->idx[pos] = i;
}

static void topk_fill(topk_t *t, int64_t *idx, double *dist)
{
    for (int64_t j = 0; j < t->k; ++j) {
        if (j < t->count) { idx[j] = t->idx[j]; dist[j] = t->dist[j]; }
        else { idx[j] = -1; dist[j] = ORC_INF; }
    }
}

/* ------------------------------------------------------------------ */
/* Search                                                               */
/* ------------------------------------------------------------------ */

/*
 * Brute force: the problem statement itself (Sec. 2.1, Eq. 3): DTW of the
 * z-normalised query against every z-normalised window of windows
 * [first, first+count), keep the k smallest (distance, index) pairs.
 * Returns 0, or -1 on bad arguments / no memory.
 */
int orc_search_brute(const float *x, int64_t n, const float *Q, int64_t m, int64_t r,
                     int64_t k, int64_t first, int64_t count, int64_t *idx, double *dist)
{
    if (m < 2 || m > n || r < 0 || k < 1 || first < 0 || count < 0 ||
        first + count > n - m + 1)
        return -1;
    double *qh = (double *)malloc(sizeof(double) * (size_t)m);
    double *ch = (double *)malloc(sizeof(double) * (size_t)m);
    double *work = (double *)malloc(sizeof(double) * (size_t)(m + 1) * (size_t)(m + 1));
    double *td = (double *)malloc(sizeof(double) * (size_t)k);
    int64_t *ti = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (!qh || !ch || !work || !td || !ti) {
        free(qh); free(ch); free(work); free(td); free(ti);
        return -1;
    }
    topk_t t = {k, 0, td, ti};
    orc_znorm(Q, m, qh);
    for (int64_t i = first; i < first + count; ++i) {
        orc_znorm(x + i, m, ch);
        topk_offer(&t, orc_dtw(qh, ch, m, r, ORC_INF, work), i);
    }
    topk_fill(&t, idx, dist);
    free(qh); free(ch); free(work); free(td); free(ti);
    return 0;
}

/*
 * UCR-DTW-style cascade (Sec. 2.2, the scan described at the end of the
 * subsection; the per-window steps of PREPARE/IMPROVE in Sec. 3.3 compute the
 * same quantities): normalise Q, build its envelope, bsf = +inf; scan the
 * windows in ascending order; for each window apply LB_KimFL, then
 * LB_Keogh with the query envelope (Eq. 8), then LB_Keogh with the window's
 * envelope (Eq. 10), pruning when a bound exceeds bsf (R5); otherwise compute
 * DTW with early abandoning (R7) and update the top-k (R6).
 *
 * stats_mode 0: two-pass stats per window; 1: anchored block prefix sums with
 * block length B (>= m).  counters (optional, 5 entries): windows pruned by
 * KimFL, by LB_Keogh(query envelope), by LB_Keogh(window envelope), DTW
 * computed, DTW abandoned.
 */
int orc_search_cascade(const float *x, int64_t n, const float *Q, int64_t m, int64_t r,
                       int64_t k, int64_t first, int64_t count, int stats_mode, int64_t B,
                       int64_t *idx, double *dist, int64_t *counters)
{
    if (m < 2 || m > n || r < 0 || k < 1 || first < 0 || count < 0 ||
        first + count > n - m + 1)
        return -1;
    int64_t rr = r > m - 1 ? m - 1 : r;
    double *qh = (double *)malloc(sizeof(double) * (size_t)m);
    double *ch = (double *)malloc(sizeof(double) * (size_t)m);
    double *Uq = (double *)malloc(sizeof(double) * (size_t)m);
    double *Lq = (double *)malloc(sizeof(double) * (size_t)m);
    double *Uc = (double *)malloc(sizeof(double) * (size_t)m);
    double *Lc = (double *)malloc(sizeof(double) * (size_t)m);
    double *work = (double *)malloc(sizeof(double) * (size_t)(m + 1) * (size_t)(m + 1));
    double *td = (double *)malloc(sizeof(double) * (size_t)k);
    int64_t *ti = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    double *mu = NULL, *sg = NULL;
    int rc = 0;
    if (!qh || !ch || !Uq || !Lq || !Uc || !Lc || !work || !td || !ti) { rc = -1; goto out; }
    if (stats_mode == 1) {
        /* stats of the windows of the fragment's own sub-series */
        int64_t len = count + m - 1;
        mu = (double *)malloc(sizeof(double) * (size_t)count);
        sg = (double *)malloc(sizeof(double) * (size_t)count);
        if (!mu || !sg || count == 0) { rc = count == 0 ? 0 : -1; goto out; }
        if (orc_window_stats_anchored(x + first, len, m, B, mu, sg) != 0) { rc = -1; goto out; }
    }
    int64_t c_kim = 0, c_eq = 0, c_ec = 0, c_dtw = 0, c_ab = 0;
    topk_t t = {k, 0, td, ti};
    orc_znorm(Q, m, qh);
    orc_envelope(qh, m, rr, Uq, Lq);
    for (int64_t i = first; i < first + count; ++i) {
        double mu_i, sg_i;
        if (stats_mode == 1) { mu_i = mu[i - first]; sg_i = sg[i - first]; }
        else orc_stats_twopass(x + i, m, &mu_i, &sg_i);
        orc_normalize(x + i, m, mu_i, sg_i, ch);
        double bsf = topk_bsf(&t);
        if (orc_lb_kim_fl(qh, ch, m) > bsf) { ++c_kim; continue; }
        if (orc_lb_keogh(ch, Uq, Lq, m, bsf) > bsf) { ++c_eq; continue; }
        orc_envelope(ch, m, rr, Uc, Lc);
        if (orc_lb_keogh(qh, Uc, Lc, m, bsf) > bsf) { ++c_ec; continue; }
        ++c_dtw;
        double d = orc_dtw(qh, ch, m, rr, bsf, work);
        if (d == ORC_INF) { ++c_ab; continue; }
        topk_offer(&t, d, i);
    }
    topk_fill(&t, idx, dist);
    if (counters) {
        counters[0] = c_kim; counters[1] = c_eq; counters[2] = c_ec;
        counters[3] = c_dtw; counters[4] = c_ab;
    }
out:
    free(qh); free(ch); free(Uq); free(Lq); free(Uc); free(Lc);
    free(work); free(td); free(ti); free(mu); free(sg);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Per-offset helpers for element-wise kernel parity                   */
/* ------------------------------------------------------------------ */

/* FP64 DTW of the z-normalised query against the z-normalised windows at
   the given offsets (no pruning).  Returns 0 or -1. */
int orc_dtw_at(const float *x, int64_t n, const float *Q, int64_t m, int64_t r,
               const int64_t *offsets, int64_t count, double *out)
{
    double *qh = (double *)malloc(sizeof(double) * (size_t)m);
    double *ch = (double *)malloc(sizeof(double) * (size_t)m);
    double *work = (double *)malloc(sizeof(double) * (size_t)(m + 1) * (size_t)(m + 1));
    if (!qh || !ch || !work) { free(qh); free(ch); free(work); return -1; }
    orc_znorm(Q, m, qh);
    for (int64_t t = 0; t < count; ++t) {
        int64_t i = offsets[t];
        if (i < 0 || i + m > n) { out[t] = -1.0; continue; }
        orc_znorm(x + i, m, ch);
        out[t] = orc_dtw(qh, ch, m, r, ORC_INF, work);
    }
    free(qh); free(ch); free(work);
    return 0;
}

/* Raw sliding envelope of the whole series with half-width r, clipped to the
   series (the candidate-envelope reading that the series-wide LB uses). */
void orc_series_envelope(const float *x, int64_t n, int64_t r, float *U, float *L)
{
    for (int64_t t = 0; t < n; ++t) {
        int64_t lo = t - r > 0 ? t - r : 0, hi = t + r < n - 1 ? t + r : n - 1;
        float u = x[lo], l = x[lo];
        for (int64_t s = lo + 1; s <= hi; ++s) {
            if (x[s] > u) u = x[s];
            if (x[s] < l) l = x[s];
        }
        U[t] = u;
        L[t] = l;
    }
}

/*
 * Lower bounds at given offsets, FP64: LB_KimFL (Eq. 7), LB_Keogh of the
 * window against the query envelope (Eq. 8), LB_Keogh of the query against
 * the window's own clipped envelope (Eq. 10, R4), and the same with the
 * series-wide envelope (raw envelope over [i+j-r, i+j+r] clipped to the
 * series, then normalised with the window's stats), which is looser and
 * still admissible because normalisation with sigma > 0 is monotone.
 */
int orc_lbs_at(const float *x, int64_t n, const float *Q, int64_t m, int64_t r,
               const int64_t *offsets, int64_t count,
               double *kim, double *keogh_q, double *keogh_c, double *keogh_series)
{
    int64_t rr = r > m - 1 ? m - 1 : r;
    double *qh = (double *)malloc(sizeof(double) * (size_t)m);
    double *ch = (double *)malloc(sizeof(double) * (size_t)m);
    double *Uq = (double *)malloc(sizeof(double) * (size_t)m);
    double *Lq = (double *)malloc(sizeof(double) * (size_t)m);
    double *Uc = (double *)malloc(sizeof(double) * (size_t)m);
    double *Lc = (double *)malloc(sizeof(double) * (size_t)m);
    if (!qh || !ch || !Uq || !Lq || !Uc || !Lc) {
        free(qh); free(ch); free(Uq); free(Lq); free(Uc); free(Lc);
        return -1;
    }
    orc_znorm(Q, m, qh);
    orc_envelope(qh, m, rr, Uq, Lq);
    for (int64_t t = 0; t < count; ++t) {
        int64_t i = offsets[t];
        double mu, sg;
        orc_stats_twopass(x + i, m, &mu, &sg);
        orc_normalize(x + i, m, mu, sg, ch);
        kim[t] = orc_lb_kim_fl(qh, ch, m);
        keogh_q[t] = orc_lb_keogh(ch, Uq, Lq, m, ORC_INF);
        orc_envelope(ch, m, rr, Uc, Lc);
        keogh_c[t] = orc_lb_keogh(qh, Uc, Lc, m, ORC_INF);
        for (int64_t j = 0; j < m; ++j) {
            int64_t lo = i + j - rr > 0 ? i + j - rr : 0;
            int64_t hi = i + j + rr < n - 1 ? i + j + rr : n - 1;
            double u = x[lo], l = x[lo];
            for (int64_t s = lo + 1; s <= hi; ++s) {
                if (x[s] > u) u = x[s];
                if (x[s] < l) l = x[s];
            }
            Uc[j] = sg == 0.0 ? 0.0 : (u - mu) / sg;
            Lc[j] = sg == 0.0 ? 0.0 : (l - mu) / sg;
        }
        keogh_series[t] = orc_lb_keogh(qh, Uc, Lc, m, ORC_INF);
    }
    free(qh); free(ch); free(Uq); free(Lq); free(Uc); free(Lc);
    return 0;
}
