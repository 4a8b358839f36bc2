// dtw_band.cuh -- the systolic banded-DTW core shared by the DTW kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dtws_common.cuh"

namespace dtws {

// ------------------------------------------------------------------ banded DTW core
// Systolic evaluation of d(i,j) = (q_i - c_j)^2 + min(d(i-1,j), d(i,j-1),
// d(i-1,j-1)) on the band |i - j| <= r (Sec. 2.1, Eq. 1), by a group of L
// lanes.  Lane l owns rows l, l+L, l+2L, ...; in a row it walks the band
// index k = j - i + r from 0 to W-1 (W = 2r+1), one cell per step, and lane
// l runs two steps behind lane l-1: at step s it holds cell k = s - tW - 2l
// of row tL + l.  So d(i-1, j) is lane l-1's value of the previous step
// (one shuffle) and d(i-1, j-1) the value shuffled one step earlier; lane 0
// reads row tL-1 from a ring in shared memory that lane L-1 wrote a block
// earlier, which is safe while W > 2L-1, i.e. L <= r (or L = 1).  Costs
// outside the band or the window are +inf.  d(-1,-1) = 0 is ring[r].
//
// Early abandon (ABANDON): every warping path crosses every row, so when a
// lane finishes row i, min_j d(i, j) plus a lower bound of the rows i+1..m-1
// exceeding thr proves DTW > thr.  The bound of the remaining rows (TAIL) is
// the sum over them of the LB_Keogh term of q_hat_i against the window's
// normalised series envelope at i, which bounds that row's cheapest cell.
template <typename T>
__device__ __forceinline__ T tinf();
template <>
__device__ __forceinline__ float tinf<float>() { return __int_as_float(0x7f800000); }
template <>
__device__ __forceinline__ double tinf<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }

template <int L>
__device__ __forceinline__ float group_sum(float v, unsigned gmask) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o, L);
    return v;
}
template <int L>
__device__ __forceinline__ float group_incl_scan(float v, unsigned gmask, int lane) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
        float u = __shfl_up_sync(gmask, v, o, L);
        if (lane >= o) v += u;
    }
    return v;
}

struct TailCtx {
    const float *Uw, *Lw;  // exact series envelope at the window's first sample, or null:
    const float *stmax, *stmin;  // the block envelope (sparse table, kEnvLevels x nblk)
    int64_t nblk, n, t0;   // blocks, series length, the window's first sample
    int r;
    const float *qs;       // q_hat (shared)
    float mh, is, ls;
};

// Raw envelope bounds of series position t0 + i: the exact U_x, L_x (Eq. 9
// over the series, clipped), or max / min over the kEnvG-sample blocks that
// cover [t - r, t + r] clipped -- a superset of that range, so U' >= U_x and
// L' <= L_x and the bound stays admissible.
__device__ __forceinline__ void env_at(const TailCtx &c, int i, float &u, float &l) {
    if (c.Uw) {
        u = c.Uw[i];
        l = c.Lw[i];
        return;
    }
    const int64_t t = c.t0 + i;
    const int64_t lo = t - c.r > 0 ? t - c.r : 0, hi = t + c.r < c.n - 1 ? t + c.r : c.n - 1;
    const int64_t a = lo / kEnvG, bb = hi / kEnvG;
    const int k = 31 - __clz((int)(bb - a + 1));
    const int64_t b2 = bb - (1ll << k) + 1;
    const float *mx = c.stmax + (size_t)k * c.nblk, *mn = c.stmin + (size_t)k * c.nblk;
    u = fmaxf(mx[a], mx[b2]);
    l = fminf(mn[a], mn[b2]);
}

// LB_Keogh term of row i: squared distance of q_hat_i to the normalised
// envelope interval of the window at position i.
__device__ __forceinline__ float tail_term(const TailCtx &c, int i) {
    float U, L;
    env_at(c, i, U, L);
    float u = fmaf(U - c.mh, c.is, -c.ls);
    float l = fmaf(L - c.mh, c.is, -c.ls);
    float q = c.qs[i];
    float d = fmaxf(q - u, 0.0f) + fmaxf(l - q, 0.0f);
    return d * d;
}

// Candidate sample j of the window, normalised: from the group's staged copy
// in shared memory (cs != nullptr) or from the series with the window's
// normalisation (x - na) * nb - nc.
template <typename T>
__device__ __forceinline__ T cand_value(const T *cs, const float *xw, T na, T nb, T nc, int j) {
    return cs ? cs[j] : tfma((T)xw[j] - na, nb, -nc);
}

template <typename T, int L, bool ABANDON>
__device__ T dtw_band(const T *__restrict__ qs, const float *__restrict__ xw, const T *cs, T na, T nb,
                      T nc, const TailCtx *tail, T *ring, int m, int r, T thr, unsigned gmask, int lane,
                      int &cells) {
    const T INF = tinf<T>();
    const int W = 2 * r + 1;
    const int R = (m + L - 1) / L;
    const int total = R * W + 2 * (L - 1);
    for (int t = lane; t <= W; t += L) ring[t] = (t == r) ? (T)0 : INF;

    float tot = 0.0f, pref_cur = 0.0f, pref_next = 0.0f, carry = 0.0f;
    if (ABANDON && tail) {
        float s = 0.0f;
        for (int i = lane; i < m; i += L) s += tail_term(*tail, i);
        tot = group_sum<L>(s, gmask);
        float e = lane < m ? tail_term(*tail, lane) : 0.0f;
        float inc = group_incl_scan<L>(e, gmask, lane);
        pref_cur = inc;
        carry = __shfl_sync(gmask, inc, L - 1, L);
    }
    __syncwarp(gmask);

    int k = -2 * lane, i = lane, wcount = 0;
    T qi = i < m ? qs[i] : (T)0;
    T out = INF, upPrev = INF, rmin = INF, res = INF;
    bool stop = false;
    // operands of the current step, loaded one step ahead: lane 0's ring
    // cells (written by lane L-1 at least two steps earlier, since L <= r)
    // and the candidate sample of this lane's cell
    T rk0 = INF, rk1 = INF, cj = (T)0;
    bool valid = false;
    {
        const bool act = (k >= 0) && (i < m);
        const int kk = act ? k : 0, j = i - r + k;
        if (lane == 0) { rk0 = ring[kk]; rk1 = ring[kk + 1]; }
        valid = act && j >= 0 && j < m;
        if (valid) cj = cand_value(cs, xw, na, nb, nc, j);
    }
    for (int s = 0; s < total; ++s) {
        const T upIn = __shfl_up_sync(gmask, out, 1, L);
        const bool act = (k >= 0) && (i < m);
        T up, diag;
        if (lane == 0) {
            up = rk1;
            diag = rk0;
        } else {
            up = (k + 1 < W) ? upIn : INF;
            diag = upPrev;
        }
        upPrev = upIn;
        const T left = (k > 0) ? out : INF;
        T v = INF;
        if (valid) {
            const T c = qi - cj;
            v = tfma(c, c, tmin(tmin(up, diag), left));
            ++cells;
        }
        out = v;
        if (lane == L - 1 && act) ring[k] = v;
        rmin = tmin(rmin, v);
        if (act && i == m - 1 && k == r) res = v;
        if (ABANDON && tail) {
            if (++wcount == W) {  // all lanes together: prefix of the next block's rows
                wcount = 0;
                const int row = ((s + 1) / W) * L + lane;
                const float e = row < m ? tail_term(*tail, row) : 0.0f;
                const float inc = group_incl_scan<L>(e, gmask, lane);
                pref_next = carry + inc;
                carry += __shfl_sync(gmask, inc, L - 1, L);
            }
        }
        if (++k == W) {
            if (ABANDON && act) {
                float rest = 0.0f;
                if (tail) rest = fmaxf(0.0f, (tot - pref_cur) - 1e-5f * tot);
                if ((float)rmin + rest > (float)thr) stop = true;
            }
            rmin = INF;
            k = 0;
            i += L;
            qi = i < m ? qs[i] : (T)0;
            pref_cur = pref_next;
        }
        {  // next step's operands
            const bool nact = (k >= 0) && (i < m);
            const int kk = nact ? k : 0, j = i - r + k;
            if (lane == 0) { rk0 = ring[kk]; rk1 = ring[kk + 1]; }
            valid = nact && j >= 0 && j < m;
            if (valid) cj = cand_value(cs, xw, na, nb, nc, j);
        }
        __syncwarp(gmask);
        if (ABANDON && (s & 15) == 15) {
            if (__any_sync(gmask, stop)) return INF;
        }
    }
    return __shfl_sync(gmask, res, (m - 1) % L, L);
}

// ------------------------------------------------------------------ anti-diagonal DTW
// The same recurrence (Eq. 1 on the band |i - j| <= r) evaluated along
// anti-diagonals a = i + j.  On anti-diagonal a the band holds the cells
// e = j - i in [-r, r] with e = a (mod 2); cell p (0-based) has
// e = e_min(a) + 2p, e_min(a) = -r + ((a + r) & 1), i = (a - e)/2,
// j = (a + e)/2.  Its neighbours are (i, j-1) and (i-1, j) on anti-diagonal
// a-1 and (i-1, j-1) on a-2; in cell indices that is
//   even (a + r):  left = prev1[p-1], up = prev1[p],   diag = prev2[p]
//   odd  (a + r):  left = prev1[p],   up = prev1[p+1], diag = prev2[p].
// A group of L lanes holds the r+1 cells of an anti-diagonal, K consecutive
// cells per lane in registers; the one neighbour held by the adjacent lane
// arrives by one shuffle per anti-diagonal.  2m - 1 steps, K independent
// cells per lane per step.  The base d(-1,-1) = 0 sits on anti-diagonal -2.
//
// Early abandon (ABANDON): every warping path visits anti-diagonal a or a+1,
// so min over the cells of two consecutive anti-diagonals of d(cell) plus a
// lower bound of the rows after the cell's row bounds DTW from below.  The
// rows' bound is a suffix sum of the rows' LB_Keogh terms (q_hat_i' against
// the window's envelope), kept every kTailG rows in shared memory
// (tail_suffix); tested once per unrolled iteration (at least 16 steps).
// Padding on each side of the query / window arrays the anti-diagonal kernel
// reads: cell indices run r/2 + L*K past either end.  The query is padded
// with +inf and the window with -inf, so every cell outside [0, m)^2 costs
// +inf (never NaN) and needs no bounds test.
__host__ __device__ inline int diag_pad(int r, int L, int K) { return (r >> 1) + L * K + 4; }

// Named barrier `id` over `nthreads` threads (a multiple of 32): the warps
// of one lane group meet without stopping the rest of the CTA.
__device__ __forceinline__ void group_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Three-input minimum (one instruction on sm_100 and later).  The DTW
// values are never NaN (out-of-band cells are +inf), so its NaN rule does
// not matter here.
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Band cells (the band |i - j| <= r of Eq. 1 inside [0, m)^2) on the
// anti-diagonals 0..A, in closed form.  G(B) counts the band's cells with
// i + j <= B for B <= m - 1, where only i, j >= 0 bind: anti-diagonal a
// holds a + 1 of them while a <= r, then r or r + 1 by parity.  Past the
// middle the complement follows from the symmetry (i, j) -> (m-1-i, m-1-j).
__host__ __device__ inline long long band_cells_upto(int A, int m, int r) {
    if (r > m - 1) r = m - 1;
    const long long T = (long long)m * (2 * r + 1) - (long long)r * (r + 1);
    if (A < 0) return 0;
    if (A >= 2 * m - 2) return T;
    auto G = [r](long long B) -> long long {
        if (B < 0) return 0;
        if (B <= r) return (B + 1) * (B + 2) / 2;
        return (long long)(r + 1) * (r + 2) / 2 + (B - r) * r + (B - r) / 2;
    };
    return A <= m - 1 ? G(A) : T - G(2LL * m - 3 - A);
}

// Anti-diagonal pairs per unrolled iteration of dtw_diag: a multiple of K
// (the register windows rotate by one slot per pair, so after K pairs every
// value is back in its own register) and at least 8.
__host__ __device__ constexpr int diag_unroll(int K) { return K * ((8 + K - 1) / K); }

// Rows per entry of the coarse tail bound cbs that dtw_diag reads: entry g
// holds the bound of the rows from kTailG*g on.
constexpr int kTailG = 8;
__host__ __device__ inline int tail_entries(int m) { return (m + kTailG - 1) / kTailG + 1; }

// One anti-diagonal step of dtw_diag: lane cell t (position p = lane*K + t
// along the anti-diagonal) takes its left / up neighbours from the previous
// anti-diagonal (p1, with one value from the adjacent lane), its diagonal
// one from the one before (p2), and the query / window values from the
// register windows, whose logical element t sits in physical slot
// (t - QP) mod K (query) and (t + CP) mod K (window).
//
// Cells past the band: with every cell past the band held at +inf, an
// even (a + r) step's cells p > r see only such cells, and an odd step's
// cells p > r as well; the odd step's cell p = r alone has a neighbour in
// the band (its left, cell r of the even anti-diagonal), so only that cell
// is forced to +inf, by the per-lane penalty pen (K <= 8) or a compare.
template <int L, int K, int ODD, int QP, int CP>
__device__ __forceinline__ void diag_step(const float (&qv)[K], const float (&cv)[K], float (&p1)[K],
                                          float (&p2)[K], const float (&pen)[K], int lane, int r, unsigned gmask) {
    const float INF = __int_as_float(0x7f800000);
    // the one neighbour held by the adjacent lane: p-1 (even) / p+1 (odd)
    float nb = __shfl_sync(gmask, ODD ? p1[0] : p1[K - 1], ODD ? ((lane + 1) & (L - 1)) : ((lane - 1) & (L - 1)), L);
    if (ODD ? (lane == L - 1) : (lane == 0)) nb = INF;
    float cur[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const float left = ODD ? p1[t] : (t == 0 ? nb : p1[t > 0 ? t - 1 : 0]);
        const float up = ODD ? (t == K - 1 ? nb : p1[t < K - 1 ? t + 1 : 0]) : p1[t];
        const float d = qv[((t - QP) % K + K) % K] - cv[(t + CP) % K];
        float v = fmaf(d, d, min3f(left, up, p2[t]));
        if (ODD) {
            // pen is 0 or +inf and v >= 0: an add, which the FMA pipe takes,
            // instead of a maximum on the ALU pipe, the walk's busiest
            if constexpr (K <= 8) v = v + pen[t];
            else if (lane * K + t == r) v = INF;
        }
        cur[t] = v;
    }
#pragma unroll
    for (int t = 0; t < K; ++t) {
        p2[t] = p1[t];
        p1[t] = cur[t];
    }
}

// Register windows of the anti-diagonal walk: cell p of a step reads
// q[qbase - p] and c[cbase + p].  After an even step cbase grows by one (the
// window values move one cell down, the last lane loads the new one); after
// an odd step qbase grows by one (the query values move one cell up, lane 0
// loads the new one).  The move is a rotation: the slot whose value leaves
// the lane takes the arriving one, and the phase (CP, QP) advances.
template <int L, int K, int CP>
__device__ __forceinline__ void rot_c(float (&cv)[K], const float *cp, int cbase_new, int lane, unsigned gmask) {
    constexpr int s = CP % K;  // logical 0: leaves downwards, becomes logical K-1
    const float from_next = __shfl_down_sync(gmask, cv[s], 1, L);
    const float fresh = cp[cbase_new + L * K - 1];
    cv[s] = lane == L - 1 ? fresh : from_next;
}
template <int L, int K, int QP>
__device__ __forceinline__ void rot_q(float (&qv)[K], const float *qp, int qbase_new, int lane, unsigned gmask) {
    constexpr int s = ((K - 1 - QP) % K + K) % K;  // logical K-1: leaves upwards, becomes logical 0
    const float from_prev = __shfl_up_sync(gmask, qv[s], 1, L);
    const float fresh = qp[qbase_new];
    qv[s] = lane == 0 ? fresh : from_prev;
}

// The same moves without rotation (phase 0 before and after): the values
// move one register along, the leaving one goes to the adjacent lane.
template <int L, int K>
__device__ __forceinline__ void shift_c(float (&cv)[K], const float *cp, int cbase_new, int lane, unsigned gmask) {
    const float from_next = __shfl_down_sync(gmask, cv[0], 1, L);
    const float fresh = cp[cbase_new + L * K - 1];
#pragma unroll
    for (int t = 0; t < K - 1; ++t) cv[t] = cv[t + 1];
    cv[K - 1] = lane == L - 1 ? fresh : from_next;
}
template <int L, int K>
__device__ __forceinline__ void shift_q(float (&qv)[K], const float *qp, int qbase_new, int lane, unsigned gmask) {
    const float from_prev = __shfl_up_sync(gmask, qv[K - 1], 1, L);
    const float fresh = qp[qbase_new];
#pragma unroll
    for (int t = K - 1; t > 0; --t) qv[t] = qv[t - 1];
    qv[0] = lane == 0 ? fresh : from_prev;
}

// The end of the walk: d(m-1, m-1) is cell pe of the last anti-diagonal.
template <int K>
__device__ __forceinline__ float diag_result(const float (&p1)[K], int lane, int pe) {
    float res = __int_as_float(0x7f800000);
#pragma unroll
    for (int t = 0; t < K; ++t)
        if (lane * K + t == pe) res = p1[t];
    return res;
}

// qp, cp: the query and the group's normalised window, each padded by
// diag_pad(r, L, K) elements (+inf / -inf) on both sides, pointing at
// element 0.  cbs: the rows' coarse tail bound for ABANDON (or nullptr):
// cbs[g] bounds the cost of the rows kTailG*g .. m-1 from below, so the
// rows after row i are bounded by cbs[ceil((i+1)/kTailG)] (fewer rows, a
// smaller sum).  cells: lane 0 accumulates the cells evaluated (in the band
// and the matrix).  The walk takes diag_unroll(K) anti-diagonal pairs per
// iteration; the abandon test runs once per iteration.
template <typename T, int L, int K, bool ABANDON>
__device__ T dtw_diag(const T *__restrict__ qp, const T *__restrict__ cp, const float *cbs, int m, int r, T thr,
                      unsigned gmask, int lane, int &cells) {
    static_assert(sizeof(T) == 4, "the FP32 walk");
    constexpr int U = diag_unroll(K);
    const float INF = __int_as_float(0x7f800000);
    const int p0 = (r - (r & 1)) >> 1;
    float p1[K], p2[K], qv[K], cv[K], pen[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        p1[t] = INF;
        p2[t] = (lane * K + t == p0) ? 0.0f : INF;
        pen[t] = (lane * K + t == r) ? INF : 0.0f;
    }
    const int last = 2 * m - 2;
    const int pe_even = r >> 1, pe_odd = (r - 1) >> 1;  // cell e = 0 by the parity of (last + r)
    // anti-diagonal a has e_min = -r + ((a + r) & 1); its first cell is
    // (bi, bj) = ((a - e_min)/2, (a + e_min)/2).  Along an (even, odd) pair
    // bi stays and bj grows by one; from pair to pair both grow by one.
    int a = 0;
    if (r & 1) {  // a = 0 is odd: e_min = 1 - r; one odd step, then the query window shifts
        const int qb = (r - 1) >> 1, cb = (1 - r) >> 1;
#pragma unroll
        for (int t = 0; t < K; ++t) {
            qv[t] = qp[qb - (lane * K + t)];
            cv[t] = cp[cb + (lane * K + t)];
        }
        diag_step<L, K, 1, 0, 0>(qv, cv, p1, p2, pen, lane, r, gmask);
        a = 1;
        shift_q<L, K>(qv, qp, qb + 1, lane, gmask);
    } else {
        const int qb = r >> 1, cb = -(r >> 1);
#pragma unroll
        for (int t = 0; t < K; ++t) {
            qv[t] = qp[qb - (lane * K + t)];
            cv[t] = cp[cb + (lane * K + t)];
        }
    }
    int bi = (a + r) >> 1, bj = (a - r) >> 1;
    float res = INF;
    // iterations that end before the last anti-diagonal need no end test
    while (a + 2 * U - 1 < last) {
        static_for<U>([&](auto uc) {
            constexpr int u = decltype(uc)::value;
            diag_step<L, K, 0, u % K, u % K>(qv, cv, p1, p2, pen, lane, r, gmask);
            rot_c<L, K, u % K>(cv, cp, bj + u + 1, lane, gmask);
            diag_step<L, K, 1, u % K, (u + 1) % K>(qv, cv, p1, p2, pen, lane, r, gmask);
            rot_q<L, K, u % K>(qv, qp, bi + u + 1, lane, gmask);
        });
        a += 2 * U;
        bi += U;
        bj += U;
        if (ABANDON) {
            // p1: anti-diagonal a-1, p2: a-2, both on rows bi - 1 - p
            float low = INF;
#pragma unroll
            for (int t = 0; t < K; ++t) {
                const int i = bi - 1 - (lane * K + t);
                const float tail = (cbs && i >= 0 && i < m) ? cbs[(i + kTailG) / kTailG] : 0.0f;
                low = fminf(low, fminf(p1[t], p2[t]) + tail);
            }
#pragma unroll
            for (int o = L / 2; o > 0; o >>= 1) low = fminf(low, __shfl_xor_sync(gmask, low, o, L));
            if (low > (float)thr) {
                if (lane == 0) cells += (int)band_cells_upto(a - 1, m, r);  // anti-diagonals 0..a-1
                return (T)INF;
            }
        }
    }
    // the rest (fewer than U pairs), one pair at a time: the rotation phase
    // is 0 here (the loop above took whole multiples of K pairs), so the
    // windows shift by register moves and keep that phase
    for (;; a += 2, ++bi, ++bj) {
        diag_step<L, K, 0, 0, 0>(qv, cv, p1, p2, pen, lane, r, gmask);
        if (a == last) {
            res = diag_result<K>(p1, lane, pe_even);
            break;
        }
        shift_c<L, K>(cv, cp, bj + 1, lane, gmask);
        diag_step<L, K, 1, 0, 0>(qv, cv, p1, p2, pen, lane, r, gmask);
        if (a + 1 == last) {
            res = diag_result<K>(p1, lane, pe_odd);
            break;
        }
        shift_q<L, K>(qv, qp, bi + 1, lane, gmask);
    }
    if (lane == 0) cells += (int)band_cells_upto(last, m, r);
    // d(m-1, m-1): e = 0 on the last anti-diagonal
    const int pe = ((last + r) & 1) ? pe_odd : pe_even;
    return (T)__shfl_sync(gmask, res, pe / K, L);
}

// ------------------------------------------------------------------ multi-warp FP32 walk
// dtw_diag with the r+1 cells of an anti-diagonal spread over W warps of one
// group (32 W lanes, K cells each): bands up to 32 W K - 1 (2047 with four
// warps of 16 cells).  Inside a warp the neighbour cell arrives by shuffle;
// across a warp boundary through shared memory: after each step every warp's
// first and last lane publish their newest cell into the other half of a
// double buffer and the group meets at its named barrier, so a step's reads
// (this half) never race the next step's writes (the other half).  The
// register windows rotate as in dtw_diag; each warp's boundary lane loads
// its fresh value from the padded arrays instead of a neighbour warp.
struct MwXchg {
    float first[2][8], last[2][8];  // [buffer][warp]: lane 0's p1[0], lane 31's p1[K-1]
    float red[2][8];                // per-warp partial sums / minima
    float res;
};

template <int W, int K, int ODD, int QP, int CP>
__device__ __forceinline__ void diag_step_mw(const float (&qv)[K], const float (&cv)[K], float (&p1)[K],
                                             float (&p2)[K], const float (&pen)[K], int gl, int lane, int w, int r,
                                             const MwXchg &x, int buf) {
    const float INF = __int_as_float(0x7f800000);
    float nb = __shfl_sync(0xffffffffu, ODD ? p1[0] : p1[K - 1], ODD ? ((lane + 1) & 31) : ((lane - 1) & 31));
    if (ODD) {
        if (lane == 31) nb = (w == W - 1) ? INF : x.first[buf][w + 1];
    } else {
        if (lane == 0) nb = (w == 0) ? INF : x.last[buf][w - 1];
    }
    float cur[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const float left = ODD ? p1[t] : (t == 0 ? nb : p1[t > 0 ? t - 1 : 0]);
        const float up = ODD ? (t == K - 1 ? nb : p1[t < K - 1 ? t + 1 : 0]) : p1[t];
        const float d = qv[((t - QP) % K + K) % K] - cv[(t + CP) % K];
        float v = fmaf(d, d, min3f(left, up, p2[t]));
        if (ODD) {
            if constexpr (K <= 8) v = v + pen[t];  // (as in diag_step)
            else if (gl * K + t == r) v = INF;
        }
        cur[t] = v;
    }
#pragma unroll
    for (int t = 0; t < K; ++t) {
        p2[t] = p1[t];
        p1[t] = cur[t];
    }
}

template <int W, int K>
__device__ __forceinline__ void mw_publish(const float (&p1)[K], int lane, int w, MwXchg &x, int &buf, int bar) {
    const int nbuf = buf ^ 1;
    if (lane == 0) x.first[nbuf][w] = p1[0];
    if (lane == 31) x.last[nbuf][w] = p1[K - 1];
    group_bar(bar, 32 * W);
    buf = nbuf;
}

template <int K, int CP>
__device__ __forceinline__ void rot_c_mw(float (&cv)[K], const float *cp, int cbase_new, int gl, int lane) {
    constexpr int s = CP % K;
    const float from_next = __shfl_down_sync(0xffffffffu, cv[s], 1);
    const float fresh = cp[cbase_new + (gl + 1) * K - 1];
    cv[s] = lane == 31 ? fresh : from_next;
}
template <int K, int QP>
__device__ __forceinline__ void rot_q_mw(float (&qv)[K], const float *qp, int qbase_new, int gl, int lane) {
    constexpr int s = ((K - 1 - QP) % K + K) % K;
    const float from_prev = __shfl_up_sync(0xffffffffu, qv[s], 1);
    const float fresh = qp[qbase_new - gl * K];
    qv[s] = lane == 0 ? fresh : from_prev;
}
template <int K>
__device__ __forceinline__ void shift_c_mw(float (&cv)[K], const float *cp, int cbase_new, int gl, int lane) {
    const float from_next = __shfl_down_sync(0xffffffffu, cv[0], 1);
    const float fresh = cp[cbase_new + (gl + 1) * K - 1];
#pragma unroll
    for (int t = 0; t < K - 1; ++t) cv[t] = cv[t + 1];
    cv[K - 1] = lane == 31 ? fresh : from_next;
}
template <int K>
__device__ __forceinline__ void shift_q_mw(float (&qv)[K], const float *qp, int qbase_new, int gl, int lane) {
    const float from_prev = __shfl_up_sync(0xffffffffu, qv[K - 1], 1);
    const float fresh = qp[qbase_new - gl * K];
#pragma unroll
    for (int t = K - 1; t > 0; --t) qv[t] = qv[t - 1];
    qv[0] = lane == 0 ? fresh : from_prev;
}

// qp, cp: element 0 of the query / the group's normalised window, padded by
// diag_pad(r, 32*W, K) on both sides (+inf / -inf); cbs: the coarse tail
// bound (as dtw_diag) or nullptr.  Called by all 32 W threads of warps
// w = 0..W-1 of the group; bar: the group's named barrier.  Every thread
// returns the distance (+inf when abandoned); thread 0 of the group adds the
// cells evaluated to `cells`.
template <int W, int K, bool ABANDON>
__device__ float dtw_diag_mw(const float *__restrict__ qp, const float *__restrict__ cp, const float *cbs, int m,
                             int r, float thr, int w, int lane, MwXchg &x, int bar, int &cells) {
    static_assert(W >= 2 && W <= 8, "two to eight warps");
    constexpr int U = diag_unroll(K);
    const float INF = __int_as_float(0x7f800000);
    const int gl = w * 32 + lane;
    const int p0 = (r - (r & 1)) >> 1;
    float p1[K], p2[K], qv[K], cv[K], pen[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        p1[t] = INF;
        p2[t] = (gl * K + t == p0) ? 0.0f : INF;
        pen[t] = (gl * K + t == r) ? INF : 0.0f;
    }
    int buf = 1;
    mw_publish<W, K>(p1, lane, w, x, buf, bar);  // buffer 0 := the all-inf anti-diagonal -1
    const int last = 2 * m - 2;
    const int pe_even = r >> 1, pe_odd = (r - 1) >> 1;
    int a = 0;
    if (r & 1) {
        const int qb = (r - 1) >> 1, cb = (1 - r) >> 1;
#pragma unroll
        for (int t = 0; t < K; ++t) {
            qv[t] = qp[qb - (gl * K + t)];
            cv[t] = cp[cb + (gl * K + t)];
        }
        diag_step_mw<W, K, 1, 0, 0>(qv, cv, p1, p2, pen, gl, lane, w, r, x, buf);
        mw_publish<W, K>(p1, lane, w, x, buf, bar);
        a = 1;
        shift_q_mw<K>(qv, qp, qb + 1, gl, lane);
    } else {
        const int qb = r >> 1, cb = -(r >> 1);
#pragma unroll
        for (int t = 0; t < K; ++t) {
            qv[t] = qp[qb - (gl * K + t)];
            cv[t] = cp[cb + (gl * K + t)];
        }
    }
    int bi = (a + r) >> 1, bj = (a - r) >> 1;
    while (a + 2 * U - 1 < last) {
        static_for<U>([&](auto uc) {
            constexpr int u = decltype(uc)::value;
            diag_step_mw<W, K, 0, u % K, u % K>(qv, cv, p1, p2, pen, gl, lane, w, r, x, buf);
            mw_publish<W, K>(p1, lane, w, x, buf, bar);
            rot_c_mw<K, u % K>(cv, cp, bj + u + 1, gl, lane);
            diag_step_mw<W, K, 1, u % K, (u + 1) % K>(qv, cv, p1, p2, pen, gl, lane, w, r, x, buf);
            mw_publish<W, K>(p1, lane, w, x, buf, bar);
            rot_q_mw<K, u % K>(qv, qp, bi + u + 1, gl, lane);
        });
        a += 2 * U;
        bi += U;
        bj += U;
        if (ABANDON) {
            float low = INF;
#pragma unroll
            for (int t = 0; t < K; ++t) {
                const int i = bi - 1 - (gl * K + t);
                const float tail = (cbs && i >= 0 && i < m) ? cbs[(i + kTailG) / kTailG] : 0.0f;
                low = fminf(low, fminf(p1[t], p2[t]) + tail);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) low = fminf(low, __shfl_xor_sync(0xffffffffu, low, o));
            if (lane == 0) x.red[0][w] = low;
            group_bar(bar, 32 * W);
#pragma unroll
            for (int v = 0; v < W; ++v) low = fminf(low, x.red[0][v]);
            if (low > thr) {
                if (gl == 0) cells += (int)band_cells_upto(a - 1, m, r);
                group_bar(bar, 32 * W);  // x.red is read before anyone writes it again
                return INF;
            }
        }
    }
    bool at_end = false;
    for (;; a += 2, ++bi, ++bj) {
        diag_step_mw<W, K, 0, 0, 0>(qv, cv, p1, p2, pen, gl, lane, w, r, x, buf);
        mw_publish<W, K>(p1, lane, w, x, buf, bar);
        if (a == last) {
#pragma unroll
            for (int t = 0; t < K; ++t)
                if (gl * K + t == pe_even) x.res = p1[t];
            at_end = true;
        }
        if (at_end) break;
        shift_c_mw<K>(cv, cp, bj + 1, gl, lane);
        diag_step_mw<W, K, 1, 0, 0>(qv, cv, p1, p2, pen, gl, lane, w, r, x, buf);
        mw_publish<W, K>(p1, lane, w, x, buf, bar);
        if (a + 1 == last) {
#pragma unroll
            for (int t = 0; t < K; ++t)
                if (gl * K + t == pe_odd) x.res = p1[t];
            at_end = true;
        }
        if (at_end) break;
        shift_q_mw<K>(qv, qp, bi + 1, gl, lane);
    }
    group_bar(bar, 32 * W);
    const float res = x.res;
    if (gl == 0) cells += (int)band_cells_upto(last, m, r);
    group_bar(bar, 32 * W);  // x.res is read before the next walk writes it
    return res;
}

// Knuth's error-free transformations (TwoSum, FastTwoSum, FMA-based
// products).  It runs on the FP32 pipes, which on this part issue far more
// than its FP64 units; accumulated relative error over a DTW is ~1e-14.
struct dfloat {
    float hi, lo;
};
__device__ __forceinline__ dfloat df_from(double v) {
    const float h = (float)v;
    return dfloat{h, (float)(v - (double)h)};
}
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return dfloat{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
    const float s = a + b;
    return dfloat{s, b - (s - a)};
}
// x + y for x, y >= 0 (all DTW partial sums are)
__device__ __forceinline__ dfloat df_add_pos(dfloat x, dfloat y) {
    const dfloat s = df_two_sum(x.hi, y.hi);
    return df_fast_two_sum(s.hi, (s.lo + x.lo) + y.lo);
}
__device__ __forceinline__ dfloat df_sub(dfloat x, dfloat y) {
    const dfloat s = df_two_sum(x.hi, -y.hi);
    return df_fast_two_sum(s.hi, s.lo + (x.lo - y.lo));
}
__device__ __forceinline__ dfloat df_sqr(dfloat d) {
    const float p = d.hi * d.hi;
    float e = fmaf(d.hi, d.hi, -p);
    e = fmaf(2.0f * d.hi, d.lo, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfloat df_min(dfloat x, dfloat y) {
    return (y.hi < x.hi || (y.hi == x.hi && y.lo < x.lo)) ? y : x;
}
__device__ __forceinline__ dfloat df_shfl(unsigned mask, dfloat v, int src, int width) {
    return dfloat{__shfl_sync(mask, v.hi, src, width), __shfl_sync(mask, v.lo, src, width)};
}

// One anti-diagonal step of dtw_diag_df: as diag_step, in double-float
// arithmetic, with the query / window values in the register windows qv, cv.
template <int L, int K, int ODD>
__device__ __forceinline__ void diag_step_df(const dfloat (&qv)[K], const dfloat (&cv)[K], dfloat (&p1)[K],
                                             dfloat (&p2)[K], int lane, int r, unsigned gmask) {
    // a large finite stand-in for +inf: sums of such values stay finite
    const dfloat INF = dfloat{1e30f, 0.0f};
    dfloat nb = df_shfl(gmask, ODD ? p1[0] : p1[K - 1], ODD ? ((lane + 1) & (L - 1)) : ((lane - 1) & (L - 1)), L);
    if (ODD ? (lane == L - 1) : (lane == 0)) nb = INF;
    dfloat cur[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const int p = lane * K + t;
        const dfloat left = ODD ? p1[t] : (t == 0 ? nb : p1[t > 0 ? t - 1 : 0]);
        const dfloat up = ODD ? (t == K - 1 ? nb : p1[t < K - 1 ? t + 1 : 0]) : p1[t];
        // the query / window arrays are padded with finite poison values
        // (+/-1e15): a cell outside [0, m)^2 costs ~4e30, far above any DTW
        // and far below FP32 overflow over 2m steps, and never turns
        // TwoSum into NaN
        // (the cell's own predecessor and the diagonal first: only the last
        // minimum waits for the neighbour lane's value; the minimum of
        // double-floats is exact, so the order does not change the result)
        const dfloat best = ODD ? df_min(up, df_min(left, p2[t])) : df_min(left, df_min(up, p2[t]));
        dfloat v = df_add_pos(df_sqr(df_sub(qv[t], cv[t])), best);
        if (ODD ? (p >= r) : (p > r)) v = INF;  // past the band's cells
        cur[t] = v;
    }
#pragma unroll
    for (int t = 0; t < K; ++t) {
        p2[t] = p1[t];
        p1[t] = cur[t];
    }
}

// Register windows of the double-float walk (as shift_c / shift_q).
template <int L, int K>
__device__ __forceinline__ void shift_c_df(dfloat (&cv)[K], const dfloat *cp, int cbase_new, int lane,
                                           unsigned gmask) {
    const dfloat from_next =
        dfloat{__shfl_down_sync(gmask, cv[0].hi, 1, L), __shfl_down_sync(gmask, cv[0].lo, 1, L)};
    const dfloat fresh = cp[cbase_new + L * K - 1];
#pragma unroll
    for (int t = 0; t < K - 1; ++t) cv[t] = cv[t + 1];
    cv[K - 1] = lane == L - 1 ? fresh : from_next;
}
template <int L, int K>
__device__ __forceinline__ void shift_q_df(dfloat (&qv)[K], const dfloat *qp, int qbase_new, int lane,
                                           unsigned gmask) {
    const dfloat from_prev =
        dfloat{__shfl_up_sync(gmask, qv[K - 1].hi, 1, L), __shfl_up_sync(gmask, qv[K - 1].lo, 1, L)};
    const dfloat fresh = qp[qbase_new];
#pragma unroll
    for (int t = K - 1; t > 0; --t) qv[t] = qv[t - 1];
    qv[0] = lane == 0 ? fresh : from_prev;
}

// Double-float counterpart of dtw_diag (no abandon), the same walk and the
// same register windows.  qs, cs point at element 0 of arrays padded by
// diag_pad(r, L, K) on both sides with +1e15 (query) and -1e15 (window).
template <int L, int K>
__device__ double dtw_diag_df(const dfloat *__restrict__ qs, const dfloat *__restrict__ cs, int m, int r,
                              unsigned gmask, int lane) {
    const dfloat INF = dfloat{1e30f, 0.0f};
    const int p0 = (r - (r & 1)) >> 1;
    dfloat p1[K], p2[K], qv[K], cv[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        p1[t] = INF;
        p2[t] = (lane * K + t == p0) ? dfloat{0.0f, 0.0f} : INF;
    }
    const int last = 2 * m - 2;
    int a = 0, bi, bj;
    if (r & 1) {
        const int qb = (r - 1) >> 1, cb = (1 - r) >> 1;
#pragma unroll
        for (int t = 0; t < K; ++t) {
            qv[t] = qs[qb - (lane * K + t)];
            cv[t] = cs[cb + (lane * K + t)];
        }
        diag_step_df<L, K, 1>(qv, cv, p1, p2, lane, r, gmask);
        a = 1;
        shift_q_df<L, K>(qv, qs, qb + 1, lane, gmask);
    } else {
        const int qb = r >> 1, cb = -(r >> 1);
#pragma unroll
        for (int t = 0; t < K; ++t) {
            qv[t] = qs[qb - (lane * K + t)];
            cv[t] = cs[cb + (lane * K + t)];
        }
    }
    bi = (a + r) >> 1;
    bj = (a - r) >> 1;
    for (; a + 1 <= last; a += 2, ++bi, ++bj) {
        diag_step_df<L, K, 0>(qv, cv, p1, p2, lane, r, gmask);
        shift_c_df<L, K>(cv, cs, bj + 1, lane, gmask);
        diag_step_df<L, K, 1>(qv, cv, p1, p2, lane, r, gmask);
        shift_q_df<L, K>(qv, qs, bi + 1, lane, gmask);
    }
    if (a == last) diag_step_df<L, K, 0>(qv, cv, p1, p2, lane, r, gmask);
    const int pe = (r - ((last + r) & 1)) >> 1;
    dfloat res = INF;
#pragma unroll
    for (int t = 0; t < K; ++t)
        if (lane * K + t == pe) res = p1[t];
    res = df_shfl(gmask, res, pe / K, L);
    return (double)res.hi + (double)res.lo;
}

// ------------------------------------------------------------------ multi-warp double-float walk
// The same walk with the r+1 cells of an anti-diagonal spread over W warps
// (32*W lanes, K cells each; W <= 8).  Inside a warp the neighbour arrives by
// shuffle as in dtw_diag_df; across a warp boundary it goes through shared
// memory: after each step every warp's first and last lane publish their
// newest cell into the other half of a double buffer and the W warps meet at
// one named barrier, so a step's reads (this half) never race the next
// step's writes (the other half).  The register windows' boundary lanes load
// their fresh value from the padded arrays instead of a neighbour warp.
struct DfXchg {
    dfloat first[2][8], last[2][8];  // [buffer][warp]: lane 0's p1[0], lane 31's p1[K-1]
    dfloat res;
};


// The cells' costs (q_hat_i - c_j)^2 of a step, from its register windows.
template <int K>
__device__ __forceinline__ void df_costs(const dfloat (&qv)[K], const dfloat (&cv)[K], dfloat (&cst)[K]) {
#pragma unroll
    for (int t = 0; t < K; ++t) cst[t] = df_sqr(df_sub(qv[t], cv[t]));
}

// A step of the multi-warp walk with its cells' costs given (computed while
// the previous step's values were still on their way: only the minimum and
// the addition wait for them).
template <int W, int K, int ODD>
__device__ __forceinline__ void diag_step_df_mw(const dfloat (&cst)[K], dfloat (&p1)[K],
                                                dfloat (&p2)[K], int gl, int lane, int w, int r,
                                                const DfXchg &x, int buf) {
    const dfloat INF = dfloat{1e30f, 0.0f};
    dfloat nb = df_shfl(0xffffffffu, ODD ? p1[0] : p1[K - 1], ODD ? ((lane + 1) & 31) : ((lane - 1) & 31), 32);
    if (ODD) {
        if (lane == 31) nb = (w == W - 1) ? INF : x.first[buf][w + 1];
    } else {
        if (lane == 0) nb = (w == 0) ? INF : x.last[buf][w - 1];
    }
    dfloat cur[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const int p = gl * K + t;
        const dfloat left = ODD ? p1[t] : (t == 0 ? nb : p1[t > 0 ? t - 1 : 0]);
        const dfloat up = ODD ? (t == K - 1 ? nb : p1[t < K - 1 ? t + 1 : 0]) : p1[t];
        const dfloat best = ODD ? df_min(up, df_min(left, p2[t])) : df_min(left, df_min(up, p2[t]));
        dfloat v = df_add_pos(cst[t], best);
        if (ODD ? (p >= r) : (p > r)) v = INF;
        cur[t] = v;
    }
#pragma unroll
    for (int t = 0; t < K; ++t) {
        p2[t] = p1[t];
        p1[t] = cur[t];
    }
}

template <int W, int K>
__device__ __forceinline__ void df_mw_publish(const dfloat (&p1)[K], int lane, int w, DfXchg &x, int &buf,
                                              int bar_id) {
    if constexpr (W == 1) {  // one warp: no other warp reads the boundary cells
        buf ^= 1;
        return;
    }
    const int nbuf = buf ^ 1;
    if (lane == 0) x.first[nbuf][w] = p1[0];
    if (lane == 31) x.last[nbuf][w] = p1[K - 1];
    group_bar(bar_id, 32 * W);
    buf = nbuf;
}

// Register windows of the multi-warp walk (as shift_c_df / shift_q_df);
// each warp's boundary lane loads its fresh value from the padded array.
template <int K>
__device__ __forceinline__ void shift_c_df_mw(dfloat (&cv)[K], const dfloat *cs, int cbase_new, int gl, int lane) {
    const dfloat from_next =
        dfloat{__shfl_down_sync(0xffffffffu, cv[0].hi, 1), __shfl_down_sync(0xffffffffu, cv[0].lo, 1)};
    const dfloat fresh = cs[cbase_new + (gl + 1) * K - 1];
#pragma unroll
    for (int t = 0; t < K - 1; ++t) cv[t] = cv[t + 1];
    cv[K - 1] = lane == 31 ? fresh : from_next;
}
template <int K>
__device__ __forceinline__ void shift_q_df_mw(dfloat (&qv)[K], const dfloat *qs, int qbase_new, int gl, int lane) {
    const dfloat from_prev =
        dfloat{__shfl_up_sync(0xffffffffu, qv[K - 1].hi, 1), __shfl_up_sync(0xffffffffu, qv[K - 1].lo, 1)};
    const dfloat fresh = qs[qbase_new - gl * K];
#pragma unroll
    for (int t = K - 1; t > 0; --t) qv[t] = qv[t - 1];
    qv[0] = lane == 0 ? fresh : from_prev;
}

// qs, cs: element 0 of arrays padded by diag_pad(r, 32*W, K) on both sides
// with +1e15 / -1e15.  Called by all 32*W threads of warps w = 0..W-1 of the
// group (w: the warp's index in the group); bar_id: a named barrier the group
// owns.  Every lane returns the distance.
template <int W, int K>
__device__ double dtw_diag_df_mw(const dfloat *__restrict__ qs, const dfloat *__restrict__ cs, int m, int r, int w,
                                 int lane, DfXchg &x, int bar_id) {
    static_assert(W >= 1 && W <= 8, "at most eight warps");
    const dfloat INF = dfloat{1e30f, 0.0f};
    const int gl = w * 32 + lane;
    const int p0 = (r - (r & 1)) >> 1;
    dfloat p1[K], p2[K], qv[K], cv[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        p1[t] = INF;
        p2[t] = (gl * K + t == p0) ? dfloat{0.0f, 0.0f} : INF;
        qv[t] = cv[t] = INF;  // (loaded below)
    }
    int buf = 1;
    df_mw_publish<W, K>(p1, lane, w, x, buf, bar_id);  // buffer 0 := the all-inf anti-diagonal -1
    const int last = 2 * m - 2;
    int a = 0, bi, bj;
    // each step's costs are formed before the previous step's exchange, so
    // the chain from one step's values to the next holds only the minimum,
    // the addition and the exchange
    dfloat cst[K], cst2[K];
    if (r & 1) {
        const int qb = (r - 1) >> 1, cb = (1 - r) >> 1;
#pragma unroll
        for (int t = 0; t < K; ++t) {
            qv[t] = qs[qb - (gl * K + t)];
            cv[t] = cs[cb + (gl * K + t)];
        }
        df_costs<K>(qv, cv, cst);
        diag_step_df_mw<W, K, 1>(cst, p1, p2, gl, lane, w, r, x, buf);
        shift_q_df_mw<K>(qv, qs, qb + 1, gl, lane);
        df_costs<K>(qv, cv, cst);
        df_mw_publish<W, K>(p1, lane, w, x, buf, bar_id);
        a = 1;
    } else {
        const int qb = r >> 1, cb = -(r >> 1);
#pragma unroll
        for (int t = 0; t < K; ++t) {
            qv[t] = qs[qb - (gl * K + t)];
            cv[t] = cs[cb + (gl * K + t)];
        }
        df_costs<K>(qv, cv, cst);
    }
    bi = (a + r) >> 1;
    bj = (a - r) >> 1;
    for (; a + 1 <= last; a += 2, ++bi, ++bj) {
        if constexpr (K <= 2 || W >= 8) {
            // even step a (costs in cst); the odd step's operands and costs
            shift_c_df_mw<K>(cv, cs, bj + 1, gl, lane);
            df_costs<K>(qv, cv, cst2);
            diag_step_df_mw<W, K, 0>(cst, p1, p2, gl, lane, w, r, x, buf);
            df_mw_publish<W, K>(p1, lane, w, x, buf, bar_id);
            // odd step a + 1 (costs in cst2); the next even step's
            shift_q_df_mw<K>(qv, qs, bi + 1, gl, lane);
            df_costs<K>(qv, cv, cst);
            diag_step_df_mw<W, K, 1>(cst2, p1, p2, gl, lane, w, r, x, buf);
            df_mw_publish<W, K>(p1, lane, w, x, buf, bar_id);
        } else {
            // (measured per window: ahead, 148 us instead of 173 at m = 512,
            // r = 51 on 2 warps x 1 cell and 2.14 ms instead of 2.25 at
            // m = 2048, r = 1843 on 8 warps x 8 cells, but 0.29 ms instead
            // of 0.18 at m = 1024, r = 921 on 4 warps x 8 cells)
            diag_step_df_mw<W, K, 0>(cst, p1, p2, gl, lane, w, r, x, buf);
            df_mw_publish<W, K>(p1, lane, w, x, buf, bar_id);
            shift_c_df_mw<K>(cv, cs, bj + 1, gl, lane);
            df_costs<K>(qv, cv, cst2);
            diag_step_df_mw<W, K, 1>(cst2, p1, p2, gl, lane, w, r, x, buf);
            df_mw_publish<W, K>(p1, lane, w, x, buf, bar_id);
            shift_q_df_mw<K>(qv, qs, bi + 1, gl, lane);
            df_costs<K>(qv, cv, cst);
        }
    }
    if (a == last) diag_step_df_mw<W, K, 0>(cst, p1, p2, gl, lane, w, r, x, buf);
    const int pe = (r - ((last + r) & 1)) >> 1;
#pragma unroll
    for (int t = 0; t < K; ++t)
        if (gl * K + t == pe) x.res = p1[t];
    group_bar(bar_id, 32 * W);
    const dfloat res = x.res;
    return (double)res.hi + (double)res.lo;
}

// Suffix sums of the rows' LB_Keogh terms for the abandon test of dtw_diag,
// kept every kTailG rows: cbs[g] = sum_{i >= kTailG*g} (q_hat_i against the
// window's normalised envelope interval at i)^2, cbs[tail_entries(m) - 1] =
// 0, shrunk by 1e-5 of the total so FP32 rounding of the sums can only
// weaken the bound.  cbs[0] is the whole Eq. 10 bound.  Rows are taken L at
// a time (coalesced loads), from the last chunk to the first, with a suffix
// scan across the group per chunk.
template <int L>
__device__ void tail_suffix(const TailCtx &tc, float *cbs, int m, unsigned gmask, int lane) {
    const int chunks = (m + L - 1) / L;
    float carry = 0.0f;
    for (int c = chunks - 1; c >= 0; --c) {
        const int i = c * L + lane;
        float v = i < m ? tail_term(tc, i) : 0.0f;
#pragma unroll
        for (int o = 1; o < L; o <<= 1) {
            const float u = __shfl_down_sync(gmask, v, o, L);
            if (lane + o < L) v += u;
        }
        if (i < m && (i % kTailG) == 0) cbs[i / kTailG] = carry + v;
        carry += __shfl_sync(gmask, v, 0, L);
    }
    __syncwarp(gmask);  // entries written by other lanes of the group
    const float slack = 1e-5f * carry;
    const int ne = tail_entries(m);
    for (int g = lane; g < ne - 1; g += L) cbs[g] = fmaxf(0.0f, cbs[g] - slack);
    if (lane == 0) cbs[ne - 1] = 0.0f;
    __syncwarp(gmask);
}

// Cells per lane for the anti-diagonal kernel: r+1 cells over L lanes.
__host__ __device__ inline void diag_shape(int r, int *L, int *K) {
    const int need = r + 1;
    if (need <= 32) {
        int l = 1;
        while (l < need) l *= 2;
        *L = l;
        *K = 1;
        return;
    }
    // 32 lanes and the smallest instantiated K with 32*K >= r+1 cells: a
    // non-power-of-two K cuts the cells past the band (e.g. r = 276: 320
    // cells instead of 512)
    *L = 32;
    const int ks[9] = {1, 2, 3, 4, 6, 8, 10, 12, 16};
    int k = 16;
    for (int i = 0; i < 9; ++i)
        if (32 * ks[i] >= need) {
            k = ks[i];
            break;
        }
    *K = k;  // 0 < K <= 16 for r <= 511
}

// Cells per lane for the FP32 anti-diagonal kernel: as diag_shape, except
// that bands of 4 < r+1 <= 32 cells take two cells per lane on half as many
// lanes (a power of two), so that each lane's pair of shuffles and window
// loads per anti-diagonal pair serves two cells and a warp walks two or
// more candidates at once.
__host__ __device__ inline void diag_shape_f32(int r, int *L, int *K) {
    const int need = r + 1;
    if (need > 4 && need <= 32) {
        int l = 1;
        while (2 * l < need) l *= 2;
        *L = l;
        *K = 2;
        return;
    }
    diag_shape(r, L, K);
}

// Lanes per group for band half-width r: the largest power of two <= r
// (<= 32), 1 for r = 0.
__host__ __device__ inline int lanes_for(int r) {
    int L = 1;
    while (L * 2 <= r && L < 32) L *= 2;
    return L;
}

}  // namespace dtws
