// dtw_band.cuh -- the systolic banded-DTW core shared by the DTW kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

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
    const float *Uw, *Lw;  // series envelope at the window's first sample
    const float *qs;       // q_hat (shared)
    float mh, is, ls;
};

// LB_Keogh term of row i: squared distance of q_hat_i to the normalised
// envelope interval of the window at position i.
__device__ __forceinline__ float tail_term(const TailCtx &c, int i) {
    float u = fmaf(c.Uw[i] - c.mh, c.is, -c.ls);
    float l = fmaf(c.Lw[i] - c.mh, c.is, -c.ls);
    float q = c.qs[i];
    float d = fmaxf(q - u, 0.0f) + fmaxf(l - q, 0.0f);
    return d * d;
}

template <typename T, int L, bool ABANDON>
__device__ T dtw_band(const T *__restrict__ qs, const float *__restrict__ xw, T na, T nb, T nc,
                      const TailCtx *tail, T *ring, int m, int r, T thr, unsigned gmask, int lane,
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
    for (int s = 0; s < total; ++s) {
        T upIn = __shfl_up_sync(gmask, out, 1, L);
        const bool act = (k >= 0) && (i < m);
        const int kk = act ? k : 0;
        T up, diag;
        if (lane == 0) {
            up = ring[kk + 1];
            diag = ring[kk];
        } else {
            up = (k + 1 < W) ? upIn : INF;
            diag = upPrev;
        }
        upPrev = upIn;
        const T left = (k > 0) ? out : INF;
        const int j = i - r + k;
        T v = INF;
        if (act && j >= 0 && j < m) {
            T c = qi - tfma((T)xw[j] - na, nb, -nc);
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
                int row = ((s + 1) / W) * L + lane;
                float e = row < m ? tail_term(*tail, row) : 0.0f;
                float inc = group_incl_scan<L>(e, gmask, lane);
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
        __syncwarp(gmask);
        if (ABANDON && (s & 15) == 15) {
            if (__any_sync(gmask, stop)) return INF;
        }
    }
    return __shfl_sync(gmask, res, (m - 1) % L, L);
}

// Lanes per group for band half-width r: the largest power of two <= r
// (<= 32), 1 for r = 0.
__host__ __device__ inline int lanes_for(int r) {
    int L = 1;
    while (L * 2 <= r && L < 32) L *= 2;
    return L;
}

}  // namespace dtws
