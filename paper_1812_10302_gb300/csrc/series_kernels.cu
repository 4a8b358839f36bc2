// series_kernels.cu -- per-series and per-(series, m | r) kernels:
//   * finiteness check of the series;
//   * anchored FP64 prefix sums of the series (once per series);
//   * window statistics for a query length m (Sec. 2.2, Eq. 5, population
//     sigma) from those sums;
//   * the raw sliding envelope of the series for a band half-width r
//     (Sec. 2.2, Eq. 9 applied to the series, clipped to [0, n)).
#include <cmath>

#include "dtws_internal.h"

namespace dtws {

// ------------------------------------------------------------------ finite
__global__ void k_check_finite(const float *__restrict__ x, int64_t n, int *flag) {
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[t]);
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(flag, 1);
}

cudaError_t launch_check_finite(const float *x, int64_t n, int *flag, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_check_finite<<<blocks, 256, 0, s>>>(x, n, flag);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ prefix
// One thread per block b of kBlockB samples.  The anchor a_b = x[b*B]; every
// sum inside the block runs over d = x - a_b, in FP64, so no sum grows with
// the series.  The running sums are compensated (Neumaier's variant of Kahan
// summation), so each stored prefix is within about one FP64 ulp of the
// exact sum of the (rounded) terms, whatever the block length -- plain
// sequential sums could drift by up to B/2 ulps.  Outputs, for t in block b:
//   P1[t] = sum_{bB <= u < t} d_u,  P2[t] = sum d_u^2   (exclusive prefix)
//   T1[b], T2[b] = block totals, A[b] = a_b.
__device__ __forceinline__ void neumaier_add(double &s, double &c, double v) {
    const double t = s + v;
    c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
}

__global__ void k_prefix(const float *__restrict__ x, int64_t n, double *__restrict__ P1,
                         double *__restrict__ P2, double *__restrict__ T1, double *__restrict__ T2,
                         double *__restrict__ A, int64_t nb) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int64_t t0 = b * kBlockB;
    const int64_t t1 = t0 + kBlockB < n ? t0 + kBlockB : n;
    const double a = (double)x[t0];
    double s1 = 0.0, c1 = 0.0, s2 = 0.0, c2 = 0.0;
    for (int64_t t = t0; t < t1; ++t) {
        P1[t] = s1 + c1;
        P2[t] = s2 + c2;
        const double d = (double)x[t] - a;
        neumaier_add(s1, c1, d);
        neumaier_add(s2, c2, d * d);
    }
    T1[b] = s1 + c1;
    T2[b] = s2 + c2;
    A[b] = a;
}

cudaError_t launch_prefix(const float *x, int64_t n, double *P1, double *P2, double *T1,
                          double *T2, double *A, cudaStream_t s) {
    int64_t nb = (n + kBlockB - 1) / kBlockB;
    k_prefix<<<(unsigned)((nb + 63) / 64), 64, 0, s>>>(x, n, P1, P2, T1, T2, A, nb);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ window stats
// Sum over [bB, e) of block b's anchored terms, bB < e <= end of block b.
__device__ __forceinline__ double upto(const double *P, const double *T, int64_t n, int64_t b,
                                       int64_t e) {
    int64_t end = (b + 1) * kBlockB < n ? (b + 1) * kBlockB : n;
    return e == end ? T[b] : P[e];
}

// Eq. 5 statistics of window i = [i, i+m) from the anchored sums.  A window
// spans at most two blocks (m <= kBlockB); the second block's sums are moved
// to the first anchor with the exact shift identities
//   sum(x - a0)   = sum(x - a1) + k (a1 - a0)
//   sum(x - a0)^2 = sum(x - a1)^2 + 2 (a1 - a0) sum(x - a1) + k (a1 - a0)^2.
// var = S2/m - (S1/m)^2.  The window is evaluated two-pass from its samples
// instead when the prefix differences cannot carry var to FP32 accuracy:
//   * the subtraction cancelled, var <= 1e-6 * S2/m, or
//   * var is below the bound the prefix rounding implies.  Each compensated
//     prefix is within ~2^-53 of its magnitude, so S2 is off by at most
//     ~3*2^-53*M2 and S1 by ~2*2^-53*sqrt(B*M2), with M2 the block totals of
//     the squares (plus the shift terms); var then holds 2^-26 relative
//     accuracy only if m*var >= 2^-27*(3*M2 + 4|S1/m|*sqrt(B*M2)).
// Zero-variance rule: var <= 1e-24*max(1, mu^2) gives inv_sigma = 0 (the
// window normalises to all zeros).
__global__ void k_window_stats(const float *__restrict__ x, int64_t n, int m,
                               const double *__restrict__ P1, const double *__restrict__ P2,
                               const double *__restrict__ T1, const double *__restrict__ T2,
                               const double *__restrict__ A, float *__restrict__ mu_hi,
                               float *__restrict__ mu_lo, float *__restrict__ inv_sigma,
                               float *__restrict__ smu_hi, float *__restrict__ smu_lo,
                               float *__restrict__ sinv_sigma) {
    const int64_t N = n - m + 1;
    const double inv_m = 1.0 / (double)m;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b0 = i / kBlockB, e = i + m;
        const double a0 = A[b0];
        double S1, S2;
        float M2;  // magnitude of the squared sums the prefix differences used
        if (e <= (b0 + 1) * kBlockB) {
            S1 = upto(P1, T1, n, b0, e) - P1[i];
            S2 = upto(P2, T2, n, b0, e) - P2[i];
            M2 = (float)T2[b0];
        } else {
            const int64_t b1 = b0 + 1;
            const double k = (double)(e - b1 * kBlockB), da = A[b1] - a0;
            const double e1 = upto(P1, T1, n, b1, e), e2 = upto(P2, T2, n, b1, e);
            S1 = (T1[b0] - P1[i]) + fma(k, da, e1);
            S2 = (T2[b0] - P2[i]) + fma(2.0 * da, e1, fma(k * da, da, e2));
            M2 = (float)(T2[b0] + T2[b1]) + 2.0f * fabsf((float)da) * sqrtf((float)kBlockB * (float)T2[b1]) +
                 (float)(k * da * da);
        }
        double mr = S1 * inv_m;
        double ms = S2 * inv_m;
        double var = fma(-mr, mr, ms);
        double mu = a0 + mr;
        const float bound = 7.450580596923828e-09f *  // 2^-27
                            (3.0f * M2 + 4.0f * fabsf((float)mr) * sqrtf((float)kBlockB * M2));
        if (var <= 1e-6 * ms || (float)var * (float)m < bound) {
            // two-pass from the samples (rare: near-constant windows)
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += (double)x[i + j];
            mu = s / (double)m;
            double v = 0.0;
            for (int j = 0; j < m; ++j) {
                double d = (double)x[i + j] - mu;
                v += d * d;
            }
            var = v / (double)m;
        }
        const float mh = (float)mu, ml = (float)(mu - (double)mh);
        const double mm = mu * mu;
        float is = 0.0f;
        if (!(var <= 1e-24 * (mm > 1.0 ? mm : 1.0))) {
            // 1/sqrt(var): FP32 estimate refined by one Newton step in FP64
            double y = (double)rsqrtf((float)var);
            y = y * fma(-0.5 * var * y, y, 1.5);
            is = (float)y;
        }
        mu_hi[i] = mh;
        mu_lo[i] = ml;
        inv_sigma[i] = is;
        if ((i & (kProxyStride - 1)) == 0) {  // every kProxyStride-th window, for the proxy scan
            smu_hi[i / kProxyStride] = mh;
            smu_lo[i / kProxyStride] = ml;
            sinv_sigma[i / kProxyStride] = is;
        }
    }
}

cudaError_t launch_window_stats(const float *x, int64_t n, int m, const double *P1,
                                const double *P2, const double *T1, const double *T2,
                                const double *A, float *mu_hi, float *mu_lo, float *inv_sigma,
                                float *smu_hi, float *smu_lo, float *sinv_sigma, cudaStream_t s) {
    int64_t N = n - m + 1;
    int64_t blocks = (N + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_window_stats<<<(unsigned)blocks, 256, 0, s>>>(x, n, m, P1, P2, T1, T2, A, mu_hi, mu_lo,
                                                    inv_sigma, smu_hi, smu_lo, sinv_sigma);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ envelope
// U[t] = max x[max(0,t-r) .. min(n-1,t+r)], L[t] = min (clipped to the
// series).  A CTA produces kEnvTile outputs from the samples
// [t0 - r, t0 + kEnvTile + r) held in shared memory (outside [0, n) as
// -inf / +inf, which never wins the max / min, so clipping is automatic).
// Doubling: after pass p, M[u] = max over [u, u + 2^p); a window of length
// w = 2r+1 is the max of two overlapping runs of length 2^P <= w.
constexpr int kEnvTile = 4096;
constexpr int kEnvThreads = 512;

__global__ void __launch_bounds__(kEnvThreads)
k_envelope(const float *__restrict__ x, int64_t n, int r, float *__restrict__ U,
           float *__restrict__ L) {
    extern __shared__ float sm[];
    const int len = kEnvTile + 2 * r;
    float *mx = sm, *mn = sm + len;
    const int64_t t0 = (int64_t)blockIdx.x * kEnvTile;
    const float inf = __int_as_float(0x7f800000);
    for (int u = threadIdx.x; u < len; u += blockDim.x) {
        int64_t t = t0 - r + u;
        bool in = t >= 0 && t < n;
        float v = in ? x[t] : 0.0f;
        mx[u] = in ? v : -inf;
        mn[u] = in ? v : inf;
    }
    __syncthreads();
    const int w = 2 * r + 1;
    int span = 1;
    // grow runs while 2*span <= w; the run at u may read past `len` only
    // for u that no output needs, so clamp the partner index
    while (2 * span <= w) {
        // read phase into registers then write, so the update is in place
        for (int base = 0; base < len; base += blockDim.x * 8) {
            float a[8], c[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int u = base + q * blockDim.x + threadIdx.x;
                if (u < len) {
                    int v = u + span < len ? u + span : len - 1;
                    a[q] = fmaxf(mx[u], mx[v]);
                    c[q] = fminf(mn[u], mn[v]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int u = base + q * blockDim.x + threadIdx.x;
                if (u < len) { mx[u] = a[q]; mn[u] = c[q]; }
            }
            __syncthreads();
        }
        span *= 2;
    }
    for (int u = threadIdx.x; u < kEnvTile; u += blockDim.x) {
        int64_t t = t0 + u;
        if (t >= n) break;
        int v = u + w - span;  // second run ends exactly at u + w - 1
        U[t] = fmaxf(mx[u], mx[v]);
        L[t] = fminf(mn[u], mn[v]);
    }
}

cudaError_t launch_envelope(const float *x, int64_t n, int r, float *U, float *L, cudaStream_t s) {
    int64_t blocks = (n + kEnvTile - 1) / kEnvTile;
    size_t smem = (size_t)2 * (kEnvTile + 2 * r) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_envelope, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_envelope<<<(unsigned)blocks, kEnvThreads, smem, s>>>(x, n, r, U, L);
    return cudaGetLastError();
}

}  // namespace dtws
