// series_kernels.cu -- per-series and per-(series, m | r) kernels:
//   * finiteness check of the series;
//   * anchored, compensated FP64 prefix sums of the series (once per
//     series), stored as FP32 pairs;
//   * window statistics for a query length m (Sec. 2.2, Eq. 5, population
//     sigma) from those sums;
//   * the raw sliding envelope of the series for a band half-width r
//     (Sec. 2.2, Eq. 9 applied to the series, clipped to [0, n)).
#include <cmath>

#include "dtws_internal.h"

namespace dtws {

// ------------------------------------------------------------------ finite
// Also the largest |x| (as its FP32 bit pattern, which orders like the value
// for non-negative floats; meaningful when no value is NaN or Inf).
__global__ void k_check_finite(const float *__restrict__ x, int64_t n, int *flag, unsigned *absmax) {
    bool bad = false;
    unsigned amax = 0u;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[t];
        bad |= !isfinite(v);
        amax = max(amax, __float_as_uint(fabsf(v)));
    }
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(flag, 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane_id() == 0 && amax) atomicMax(absmax, amax);
}

cudaError_t launch_check_finite(const float *x, int64_t n, int *flag, unsigned *absmax, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_check_finite<<<blocks, 256, 0, s>>>(x, n, flag, absmax);
    return cudaGetLastError();
}

__global__ void k_fill(float *__restrict__ p, int64_t count, float v) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        p[t] = v;
}

cudaError_t launch_fill(float *p, int64_t count, float v, int num_sms, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 8LL * num_sms) blocks = 8LL * num_sms;
    k_fill<<<(int)blocks, 256, 0, s>>>(p, count, v);
    return cudaGetLastError();
}

// The series' every kProxyStride-th sample, xs[j] = x[kProxyStride j] for
// j < count (the proxy scan scores every kProxyStride-th window at term
// positions that are multiples of kProxyStride, so it reads only these).
__global__ void k_subsample(const float *__restrict__ x, int64_t count, float *__restrict__ xs) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x)
        xs[j] = x[kProxyStride * j];
}

cudaError_t launch_subsample(const float *x, int64_t count, float *xs, int num_sms, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 8LL * num_sms) blocks = 8LL * num_sms;
    k_subsample<<<(int)blocks, 256, 0, s>>>(x, count, xs);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ prefix
// One thread per block b of kBlockB samples.  The anchor a_b = x[b*B]; every
// sum inside the block runs over d = x - a_b, in FP64, so no sum grows with
// the series.  The running sums are compensated (Neumaier's variant of Kahan
// summation), so each prefix is within about one FP64 ulp of the exact sum of
// the (rounded) terms, whatever the block length -- plain sequential sums
// could drift by up to B/2 ulps.  Each FP64 prefix is stored as the exact
// pair hi = fl32(v), lo = fl32(v - hi) (|v - hi - lo| <= 2^-48 |v|), so the
// per-window arithmetic runs in FP32 pairs instead of FP64 (GB300 issues
// FP64 at a small fraction of its FP32 rate).  Outputs, for t in block b:
//   P1[t] = sum_{bB <= u < t} d_u,  P2[t] = sum d_u^2   (exclusive prefix)
//   T1[b], T2[b] = block totals, A[b] = a_b,
//   ok[b] = 1 when every nonzero |d| in the block lies in [2^-40, 2^40], so
//   that no pair over- or underflows FP32 (else windows touching the block
//   take the two-pass FP64 path).
// All of it in units scaled by one power of two per series, 2^s with s such
// that the largest in-block excursion max|x - a_b| lies in [1, 2) (exact
// scaling; it keeps the pairs away from FP32 over- and underflow whatever the
// series' units).  Layout: pf = [P1h | P1l | P2h | P2l] (n floats each),
// bf = [T1h | T1l | T2h | T2l | A] (nb floats each, A scaled), scale[0] = 2^s.
__device__ __forceinline__ void neumaier_add(double &s, double &c, double v) {
    const double t = s + v;
    c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
}

__device__ __forceinline__ void split_store(double v, float *hi, float *lo, int64_t t) {
    const float h = (float)v;
    hi[t] = h;
    lo[t] = (float)(v - (double)h);
}

// largest |x[t] - x[block start]| of the series, as float bits (non-negative
// floats order like their bits)
__global__ void k_block_maxabs(const float *__restrict__ x, int64_t n, unsigned *out) {
    float mx = 0.0f;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float d = (float)fabs((double)x[t] - (double)x[t / kBlockB * kBlockB]);
        mx = fmaxf(mx, d);
    }
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane_id() == 0) atomicMax(out, __float_as_uint(mx));
}

__global__ void k_prefix(const float *__restrict__ x, int64_t n, float *__restrict__ pf,
                         float *__restrict__ bf, int *__restrict__ ok, int64_t nb,
                         const unsigned *__restrict__ maxabs, float *__restrict__ scale_out) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const float mx = __uint_as_float(*maxabs);
    // 2^s with mx * 2^s in [1, 2); 1 for a constant series
    const double sc = mx > 0.0f ? ldexp(1.0, -ilogbf(mx)) : 1.0;
    if (b == 0) scale_out[0] = (float)sc;
    if (b >= nb) return;
    const int64_t t0 = b * kBlockB;
    const int64_t t1 = t0 + kBlockB < n ? t0 + kBlockB : n;
    float *p1h = pf, *p1l = pf + n, *p2h = pf + 2 * n, *p2l = pf + 3 * n;
    const float af = x[t0];
    const double a = (double)af;
    double s1 = 0.0, c1 = 0.0, s2 = 0.0, c2 = 0.0;
    bool good = true;
    for (int64_t t = t0; t < t1; ++t) {
        split_store(s1 + c1, p1h, p1l, t);
        split_store(s2 + c2, p2h, p2l, t);
        const double d = ((double)x[t] - a) * sc;
        const double ad = fabs(d);
        good &= d == 0.0 || (ad >= 9.094947017729282e-13 && ad <= 1099511627776.0);  // 2^-40, 2^40
        neumaier_add(s1, c1, d);
        neumaier_add(s2, c2, d * d);
    }
    split_store(s1 + c1, bf, bf + nb, b);
    split_store(s2 + c2, bf + 2 * nb, bf + 3 * nb, b);
    const double as = a * sc;
    bf[4 * nb + b] = (float)as;
    ok[b] = good && (double)(float)as == as && fabs(as) < 1e30 ? 1 : 0;
}

cudaError_t launch_prefix(const float *x, int64_t n, float *pf, float *bf, int *ok, unsigned *maxabs,
                          float *scale, cudaStream_t s) {
    int64_t nb = (n + kBlockB - 1) / kBlockB;
    cudaError_t e = cudaMemsetAsync(maxabs, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_block_maxabs<<<(unsigned)blocks, 256, 0, s>>>(x, n, maxabs);
    k_prefix<<<(unsigned)((nb + 63) / 64), 64, 0, s>>>(x, n, pf, bf, ok, nb, maxabs, scale);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ FP32 pairs
// Unevaluated sums hi + lo of two floats with error-free transformations
// (Knuth's TwoSum, Dekker's Fast2Sum, the FMA product error).
struct f2 {
    float hi, lo;
};
__device__ __forceinline__ f2 two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ f2 f2_add(f2 x, f2 y) {
    f2 s = two_sum(x.hi, y.hi);
    const f2 t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ f2 f2_neg(f2 x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ f2 f2_mul(f2 x, f2 y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    return fast_two_sum(p, e);
}
__device__ __forceinline__ f2 f2_mul_f(f2 x, float f) {
    const float p = x.hi * f;
    const float e = fmaf(x.lo, f, fmaf(x.hi, f, -p));
    return fast_two_sum(p, e);
}
__device__ __forceinline__ f2 ld2(const float *h, const float *l, int64_t t) { return {h[t], l[t]}; }

// ------------------------------------------------------------------ window stats
// Eq. 5 statistics of window i = [i, i+m) from the anchored sums.  A window
// spans at most two blocks (m <= kBlockB); the second block's sums are moved
// to the first anchor with the exact shift identities
//   sum(x - a0)   = sum(x - a1) + k (a1 - a0)
//   sum(x - a0)^2 = sum(x - a1)^2 + 2 (a1 - a0) sum(x - a1) + k (a1 - a0)^2,
// all in FP32 pairs (about 2^-47 relative per operation).  var = S2/m - (S1/m)^2.
// The window is evaluated two-pass from its samples in FP64 instead when
//   * a block it touches is not ok (see k_prefix), or
//   * the subtraction cancelled, var <= 1e-6 * S2/m, or
//   * var is below the bound the stored sums' rounding implies.  Each stored
//     prefix is within ~2^-48 of its magnitude, so S2 is off by at most
//     ~3*2^-48*M2 and S1 by ~2*2^-48*sqrt(B*M2), with M2 the block totals of
//     the squares (plus the shift terms); var then holds 2^-26 relative
//     accuracy only if m*var >= 2^-22*(3*M2 + 4|S1/m|*sqrt(B*M2)).
// Zero-variance rule: var <= 1e-24*max(1, mu^2) gives inv_sigma = 0 (the
// window normalises to all zeros).
__global__ void k_window_stats(const float *__restrict__ x, int64_t n, int m, const float *__restrict__ pf,
                               const float *__restrict__ bf, const int *__restrict__ ok,
                               const float *__restrict__ scale, int64_t nb,
                               float *__restrict__ mu_hi, float *__restrict__ mu_lo,
                               float *__restrict__ inv_sigma, float *__restrict__ smu_hi,
                               float *__restrict__ sinv_sigma) {
    const int64_t N = n - m + 1;
    const float sc = scale[0], isc = 1.0f / sc;  // powers of two
    const float *p1h = pf, *p1l = pf + n, *p2h = pf + 2 * n, *p2l = pf + 3 * n;
    const float *t1h = bf, *t1l = bf + nb, *t2h = bf + 2 * nb, *t2l = bf + 3 * nb, *A = bf + 4 * nb;
    // 1/m as a pair: hi = fl(1/m), lo = (1 - hi*m)/m (the FMA residual is exact)
    const float ih = 1.0f / (float)m;
    const f2 inv_m = {ih, fmaf(-ih, (float)m, 1.0f) * ih};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b0 = i / kBlockB, e = i + m, end0 = (b0 + 1) * kBlockB;
        const float a0 = A[b0];
        f2 S1, S2;
        float M2;  // magnitude of the squared sums the prefix differences used
        bool good = ok[b0] != 0;
        const f2 P1i = ld2(p1h, p1l, i), P2i = ld2(p2h, p2l, i);
        if (e <= end0) {
            const bool tot = e == (end0 < n ? end0 : n);
            S1 = f2_add(tot ? ld2(t1h, t1l, b0) : ld2(p1h, p1l, e), f2_neg(P1i));
            S2 = f2_add(tot ? ld2(t2h, t2l, b0) : ld2(p2h, p2l, e), f2_neg(P2i));
            M2 = t2h[b0];
        } else {
            const int64_t b1 = b0 + 1, end1 = (b1 + 1) * kBlockB;
            good = good && ok[b1] != 0;
            const bool tot = e == (end1 < n ? end1 : n);
            const float k = (float)(e - b1 * kBlockB);
            const f2 da = two_sum(A[b1], -a0);
            const f2 e1 = tot ? ld2(t1h, t1l, b1) : ld2(p1h, p1l, e);
            const f2 e2 = tot ? ld2(t2h, t2l, b1) : ld2(p2h, p2l, e);
            S1 = f2_add(f2_add(ld2(t1h, t1l, b0), f2_neg(P1i)), f2_add(f2_mul_f(da, k), e1));
            const f2 da_e1 = f2_mul(da, e1);
            const f2 sh = f2_add(f2_add({2.0f * da_e1.hi, 2.0f * da_e1.lo}, f2_mul_f(f2_mul(da, da), k)), e2);
            S2 = f2_add(f2_add(ld2(t2h, t2l, b0), f2_neg(P2i)), sh);
            M2 = t2h[b0] + t2h[b1] + 2.0f * fabsf(da.hi) * sqrtf((float)kBlockB * t2h[b1]) + k * da.hi * da.hi;
        }
        const f2 mr = f2_mul(S1, inv_m);
        const f2 ms = f2_mul(S2, inv_m);
        const f2 var2 = f2_add(ms, f2_neg(f2_mul(mr, mr)));
        const f2 mu2 = f2_add(mr, {a0, 0.0f});
        const float bound = 2.384185791015625e-07f *  // 2^-22
                            (3.0f * M2 + 4.0f * fabsf(mr.hi) * sqrtf((float)kBlockB * M2));
        float mh = mu2.hi * isc, ml = mu2.lo * isc, is = 0.0f;
        if (!good || var2.hi <= 1e-6f * ms.hi || var2.hi * (float)m < bound) {
            // two-pass from the samples in FP64 (rare: near-constant windows,
            // or blocks whose values the FP32 pairs cannot carry)
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += (double)x[i + j];
            const double mu = s / (double)m;
            double v = 0.0;
            for (int j = 0; j < m; ++j) {
                const double d = (double)x[i + j] - mu;
                v += d * d;
            }
            const double var = v / (double)m;
            mh = (float)mu;
            ml = (float)(mu - (double)mh);
            const double mm = mu * mu;
            if (!(var <= 1e-24 * (mm > 1.0 ? mm : 1.0))) {
                double y = (double)rsqrtf((float)var);
                y = y * fma(-0.5 * var * y, y, 1.5);
                is = (float)y;
            }
        } else if (!(sqrtf(var2.hi) <= 1e-12f * fmaxf(sc, fabsf(mu2.hi)))) {
            // (the zero-variance rule in scaled units.)  1/sqrt(var): FP32
            // estimate refined by one Newton step whose residual 1 - var*y^2
            // is taken in pairs; then back to the series' units
            const float y = rsqrtf(var2.hi);
            const f2 yy = {y * y, fmaf(y, y, -y * y)};
            const f2 r = f2_add({1.0f, 0.0f}, f2_neg(f2_mul(var2, yy)));
            is = fmaf(0.5f * y, r.hi, y) * sc;
        }
        mu_hi[i] = mh;
        mu_lo[i] = ml;
        inv_sigma[i] = is;
        if ((i & (kProxyStride - 1)) == 0) {  // every kProxyStride-th window, for the proxy scan
            // (the mean's high part alone: the proxy only ranks proposals)
            smu_hi[i / kProxyStride] = mh;
            sinv_sigma[i / kProxyStride] = is;
        }
    }
}

cudaError_t launch_window_stats(const float *x, int64_t n, int m, const float *pf, const float *bf,
                                const int *ok, const float *scale, float *mu_hi, float *mu_lo, float *inv_sigma,
                                float *smu_hi, float *sinv_sigma, int num_sms, cudaStream_t s) {
    const int64_t N = n - m + 1, nb = (n + kBlockB - 1) / kBlockB;
    int64_t blocks = (N + 255) / 256;
    if (blocks > (int64_t)num_sms * 16) blocks = (int64_t)num_sms * 16;
    k_window_stats<<<(unsigned)blocks, 256, 0, s>>>(x, n, m, pf, bf, ok, scale, nb, mu_hi, mu_lo, inv_sigma, smu_hi,
                                                    sinv_sigma);
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

// ------------------------------------------------------------------ block envelope
// Sparse table over blocks of kEnvG samples: level 0 holds each block's max
// (min), level k the max (min) of blocks [j, j + 2^k); entries whose range
// passes the last block are left unset and never read.
__global__ void k_env_level0(const float *__restrict__ x, int64_t n, float *__restrict__ mx,
                             float *__restrict__ mn, int64_t nblk) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nblk;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t0 = j * kEnvG, t1 = t0 + kEnvG < n ? t0 + kEnvG : n;
        float u = x[t0], l = u;
        for (int64_t t = t0 + 1; t < t1; ++t) {
            u = fmaxf(u, x[t]);
            l = fminf(l, x[t]);
        }
        mx[j] = u;
        mn[j] = l;
    }
}

__global__ void k_env_level(float *__restrict__ mx, float *__restrict__ mn, int64_t nblk, int k) {
    const int64_t h = 1ll << (k - 1), last = nblk - (1ll << k);
    const float *pm = mx + (size_t)(k - 1) * nblk, *pn = mn + (size_t)(k - 1) * nblk;
    float *qm = mx + (size_t)k * nblk, *qn = mn + (size_t)k * nblk;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= last;
         j += (int64_t)gridDim.x * blockDim.x) {
        qm[j] = fmaxf(pm[j], pm[j + h]);
        qn[j] = fminf(pn[j], pn[j + h]);
    }
}

cudaError_t launch_block_envelope(const float *x, int64_t n, float *st, int64_t nblk, cudaStream_t s) {
    float *mx = st, *mn = st + (size_t)kEnvLevels * nblk;
    int64_t blocks = (nblk + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_env_level0<<<(unsigned)blocks, 256, 0, s>>>(x, n, mx, mn, nblk);
    for (int k = 1; k < kEnvLevels && (1ll << k) <= nblk; ++k)
        k_env_level<<<(unsigned)blocks, 256, 0, s>>>(mx, mn, nblk, k);
    return cudaGetLastError();
}

}  // namespace dtws
