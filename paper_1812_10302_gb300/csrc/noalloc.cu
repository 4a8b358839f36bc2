// noalloc.cu -- dtws_dtw_at_noalloc: banded DTW at given offsets without any
// device allocation by the library.
//
// Some callers cannot let a library allocate device memory: code that must
// not call cudaMalloc once it is running (it synchronises the device and can
// stall other streams), hosts whose framework owns every byte of device
// memory through its own pool, and fixed-footprint deployments that size
// memory once at start-up.  For them this entry point takes only caller-owned
// inputs and outputs; its one piece of working memory -- the normalised
// query and a work cursor -- lives in a fixed file-scope device array of
// kNoAllocFloats floats (about 33 KB), which every GPU that loads this
// library holds until the process exits.
//
// Host code may not pass the array's name to a kernel (on the host it is
// only a stand-in for the symbol, not a device address).  The device address
// is looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on it; that first call should therefore
// come before any stream capture.  All calls share the array and it keeps
// the previous call's contents: each call re-initialises what it reads (the
// normalised query, the cursor) before use, and calls whose kernels overlap
// on the GPU race on it, so a caller must not run two of them concurrently.
#include <cstdio>
#include <mutex>

#include "../../include/dtws.h"
#include "dtw_band.cuh"
#include "dtws_common.cuh"
#include "dtws_internal.h"

namespace {

constexpr int kNoAllocCursor = DTWS_NOALLOC_M_MAX;      // 64-bit slot after q_hat (8-byte aligned)
constexpr int kNoAllocFloats = DTWS_NOALLOC_M_MAX + 64;  // q_hat, cursor, padding

// The largest launch this entry point makes is one warp (a group of 32
// lanes) at m = DTWS_NOALLOC_M_MAX and r = m - 1: the normalised query
// (4 m bytes) plus one ring of 2r + 2 floats (8 m bytes).  It must fit the
// 227 KB a CTA may opt into on this part; the run-time check below also
// compares it with the device's own limit.
static_assert(12 * DTWS_NOALLOC_M_MAX <= 227 * 1024, "scratch query length too long for one warp's shared memory");

}  // namespace

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

namespace dtws {
namespace {

// z-normalise Q into scratch[0, m) (Sec. 2.2, Eq. 5, FP64 two-pass, same
// zero-variance rule as the search) and reset the work cursor.  A
// non-finite query leaves a NaN in scratch[0] so the DTW kernel writes NaN.
__global__ void __launch_bounds__(1024) k_noalloc_prep(const float *__restrict__ Q, int m,
                                                       float *scratch) {
    __shared__ double red[32];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    bool nf = false;
    for (int j = threadIdx.x; j < m; j += blockDim.x) nf |= !isfinite(Q[j]);
    if (nf) atomicOr(&bad, 1);
    __syncthreads();
    if (threadIdx.x == 0) *(unsigned long long *)(scratch + kNoAllocCursor) = 0ull;
    if (bad) {
        if (threadIdx.x == 0) scratch[0] = __int_as_float(0x7fc00000);
        return;
    }
    auto bsum = [&](double v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        return s;
    };
    double s = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) s += (double)Q[j];
    const double mu = bsum(s) / (double)m;
    double v = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const double d = (double)Q[j] - mu;
        v = fma(d, d, v);
    }
    const double var = bsum(v) / (double)m, mm = mu * mu;
    const bool zero = var <= 1e-24 * (mm > 1.0 ? mm : 1.0);
    const double sg = zero ? 0.0 : sqrt(var);
    for (int j = threadIdx.x; j < m; j += blockDim.x)
        scratch[j] = zero ? 0.0f : (float)(((double)Q[j] - mu) / sg);
}

// FP32 banded DTW of the normalised query (scratch) against the windows at
// offsets; each window's Eq. 5 statistics are computed two-pass in FP64 by
// its lane group.  Groups of L lanes pull offsets from the scratch cursor.
template <int L>
__global__ void __launch_bounds__(256) k_noalloc_dtw(const float *__restrict__ x, int64_t n, int m, int r,
                                                     const int64_t *__restrict__ offsets, int64_t count,
                                                     float *__restrict__ out, float *scratch) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int W = 2 * r + 1;
    const int64_t N = n - m + 1;
    float *qs = (float *)smraw;
    for (int t = threadIdx.x; t < m; t += blockDim.x) qs[t] = scratch[t];
    __syncthreads();
    const bool qbad = !(qs[0] == qs[0]);
    const int warp = threadIdx.x >> 5, ln = threadIdx.x & 31;
    const int g = ln / L, lane = ln % L;
    const int gid = warp * (32 / L) + g;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g * L));
    float *ring = qs + ((m + 3) & ~3) + gid * (W + 1);
    // 64-bit cursor: count may exceed INT_MAX
    unsigned long long *cursor = (unsigned long long *)(scratch + kNoAllocCursor);
    while (true) {
        unsigned long long cu = 0;
        if (lane == 0) cu = atomicAdd(cursor, 1ull);
        cu = __shfl_sync(gmask, cu, 0, L);
        if (cu >= (unsigned long long)count) break;
        const int64_t c = (int64_t)cu;
        const int64_t o = offsets[c];
        if (qbad || o < 0 || o >= N) {
            if (lane == 0) out[c] = __int_as_float(0x7fc00000);
            continue;
        }
        const float *xw = x + o;
        double s = 0.0;
        for (int j = lane; j < m; j += L) s += (double)xw[j];
        for (int q = L / 2; q > 0; q >>= 1) s += __shfl_xor_sync(gmask, s, q, L);
        const double mu = s / (double)m;
        double v = 0.0;
        for (int j = lane; j < m; j += L) {
            const double d = (double)xw[j] - mu;
            v = fma(d, d, v);
        }
        for (int q = L / 2; q > 0; q >>= 1) v += __shfl_xor_sync(gmask, v, q, L);
        const double var = v / (double)m, mm = mu * mu;
        const bool zero = var <= 1e-24 * (mm > 1.0 ? mm : 1.0);
        const double inv = zero ? 0.0 : 1.0 / sqrt(var);
        const float mh = (float)mu, is = (float)inv, ls = (float)(mu - (double)mh) * is;
        int cells = 0;
        const float d = dtw_band<float, L, false>(qs, xw, (const float *)nullptr, mh, is, ls, nullptr, ring, m, r,
                                                  __int_as_float(0x7f800000), gmask, lane, cells);
        if (lane == 0) out[c] = d;
        __syncwarp(gmask);
    }
}

std::mutex g_scratch_mu;
constexpr int kMaxDevices = 64;
float *g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this set-up).
dtws_status scratch_address(float **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error_detail("dtws_dtw_at_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
        return DTWS_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error_detail("dtws_dtw_at_noalloc: device %d beyond %d", dev, kMaxDevices);
        return DTWS_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error_detail("dtws_dtw_at_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return DTWS_ECUDA;
        }
        g_scratch_addr[dev] = (float *)p;
    }
    *out = g_scratch_addr[dev];
    return DTWS_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Shared memory of a k_noalloc_dtw CTA of `warps` warps: the normalised
// query and one ring of W + 1 floats per lane group.
inline size_t noalloc_smem(int m, int r, int L, int warps) {
    const size_t qbytes = (size_t)((m + 3) & ~3) * 4;
    const size_t per_warp = (size_t)(32 / L) * (2 * r + 2) * 4;
    return qbytes + (size_t)warps * per_warp;
}

template <int L>
cudaError_t launch_noalloc_dtw(const float *x, int64_t n, int m, int r, const int64_t *offsets,
                               int64_t count, float *out, float *scratch, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int warps = 8;
    while (warps > 1 && noalloc_smem(m, r, L, warps) > 100 * 1024) --warps;
    const size_t smem = noalloc_smem(m, r, L, warps);
    const int groups = warps * (32 / L);
    int64_t blocks = (count + groups - 1) / groups;
    if (blocks > (int64_t)sms * 4) blocks = (int64_t)sms * 4;
    if (blocks < 1) blocks = 1;
    cudaError_t e = cudaFuncSetAttribute(k_noalloc_dtw<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_noalloc_dtw<L><<<(unsigned)blocks, warps * 32, smem, s>>>(x, n, m, r, offsets, count, out, scratch);
    return cudaGetLastError();
}

}  // namespace
}  // namespace dtws

extern "C" dtws_status dtws_dtw_at_noalloc(const float *series, int64_t n, const float *Q, int32_t m,
                                           int32_t r, const int64_t *offsets, int64_t count, float *out,
                                           void *stream) {
    using namespace dtws;
    if (!series || !Q || !out || (!offsets && count > 0) || count < 0) {
        set_error_detail("dtws_dtw_at_noalloc: null pointer or count < 0");
        return DTWS_EINVAL;
    }
    if (n < 2 || n > DTWS_N_MAX) {
        set_error_detail("dtws_dtw_at_noalloc: n=%lld out of range [2, %lld]", (long long)n,
                         (long long)DTWS_N_MAX);
        return DTWS_EINVAL;
    }
    if (m < 2 || (int64_t)m > n || m > DTWS_NOALLOC_M_MAX) {
        set_error_detail("dtws_dtw_at_noalloc: m=%d exceeds the fixed scratch (m must be in [2, min(n, %d)])",
                         m, DTWS_NOALLOC_M_MAX);
        return DTWS_EINVAL;
    }
    if (r < 0) {
        set_error_detail("dtws_dtw_at_noalloc: r=%d < 0", r);
        return DTWS_EINVAL;
    }
    if (!on_device(series) || !on_device(Q) || !on_device(out) || (count > 0 && !on_device(offsets))) {
        set_error_detail("dtws_dtw_at_noalloc: every array must be device memory (nothing is staged)");
        return DTWS_EINVAL;
    }
    float *scratch = nullptr;
    dtws_status st = scratch_address(&scratch);
    if (st != DTWS_OK) return st;
    if (count == 0) return DTWS_OK;
    const int rr = r > m - 1 ? m - 1 : r;
    {  // one warp's shared memory must fit the device's per-block limit
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const size_t need = noalloc_smem(m, rr, lanes_for(rr), 1);
        if (optin > 0 && need > (size_t)optin) {
            set_error_detail("dtws_dtw_at_noalloc: m=%d, r=%d need %zu bytes of shared memory per warp, "
                             "beyond the device's %d", m, rr, need, optin);
            return DTWS_EINVAL;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    k_noalloc_prep<<<1, 1024, 0, s>>>(Q, m, scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        switch (lanes_for(rr)) {
        case 1: e = launch_noalloc_dtw<1>(series, n, m, rr, offsets, count, out, scratch, s); break;
        case 2: e = launch_noalloc_dtw<2>(series, n, m, rr, offsets, count, out, scratch, s); break;
        case 4: e = launch_noalloc_dtw<4>(series, n, m, rr, offsets, count, out, scratch, s); break;
        case 8: e = launch_noalloc_dtw<8>(series, n, m, rr, offsets, count, out, scratch, s); break;
        case 16: e = launch_noalloc_dtw<16>(series, n, m, rr, offsets, count, out, scratch, s); break;
        default: e = launch_noalloc_dtw<32>(series, n, m, rr, offsets, count, out, scratch, s); break;
        }
    }
    if (e != cudaSuccess) {
        set_error_detail("dtws_dtw_at_noalloc: launch: %s", cudaGetErrorString(e));
        return DTWS_ECUDA;
    }
    return DTWS_OK;
}
