// encoder.cu -- the learned proposal encoder: a bias-free 1-D CNN over the
// block-mean differences of a z-normalised window (4 convolution layers of 32
// channels and kernel 7, valid padding, ReLU after the first three; mean pool
// over 8 segments; linear projection to 64 dimensions).  The paper has no
// learned component: it orders candidates only to seed the best-so-far of
// the exact search (Sec. 2.2's random first bsf, Algorithm 1); pruning never
// uses it.
//
// Input of a window y of length m: b = floor(m/64); block means a_j of
// y[j*b, (j+1)*b), j < 64; u_j = (a_{j+1} - a_j) / sigma(y), j < 63 (sigma
// of all m samples, Eq. 5; 0 when sigma is 0).  Without biases every layer is
// positively homogeneous, so the embedding of a window is 1/sigma times the
// embedding of its raw block-mean differences: one series-wide feature map
// per (series, m) serves every window at offsets that are multiples of b.
//
// Arithmetic: convolutions 2-4, their backward passes and the series
// projection on tensor cores (mma.sync m16n8k16, BF16 operands, FP32
// accumulation); the layer-1 convolution and reductions in FP32.  Each
// convolution is a GEMM whose reduction index is (tap, input channel): the
// A operand of tap t is the activation tile shifted by t rows, read straight
// from shared memory (no im2col copy).
//
// Parameters (flat FP32, 38112): W1[32][7], W2..W4[32][7][32] ([co][t][ci]),
// P[64][256] ([d][s*32 + c]).  Kernels use a packed copy: W1 (FP32), W2..W4
// in BF16 as [co][t*32+ci] (forward) and as [ci][t'*32+co] = W[co][6-t'][ci]
// (the transposed convolution of the backward pass), P in BF16.
#include <cuda_bf16.h>

#include <cstdint>

#include "dtws_internal.h"

namespace dtws {
namespace enc {

constexpr int C = 32, KW = 7, NB = 64, NU = 63;
constexpr int L1 = NU - 6, L2 = NU - 12, L3 = NU - 18, L4 = NU - 24;  // 57, 51, 45, 39
constexpr int NSEG = 8, DIM = 64, KD = C * KW;                        // KD = 224
constexpr int oW1 = 0, oW2 = oW1 + C * KW, oW3 = oW2 + C * KD, oW4 = oW3 + C * KD;
constexpr int oP = oW4 + C * KD, NPAR = oP + DIM * NSEG * C;  // 38112
static_assert(NPAR == kEncParams, "parameter count");

// packed blob (bytes)
constexpr int bW1 = 0;                          // FP32 [224]
constexpr int bWf = 1024;                       // BF16 [3][32][224]
constexpr int bWt = bWf + 3 * C * KD * 2;       // BF16 [3][32][224]
constexpr int bP = bWt + 3 * C * KD * 2;        // BF16 [64][256]
constexpr int kBlobBytes = bP + DIM * NSEG * C * 2;
static_assert(kBlobBytes == kEncBlobBytes, "blob size");

// shared-memory row strides (elements) chosen so that the 8 rows one
// fragment load touches fall in distinct banks
constexpr int LDW = KD + 8;       // 232 bf16 per weight row
constexpr int LDX = C + 8;        // 40 bf16 per activation row
constexpr int LDP = NSEG * C + 8; // 264 bf16 per projection row
constexpr int kSeqThreads = 128;  // per-sequence kernels: 4 warps

__host__ __device__ constexpr int seg_lo(int s) { return L4 * s / NSEG; }

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t ld32(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ uint32_t pack2b(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
__device__ __forceinline__ float rbf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// D = A * B + D, A 16x16 (row), B 16x8 (col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Y[p][n] = sum_{t<7, c<32} X[p+t][c] * W[n][t*32+c] for the 32 outputs n of
// m16 tiles mt = warp, warp+nwarps, ... < m_tiles.  X: [rows][LDX] with at
// least 16*m_tiles + 6 rows; W: [32][LDW].  epi(row, col, v0, v1) receives
// the outputs (row, col) and (row, col+1).
template <typename Epi>
__device__ __forceinline__ void conv_mma(const bf16 *X, const bf16 *W, int m_tiles, int warp, int nwarps,
                                         Epi epi) {
    const int lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
    for (int mt = warp; mt < m_tiles; mt += nwarps) {
        float acc[4][4] = {};
#pragma unroll 2
        for (int kk = 0; kk < KD / 16; ++kk) {
            const int t = kk >> 1, cb = (kk & 1) * 16;
            const bf16 *x0 = X + (mt * 16 + g + t) * LDX + cb + 2 * tg;
            uint32_t a[4];
            a[0] = ld32(x0);
            a[1] = ld32(x0 + 8 * LDX);
            a[2] = ld32(x0 + 8);
            a[3] = ld32(x0 + 8 * LDX + 8);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const bf16 *w0 = W + (nt * 8 + g) * LDW + kk * 16 + 2 * tg;
                mma16816(acc[nt], a, ld32(w0), ld32(w0 + 8));
            }
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            epi(mt * 16 + g, nt * 8 + 2 * tg, acc[nt][0], acc[nt][1]);
            epi(mt * 16 + g + 8, nt * 8 + 2 * tg, acc[nt][2], acc[nt][3]);
        }
    }
}

// copy `rows` rows of `cols` bf16 (cols*2 a multiple of 16 bytes) from a
// dense global array into shared memory rows of stride `ld`
__device__ __forceinline__ void load_rows(bf16 *dst, int ld, const bf16 *src, int rows, int cols) {
    const int chunks = cols / 8;
    for (int i = threadIdx.x; i < rows * chunks; i += blockDim.x) {
        const int r = i / chunks, c = i - r * chunks;
        *reinterpret_cast<uint4 *>(dst + r * ld + c * 8) =
            *reinterpret_cast<const uint4 *>(src + (size_t)r * cols + c * 8);
    }
}

__device__ __forceinline__ void zero_smem(void *p, int bytes) {
    for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) reinterpret_cast<uint4 *>(p)[i] = make_uint4(0, 0, 0, 0);
}

// ------------------------------------------------------------------ packing
// params (FP32) -> blob; when `adam` is set, first one Adam step on params
// with `grad` (moments m1, v1; bias corrections c1 = 1 - beta1^t, c2 = 1 - beta2^t).
__global__ void k_pack(float *params, const float *grad, float *m1, float *v1, uint8_t *blob, int adam,
                       float lr, float beta1, float beta2, float eps, float c1, float c2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NPAR) return;
    float p = params[j];
    if (adam) {
        const float gr = grad[j];
        const float m = beta1 * m1[j] + (1.0f - beta1) * gr;
        const float v = beta2 * v1[j] + (1.0f - beta2) * gr * gr;
        m1[j] = m;
        v1[j] = v;
        p -= lr * (m / c1) / (sqrtf(v / c2) + eps);
        params[j] = p;
    }
    if (j < oW2) {
        reinterpret_cast<float *>(blob + bW1)[j] = p;
    } else if (j < oP) {
        const int l = (j - oW2) / (C * KD), r = (j - oW2) % (C * KD);
        const int co = r / KD, t = (r % KD) / C, ci = r % C;
        bf16 *wf = reinterpret_cast<bf16 *>(blob + bWf) + l * C * KD;
        bf16 *wt = reinterpret_cast<bf16 *>(blob + bWt) + l * C * KD;
        wf[co * KD + t * C + ci] = __float2bfloat16_rn(p);
        wt[ci * KD + (KW - 1 - t) * C + co] = __float2bfloat16_rn(p);
    } else {
        reinterpret_cast<bf16 *>(blob + bP)[j - oP] = __float2bfloat16_rn(p);
    }
}

// ------------------------------------------------------------------ input
// u of `rows` windows X[off[i] .. off[i]+m) (FP64 statistics, anchored at the
// window's first sample); one warp per row.
__global__ void k_prep(const float *X, const int64_t *off, int rows, int m, float *u) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= rows) return;
    const float *y = X + off[w];
    const double a0 = y[0];
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s += (double)y[i] - a0;
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double mu_rel = s / m;
    double v = 0.0;
    for (int i = lane; i < m; i += 32) {
        const double d = (double)y[i] - a0 - mu_rel;
        v += d * d;
    }
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    v /= m;
    const double mu = a0 + mu_rel;
    const double mm = mu * mu;
    const bool zero = v <= 1e-24 * (mm > 1.0 ? mm : 1.0);
    const double inv = zero ? 0.0 : 1.0 / sqrt(v);
    const int b = m / NB;
    // block sums relative to the anchor: lane j holds blocks j and j + 32
    double bs[2];
    for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        double acc = 0.0;
        for (int i = 0; i < b; ++i) acc += (double)y[j * b + i] - a0;
        bs[h] = acc;
    }
    // u_j = (S_{j+1} - S_j) / (b sigma); lane j needs S_{j+1}
    const double nxt0 = __shfl_down_sync(0xffffffffu, bs[0], 1);
    const double first1 = __shfl_sync(0xffffffffu, bs[1], 0);
    const double nxt1 = __shfl_down_sync(0xffffffffu, bs[1], 1);
    float *uo = u + (size_t)w * NB;
    const double sc = inv / b;
    uo[lane] = (float)(((lane < 31 ? nxt0 : first1) - bs[0]) * sc);
    if (lane < 31) uo[lane + 32] = (float)((nxt1 - bs[1]) * sc);
    else uo[63] = 0.0f;
}

// ------------------------------------------------------------------ per-sequence kernels
struct SeqSmem {
    // byte offsets
    static constexpr int W = 0;                                   // 3 x [32][LDW] bf16
    static constexpr int P = W + 3 * C * LDW * 2;                 // [64][LDP] bf16
    static constexpr int W1 = P + DIM * LDP * 2;                  // [224] f32
    static constexpr int U = W1 + 224 * 4;                        // [64] f32
    static constexpr int HA = U + 64 * 4;                         // [72][LDX] bf16
    static constexpr int HB = HA + 72 * LDX * 2;
    static constexpr int HC = HB + 72 * LDX * 2;
    static constexpr int H4 = HC + 72 * LDX * 2;                  // [48][32] f32
    static constexpr int G = H4 + 48 * C * 4;                     // [256] f32
    static constexpr int E = G + 256 * 4;                         // [64] f32
    static constexpr int BYTES = E + 64 * 4;
};

// stage the forward (or, with `transposed`, the backward) weights and P
__device__ void stage_weights(uint8_t *sm, const uint8_t *blob, bool transposed) {
    const bf16 *wsrc = reinterpret_cast<const bf16 *>(blob + (transposed ? bWt : bWf));
    for (int l = 0; l < 3; ++l)
        load_rows(reinterpret_cast<bf16 *>(sm + SeqSmem::W) + l * C * LDW, LDW, wsrc + l * C * KD, C, KD);
    load_rows(reinterpret_cast<bf16 *>(sm + SeqSmem::P), LDP, reinterpret_cast<const bf16 *>(blob + bP), DIM,
              NSEG * C);
    float *w1 = reinterpret_cast<float *>(sm + SeqSmem::W1);
    for (int i = threadIdx.x; i < 224; i += blockDim.x) w1[i] = reinterpret_cast<const float *>(blob + bW1)[i];
}

// Forward of one sequence whose u is in shared memory; leaves h1..h3 (BF16,
// post-ReLU) in HA, HB, HC, g (BF16-rounded, FP32) in G and e in E.
__device__ void seq_forward(uint8_t *sm) {
    const int warp = threadIdx.x >> 5;
    const float *u = reinterpret_cast<const float *>(sm + SeqSmem::U);
    const float *w1 = reinterpret_cast<const float *>(sm + SeqSmem::W1);
    const bf16 *W = reinterpret_cast<const bf16 *>(sm + SeqSmem::W);
    bf16 *h1 = reinterpret_cast<bf16 *>(sm + SeqSmem::HA);
    bf16 *h2 = reinterpret_cast<bf16 *>(sm + SeqSmem::HB);
    bf16 *h3 = reinterpret_cast<bf16 *>(sm + SeqSmem::HC);
    float *h4 = reinterpret_cast<float *>(sm + SeqSmem::H4);
    float *g = reinterpret_cast<float *>(sm + SeqSmem::G);
    float *e = reinterpret_cast<float *>(sm + SeqSmem::E);
    // conv1 (FP32), rows >= L1 stay zero
    for (int i = threadIdx.x; i < L1 * C; i += blockDim.x) {
        const int p = i / C, c = i - p * C;
        float z = 0.0f;
#pragma unroll
        for (int t = 0; t < KW; ++t) z = fmaf(w1[c * KW + t], u[p + t], z);
        h1[p * LDX + c] = __float2bfloat16_rn(fmaxf(z, 0.0f));
    }
    __syncthreads();
    conv_mma(h1, W, 4, warp, 4, [&](int p, int n, float v0, float v1) {
        const bool ok = p < L2;
        *reinterpret_cast<uint32_t *>(h2 + p * LDX + n) = pack2(ok ? fmaxf(v0, 0.f) : 0.f, ok ? fmaxf(v1, 0.f) : 0.f);
    });
    __syncthreads();
    conv_mma(h2, W + C * LDW, 3, warp, 4, [&](int p, int n, float v0, float v1) {
        const bool ok = p < L3;
        *reinterpret_cast<uint32_t *>(h3 + p * LDX + n) = pack2(ok ? fmaxf(v0, 0.f) : 0.f, ok ? fmaxf(v1, 0.f) : 0.f);
    });
    __syncthreads();
    conv_mma(h3, W + 2 * C * LDW, 3, warp, 4, [&](int p, int n, float v0, float v1) {
        h4[p * C + n] = v0;
        h4[p * C + n + 1] = v1;
    });
    __syncthreads();
    for (int j = threadIdx.x; j < NSEG * C; j += blockDim.x) {
        const int s = j / C, c = j - s * C, lo = seg_lo(s), hi = seg_lo(s + 1);
        float acc = 0.0f;
        for (int p = lo; p < hi; ++p) acc += h4[p * C + c];
        g[j] = rbf(acc / (float)(hi - lo));
    }
    __syncthreads();
    {
        const bf16 *P = reinterpret_cast<const bf16 *>(sm + SeqSmem::P);
        const int d = threadIdx.x >> 1, half = threadIdx.x & 1;
        float acc = 0.0f;
        for (int j = half * 128; j < half * 128 + 128; ++j) acc = fmaf(__bfloat162float(P[d * LDP + j]), g[j], acc);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (!half) e[d] = acc;
    }
    __syncthreads();
}

// Per-sequence workspace of the trainer (bytes per sequence).
struct SeqWs {
    static constexpr int ACT = 0;                  // h1, h2, h3: [3][64][32] bf16
    static constexpr int DZ = ACT + 3 * 64 * C * 2; // dz1..dz4: [4][64][32] bf16
    static constexpr int G = DZ + 4 * 64 * C * 2;   // [256] f32
    static constexpr int E = G + 256 * 4;           // [64] f32
    static constexpr int DE = E + 64 * 4;           // [64] f32
    static constexpr int U = DE + 64 * 4;           // [64] f32
    static constexpr int BYTES = U + 64 * 4;
};

// Forward of `rows` sequences (u: [rows][64] f32).  TRAIN: store the
// activations for the backward pass in the workspace; else write e.
template <bool TRAIN>
__global__ void __launch_bounds__(kSeqThreads) k_seq_forward(const uint8_t *blob, const float *u, int rows,
                                                             float *e_out, uint8_t *ws) {
    extern __shared__ __align__(16) uint8_t sm[];
    stage_weights(sm, blob, false);
    zero_smem(sm + SeqSmem::HA, 3 * 72 * LDX * 2);
    __syncthreads();
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        float *us = reinterpret_cast<float *>(sm + SeqSmem::U);
        for (int i = threadIdx.x; i < 64; i += blockDim.x) us[i] = i < NU ? u[(size_t)r * 64 + i] : 0.0f;
        __syncthreads();
        seq_forward(sm);
        const float *e = reinterpret_cast<const float *>(sm + SeqSmem::E);
        if (TRAIN) {
            uint8_t *w = ws + (size_t)r * SeqWs::BYTES;
            for (int l = 0; l < 3; ++l) {
                const bf16 *h = reinterpret_cast<const bf16 *>(sm + SeqSmem::HA + l * 72 * LDX * 2);
                bf16 *dst = reinterpret_cast<bf16 *>(w + SeqWs::ACT) + l * 64 * C;
                for (int i = threadIdx.x; i < 64 * C / 8; i += blockDim.x) {
                    const int p = i / (C / 8), c = (i % (C / 8)) * 8;
                    *reinterpret_cast<uint4 *>(dst + p * C + c) = *reinterpret_cast<const uint4 *>(h + p * LDX + c);
                }
            }
            const float *g = reinterpret_cast<const float *>(sm + SeqSmem::G);
            for (int i = threadIdx.x; i < 256; i += blockDim.x) reinterpret_cast<float *>(w + SeqWs::G)[i] = g[i];
            for (int i = threadIdx.x; i < 64; i += blockDim.x) {
                reinterpret_cast<float *>(w + SeqWs::E)[i] = e[i];
                reinterpret_cast<float *>(w + SeqWs::U)[i] = us[i];
            }
        } else {
            for (int i = threadIdx.x; i < DIM; i += blockDim.x) e_out[(size_t)r * DIM + i] = e[i];
        }
        __syncthreads();
    }
}

// Loss of B triples (sequence i = query, B + i = candidate) and d(loss)/de.
__global__ void k_loss(uint8_t *ws, const float *y, int B, float *loss) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= B) return;
    uint8_t *wq = ws + (size_t)i * SeqWs::BYTES, *wc = ws + (size_t)(B + i) * SeqWs::BYTES;
    const float *eq = reinterpret_cast<const float *>(wq + SeqWs::E);
    const float *ec = reinterpret_cast<const float *>(wc + SeqWs::E);
    const float d0 = eq[lane] - ec[lane], d1 = eq[lane + 32] - ec[lane + 32];
    float dist = d0 * d0 + d1 * d1;
    for (int o = 16; o; o >>= 1) dist += __shfl_xor_sync(0xffffffffu, dist, o);
    const float eps = 1e-3f;
    const float lr = logf(dist + eps) - logf(y[i] + eps);
    const float dd = 2.0f * lr / (dist + eps) / (float)B;
    float *deq = reinterpret_cast<float *>(wq + SeqWs::DE), *dec = reinterpret_cast<float *>(wc + SeqWs::DE);
    deq[lane] = 2.0f * d0 * dd;
    deq[lane + 32] = 2.0f * d1 * dd;
    dec[lane] = -2.0f * d0 * dd;
    dec[lane + 32] = -2.0f * d1 * dd;
    if (lane == 0) atomicAdd(loss, lr * lr / (float)B);
}

// Backward through projection, pooling and the convolutions of each
// sequence (data gradients); stores dz1..dz4 (gradients of the layers'
// pre-activations, zero beyond each layer's length) in the workspace.
__global__ void __launch_bounds__(kSeqThreads) k_seq_backward(const uint8_t *blob, int rows, uint8_t *ws) {
    extern __shared__ __align__(16) uint8_t sm[];
    stage_weights(sm, blob, true);
    zero_smem(sm + SeqSmem::HA, 3 * 72 * LDX * 2);
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const bf16 *Wt = reinterpret_cast<const bf16 *>(sm + SeqSmem::W);
    const bf16 *P = reinterpret_cast<const bf16 *>(sm + SeqSmem::P);
    bf16 *dA = reinterpret_cast<bf16 *>(sm + SeqSmem::HA);  // padded gradient tiles: row 6 + p holds position p
    bf16 *dB = reinterpret_cast<bf16 *>(sm + SeqSmem::HB);
    bf16 *act = reinterpret_cast<bf16 *>(sm + SeqSmem::HC);  // [72][LDX]: the current layer's h for the mask
    float *de = reinterpret_cast<float *>(sm + SeqSmem::E);
    float *dg = reinterpret_cast<float *>(sm + SeqSmem::G);
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        uint8_t *w = ws + (size_t)r * SeqWs::BYTES;
        const bf16 *hg = reinterpret_cast<const bf16 *>(w + SeqWs::ACT);
        bf16 *dz = reinterpret_cast<bf16 *>(w + SeqWs::DZ);
        for (int i = threadIdx.x; i < 64; i += blockDim.x) de[i] = reinterpret_cast<const float *>(w + SeqWs::DE)[i];
        __syncthreads();
        for (int j = threadIdx.x; j < NSEG * C; j += blockDim.x) {
            float acc = 0.0f;
            for (int d = 0; d < DIM; ++d) acc = fmaf(__bfloat162float(P[d * LDP + j]), de[d], acc);
            dg[j] = acc;
        }
        __syncthreads();
        // dz4 = pool backward, placed at rows 6 + p of dA; rows 0..5 and >= 6 + L4 zero
        for (int i = threadIdx.x; i < 72 * C; i += blockDim.x) {
            const int row = i / C, c = i - row * C, p = row - 6;
            float v = 0.0f;
            if (p >= 0 && p < L4) {
                int s = 0;
                while (s < NSEG - 1 && p >= seg_lo(s + 1)) ++s;
                v = dg[s * C + c] / (float)(seg_lo(s + 1) - seg_lo(s));
            }
            dA[row * LDX + c] = __float2bfloat16_rn(v);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 64 * C; i += blockDim.x) {  // global dz4: position p at row p
            const int p = i / C, c = i - p * C;
            dz[3 * 64 * C + i] = p < L4 ? dA[(p + 6) * LDX + c] : __float2bfloat16_rn(0.f);
        }
        // l = 3, 2, 1: dh_l = transposed convolution of dz_{l+1} with W_{l+1};
        // dz_l = dh_l masked by h_l > 0.  Buffers alternate dA -> dB -> dA -> dB.
        for (int l = 3; l >= 1; --l) {
            const int Lout = l == 3 ? L3 : (l == 2 ? L2 : L1);
            const int mtiles = (Lout + 15) / 16;
            const bf16 *src = (l == 2) ? dB : dA;
            bf16 *dst = (l == 2) ? dA : dB;
            for (int i = threadIdx.x; i < 64 * C / 8; i += blockDim.x) {
                const int p = i / (C / 8), c = (i % (C / 8)) * 8;
                *reinterpret_cast<uint4 *>(act + p * LDX + c) =
                    *reinterpret_cast<const uint4 *>(hg + (l - 1) * 64 * C + p * C + c);
            }
            __syncthreads();
            bf16 *dzl = dz + (l - 1) * 64 * C;
            conv_mma(src, Wt + (l - 1) * C * LDW, mtiles, warp, 4, [&](int q, int n, float v0, float v1) {
                const bool ok = q < Lout;
                const float m0 = ok && __bfloat162float(act[q * LDX + n]) > 0.f ? v0 : 0.f;
                const float m1 = ok && __bfloat162float(act[q * LDX + n + 1]) > 0.f ? v1 : 0.f;
                const uint32_t pk = pack2(m0, m1);
                *reinterpret_cast<uint32_t *>(dst + (q + 6) * LDX + n) = pk;
                *reinterpret_cast<uint32_t *>(dzl + q * C + n) = pk;
            });
            __syncthreads();
            // the next layer reads rows 0..69 of dst: zero the rows no tile wrote
            for (int i = threadIdx.x; i < 72 * C; i += blockDim.x) {
                const int row = i / C;
                if (row < 6 || row >= 6 + mtiles * 16) dst[i / C * LDX + (i % C)] = __float2bfloat16_rn(0.f);
            }
            for (int i = threadIdx.x; i < 64 * C; i += blockDim.x)
                if (i / C >= mtiles * 16) dzl[i] = __float2bfloat16_rn(0.f);
            __syncthreads();
        }
    }
}

// Weight gradients.  blockIdx.y = 0: dW1 (FP32); 1..3: dW2..dW4 on tensor
// cores, dW[co][t*32+ci] = sum over sequences and positions p of
// dz_l[p][co] * h_{l-1}[p+t][ci]; each CTA sums its sequences, then adds to
// `grad` atomically.
__global__ void __launch_bounds__(kSeqThreads) k_wgrad(const uint8_t *ws, int rows, float *grad) {
    __shared__ __align__(16) bf16 dzT[C * 72];  // [co][p]
    __shared__ __align__(16) bf16 hT[C * 72];   // [ci][q], q < 72 (zero past 63)
    __shared__ float s_dz[64 * C];
    __shared__ float s_u[64];
    const int layer = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, tg = lane & 3;
    if (layer == 0) {
        float acc0 = 0.f, acc1 = 0.f;
        const int i0 = threadIdx.x, i1 = threadIdx.x + 128;  // (co, t) = i / 7, i % 7
        for (int r = blockIdx.x; r < rows; r += gridDim.x) {
            const uint8_t *w = ws + (size_t)r * SeqWs::BYTES;
            const bf16 *dz1 = reinterpret_cast<const bf16 *>(w + SeqWs::DZ);
            for (int i = threadIdx.x; i < 64 * C; i += blockDim.x) s_dz[i] = __bfloat162float(dz1[i]);
            for (int i = threadIdx.x; i < 64; i += blockDim.x) s_u[i] = reinterpret_cast<const float *>(w + SeqWs::U)[i];
            __syncthreads();
            {
                const int co = i0 / KW, t = i0 % KW;
                for (int p = 0; p < L1; ++p) acc0 = fmaf(s_dz[p * C + co], s_u[p + t], acc0);
            }
            if (i1 < C * KW) {
                const int co = i1 / KW, t = i1 % KW;
                for (int p = 0; p < L1; ++p) acc1 = fmaf(s_dz[p * C + co], s_u[p + t], acc1);
            }
            __syncthreads();
        }
        atomicAdd(grad + oW1 + i0, acc0);
        if (i1 < C * KW) atomicAdd(grad + oW1 + i1, acc1);
        return;
    }
    // layer l = layer + 1 in 2..4: dz_l is dz index l-1, h_{l-1} is act index l-2
    const int dzi = layer, hi = layer - 1;
    float acc[2][7][4] = {};
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const uint8_t *w = ws + (size_t)r * SeqWs::BYTES;
        const bf16 *dz = reinterpret_cast<const bf16 *>(w + SeqWs::DZ) + dzi * 64 * C;
        const bf16 *h = reinterpret_cast<const bf16 *>(w + SeqWs::ACT) + hi * 64 * C;
        for (int i = threadIdx.x; i < 64 * C; i += blockDim.x) {
            const int p = i / C, c = i - p * C;
            dzT[c * 72 + p] = dz[i];
            hT[c * 72 + p] = h[i];
        }
        for (int i = threadIdx.x; i < C * 8; i += blockDim.x) hT[(i >> 3) * 72 + 64 + (i & 7)] = __float2bfloat16_rn(0.f);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const bf16 *p0 = dzT + (mt * 16 + g) * 72 + kk * 16 + 2 * tg;
                a[mt][0] = ld32(p0);
                a[mt][1] = ld32(p0 + 8 * 72);
                a[mt][2] = ld32(p0 + 8);
                a[mt][3] = ld32(p0 + 8 * 72 + 8);
            }
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                const int n = (warp * 7 + j) * 8 + g, t = n >> 5, ci = n & 31;
                const bf16 *q0 = hT + ci * 72 + kk * 16 + 2 * tg + t;
                const uint32_t b0 = pack2b(q0[0], q0[1]), b1 = pack2b(q0[8], q0[9]);
                mma16816(acc[0][j], a[0], b0, b1);
                mma16816(acc[1][j], a[1], b0, b1);
            }
        }
        __syncthreads();
    }
    float *gw = grad + oW2 + (layer - 1) * C * KD;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const int co = mt * 16 + g, n = (warp * 7 + j) * 8 + 2 * tg;
            atomicAdd(gw + co * KD + n, acc[mt][j][0]);
            atomicAdd(gw + co * KD + n + 1, acc[mt][j][1]);
            atomicAdd(gw + (co + 8) * KD + n, acc[mt][j][2]);
            atomicAdd(gw + (co + 8) * KD + n + 1, acc[mt][j][3]);
        }
}

// dP[d][j] = sum over sequences of de[d] * g[j] (g as used by the forward)
__global__ void k_dP(const uint8_t *ws, int rows, float *grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= DIM * NSEG * C) return;
    const int d = i / (NSEG * C), j = i - d * (NSEG * C);
    float acc = 0.0f;
    for (int r = 0; r < rows; ++r) {
        const uint8_t *w = ws + (size_t)r * SeqWs::BYTES;
        acc = fmaf(reinterpret_cast<const float *>(w + SeqWs::DE)[d], reinterpret_cast<const float *>(w + SeqWs::G)[j],
                   acc);
    }
    grad[oP + i] = acc;
}

// ------------------------------------------------------------------ series-wide embeddings
// For the windows at offsets j0*b (j0 < Nw): E[j0] = inv_sigma[j0*b] * e(raw
// block-mean differences of the window), BF16 [Nw][64].  One CTA (8 warps)
// per tile of 128 windows, persistent over tiles.
constexpr int kSerThreads = 256, kSerTile = 128;
constexpr int kSerD = kSerTile + 62 + 2;      // 192 differences (190 needed)
struct SerSmem {
    static constexpr int W = 0;                              // 3 x [32][LDW] bf16
    static constexpr int P = W + 3 * C * LDW * 2;            // [64][LDP] bf16
    static constexpr int W1 = P + DIM * LDP * 2;             // [224] f32
    static constexpr int D = W1 + 224 * 4;                   // [kSerD + 2] f32 (block sums, then differences)
    static constexpr int HA = D + (kSerD + 2 + 2) * 4;        // [200][LDX] bf16: h1, then h3
    static constexpr int HB = HA + 200 * LDX * 2;            // [192][LDX] bf16: h2
    static constexpr int C4 = HB + 192 * LDX * 2;            // [178][32] f32: prefix sums of h4
    static constexpr int BYTES = C4 + 178 * C * 4;
};
static_assert(SerSmem::D % 16 == 0 && SerSmem::HA % 16 == 0 && SerSmem::HB % 16 == 0 && SerSmem::C4 % 16 == 0, "align");

__global__ void __launch_bounds__(kSerThreads) k_series(const uint8_t *blob, const float *x, int64_t n, int b,
                                                        const float *inv_sigma, int64_t Nw, bf16 *E) {
    extern __shared__ __align__(16) uint8_t sm[];
    stage_weights(sm, blob, false);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bf16 *W = reinterpret_cast<const bf16 *>(sm + SerSmem::W);
    const bf16 *P = reinterpret_cast<const bf16 *>(sm + SerSmem::P);
    const float *w1 = reinterpret_cast<const float *>(sm + SerSmem::W1);
    float *D = reinterpret_cast<float *>(sm + SerSmem::D);
    bf16 *hA = reinterpret_cast<bf16 *>(sm + SerSmem::HA);
    bf16 *hB = reinterpret_cast<bf16 *>(sm + SerSmem::HB);
    float *c4 = reinterpret_cast<float *>(sm + SerSmem::C4);
    const int64_t nblocks = n / b;
    const int64_t tiles = (Nw + kSerTile - 1) / kSerTile;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t j0 = tile * kSerTile;
        __syncthreads();
        // block sums S_j (j0 <= j < j0 + 193) relative to the tile's first sample
        const float anchor = x[j0 * b];
        for (int r = warp; r < kSerD + 1; r += kSerThreads / 32) {
            const int64_t j = j0 + r;
            float acc = 0.0f;
            if (j < nblocks)
                for (int i = lane; i < b; i += 32) acc += x[j * b + i] - anchor;
            for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) D[r] = acc;
        }
        __syncthreads();
        float dv = 0.0f;
        if (threadIdx.x < kSerD) dv = (D[threadIdx.x + 1] - D[threadIdx.x]) / (float)b;
        __syncthreads();
        if (threadIdx.x < kSerD) D[threadIdx.x] = dv;
        __syncthreads();
        // conv1 -> h1 rows 0..185 (valid 184), rows >= 186 zero
        for (int i = threadIdx.x; i < 200 * C; i += kSerThreads) {
            const int p = i / C, c = i - p * C;
            float z = 0.0f;
            if (p < kSerD - 6) {
#pragma unroll
                for (int t = 0; t < KW; ++t) z = fmaf(w1[c * KW + t], D[p + t], z);
            }
            hA[p * LDX + c] = __float2bfloat16_rn(fmaxf(z, 0.0f));
        }
        __syncthreads();
        conv_mma(hA, W, 12, warp, 8, [&](int p, int nn, float v0, float v1) {
            *reinterpret_cast<uint32_t *>(hB + p * LDX + nn) = pack2(fmaxf(v0, 0.f), fmaxf(v1, 0.f));
        });
        __syncthreads();
        conv_mma(hB, W + C * LDW, 11, warp, 8, [&](int p, int nn, float v0, float v1) {
            *reinterpret_cast<uint32_t *>(hA + p * LDX + nn) = pack2(fmaxf(v0, 0.f), fmaxf(v1, 0.f));
        });
        for (int i = threadIdx.x; i < 8 * C; i += kSerThreads) hA[(176 + i / C) * LDX + (i % C)] = __float2bfloat16_rn(0.f);
        __syncthreads();
        conv_mma(hA, W + 2 * C * LDW, 11, warp, 8, [&](int p, int nn, float v0, float v1) {
            c4[(p + 1) * C + nn] = v0;
            c4[(p + 1) * C + nn + 1] = v1;
        });
        __syncthreads();
        if (threadIdx.x < C) {  // prefix over positions, per channel: c4[p] = sum_{p' < p} h4[p']
            float acc = 0.0f;
            c4[threadIdx.x] = 0.0f;
            for (int p = 1; p <= 166; ++p) {
                acc += c4[p * C + threadIdx.x];
                c4[p * C + threadIdx.x] = acc;
            }
        }
        __syncthreads();
        // projection: warp w -> windows w*16 .. w*16+15, all 64 outputs
        {
            const int g = lane >> 2, tg = lane & 3;
            float acc[8][4] = {};
            const int wr0 = warp * 16 + g, wr1 = wr0 + 8;
#pragma unroll 2
            for (int kk = 0; kk < 16; ++kk) {
                const int s = kk >> 1, lo = seg_lo(s), hi = seg_lo(s + 1);
                const float il = 1.0f / (float)(hi - lo);
                const int c0 = (kk & 1) * 16 + 2 * tg;
                uint32_t a[4];
                auto seg = [&](int w, int c) {
                    return pack2(rbf((c4[(w + hi) * C + c] - c4[(w + lo) * C + c]) * il),
                                 rbf((c4[(w + hi) * C + c + 1] - c4[(w + lo) * C + c + 1]) * il));
                };
                a[0] = seg(wr0, c0);
                a[1] = seg(wr1, c0);
                a[2] = seg(wr0, c0 + 8);
                a[3] = seg(wr1, c0 + 8);
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const bf16 *p0 = P + (nt * 8 + g) * LDP + kk * 16 + 2 * tg;
                    mma16816(acc[nt], a, ld32(p0), ld32(p0 + 8));
                }
            }
            const int64_t r0 = j0 + wr0, r1 = j0 + wr1;
            const float s0 = r0 < Nw ? inv_sigma[r0 * b] : 0.f, s1 = r1 < Nw ? inv_sigma[r1 * b] : 0.f;
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int d = nt * 8 + 2 * tg;
                if (r0 < Nw) *reinterpret_cast<uint32_t *>(E + r0 * DIM + d) = pack2(acc[nt][0] * s0, acc[nt][1] * s0);
                if (r1 < Nw) *reinterpret_cast<uint32_t *>(E + r1 * DIM + d) = pack2(acc[nt][2] * s1, acc[nt][3] * s1);
            }
        }
    }
}

// ------------------------------------------------------------------ query side
// e_q of the normalised query (qh32) into the query state; one CTA.
__global__ void __launch_bounds__(kSeqThreads) k_query_embed(const uint8_t *blob, QueryBufs bq, int m) {
    extern __shared__ __align__(16) uint8_t sm[];
    if (!bq.st->valid) return;
    stage_weights(sm, blob, false);
    zero_smem(sm + SeqSmem::HA, 3 * 72 * LDX * 2);
    float *us = reinterpret_cast<float *>(sm + SeqSmem::U);
    float *tmp = reinterpret_cast<float *>(sm + SeqSmem::G);  // block means
    const int b = m / NB;
    for (int j = threadIdx.x; j < NB; j += blockDim.x) {
        float acc = 0.0f;
        for (int i = 0; i < b; ++i) acc += bq.qh32[j * b + i];
        tmp[j] = acc / (float)b;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < 64; j += blockDim.x) us[j] = j < NU ? tmp[j + 1] - tmp[j] : 0.0f;
    __syncthreads();
    seq_forward(sm);
    for (int i = threadIdx.x; i < DIM; i += blockDim.x) bq.st->e_q[i] = reinterpret_cast<const float *>(sm + SeqSmem::E)[i];
}

// Per-row int8 copy of the embeddings for the scan: q = round(e * 127 / max|e|)
// with the row's scale s = max|e| / 127 (q = 0, s = 0 for an all-zero row),
// and the squared norm of the quantised row, s^2 * sum q^2: S[row] = (s, norm).
// Eight lanes per row (8 values each), the row maximum by shuffles.
__global__ void k_quant_rows(const bf16 *__restrict__ E, int64_t rows, int8_t *__restrict__ Q,
                             float2 *__restrict__ S) {
    const int lane = threadIdx.x & 31, sub = lane & 7;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (gridDim.x * (int64_t)blockDim.x) >> 5;
    for (int64_t r0 = gw * 4; r0 < rows; r0 += nw * 4) {  // four rows per warp, warp-uniform
        const int64_t r = r0 + (lane >> 3);
        float v[8];
        float mx = 0.0f;
        if (r < rows) {
            const uint4 raw = *reinterpret_cast<const uint4 *>(E + r * DIM + sub * 8);
            const bf16 *h = reinterpret_cast<const bf16 *>(&raw);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                v[k] = __bfloat162float(h[k]);
                mx = fmaxf(mx, fabsf(v[k]));
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = 0.0f;
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float inv = mx > 0.0f ? 127.0f / mx : 0.0f;
        unsigned w[2] = {0u, 0u};
        int q2 = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int q = max(-127, min(127, __float2int_rn(v[k] * inv)));
            q2 += q * q;
            w[k >> 2] |= (unsigned)(q & 0xff) << (8 * (k & 3));
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) q2 += __shfl_xor_sync(0xffffffffu, q2, o);
        if (r < rows) {
            *reinterpret_cast<uint2 *>(Q + r * DIM + sub * 8) = make_uint2(w[0], w[1]);
            if (sub == 0) {
                const float sc = mx * (1.0f / 127.0f);
                S[r] = make_float2(sc, sc * sc * (float)q2);
            }
        }
    }
}

// Score every window at stride b by |e_q - s_j v_j|^2, v_j, s_j the row's
// int8 embedding and scale, expanded as |e_q|^2 - 2 s_j s_q (e8 . v_j) +
// s_j^2 |v_j|^2 with e8, s_q the query embedding quantised the same way:
// the dot product of two int8 vectors in four DP4A instructions per lane
// (4 lanes per window, 16 dimensions each), |v_j|^2 stored with the row.
// The expansion cancels for near matches (a few 1e-3 of |e_q|^2), which
// only perturbs the order among the closest windows; negative results are
// clamped to 0.  Each warp scans one contiguous segment of the windows with
// eight 16-byte loads in flight per lane; each CTA writes its best window
// (one barrier, at the end) to its slot for the proposal merge.
constexpr int kLsThreads = 256, kLsU = 8;
__global__ void __launch_bounds__(kLsThreads) k_learn_scan(QueryBufs bq, const int8_t *Q, const float2 *S,
                                                           int64_t Nw, int b, int phase, int slot, int64_t seg) {
    __shared__ unsigned long long wbest[kLsThreads / 32];
    QueryState *st = bq.st;
    if (!st->valid) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, sub = lane & 3, grp = lane >> 2;
    const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    // the query's embedding: |e_q|^2, its int8 copy (this lane's 16 values)
    float qn = 0.0f, qmx = 0.0f;
    for (int i = 0; i < DIM; ++i) {
        const float e = st->e_q[i];
        qn = fmaf(e, e, qn);
        qmx = fmaxf(qmx, fabsf(e));
    }
    const float qinv = qmx > 0.0f ? 127.0f / qmx : 0.0f, two_sq = 2.0f * qmx * (1.0f / 127.0f);
    int e8[4];
#pragma unroll
    for (int wi = 0; wi < 4; ++wi) {
        unsigned wd = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int q = max(-127, min(127, __float2int_rn(st->e_q[sub * 16 + wi * 4 + k] * qinv)));
            wd |= (unsigned)(q & 0xff) << (8 * k);
        }
        e8[wi] = (int)wd;
    }
    const int64_t lo = gwarp * seg, hi = lo + seg < Nw ? lo + seg : Nw;
    unsigned long long mine = ~0ull;
    // every lane runs the same number of steps (the shuffles below need the whole warp)
    for (int64_t base = lo; base < hi; base += 8 * kLsU) {
        const int64_t j0 = base + grp;
        uint4 v[kLsU];
        float2 sn[kLsU];  // (scale, norm) of the row, loaded with it
#pragma unroll
        for (int u = 0; u < kLsU; ++u) {
            const int64_t j = j0 + 8 * u;
            const bool in = j < hi;
            v[u] = in ? *reinterpret_cast<const uint4 *>(Q + j * DIM + sub * 16) : make_uint4(0, 0, 0, 0);
            sn[u] = in && sub == 0 ? S[j] : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < kLsU; ++u) {
            const int64_t j = j0 + 8 * u;
            int dot = __dp4a((int)v[u].x, e8[0], 0);
            dot = __dp4a((int)v[u].y, e8[1], dot);
            dot = __dp4a((int)v[u].z, e8[2], dot);
            dot = __dp4a((int)v[u].w, e8[3], dot);
            dot += __shfl_xor_sync(0xffffffffu, dot, 1);
            dot += __shfl_xor_sync(0xffffffffu, dot, 2);
            if (j < hi && sub == 0) {
                const float s = fmaxf(0.0f, fmaf(-two_sq * sn[u].x, (float)dot, qn + sn[u].y));
                const unsigned long long k = make_key(s, (unsigned)(j * b + phase));
                mine = k < mine ? k : mine;
            }
        }
    }
    for (int o = 16; o; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, mine, o);
        mine = v < mine ? v : mine;
    }
    if (lane == 0) wbest[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long k = wbest[0];
        for (int w = 1; w < kLsThreads / 32; ++w) k = wbest[w] < k ? wbest[w] : k;
        st->cta_best[slot * kCtaSlots + blockIdx.x] = k;
    }
}

}  // namespace enc

// ------------------------------------------------------------------ launchers
static cudaError_t set_smem(const void *f, int bytes) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_enc_pack(float *params, const float *grad, float *m1, float *v1, uint8_t *blob, bool adam,
                            float lr, float beta1, float beta2, float eps, float c1, float c2, cudaStream_t s) {
    enc::k_pack<<<(enc::NPAR + 255) / 256, 256, 0, s>>>(params, grad, m1, v1, blob, adam ? 1 : 0, lr, beta1,
                                                        beta2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_enc_prep(const float *X, const int64_t *off, int rows, int m, float *u, cudaStream_t s) {
    enc::k_prep<<<(rows * 32 + 255) / 256, 256, 0, s>>>(X, off, rows, m, u);
    return cudaGetLastError();
}

cudaError_t launch_enc_forward(const uint8_t *blob, const float *u, int rows, float *e, uint8_t *ws, int num_sms,
                               cudaStream_t s) {
    const int smem = enc::SeqSmem::BYTES;
    const int grid = rows < 2 * num_sms ? rows : 2 * num_sms;
    cudaError_t err;
    if (ws) {
        if ((err = set_smem((const void *)enc::k_seq_forward<true>, smem)) != cudaSuccess) return err;
        enc::k_seq_forward<true><<<grid, enc::kSeqThreads, smem, s>>>(blob, u, rows, e, ws);
    } else {
        if ((err = set_smem((const void *)enc::k_seq_forward<false>, smem)) != cudaSuccess) return err;
        enc::k_seq_forward<false><<<grid, enc::kSeqThreads, smem, s>>>(blob, u, rows, e, ws);
    }
    return cudaGetLastError();
}

cudaError_t launch_enc_backward(const uint8_t *blob, const float *y, int B, float *loss, float *grad,
                                uint8_t *ws, int num_sms, cudaStream_t s) {
    const int rows = 2 * B;
    enc::k_loss<<<(B * 32 + 255) / 256, 256, 0, s>>>(ws, y, B, loss);
    cudaError_t err = set_smem((const void *)enc::k_seq_backward, enc::SeqSmem::BYTES);
    if (err != cudaSuccess) return err;
    const int grid = rows < 2 * num_sms ? rows : 2 * num_sms;
    enc::k_seq_backward<<<grid, enc::kSeqThreads, enc::SeqSmem::BYTES, s>>>(blob, rows, ws);
    if ((err = cudaMemsetAsync(grad, 0, sizeof(float) * enc::oP, s)) != cudaSuccess) return err;
    const int gx = rows < num_sms ? rows : num_sms;
    enc::k_wgrad<<<dim3(gx, 4), enc::kSeqThreads, 0, s>>>(ws, rows, grad);
    enc::k_dP<<<(enc::DIM * enc::NSEG * enc::C + 127) / 128, 128, 0, s>>>(ws, rows, grad);
    return cudaGetLastError();
}

cudaError_t launch_enc_series(const uint8_t *blob, const float *x, int64_t n, int b, const float *inv_sigma,
                              int64_t Nw, void *E, int num_sms, cudaStream_t s) {
    cudaError_t err = set_smem((const void *)enc::k_series, enc::SerSmem::BYTES);
    if (err != cudaSuccess) return err;
    const int64_t tiles = (Nw + enc::kSerTile - 1) / enc::kSerTile;
    const int grid = (int)(tiles < num_sms ? tiles : num_sms);
    enc::k_series<<<grid, enc::kSerThreads, enc::SerSmem::BYTES, s>>>(blob, x, n, b, inv_sigma, Nw,
                                                                       reinterpret_cast<enc::bf16 *>(E));
    return cudaGetLastError();
}

cudaError_t launch_enc_query(const uint8_t *blob, const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    cudaError_t err = set_smem((const void *)enc::k_query_embed, enc::SeqSmem::BYTES);
    if (err != cudaSuccess) return err;
    enc::k_query_embed<<<1, enc::kSeqThreads, enc::SeqSmem::BYTES, s>>>(blob, b, a.m);
    return cudaGetLastError();
}

size_t enc_workspace_bytes(int rows) { return (size_t)rows * enc::SeqWs::BYTES; }

static __global__ void k_bf16_to_f32(const enc::bf16 *src, int64_t count, float *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __bfloat162float(src[i]);
}

cudaError_t launch_bf16_to_f32(const void *src, int64_t count, float *dst, cudaStream_t s) {
    const int64_t blocks = (count + 255) / 256;
    k_bf16_to_f32<<<(int)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096), 256, 0, s>>>(
        reinterpret_cast<const enc::bf16 *>(src), count, dst);
    return cudaGetLastError();
}

cudaError_t launch_enc_quant(const void *E, int64_t rows, void *Q, void *S, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    int64_t blocks = (rows * 8 + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    enc::k_quant_rows<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const enc::bf16 *>(E), rows,
                                                       reinterpret_cast<int8_t *>(Q), reinterpret_cast<float2 *>(S));
    return cudaGetLastError();
}

cudaError_t launch_learn_scan(const QueryBufs &b, const void *Q, const void *S, int64_t Nw, int stride,
                              int phase, int slot, int *ctas, cudaStream_t s) {
    // one wave: as many CTAs as are resident at once, each warp a segment of
    // >= 256 windows (a second wave would leave the first wave's SMs idle)
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enc::k_learn_scan, enc::kLsThreads, 0) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int64_t per_cta = (int64_t)(enc::kLsThreads / 32) * 256;
    int64_t grid = (Nw + per_cta - 1) / per_cta;
    if (grid > (int64_t)per_sm * b.num_sms) grid = (int64_t)per_sm * b.num_sms;
    if (grid > kCtaSlots) grid = kCtaSlots;
    if (grid < 1) grid = 1;
    const int64_t warps = grid * (enc::kLsThreads / 32);
    const int64_t seg = ((Nw + warps - 1) / warps + 31) / 32 * 32;
    enc::k_learn_scan<<<(unsigned)grid, enc::kLsThreads, 0, s>>>(b, reinterpret_cast<const int8_t *>(Q),
                                                                 reinterpret_cast<const float2 *>(S), Nw,
                                                                 stride, phase, slot, seg);
    *ctas = (int)grid;
    return cudaGetLastError();
}

}  // namespace dtws
