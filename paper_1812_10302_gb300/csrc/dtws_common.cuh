// dtws_common.cuh -- device helpers shared by the dtws kernels (sm_103a).
//
// * packed top-k keys: (float bits of a non-negative distance << 32) | offset,
//   so unsigned order is (distance, offset) order, the tie rule of the search
//   (lowest offset wins);
// * a lock-free bounded top-k list built from atomicMin on such keys;
// * inline-PTX wrappers for mbarriers and 1-D bulk (TMA) copies;
// * bounded waits that record DTWS_ETIMEOUT instead of spinning forever.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>
#include <cuda_runtime.h>

namespace dtws {

// Compile-time loop: f(std::integral_constant<int, I>{}) for I = 0..N-1, so
// the body can use I as a template argument (register indices, rotations).
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------- limits
constexpr int kBlockB = 8192;       // anchored prefix block length (= DTWS_M_MAX)
constexpr int kMMax = 8192;
constexpr int kKMax = 64;
constexpr int kListMax = 128;       // result list capacity (k + near-tie margin)
constexpr int kSeedMax = 128;       // random seeds + proxy proposals
constexpr int kPropMax = 64;
constexpr int kCtaSlots = 1024;     // per-CTA best windows of one proposal scan (at most this many CTAs)
constexpr int kProxyStride = 4;     // the proxy scan looks at every fourth window
// Euclidean seeds around each proxy proposal: offsets within +-kProxyHalf.
// A match off the proxy's grid is never scored by the proxy itself; on a
// series with strong per-sample noise the proxy can also rank a window a few
// samples off above the nearest one (one noisy copy of m = 1024 on the
// 2e7-sample walk with bursts did), so the seeds reach three samples either
// side: with one window in four scored, every window lies within two of a
// scored one.
constexpr int kProxyHalf = 3;
// Euclidean seeds: random windows + the neighbourhoods of the proposals
// (+-kProxyHalf windows for the proxy scan; +-b/2, b <= 128, for the learned scan with
// at most kLearnPropMax proposals)
constexpr int kLearnPropMax = 64;
// per-series block envelope: sparse table of max / min over blocks of
// kEnvG samples, levels 0..kEnvLevels-1 (block ranges up to 2^10 blocks,
// enough for any band of a query of at most kMMax samples)
constexpr int kEnvG = 16;
constexpr int kEnvLevels = 11;
// learned proposal encoder: parameter count and packed-weight blob size
constexpr int kEncParams = 38112;
constexpr int kEncBlobBytes = 1024 + 2 * 3 * 32 * 224 * 2 + 64 * 256 * 2;
constexpr int kEdMax = kKMax + kLearnPropMax * 129 + 64;
constexpr int kTile = 1024;         // windows per lower-bound tile
constexpr int kProxyTile = 4096;    // windows per proxy-scan tile (a multiple of kTile)
constexpr int kStages = 4;          // shared-memory stages of the scan pipeline
constexpr int kBins = 1024;         // survivor ordering bins
constexpr int kDiagRMax = 511;      // widest band of the anti-diagonal DTW kernels (all shapes)
constexpr int kDiagRMaxF32 = 1023;  // widest band of the FP32 anti-diagonal kernels (24, 32 cells per lane)
constexpr uint64_t kEmptyKey = ~0ull;
// Unnormalised DTW: the largest |value| accepted.  Path sums then stay
// below 2^66 * 2 * 8192 = 2^80, far under the 1e30 boundary of the
// double-float walk and the ~4e30 cost of its +-1e15 pads.
constexpr float kRawAbsMax = 4294967296.0f;  // 2^32

// status bits (device word in the handle)
constexpr int kStNonFinite = 1;
constexpr int kStTimeout = 2;
constexpr int kStOverflow = 4;

// per-query counters (QueryState::ctr)
enum Ctr {
    kCtrKim = 0, kCtrKeoghQ = 1, kCtrKeoghS = 2, kCtrDtwStarted = 3,
    kCtrDtwAbandoned = 4, kCtrCells = 5, kCtrRescored = 6, kCtrN = 8
};

// Device-resident state of one query (one per handle; queries of a batch
// reuse it in stream order).
struct QueryState {
    unsigned long long seed_keys[kKMax];   // k smallest seed distances
    unsigned long long res_keys[kListMax]; // smallest survivor distances
    unsigned long long prop_keys[kPropMax];// proxy-scan proposals
    unsigned long long cta_best[2 * kCtaSlots];  // each proposal-scan CTA's best window (two scans)
    unsigned long long ed_keys[kKMax];     // k smallest squared Euclidean distances
                                           // (upper bounds of DTW) of seed windows
    unsigned int ed_off[kEdMax];           // windows whose Euclidean distance is taken
    int n_ed;
    double pre_d64;                        // re-score of the pre-scored window
    int pre_done;
    int margin_skip;                       // margin entries already re-scored
    unsigned int seed_off[kSeedMax];       // offsets whose DTW seeds bsf
    int n_seeds;
    int n_cand;                            // survivors of the lower bounds
    int work;                              // work cursor (seeds, *_at, re-score)
    int work2;                             // work cursor of the survivor DTW
    int n_margin;                          // candidates to re-score in FP64
    unsigned int margin_idx[kListMax];
    double margin_d64[kListMax];
    unsigned long long ctr[kCtrN];
    float thr_scan;                        // threshold the LB scan used
    float e_q[64];                         // learned embedding of the query
    unsigned long long tile_ctr[2];        // dynamic tile cursors: proxy scan, LB scan
    int valid;                             // 0 when the query is non-finite
    int hist[kBins];
    int bin_off[kBins];
    // wide exclusion zone (QueryArgs::xz_z > 0): per bucket parity, the k
    // smallest keys with at most one window per bucket of 2z+1 offsets
    // (each bucket's best found so far), updated under xz_lock[parity]
    unsigned long long xz_keys[2][kKMax];
    int xz_lock[2];
    int xz_count;                          // windows appended to the candidate buffer
    int xz_nsel;                           // of them within the final threshold
    // batch: the survivors went to the persistent stage's pool at pool_off
    int deferred;
    long long pool_off;
    // CTAs of the proxy scan and of the survivor histogram that have
    // finished: the last one of each takes the step that needs all of them
    unsigned int prop_done, bin_done, final_done;
};

// Scalars of one query, passed by value to every kernel.
struct QueryArgs {
    int64_t N;          // windows
    int m, r, k;
    int list_cap;       // result list slots in use (k + margin)
    float delta, alpha; // prune when LB > bsf*(1+delta) + alpha
    float qgrid;        // key grid: a power of two <= alpha/4
    int prescore;       // 1: the best Euclidean seed is scored on a side stream
    int tune_l, tune_k, tune_w;  // survivor DTW shape chosen by the autotuner (0: default)
    int raw;            // 1: unnormalised DTW (the query and the re-scored windows are
                        // taken as they are: mean 0, 1/sigma 1)
    int xz_z;           // > 0: top-k with this exclusion zone, wide form (the
                        // threshold from separated windows, a candidate buffer,
                        // greedy selection at the end); 0: plain top-k
};


// ---------------------------------------------------------------- keys
__device__ __forceinline__ unsigned long long make_key(float d, unsigned int idx) {
    return ((unsigned long long)__float_as_uint(d) << 32) | idx;
}
// Distance as stored in a key: rounded DOWN to a grid coarser than FP32
// noise -- multiples of g below 2048 g, 11 mantissa bits above (the same
// spacing at the seam, so the map is monotone).  Windows whose distances
// differ only by rounding (e.g. bit-identical windows whose statistics came
// from different prefix sums) share a key distance and are ordered by
// offset, as exact ties must be.  Rounding down keeps every threshold built
// from keys within the pruning margin: with delta >= 2^-10 > 2^-11 and
// alpha >= 4 g the bound bsf*(1+delta)+alpha still covers the FP32 error.
__device__ __forceinline__ float key_quantize(float d, float g) {
    if (d < g * 2048.0f) return floorf(d / g) * g;
    return __uint_as_float(__float_as_uint(d) & ~0xfffu);
}
__device__ __forceinline__ float key_dist(unsigned long long key) {
    return key == kEmptyKey ? __int_as_float(0x7f800000) : __uint_as_float((unsigned)(key >> 32));
}
__device__ __forceinline__ unsigned int key_idx(unsigned long long key) {
    return (unsigned)(key & 0xffffffffu);
}

// The window pre-scored on the side stream: the best Euclidean seed.
__device__ __forceinline__ unsigned prescored_window(const QueryState *st, const QueryArgs &a) {
    const unsigned long long k0 = st->ed_keys[0];
    return (a.prescore && k0 != kEmptyKey) ? key_idx(k0) : 0xffffffffu;
}

// Insert a unique key into a sorted list of `cap` slots that holds the cap
// smallest keys offered so far.  Slot j keeps the minimum of what reaches it
// and hands the larger value on to slot j+1; since every atomicMin keeps one
// value and emits one, slot j ends as the (j+1)-th smallest key offered,
// whatever the interleaving.  Slots already below the key are skipped: an
// atomicMin there would return a smaller value and emit the key unchanged.
// A key already in the list (the same window offered twice) stops at the
// slot that holds it, so a window never occupies two slots.
__device__ __forceinline__ void list_insert(unsigned long long *slots, int cap,
                                            unsigned long long key) {
    for (int j = 0; j < cap && key != kEmptyKey; ++j) {
        const unsigned long long cur = *((volatile unsigned long long *)&slots[j]);
        if (cur < key) continue;
        if (cur == key) return;
        const unsigned long long old = atomicMin(&slots[j], key);
        if (old == key) return;
        key = old > key ? old : key;
    }
}

__device__ __forceinline__ float list_kth(const unsigned long long *slots, int k) {
    return key_dist(*((volatile const unsigned long long *)&slots[k - 1]));
}

// Current pruning threshold: bsf*(1+delta)+alpha, bsf = the smallest of the
// k-th seed DTW, the k-th survivor DTW found so far and the k-th squared
// Euclidean distance of the seed windows (+inf while fewer than k exist).
//
// With a wide exclusion zone z (a.xz_z > 0) those lists bound nothing (a
// match's neighbours fill them); the bound is the smaller k-th of the two
// bucket lists instead: buckets of 2z+1 offsets, one window per bucket, so
// the windows of one parity's list are pairwise more than 2z apart, and the
// k-th distance of any k windows pairwise more than 2z apart bounds the
// answer's k-th distance from above (a window the greedy selection takes
// shuts out at most one of them).
__device__ __forceinline__ float current_thr(const QueryState *st, const QueryArgs &a) {
    float b;
    if (a.xz_z > 0) {
        b = fminf(list_kth(st->xz_keys[0], a.k), list_kth(st->xz_keys[1], a.k));
    } else {
        // each list holds distinct windows, so each k-th value bounds the true
        // k-th distance from above
        b = fminf(fminf(list_kth(st->seed_keys, a.k), list_kth(st->res_keys, a.k)),
                  list_kth(st->ed_keys, a.k));
    }
    if (!(b < __int_as_float(0x7f800000))) return __int_as_float(0x7f800000);
    return fmaf(b, 1.0f + a.delta, a.alpha);
}

// ---------------------------------------------------------------- timers
__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

// ---------------------------------------------------------------- mbarrier / bulk copy
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// try_wait with a suspend-time hint: the thread sleeps in hardware until the
// phase completes or about hint_ns pass, instead of polling
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, unsigned parity, unsigned hint_ns) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of the barrier for at most limit_ns; false on
// timeout.  The retries sleep (at most 20 us each), so a waiting warp takes
// almost no issue slots from the warps that have work.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = global_ns();
    while (!mbar_try_wait_sleep(bar, parity, 20000u)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}
// 1-D bulk copy global -> shared through the TMA unit; completes `bytes`
// transaction bytes on the barrier.  dst, src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }

// Append `pass` lanes' values to a shared or global array through one atomic
// per warp.  All lanes of `mask` must call it.
__device__ __forceinline__ int warp_append(int *counter, bool pass, unsigned mask) {
    unsigned bal = __ballot_sync(mask, pass);
    if (bal == 0) return -1;
    int leader = __ffs(bal) - 1;
    int base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(counter, __popc(bal));
    base = __shfl_sync(mask, base, leader);
    unsigned lt = bal & ((1u << lane_id()) - 1u);
    return pass ? base + __popc(lt) : -1;
}

}  // namespace dtws
