// dtws_api.cu -- the C ABI of include/dtws.h: handle lifecycle, argument
// validation, device memory, per-series caches and the order in which a
// query's kernels are enqueued on the caller's stream.
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/dtws.h"
#include "dtws_internal.h"

static_assert(DTWS_M_MAX == dtws::kBlockB, "prefix block length must equal the longest query");
static_assert(DTWS_K_MAX == dtws::kKMax, "k limit mismatch");

using namespace dtws;

namespace {

thread_local char g_err[256];
int g_fail_allocs = 0;  // test hook: the next N device allocations fail

void set_err(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (g_fail_allocs > 0) {
        --g_fail_allocs;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc((void **)p, count * sizeof(T) + 256);
}

int64_t round_up(int64_t v, int64_t q) { return (v + q - 1) / q * q; }

struct StatsEntry {
    int m = 0;
    int64_t used = 0;
    float *mu_hi = nullptr, *mu_lo = nullptr, *inv_sigma = nullptr;
    float *smu_hi = nullptr, *sinv_sigma = nullptr;  // every kProxyStride-th window (proxy scan)
};
struct EnvEntry {
    int r = 0;
    int64_t used = 0;
    float *U = nullptr, *L = nullptr;
};

struct TuneEntry {
    int m = 0, r = 0, L = 0, K = 0, warps = 0;
    float ms_default = 0.f, ms_best = 0.f;
};

struct LearnEntry {
    int m = 0;
    int64_t used = 0, version = 0, rows = 0, rows2 = 0;
    void *E = nullptr;   // BF16 [rows][64]: windows at offsets j*b
    void *E2 = nullptr;  // BF16 [rows2][64]: windows at offsets j*b + b/2 (b >= 2)
    void *Q = nullptr, *Q2 = nullptr;    // their int8 copies for the scan
    float *S = nullptr, *S2 = nullptr;   // per int8 row: scale, squared norm (2 floats)
};

constexpr int kCacheSlots = 8;
constexpr int kLearnSlots = 2;

// One lane of the batched path: its own query buffers, survivor buffers and
// window-statistics slot, and its own streams, so that queries on different
// lanes overlap on the GPU.
struct Lane {
    QueryState *st = nullptr;
    float *qh32 = nullptr, *Uq = nullptr, *Lq = nullptr, *sq = nullptr, *sU = nullptr, *sL = nullptr;
    double *qh64 = nullptr;
    unsigned short *ord = nullptr;
    float *cand_lb = nullptr, *sort_lb = nullptr;
    unsigned *cand_idx = nullptr, *sort_idx = nullptr;
    StatsEntry stats;  // slot sized for the batch's smallest m
    int64_t stats_cap = 0;
    cudaStream_t stream = nullptr, side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_done = nullptr;
};

}  // namespace

void dtws::set_error_detail(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

struct dtws_ctx {
    int device = 0, num_sms = 0;
    int64_t n = 0, n_alloc = 0;
    float *x = nullptr;
    float *x_sub = nullptr;              // x[kProxyStride j] for j < n_alloc/kProxyStride, plus a zero tail
    float *pf = nullptr, *bf = nullptr;  // prefix sums as FP32 pairs, block totals and anchors
    int *pok = nullptr;                  // per-block flag: the pairs carry the block
    float *pscale = nullptr;             // [0]: the series' power-of-two scale; [1]: scratch
    float *envst = nullptr;              // block envelope (sparse table)
    int64_t nblk = 0;
    unsigned *absmax = nullptr;          // max |x| as FP32 bits (device), and its host copy:
    float xabs = 0.0f;
    std::vector<StatsEntry> stats;
    StatsEntry ident;                    // unnormalised DTW: mean 0, 1/sigma 1 for every window
    std::vector<EnvEntry> env;
    int64_t clock = 0;
    QueryState *st = nullptr;
    int *status = nullptr;
    float *qh32 = nullptr, *Uq = nullptr, *Lq = nullptr, *sq = nullptr, *sU = nullptr, *sL = nullptr;
    double *qh64 = nullptr;
    unsigned short *ord = nullptr;
    float *cand_lb = nullptr, *sort_lb = nullptr;
    unsigned *cand_idx = nullptr, *sort_idx = nullptr;
    int64_t cand_cap = 0;
    // staging of host arrays: device side, and pinned host memory for results
    void *stage = nullptr;
    size_t stage_cap = 0;
    void *hstage = nullptr;
    size_t hstage_cap = 0;
    dtws_options opt;
    cudaStream_t last_stream = nullptr;
    QueryState *last_st = nullptr;  // the state the last query's counters are in
    bool have_last = false;
    int64_t last_N = 0;
    int64_t last_launches = 0;
    cudaEvent_t ev[9] = {};
    bool ev_ok = false;
    bool ev_recorded[9] = {false};
    // side stream for work that overlaps the lower-bound scan
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // autotuned survivor-DTW shapes per (m, r)
    std::vector<TuneEntry> tune;
    // batched path
    std::vector<Lane> lanes;
    cudaEvent_t batch_fork = nullptr;
    cudaStream_t cap_stream = nullptr;  // captures a batch (the caller's stream may be the legacy one)
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<int64_t> graph_sig;  // what the cached graph was captured for
    cudaGraphExec_t qgraph_exec = nullptr;  // the same for single queries
    std::vector<int64_t> qgraph_sig;
    int64_t qgraph_launches = 0;
    // learned proposal encoder
    uint8_t *enc_blob = nullptr;
    int64_t enc_version = 0;  // 0: no encoder installed
    std::vector<LearnEntry> learn;
    // batch: per-query states and query buffers, the survivor pool of the
    // persistent stage, its query table and shape lists
    QueryState *bq_st = nullptr;
    int bq_cap = 0;
    float *bq_f = nullptr;           // qh32, Uq, Lq, sq, sU, sL: 6 runs of bq_fcap
    double *bq_d = nullptr;          // qh64
    unsigned short *bq_o = nullptr;  // ord
    int64_t bq_fcap = 0;
    SurvPool pool{};
    long long pool_limit = -1;  // test hook: survivor pool capacity (-1: sized for the batch)
    PoolQuery *pq_dev = nullptr;
    int *plist_dev = nullptr;
    int pq_cap = 0;
    // wide exclusion zone: the candidate buffer and the re-score list
    // (capacities settable for tests with dtws_debug_set_xz_capacity)
    unsigned long long *xz_buf = nullptr;
    unsigned *xz_sel = nullptr;
    double *xz_d64 = nullptr;
    int xz_cap = 1 << 20, xz_sel_cap = 8192;
};

namespace {

#define CK(call)                                                                   \
    do {                                                                           \
        cudaError_t e__ = (call);                                                  \
        if (e__ != cudaSuccess) {                                                  \
            set_err("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e__)); \
            return e__ == cudaErrorMemoryAllocation ? DTWS_ENOMEM : DTWS_ECUDA;    \
        }                                                                          \
    } while (0)

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

dtws_status ensure_stage(dtws_t h, size_t bytes) {
    if (h->stage_cap >= bytes) return DTWS_OK;
    if (h->stage) cudaFree(h->stage);
    h->stage = nullptr;
    h->stage_cap = 0;
    size_t cap = bytes < 4096 ? 4096 : bytes;
    void *p = nullptr;
    if (g_fail_allocs > 0) {
        --g_fail_allocs;
        return DTWS_ENOMEM;
    }
    CK(cudaMalloc(&p, cap));
    h->stage = p;
    h->stage_cap = cap;
    return DTWS_OK;
}

// Host-bound results: one copy of the device region that holds them (in the
// stage: offsets, then distances) into the pinned host stage, one wait, then
// plain copies into the caller's arrays.  (Copies into pageable memory are
// staged by the driver and wait on their own, once per array.)
dtws_status read_back(dtws_t h, cudaStream_t s, const int64_t *idx_d, const float *dist_d, int64_t *out_idx,
                      float *out_dist, size_t ib, size_t db, bool idev, bool ddev) {
    if (idev && ddev) return DTWS_OK;
    const char *lo = !idev ? (const char *)idx_d : (const char *)dist_d;
    const char *hi = !ddev ? (const char *)dist_d + db : (const char *)idx_d + ib;
    const size_t span = (size_t)(hi - lo);
    if (h->hstage_cap < span) {
        if (h->hstage) cudaFreeHost(h->hstage);
        h->hstage = nullptr;
        h->hstage_cap = 0;
        const size_t cap = span < 4096 ? 4096 : span;
        if (g_fail_allocs > 0) {
            --g_fail_allocs;
            return DTWS_ENOMEM;
        }
        CK(cudaMallocHost(&h->hstage, cap));
        h->hstage_cap = cap;
    }
    CK(cudaMemcpyAsync(h->hstage, lo, span, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const char *hs = (const char *)h->hstage;
    if (!idev) memcpy(out_idx, hs + ((const char *)idx_d - lo), ib);
    if (!ddev) memcpy(out_dist, hs + ((const char *)dist_d - lo), db);
    return DTWS_OK;
}

void free_stats(StatsEntry &e) {
    cudaFree(e.mu_hi);
    cudaFree(e.mu_lo);
    cudaFree(e.inv_sigma);
    cudaFree(e.smu_hi);
    cudaFree(e.sinv_sigma);
    e = StatsEntry();
}
void free_env(EnvEntry &e) {
    cudaFree(e.U);
    cudaFree(e.L);
    e = EnvEntry();
}

dtws_status get_stats(dtws_t h, int m, cudaStream_t s, StatsEntry **out, bool *computed) {
    *computed = false;
    for (auto &e : h->stats)
        if (e.m == m) {
            e.used = ++h->clock;
            *out = &e;
            return DTWS_OK;
        }
    if ((int)h->stats.size() >= kCacheSlots) {
        size_t lru = 0;
        for (size_t i = 1; i < h->stats.size(); ++i)
            if (h->stats[i].used < h->stats[lru].used) lru = i;
        CK(cudaDeviceSynchronize());  // no queued kernel may still read it
        free_stats(h->stats[lru]);
        h->stats.erase(h->stats.begin() + lru);
    }
    StatsEntry e;
    e.m = m;
    const int64_t N = h->n - m + 1;
    const int64_t cap = round_up(N, kProxyTile) + kProxyTile;
    const int64_t scap = cap / kProxyStride;
    cudaError_t a1 = dalloc(&e.mu_hi, cap), a2 = dalloc(&e.mu_lo, cap), a3 = dalloc(&e.inv_sigma, cap);
    cudaError_t a4 = dalloc(&e.smu_hi, scap), a6 = dalloc(&e.sinv_sigma, scap);
    if (a1 != cudaSuccess || a2 != cudaSuccess || a3 != cudaSuccess || a4 != cudaSuccess ||
        a6 != cudaSuccess) {
        free_stats(e);
        cudaGetLastError();
        set_err("window statistics for m=%d: out of device memory", m);
        return DTWS_ENOMEM;
    }
    cudaError_t ce = cudaMemsetAsync(e.mu_hi, 0, cap * 4, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e.mu_lo, 0, cap * 4, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e.inv_sigma, 0, cap * 4, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e.smu_hi, 0, scap * 4, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e.sinv_sigma, 0, scap * 4, s);
    if (ce == cudaSuccess)
        ce = launch_window_stats(h->x, h->n, m, h->pf, h->bf, h->pok, h->pscale, e.mu_hi, e.mu_lo, e.inv_sigma,
                                 e.smu_hi, e.sinv_sigma, h->num_sms, s);
    if (ce != cudaSuccess) {  // nothing half-initialised stays in the cache
        free_stats(e);
        cudaGetLastError();
        set_err("window statistics for m=%d: %s", m, cudaGetErrorString(ce));
        return DTWS_ECUDA;
    }
    e.used = ++h->clock;
    h->stats.push_back(e);
    *out = &h->stats.back();
    *computed = true;
    return DTWS_OK;
}

// Unnormalised DTW: statistics arrays with mean 0 and 1/sigma 1 for every
// window, so every kernel's (x - mu) * (1/sigma) is x itself, exactly.  One
// entry sized for m = 2 (the most windows) serves every m.
dtws_status get_ident(dtws_t h, cudaStream_t s, StatsEntry **out, bool *computed) {
    *computed = false;
    if (!h->ident.mu_hi) {
        StatsEntry e;
        const int64_t N = h->n - 1;
        const int64_t cap = round_up(N, kProxyTile) + kProxyTile;
        const int64_t scap = cap / kProxyStride;
        cudaError_t a1 = dalloc(&e.mu_hi, cap), a2 = dalloc(&e.mu_lo, cap), a3 = dalloc(&e.inv_sigma, cap);
        cudaError_t a4 = dalloc(&e.smu_hi, scap), a6 = dalloc(&e.sinv_sigma, scap);
        if (a1 != cudaSuccess || a2 != cudaSuccess || a3 != cudaSuccess || a4 != cudaSuccess ||
            a6 != cudaSuccess) {
            free_stats(e);
            cudaGetLastError();
            set_err("unnormalised statistics: out of device memory");
            return DTWS_ENOMEM;
        }
        cudaError_t ce = cudaMemsetAsync(e.mu_hi, 0, cap * 4, s);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(e.mu_lo, 0, cap * 4, s);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(e.smu_hi, 0, scap * 4, s);
        if (ce == cudaSuccess) ce = launch_fill(e.inv_sigma, cap, 1.0f, h->num_sms, s);
        if (ce == cudaSuccess) ce = launch_fill(e.sinv_sigma, scap, 1.0f, h->num_sms, s);
        if (ce != cudaSuccess) {
            free_stats(e);
            cudaGetLastError();
            set_err("unnormalised statistics: %s", cudaGetErrorString(ce));
            return DTWS_ECUDA;
        }
        h->ident = e;
        *computed = true;
    }
    *out = &h->ident;
    return DTWS_OK;
}

// The statistics a query reads: the window statistics for m, or the
// identity ones for unnormalised DTW.
dtws_status query_stats(dtws_t h, int m, cudaStream_t s, StatsEntry **out, bool *computed) {
    return h->opt.unnormalised ? get_ident(h, s, out, computed) : get_stats(h, m, s, out, computed);
}

dtws_status get_env(dtws_t h, int r, cudaStream_t s, EnvEntry **out, bool *computed) {
    *computed = false;
    for (auto &e : h->env)
        if (e.r == r) {
            e.used = ++h->clock;
            *out = &e;
            return DTWS_OK;
        }
    if ((int)h->env.size() >= kCacheSlots) {
        size_t lru = 0;
        for (size_t i = 1; i < h->env.size(); ++i)
            if (h->env[i].used < h->env[lru].used) lru = i;
        CK(cudaDeviceSynchronize());  // no queued kernel may still read it
        free_env(h->env[lru]);
        h->env.erase(h->env.begin() + lru);
    }
    EnvEntry e;
    e.r = r;
    cudaError_t a1 = dalloc(&e.U, h->n_alloc), a2 = dalloc(&e.L, h->n_alloc);
    if (a1 != cudaSuccess || a2 != cudaSuccess) {
        free_env(e);
        cudaGetLastError();
        set_err("series envelope for r=%d: out of device memory", r);
        return DTWS_ENOMEM;
    }
    cudaError_t ce = cudaMemsetAsync(e.U, 0, h->n_alloc * 4, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e.L, 0, h->n_alloc * 4, s);
    if (ce == cudaSuccess) ce = launch_envelope(h->x, h->n, r, e.U, e.L, s);
    if (ce != cudaSuccess) {
        free_env(e);
        cudaGetLastError();
        set_err("series envelope for r=%d: %s", r, cudaGetErrorString(ce));
        return DTWS_ECUDA;
    }
    e.used = ++h->clock;
    h->env.push_back(e);
    *out = &h->env.back();
    *computed = true;
    return DTWS_OK;
}

// Allocate whatever is still missing, so a call that failed half way (out
// of memory) leaves a handle that the next call completes or destroy frees.
template <typename T>
cudaError_t need(T **p, size_t count) {
    return *p ? cudaSuccess : dalloc(p, count);
}

void free_learn(LearnEntry &e) {
    for (void *p : {e.E, e.E2, e.Q, e.Q2, (void *)e.S, (void *)e.S2})
        if (p) cudaFree(p);
    e = LearnEntry();
}

int enc_block(int m) { return m / 64; }
int64_t enc_rows(dtws_t h, int m) { return (h->n - m) / enc_block(m) + 1; }
// the second embedding phase: windows at offsets j*b + b/2, so that every
// window lies within b/4 of an embedded one (0: no second phase, b = 1)
int enc_phase(int m) { return enc_block(m) / 2; }
int64_t enc_rows2(dtws_t h, int m) {
    const int ph = enc_phase(m);
    return ph > 0 && h->n - m >= ph ? (h->n - m - ph) / enc_block(m) + 1 : 0;
}
// Euclidean seeds around each learned proposal: +- half its grid gap
int learn_half(int m) {
    const int b = enc_block(m);
    return enc_phase(m) > 0 ? (b + 3) / 4 : b / 2;
}

// Embeddings of the windows at offsets j*b for query length m (cached).
dtws_status get_learn(dtws_t h, int m, const StatsEntry *se, cudaStream_t s, LearnEntry **out, bool *computed) {
    *computed = false;
    for (auto &e : h->learn)
        if (e.m == m && e.version == h->enc_version) {
            e.used = ++h->clock;
            *out = &e;
            return DTWS_OK;
        }
    for (size_t i = 0; i < h->learn.size();)
        if (h->learn[i].version != h->enc_version) {
            CK(cudaDeviceSynchronize());
            free_learn(h->learn[i]);
            h->learn.erase(h->learn.begin() + i);
        } else {
            ++i;
        }
    if ((int)h->learn.size() >= kLearnSlots) {
        size_t lru = 0;
        for (size_t i = 1; i < h->learn.size(); ++i)
            if (h->learn[i].used < h->learn[lru].used) lru = i;
        CK(cudaDeviceSynchronize());
        free_learn(h->learn[lru]);
        h->learn.erase(h->learn.begin() + lru);
    }
    LearnEntry e;
    e.m = m;
    e.version = h->enc_version;
    e.rows = enc_rows(h, m);
    e.rows2 = enc_rows2(h, m);
    uint16_t *E = nullptr, *E2 = nullptr;
    int8_t *Q = nullptr, *Q2 = nullptr;
    float *S = nullptr, *S2 = nullptr;
    bool ok = dalloc(&E, (size_t)e.rows * 64) == cudaSuccess && dalloc(&Q, (size_t)e.rows * 64) == cudaSuccess &&
              dalloc(&S, (size_t)e.rows * 2) == cudaSuccess;
    if (ok && e.rows2 > 0)
        ok = dalloc(&E2, (size_t)e.rows2 * 64) == cudaSuccess && dalloc(&Q2, (size_t)e.rows2 * 64) == cudaSuccess &&
             dalloc(&S2, (size_t)e.rows2 * 2) == cudaSuccess;
    e.E = E;
    e.E2 = E2;
    e.Q = Q;
    e.Q2 = Q2;
    e.S = S;
    e.S2 = S2;
    if (!ok) {
        cudaGetLastError();
        free_learn(e);
        set_err("learned embeddings for m=%d: out of device memory", m);
        return DTWS_ENOMEM;
    }
    cudaError_t ce = launch_enc_series(h->enc_blob, h->x, h->n, enc_block(m), se->inv_sigma, e.rows, e.E,
                                       h->num_sms, s);
    if (ce == cudaSuccess) ce = launch_enc_quant(e.E, e.rows, e.Q, e.S, s);
    if (ce == cudaSuccess && e.rows2 > 0) {  // the same pass over the series shifted by the phase
        const int ph = enc_phase(m);
        ce = launch_enc_series(h->enc_blob, h->x + ph, h->n - ph, enc_block(m), se->inv_sigma + ph, e.rows2, e.E2,
                               h->num_sms, s);
        if (ce == cudaSuccess) ce = launch_enc_quant(e.E2, e.rows2, e.Q2, e.S2, s);
    }
    if (ce != cudaSuccess) {
        free_learn(e);
        cudaGetLastError();
        set_err("learned embeddings for m=%d: %s", m, cudaGetErrorString(ce));
        return DTWS_ECUDA;
    }
    e.used = ++h->clock;
    h->learn.push_back(e);
    *out = &h->learn.back();
    *computed = true;
    return DTWS_OK;
}

dtws_status ensure_workspace(dtws_t h) {
    CK(need(&h->st, 1));
    CK(need(&h->qh32, kMMax));
    CK(need(&h->Uq, kMMax));
    CK(need(&h->Lq, kMMax));
    CK(need(&h->sq, kMMax));
    CK(need(&h->sU, kMMax));
    CK(need(&h->sL, kMMax));
    CK(need(&h->qh64, kMMax));
    CK(need(&h->ord, kMMax));
    return DTWS_OK;
}

dtws_status ensure_candidates(dtws_t h) {
    const int64_t cap = h->n;  // at most N <= n survivors
    CK(need(&h->cand_lb, cap));
    CK(need(&h->sort_lb, cap));
    CK(need(&h->cand_idx, cap));
    CK(need(&h->sort_idx, cap));
    h->cand_cap = cap;
    return DTWS_OK;
}

QueryBufs make_bufs(dtws_t h, const StatsEntry *se, const EnvEntry *ee) {
    QueryBufs b;
    memset(&b, 0, sizeof b);  // padding included: the bytes enter graph signatures
    b.st = h->st;
    b.x = h->x;
    b.x_sub = h->x_sub;
    b.mu_hi = se ? se->mu_hi : nullptr;
    b.mu_lo = se ? se->mu_lo : nullptr;
    b.inv_sigma = se ? se->inv_sigma : nullptr;
    b.smu_hi = se ? se->smu_hi : nullptr;
    b.sinv_sigma = se ? se->sinv_sigma : nullptr;
    b.U = ee ? ee->U : nullptr;
    b.L = ee ? ee->L : nullptr;
    b.stmax = h->envst;
    b.stmin = h->envst + (size_t)kEnvLevels * h->nblk;
    b.nblk = h->nblk;
    b.n = h->n;
    b.qh32 = h->qh32;
    b.qh64 = h->qh64;
    b.Uq = h->Uq;
    b.Lq = h->Lq;
    b.ord = h->ord;
    b.sq = h->sq;
    b.sU = h->sU;
    b.sL = h->sL;
    b.cand_lb = h->cand_lb;
    b.sort_lb = h->sort_lb;
    b.cand_idx = h->cand_idx;
    b.sort_idx = h->sort_idx;
    b.status = h->status;
    b.wait_ns = h->opt.wait_limit_ns;
    b.num_sms = h->num_sms;
    b.xz_buf = h->xz_buf;
    b.xz_sel = h->xz_sel;
    b.xz_d64 = h->xz_d64;
    b.xz_cap = h->xz_cap;
    b.xz_sel_cap = h->xz_sel_cap;
    return b;
}

// The wide exclusion zone's device buffers.
dtws_status ensure_xz(dtws_t h) {
    if (!h->xz_buf) {
        CK(dalloc(&h->xz_buf, (size_t)h->xz_cap));
        CK(dalloc(&h->xz_sel, (size_t)h->xz_sel_cap));
        CK(dalloc(&h->xz_d64, (size_t)h->xz_sel_cap));
    }
    return DTWS_OK;
}

QueryArgs make_args(dtws_t h, int m, int r, int k, bool raw) {
    QueryArgs a;
    memset(&a, 0, sizeof a);  // padding included: the bytes enter graph signatures
    a.N = h->n - m + 1;
    a.m = m;
    a.r = r > m - 1 ? m - 1 : r;
    a.k = k;
    a.list_cap = k + 64 < kListMax ? k + 64 : kListMax;
    a.delta = h->opt.delta;
    a.alpha = h->opt.alpha_per_m * (float)m;
    // Raw values (unnormalised DTW) enter the differences unscaled, so every
    // FP32 error is relative to its term and delta covers it; alpha keeps
    // its meaning, in squared units of the data.
    a.raw = raw ? 1 : 0;
    // largest power of two <= alpha/4 (alpha 0: FP32's smallest normal)
    float g = 1.17549435e-38f;
    while (g * 2.0f <= a.alpha * 0.25f) g *= 2.0f;
    a.qgrid = g;
    a.prescore = a.r <= kDiagRMaxF32 ? 1 : 0;
    a.tune_l = a.tune_k = a.tune_w = 0;
    for (const auto &t : h->tune)
        if (t.m == m && t.r == a.r) {
            a.tune_l = t.L;
            a.tune_k = t.K;
            a.tune_w = t.warps;
        }
    return a;
}
QueryArgs make_args(dtws_t h, int m, int r, int k) { return make_args(h, m, r, k, h->opt.unnormalised != 0); }

dtws_status check_query_args(dtws_t h, const float *Q, int32_t m, int32_t r, int32_t k) {
    if (!h || !Q) { set_err("null handle or query"); return DTWS_EINVAL; }
    if (m < 2 || m > DTWS_M_MAX || (int64_t)m > h->n) {
        set_err("m=%d out of range [2, min(n, %d)]", m, DTWS_M_MAX);
        return DTWS_EINVAL;
    }
    if (r < 0) { set_err("r=%d < 0", r); return DTWS_EINVAL; }
    const int64_t N = h->n - m + 1;
    if (k < 1 || k > DTWS_K_MAX || (int64_t)k > N) {
        set_err("k=%d out of range [1, min(N, %d)]", k, DTWS_K_MAX);
        return DTWS_EINVAL;
    }
    if (h->opt.unnormalised) {
        if (h->opt.ordering == DTWS_ORDER_LEARNED) {
            set_err("unnormalised DTW with the learned ordering (its embeddings are of normalised windows)");
            return DTWS_EINVAL;
        }
        if (!(h->xabs <= kRawAbsMax)) {
            set_err("unnormalised DTW needs |x| <= 2^32 (the series reaches %g)", (double)h->xabs);
            return DTWS_EINVAL;
        }
    }
    if (h->opt.ordering == DTWS_ORDER_LEARNED) {
        if (!h->enc_version) { set_err("learned ordering without an encoder (dtws_set_encoder)"); return DTWS_EINVAL; }
        if (m < 64) { set_err("learned ordering needs m >= 64 (m=%d)", m); return DTWS_EINVAL; }
        const int P = h->opt.seed_proposals, half = learn_half(m);
        if (P > kLearnPropMax || h->opt.seed_random + P * (2 * half + 1) > kEdMax) {
            set_err("learned ordering: %d proposals exceed the seed capacity", P);
            return DTWS_EINVAL;
        }
    }
    return DTWS_OK;
}

// Append the bytes of a trivially copyable value to a signature.
template <typename T>
void sig_push(std::vector<int64_t> &sig, const T &v) {
    int64_t w[(sizeof(T) + 7) / 8] = {};
    memcpy(w, &v, sizeof(T));
    sig.insert(sig.end(), w, w + (sizeof(T) + 7) / 8);
}

void record(dtws_t h, int i, cudaStream_t s) {
    if (h->opt.timing && h->ev_ok) {
        cudaEventRecord(h->ev[i], s);
        h->ev_recorded[i] = true;
    }
}

// Everything a query's kernels need besides the query itself.
struct Exec {
    QueryBufs b;
    cudaStream_t s, side;
    cudaEvent_t ev_fork, ev_join;
    const LearnEntry *le;  // learned ordering: the embeddings for m (or null)
    bool timing;           // record the handle's phase events
    // batch stages: 0 the whole query; 1 up to the survivor pass (its
    // survivors handed to the pool when `pool` is set); 2 the final stage
    int stage = 0;
    const SurvPool *pool = nullptr;
};

// Enqueue the kernels of one query (Sec. 2.2's cascade, re-planned for the
// GPU) on e.s; returns the number of kernel launches.
dtws_status enqueue_search(dtws_t h, const Exec &e, const QueryArgs &a, const float *Qd, int64_t *idx_d,
                           float *dist_d, int64_t *launches_out) {
    const QueryBufs &b = e.b;
    cudaStream_t s = e.s;
    const int m = a.m, k = a.k;
    if (e.stage == 2) {  // the final stage of a batch query (after the persistent stage)
        int nf = 0;
        CK(launch_finalize(b, a, idx_d, dist_d, s, &nf));
        *launches_out = nf;
        return DTWS_OK;
    }
    // a wide exclusion zone needs k seeds in separate buckets of each parity
    // for a first threshold: all the proposals the list holds
    const int P = (a.xz_z > 0 && h->opt.seed_proposals > 0) ? kPropMax : h->opt.seed_proposals;
    const int R = h->opt.seed_random;
    int64_t launches = 0;
    auto rec = [&](int i) {
        if (e.timing) record(h, i, s);
    };
    CK(launch_qprep(Qd, b, a, s));  // (clears the query's state first)
    rec(0);
    int half = kProxyHalf;
    if (P > 0 && e.le) {
        int c0 = 0, c1 = 0;
        CK(launch_enc_query(h->enc_blob, b, a, s));
        CK(launch_learn_scan(b, e.le->Q, e.le->S, e.le->rows, enc_block(m), 0, 0, &c0, s));
        if (e.le->rows2 > 0) {
            CK(launch_learn_scan(b, e.le->Q2, e.le->S2, e.le->rows2, enc_block(m), enc_phase(m), 1, &c1, s));
            ++launches;
        }
        CK(launch_prop_merge(b, c0, c1, P, s));
        half = learn_half(m);
        launches += 3;
    }
    if (P > 0 && !e.le) {  // (the proxy scan merges its proposals and gathers the seeds itself)
        int c0 = 0;
        CK(launch_seed_scan(b, a, P, h->opt.proxy_terms, R, half, h->opt.rng_seed, &c0, s));
        ++launches;
    } else {
        CK(launch_seed_gather(b, a, R, P, half, h->opt.rng_seed, s));
        ++launches;
    }
    CK(launch_seed_ed(b, a, R + P * (2 * half + 1), s));
    if (k > 1 && a.xz_z == 0) {  // exact DTW seeds tighten a k-th bound the Euclidean seeds leave loose
        // (the neighbours of one match, which is all these seeds are, bound
        // nothing with an exclusion zone)
        CK(launch_seed_expand(b, a, s));
        CK(launch_dtw_seeds(b, a, s));
        launches += 2;
    }
    rec(1);
    // the best Euclidean seed is scored on the side stream during the scan
    if (a.prescore) {
        CK(cudaEventRecord(e.ev_fork, s));
        CK(cudaStreamWaitEvent(e.side, e.ev_fork, 0));
        CK(launch_prescore(b, a, e.side));
        CK(cudaEventRecord(e.ev_join, e.side));
        ++launches;
    }
    CK(launch_lb_scan(b, a, s));
    rec(2);
    CK(launch_order(b, a, s));
    rec(3);
    if (e.pool) {  // batch: the survivors go to the persistent stage (unless the pool is full)
        CK(launch_defer(b, *e.pool, s));
        launches += 2;
    }
    CK(launch_dtw_survivors(b, a, s));
    rec(4);
    if (a.prescore) CK(cudaStreamWaitEvent(s, e.ev_join, 0));
    if (e.stage == 1) {
        launches += 1 + 1 + 1 + 2 + 1;  // qprep, ED seeds, scan, order x2, DTW
        *launches_out = launches;
        return DTWS_OK;
    }
    int nf = 3;
    if (a.xz_z > 0) CK(launch_xz_finalize(b, a, idx_d, dist_d, s));
    else CK(launch_finalize(b, a, idx_d, dist_d, s, &nf));
    rec(5);
    launches += 1 + 1 + 1 + 2 + 1 + nf;  // qprep, ED seeds, scan, order x2, DTW, final
    *launches_out = launches;
    return DTWS_OK;
}

// One query on the handle's own buffers (dtws_query).
dtws_status run_query(dtws_t h, const float *Qd, int m, int r, int k, int64_t *idx_d, float *dist_d,
                      cudaStream_t s, int xz_z = 0) {
    dtws_status st;
    for (bool &v : h->ev_recorded) v = false;
    record(h, 8, s);
    StatsEntry *se;
    EnvEntry *ee = nullptr;
    bool c1, c2 = false;
    if ((st = query_stats(h, m, s, &se, &c1)) != DTWS_OK) return st;
    record(h, 6, s);
    const int rr = r > m - 1 ? m - 1 : r;
    if (h->opt.exact_envelope) {
        if ((st = get_env(h, rr, s, &ee, &c2)) != DTWS_OK) return st;
    } else {  // an exact envelope already cached for this r is still used
        for (auto &en : h->env)
            if (en.r == rr) ee = &en;
    }
    record(h, 7, s);
    if ((st = ensure_workspace(h)) != DTWS_OK) return st;
    if ((st = ensure_candidates(h)) != DTWS_OK) return st;
    LearnEntry *le = nullptr;
    bool c3 = false;
    if (h->opt.seed_proposals > 0 && h->opt.ordering == DTWS_ORDER_LEARNED)
        if ((st = get_learn(h, m, se, s, &le, &c3)) != DTWS_OK) return st;
    if (xz_z > 0 && (st = ensure_xz(h)) != DTWS_OK) return st;
    Exec e{make_bufs(h, se, ee), s, h->side, h->ev_fork, h->ev_join, le, true};
    QueryArgs a = make_args(h, m, r, k);
    a.xz_z = xz_z;
    int64_t launches = 0;
    // Repeated queries with the same arguments replay one CUDA graph of the
    // search (the caches above are resolved first, on the caller's stream;
    // no phase events are recorded in a graph).  The signature holds every
    // value the captured kernels' arguments depend on.
    const bool graph = h->opt.batch_graph && !h->opt.timing;
    std::vector<int64_t> sig;
    if (graph) {
        sig = {(int64_t)(intptr_t)Qd, (int64_t)(intptr_t)idx_d, (int64_t)(intptr_t)dist_d,
               (int64_t)(intptr_t)le, le ? le->version : 0};
        sig_push(sig, h->opt);
        sig_push(sig, e.b);
        sig_push(sig, a);
        if (h->qgraph_exec && sig == h->qgraph_sig) {
            CK(cudaGraphLaunch(h->qgraph_exec, s));
            launches = h->qgraph_launches;
        } else {
            if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
            if (!h->batch_fork) CK(cudaEventCreateWithFlags(&h->batch_fork, cudaEventDisableTiming));
            // the capture stream starts after the caller's stream (the caches'
            // kernels); the graph itself is launched on the caller's stream
            CK(cudaEventRecord(h->batch_fork, s));
            CK(cudaStreamWaitEvent(h->cap_stream, h->batch_fork, 0));
            CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
            Exec ec = e;
            ec.s = h->cap_stream;
            st = enqueue_search(h, ec, a, Qd, idx_d, dist_d, &launches);
            cudaGraph_t g = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
            if (st != DTWS_OK || ce != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                if (st != DTWS_OK) return st;
                set_err("query graph capture: %s", cudaGetErrorString(ce));
                return DTWS_ECUDA;
            }
            if (h->qgraph_exec) cudaGraphExecDestroy(h->qgraph_exec);
            h->qgraph_exec = nullptr;
            h->qgraph_sig.clear();
            cudaGraphExec_t ex = nullptr;
            const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            CK(ie);
            h->qgraph_exec = ex;
            h->qgraph_sig = sig;
            h->qgraph_launches = launches;
            CK(cudaGraphLaunch(ex, s));
        }
    } else if ((st = enqueue_search(h, e, a, Qd, idx_d, dist_d, &launches)) != DTWS_OK) {
        return st;
    }
    h->last_stream = s;
    h->have_last = true;
    h->last_N = a.N;
    h->last_launches = launches + (c1 ? 1 : 0) + (c2 ? 1 : 0) + (c3 ? 1 : 0);
    h->last_st = h->st;
    return DTWS_OK;
}

void free_lane(Lane &l) {
    void *ptrs[] = {l.st, l.qh32, l.Uq, l.Lq, l.sq, l.sU, l.sL, l.qh64, l.ord, l.cand_lb, l.sort_lb, l.cand_idx,
                    l.sort_idx};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    free_stats(l.stats);
    if (l.stream) cudaStreamDestroy(l.stream);
    if (l.side) cudaStreamDestroy(l.side);
    if (l.ev_fork) cudaEventDestroy(l.ev_fork);
    if (l.ev_join) cudaEventDestroy(l.ev_join);
    if (l.ev_done) cudaEventDestroy(l.ev_done);
    l = Lane();
}

void drop_graph(dtws_t h) {
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
    h->graph_sig.clear();
    if (h->qgraph_exec) cudaGraphExecDestroy(h->qgraph_exec);
    h->qgraph_exec = nullptr;
    h->qgraph_sig.clear();
}


// Lanes with statistics slots for windows of at least m_min samples.
dtws_status ensure_lanes(dtws_t h, int count, int m_min) {
    const int64_t need_cap = round_up(h->n - m_min + 1, kProxyTile) + kProxyTile;
    for (auto &l : h->lanes)
        if (l.stats_cap < need_cap) {  // too small: rebuild all (rare)
            CK(cudaDeviceSynchronize());
            drop_graph(h);
            for (auto &x : h->lanes) free_lane(x);
            h->lanes.clear();
            break;
        }
    if (!h->batch_fork) CK(cudaEventCreateWithFlags(&h->batch_fork, cudaEventDisableTiming));
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    while ((int)h->lanes.size() < count) {
        h->lanes.emplace_back();
        Lane &l = h->lanes.back();
        const int64_t cap = h->n, scap = need_cap / kProxyStride;
        cudaError_t e = cudaSuccess;
        auto al = [&](cudaError_t r) {
            if (e == cudaSuccess) e = r;
        };
        al(dalloc(&l.st, 1));
        al(dalloc(&l.qh32, kMMax));
        al(dalloc(&l.Uq, kMMax));
        al(dalloc(&l.Lq, kMMax));
        al(dalloc(&l.sq, kMMax));
        al(dalloc(&l.sU, kMMax));
        al(dalloc(&l.sL, kMMax));
        al(dalloc(&l.qh64, kMMax));
        al(dalloc(&l.ord, kMMax));
        al(dalloc(&l.cand_lb, cap));
        al(dalloc(&l.sort_lb, cap));
        al(dalloc(&l.cand_idx, cap));
        al(dalloc(&l.sort_idx, cap));
        al(dalloc(&l.stats.mu_hi, need_cap));
        al(dalloc(&l.stats.mu_lo, need_cap));
        al(dalloc(&l.stats.inv_sigma, need_cap));
        al(dalloc(&l.stats.smu_hi, scap));
        al(dalloc(&l.stats.sinv_sigma, scap));
        al(cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking));
        al(cudaStreamCreateWithFlags(&l.side, cudaStreamNonBlocking));
        al(cudaEventCreateWithFlags(&l.ev_fork, cudaEventDisableTiming));
        al(cudaEventCreateWithFlags(&l.ev_join, cudaEventDisableTiming));
        al(cudaEventCreateWithFlags(&l.ev_done, cudaEventDisableTiming));
        l.stats_cap = need_cap;
        if (e != cudaSuccess) {
            free_lane(l);
            h->lanes.pop_back();
            cudaGetLastError();
            if (h->lanes.empty()) {
                set_err("batch lanes: %s", cudaGetErrorString(e));
                return e == cudaErrorMemoryAllocation ? DTWS_ENOMEM : DTWS_ECUDA;
            }
            break;  // fewer lanes than asked: use what fits
        }
        // statistics slots must hold finite values beyond N (bulk copies read whole tiles)
        CK(cudaMemset(l.stats.mu_hi, 0, need_cap * 4));
        CK(cudaMemset(l.stats.mu_lo, 0, need_cap * 4));
        CK(cudaMemset(l.stats.inv_sigma, 0, need_cap * 4));
        CK(cudaMemset(l.stats.smu_hi, 0, scap * 4));
        CK(cudaMemset(l.stats.sinv_sigma, 0, scap * 4));
    }
    return DTWS_OK;
}

QueryBufs lane_bufs(dtws_t h, const Lane &l, const EnvEntry *ee) {
    QueryBufs b = make_bufs(h, &l.stats, ee);
    b.st = l.st;
    b.qh32 = l.qh32;
    b.qh64 = l.qh64;
    b.Uq = l.Uq;
    b.Lq = l.Lq;
    b.ord = l.ord;
    b.sq = l.sq;
    b.sU = l.sU;
    b.sL = l.sL;
    b.cand_lb = l.cand_lb;
    b.sort_lb = l.sort_lb;
    b.cand_idx = l.cand_idx;
    b.sort_idx = l.sort_idx;
    return b;
}

// Per-query device state of a batch of nq queries with sum_m samples in all,
// and the survivor pool of the persistent stage (pool_cap survivors).
dtws_status ensure_batch(dtws_t h, int nq, int64_t sum_m, long long pool_cap) {
    if (h->bq_cap < nq) {
        if (h->bq_st) {
            CK(cudaDeviceSynchronize());
            drop_graph(h);
            cudaFree(h->bq_st);
            cudaFree(h->pq_dev);
            cudaFree(h->plist_dev);
            h->bq_st = nullptr;
            h->pq_dev = nullptr;
            h->plist_dev = nullptr;
            h->bq_cap = h->pq_cap = 0;
        }
        CK(dalloc(&h->bq_st, (size_t)nq));
        CK(dalloc(&h->pq_dev, (size_t)nq));
        CK(dalloc(&h->plist_dev, (size_t)nq));
        h->bq_cap = h->pq_cap = nq;
    }
    if (h->bq_fcap < sum_m) {
        if (h->bq_f) {
            CK(cudaDeviceSynchronize());
            drop_graph(h);
            cudaFree(h->bq_f);
            cudaFree(h->bq_d);
            cudaFree(h->bq_o);
            h->bq_f = nullptr;
            h->bq_d = nullptr;
            h->bq_o = nullptr;
            h->bq_fcap = 0;
        }
        CK(dalloc(&h->bq_f, (size_t)sum_m * 6));
        CK(dalloc(&h->bq_d, (size_t)sum_m));
        CK(dalloc(&h->bq_o, (size_t)sum_m));
        h->bq_fcap = sum_m;
    }
    if (h->pool.cap != pool_cap && (h->pool.cap < pool_cap || h->pool_limit >= 0)) {
        if (h->pool.idx || h->pool.cap) {
            CK(cudaDeviceSynchronize());
            drop_graph(h);
            void *ptrs[] = {h->pool.idx, h->pool.lb, h->pool.mh, h->pool.is, h->pool.ls, h->pool.cursor};
            for (void *p : ptrs) cudaFree(p);
            h->pool = SurvPool{};
        }
        if (pool_cap <= 0) return DTWS_OK;  // no pool: every query keeps its survivors
        SurvPool p{};
        cudaError_t e = cudaSuccess;
        auto al = [&](cudaError_t r) {
            if (e == cudaSuccess) e = r;
        };
        al(dalloc(&p.idx, (size_t)pool_cap));
        al(dalloc(&p.lb, (size_t)pool_cap));
        al(dalloc(&p.mh, (size_t)pool_cap));
        al(dalloc(&p.is, (size_t)pool_cap));
        al(dalloc(&p.ls, (size_t)pool_cap));
        al(dalloc(&p.cursor, 1));
        if (e != cudaSuccess) {
            void *ptrs[] = {p.idx, p.lb, p.mh, p.is, p.ls, p.cursor};
            for (void *q : ptrs)
                if (q) cudaFree(q);
            cudaGetLastError();
            return DTWS_OK;  // no pool: every query keeps its survivors (h->pool.cap stays 0)
        }
        p.cap = pool_cap;
        h->pool = p;
    }
    return DTWS_OK;
}

// Many queries (dtws_query_batch): queries sorted by (m, r) and dealt
// round-robin to the lanes; each lane computes the window statistics of a
// new m into its slot, in stream order, and uses the exact envelope of r
// when one is cached, else the block envelope.  Three stages:
//   1. per query, on its lane: query preparation, seeding, the lower-bound
//      scan and the survivor ordering, then the survivors and their window
//      statistics go to the batch's survivor pool (a query whose survivors do
//      not fit, or whose band takes another kernel, runs its survivor pass
//      here instead);
//   2. one persistent launch per kernel shape runs the survivor DTW of all the
//      batch's queries of that shape (k_dtw_pool);
//   3. per query, on its lane: the final stage.
// Each query has its own device state.  Unless the learned ordering is on,
// the whole batch is captured once into a CUDA graph, kept, and replayed by
// later calls with the same arguments.
dtws_status run_batch(dtws_t h, const float *Qd, const int64_t *q_off, const int32_t *m_arr, const int32_t *r_arr,
                      int32_t nq, int32_t k, int64_t *idx_d, float *dist_d, cudaStream_t s) {
    dtws_status st;
    const bool learned = h->opt.seed_proposals > 0 && h->opt.ordering == DTWS_ORDER_LEARNED;
    const int nl = std::max(1, std::min<int>(h->opt.batch_lanes, nq));
    int m_min = m_arr[0];
    int64_t sum_m = 0, sum_N = 0;
    for (int q = 0; q < nq; ++q) {
        m_min = std::min<int>(m_min, m_arr[q]);
        sum_m += m_arr[q];
        sum_N += h->n - m_arr[q] + 1;
    }
    if ((st = ensure_lanes(h, nl, m_min)) != DTWS_OK) return st;
    long long pool_want = std::min<long long>(1ll << 27, std::max<long long>(1, sum_N));
    if (h->pool_limit >= 0) pool_want = h->pool_limit;
    if ((st = ensure_batch(h, nq, sum_m, pool_want)) != DTWS_OK) return st;
    const int L = std::min<int>(nl, (int)h->lanes.size());
    std::vector<int> order(nq);
    for (int q = 0; q < nq; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return m_arr[x] != m_arr[y] ? m_arr[x] < m_arr[y] : r_arr[x] < r_arr[y];
    });
    const bool graph = h->opt.batch_graph && !learned;
    std::vector<int64_t> sig;
    if (graph) {
        // everything the captured kernels' arguments depend on
        sig = {nq, k, L, (int64_t)(intptr_t)Qd, (int64_t)(intptr_t)idx_d, (int64_t)(intptr_t)dist_d};
        const int64_t *ow = reinterpret_cast<const int64_t *>(&h->opt);
        sig.insert(sig.end(), ow, ow + sizeof(dtws_options) / 8);
        for (int q = 0; q < nq; ++q) {
            sig.push_back(q_off[q]);
            sig.push_back(((int64_t)m_arr[q] << 32) | (uint32_t)r_arr[q]);
        }
        for (auto &en : h->env) sig.push_back(((int64_t)en.r << 32) | (int64_t)(intptr_t)en.U);
        sig.push_back((int64_t)(intptr_t)h->pool.idx);
        sig.push_back(h->pool.cap);
        if (h->graph_exec && sig == h->graph_sig) {
            CK(cudaGraphLaunch(h->graph_exec, s));
            h->last_stream = s;
            return DTWS_OK;
        }
    }
    // per query: its buffers, arguments, lane, and whether its survivors go
    // to the persistent stage (the pool exists and the band takes a one-warp
    // anti-diagonal shape at its default); the persistent stage's query table
    // and per-shape lists are uploaded before any kernel is enqueued
    std::vector<int64_t> qoff(nq + 1, 0);
    for (int q = 0; q < nq; ++q) qoff[q + 1] = qoff[q] + m_arr[q];
    std::vector<QueryBufs> qb(nq);
    std::vector<QueryArgs> qa(nq);
    std::vector<PoolQuery> pq(nq);
    std::vector<char> deferq(nq, 0);
    struct Shape {
        int L, K, m_max, r_max;
        std::vector<int> list;
    };
    std::vector<Shape> shapes;
    const int64_t F = h->bq_fcap;
    for (int j = 0; j < nq; ++j) {
        const int q = order[j], li = j % L;
        Lane &l = h->lanes[li];
        const int m = m_arr[q], r = r_arr[q], rr = r > m - 1 ? m - 1 : r;
        const EnvEntry *ee = nullptr;
        for (auto &en : h->env)
            if (en.r == rr) ee = &en;
        QueryBufs b = lane_bufs(h, l, ee);
        b.st = h->bq_st + q;
        float *f = h->bq_f + qoff[q];
        b.qh32 = f;
        b.Uq = f + F;
        b.Lq = f + 2 * F;
        b.sq = f + 3 * F;
        b.sU = f + 4 * F;
        b.sL = f + 5 * F;
        b.qh64 = h->bq_d + qoff[q];
        b.ord = h->bq_o + qoff[q];
        qb[q] = b;
        qa[q] = make_args(h, m, r, k);
        pq[q] = PoolQuery{b.st, b.qh32, b.ord, b.sq, b.sU, b.sL, b.U, b.L, qa[q]};
        int sL = 0, sK = 0;
        if (h->pool.cap > 0 && qa[q].tune_l == 0 && pool_shape(qa[q].r, &sL, &sK)) {
            deferq[q] = 1;
            Shape *sh = nullptr;
            for (auto &x : shapes)
                if (x.L == sL && x.K == sK) sh = &x;
            if (!sh) {
                shapes.push_back(Shape{sL, sK, 0, 0, {}});
                sh = &shapes.back();
            }
            sh->m_max = std::max(sh->m_max, m);
            sh->r_max = std::max(sh->r_max, qa[q].r);
            sh->list.push_back(q);
        }
    }
    std::vector<int> lists;
    std::vector<int> list_off;
    for (auto &x : shapes) {
        list_off.push_back((int)lists.size());
        lists.insert(lists.end(), x.list.begin(), x.list.end());
    }
    // in the caller's stream order (after any earlier batch that read them),
    // before a capture starts; the pageable source is staged at the call.  A
    // batch without a graph rewrites the tables a cached graph reads.
    if (!graph) drop_graph(h);
    CK(cudaMemcpyAsync(h->pq_dev, pq.data(), sizeof(PoolQuery) * (size_t)nq, cudaMemcpyHostToDevice, s));
    if (!lists.empty())
        CK(cudaMemcpyAsync(h->plist_dev, lists.data(), sizeof(int) * lists.size(), cudaMemcpyHostToDevice, s));
    if (graph) {
        // the capture stream starts after the caller's stream (the uploads)
        CK(cudaEventRecord(h->batch_fork, s));
        CK(cudaStreamWaitEvent(h->cap_stream, h->batch_fork, 0));
        CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    }
    // the stream the batch forks from and joins into: the capture stream, or the caller's
    cudaStream_t root = graph ? h->cap_stream : s;
    auto fail = [&](dtws_status e) {
        if (graph) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(h->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
        }
        return e;
    };
#define CKB(call)                                                                      \
    do {                                                                               \
        cudaError_t e__ = (call);                                                      \
        if (e__ != cudaSuccess) {                                                      \
            set_err("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e__)); \
            return fail(DTWS_ECUDA);                                                   \
        }                                                                              \
    } while (0)
    auto fork = [&]() -> cudaError_t {
        cudaError_t e = cudaEventRecord(h->batch_fork, root);
        for (int i = 0; i < L && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(h->lanes[i].stream, h->batch_fork, 0);
        return e;
    };
    auto join = [&]() -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < L && e == cudaSuccess; ++i) {
            e = cudaEventRecord(h->lanes[i].ev_done, h->lanes[i].stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(root, h->lanes[i].ev_done, 0);
        }
        return e;
    };
    if (h->pool.cap > 0) CKB(cudaMemsetAsync(h->pool.cursor, 0, sizeof(unsigned long long), root));
    CKB(fork());
    std::vector<int> lane_m(L, -1);
    int64_t launches = 0;
    // stage 1
    for (int j = 0; j < nq; ++j) {
        const int q = order[j], li = j % L;
        Lane &l = h->lanes[li];
        const int m = m_arr[q];
        if (lane_m[li] != m) {
            CKB(launch_window_stats(h->x, h->n, m, h->pf, h->bf, h->pok, h->pscale, l.stats.mu_hi, l.stats.mu_lo,
                                    l.stats.inv_sigma, l.stats.smu_hi, l.stats.sinv_sigma,
                                    h->num_sms, l.stream));
            lane_m[li] = m;
            ++launches;
        }
        LearnEntry *le = nullptr;
        if (learned) {
            bool c3;
            StatsEntry *se;
            bool c1;
            // the learned embeddings are scaled by 1/sigma from the handle's statistics of m
            if ((st = get_stats(h, m, l.stream, &se, &c1)) != DTWS_OK) return fail(st);
            if ((st = get_learn(h, m, se, l.stream, &le, &c3)) != DTWS_OK) return fail(st);
        }
        Exec e{qb[q], l.stream, l.side, l.ev_fork, l.ev_join, le, false, 1, deferq[q] ? &h->pool : nullptr};
        int64_t n_l = 0;
        if ((st = enqueue_search(h, e, qa[q], Qd + q_off[q], idx_d + (int64_t)q * k, dist_d + (int64_t)q * k,
                                 &n_l)) != DTWS_OK)
            return fail(st);
        launches += n_l;
    }
    CKB(join());
    // stage 2: the persistent survivor-DTW launches, one per shape
    {
        QueryBufs base = make_bufs(h, nullptr, nullptr);
        for (size_t c = 0; c < shapes.size(); ++c) {
            const Shape &x = shapes[c];
            CKB(launch_dtw_pool(base, h->pool, h->pq_dev, h->plist_dev + list_off[c], (int)x.list.size(), x.L, x.K,
                                x.m_max, x.r_max, root));
            ++launches;
        }
    }
    // stage 3
    CKB(fork());
    for (int j = 0; j < nq; ++j) {
        const int q = order[j], li = j % L;
        Lane &l = h->lanes[li];
        Exec e{qb[q], l.stream, l.side, l.ev_fork, l.ev_join, nullptr, false, 2, nullptr};
        int64_t n_l = 0;
        if ((st = enqueue_search(h, e, qa[q], Qd + q_off[q], idx_d + (int64_t)q * k, dist_d + (int64_t)q * k,
                                 &n_l)) != DTWS_OK)
            return fail(st);
        launches += n_l;
    }
    CKB(join());
#undef CKB
    if (graph) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamEndCapture(h->cap_stream, &g));
        drop_graph(h);
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        h->graph_exec = ex;
        h->graph_sig = sig;
        CK(cudaGraphLaunch(ex, s));
    }
    h->last_stream = s;
    h->have_last = true;
    h->last_N = h->n - m_arr[order[nq - 1]] + 1;
    h->last_launches = launches;
    h->last_st = h->bq_st + order[nq - 1];
    return DTWS_OK;
}

}  // namespace

extern "C" {

void dtws_default_options(dtws_options *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->delta = 1.0f / 1024.0f;
    o->alpha_per_m = 1e-6f;
    o->seed_random = 4;
    o->seed_proposals = 16;
    o->proxy_terms = 16;
    o->ordering = DTWS_ORDER_PLAIN;
    o->timing = 0;
    o->exact_envelope = 1;
    o->batch_lanes = 4;
    o->batch_graph = 1;
    o->exclusion_zone = 0;
    o->unnormalised = 0;
    o->wait_limit_ns = 2000000000LL;
    o->rng_seed = 0;
}

const char *dtws_strerror(dtws_status s) {
    switch (s) {
    case DTWS_OK: return "ok";
    case DTWS_EINVAL: return "invalid argument";
    case DTWS_ENOMEM: return "out of memory";
    case DTWS_ECUDA: return "CUDA error";
    case DTWS_ENONFINITE: return "non-finite value in the series or the query";
    case DTWS_ETIMEOUT: return "a bounded device-side wait ran out";
    case DTWS_ENOTIMPL: return "not implemented";
    case DTWS_EOVERFLOW: return "more near-ties than the re-score list holds";
    }
    return "unknown status";
}

const char *dtws_last_error_detail(void) { return g_err; }

void dtws_debug_fail_next_allocs(int count) { g_fail_allocs = count < 0 ? 0 : count; }

dtws_status dtws_debug_set_pool_capacity(dtws_t h, int64_t cap) {
    if (!h || cap < -1) {
        set_err("dtws_debug_set_pool_capacity: need cap >= -1");
        return DTWS_EINVAL;
    }
    CK(cudaSetDevice(h->device));
    CK(cudaDeviceSynchronize());
    drop_graph(h);
    h->pool_limit = cap;
    return DTWS_OK;
}

dtws_status dtws_debug_set_xz_capacity(dtws_t h, int32_t buf_cap, int32_t sel_cap) {
    if (!h || buf_cap < 1 || sel_cap < 1 || sel_cap > 16384) {
        set_err("dtws_debug_set_xz_capacity: need buf_cap >= 1 and 1 <= sel_cap <= 16384");
        return DTWS_EINVAL;
    }
    CK(cudaSetDevice(h->device));
    CK(cudaDeviceSynchronize());
    drop_graph(h);
    void *ptrs[] = {h->xz_buf, h->xz_sel, h->xz_d64};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    h->xz_buf = nullptr;
    h->xz_sel = nullptr;
    h->xz_d64 = nullptr;
    h->xz_cap = buf_cap;
    h->xz_sel_cap = sel_cap;
    return DTWS_OK;
}

dtws_status dtws_destroy(dtws_t h) {
    if (!h) return DTWS_EINVAL;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (auto &e : h->stats) free_stats(e);
    free_stats(h->ident);
    for (auto &e : h->env) free_env(e);
    for (auto &e : h->learn) free_learn(e);
    if (h->enc_blob) cudaFree(h->enc_blob);
    drop_graph(h);
    for (auto &l : h->lanes) free_lane(l);
    if (h->batch_fork) cudaEventDestroy(h->batch_fork);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    void *ptrs[] = {h->x, h->x_sub, h->pf, h->bf, h->pok, h->pscale, h->envst, h->absmax, h->st, h->status, h->qh32, h->Uq,
                    h->Lq, h->sq, h->sU, h->sL, h->qh64, h->ord, h->cand_lb, h->sort_lb,
                    h->cand_idx, h->sort_idx, h->stage, h->xz_buf, h->xz_sel, h->xz_d64, h->bq_st, h->bq_f, h->bq_d, h->bq_o, h->pool.idx,
                    h->pool.lb, h->pool.mh, h->pool.is, h->pool.ls, h->pool.cursor, h->pq_dev, h->plist_dev};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->hstage) cudaFreeHost(h->hstage);
    if (h->ev_ok)
        for (auto &e : h->ev) cudaEventDestroy(e);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->side) cudaStreamDestroy(h->side);
    delete h;
    return DTWS_OK;
}

dtws_status dtws_create(const float *series, int64_t n, void *stream, dtws_t *out) {
    if (!out) { set_err("null output handle"); return DTWS_EINVAL; }
    *out = nullptr;
    if (!series || n < 2 || n > DTWS_N_MAX) {
        set_err("series null or n=%lld out of range", (long long)n);
        return DTWS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    dtws_ctx *h = new (std::nothrow) dtws_ctx();
    if (!h) return DTWS_ENOMEM;
    dtws_default_options(&h->opt);
    auto fail = [&](dtws_status e) {
        dtws_destroy(h);
        return e;
    };
#define CKF(call)                                                                      \
    do {                                                                               \
        cudaError_t e__ = (call);                                                      \
        if (e__ != cudaSuccess) {                                                      \
            set_err("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e__)); \
            cudaGetLastError();                                                        \
            return fail(e__ == cudaErrorMemoryAllocation ? DTWS_ENOMEM : DTWS_ECUDA);  \
        }                                                                              \
    } while (0)
    CKF(cudaGetDevice(&h->device));
    CKF(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    h->n = n;
    h->n_alloc = round_up(n, kProxyTile) + kMMax + 64;
    const int64_t nb = (n + kBlockB - 1) / kBlockB;
    CKF(dalloc(&h->x, h->n_alloc));
    CKF(dalloc(&h->x_sub, h->n_alloc / kProxyStride + kProxyTile));
    CKF(dalloc(&h->pf, 4 * n));
    CKF(dalloc(&h->bf, 5 * nb));
    CKF(dalloc(&h->pok, nb));
    CKF(dalloc(&h->pscale, 2));
    h->nblk = (n + kEnvG - 1) / kEnvG;
    CKF(dalloc(&h->envst, 2 * (size_t)kEnvLevels * h->nblk));
    CKF(dalloc(&h->status, 1));
    CKF(dalloc(&h->absmax, 1));
    CKF(cudaMemsetAsync(h->x, 0, h->n_alloc * 4, s));
    CKF(cudaMemcpyAsync(h->x, series, n * 4, cudaMemcpyDefault, s));
    CKF(cudaMemsetAsync(h->status, 0, 4, s));
    CKF(cudaMemsetAsync(h->absmax, 0, 4, s));
    CKF(launch_check_finite(h->x, n, h->status, h->absmax, s));
    int flag = 0;
    unsigned amax = 0;
    CKF(cudaMemcpyAsync(&flag, h->status, 4, cudaMemcpyDeviceToHost, s));
    CKF(cudaMemcpyAsync(&amax, h->absmax, 4, cudaMemcpyDeviceToHost, s));
    CKF(cudaStreamSynchronize(s));
    memcpy(&h->xabs, &amax, 4);
    if (flag) {
        set_err("series contains NaN or Inf");
        return fail(DTWS_ENONFINITE);
    }
    CKF(cudaMemsetAsync(h->x_sub, 0, (h->n_alloc / kProxyStride + kProxyTile) * 4, s));
    CKF(launch_subsample(h->x, h->n_alloc / kProxyStride, h->x_sub, h->num_sms, s));
    CKF(launch_prefix(h->x, n, h->pf, h->bf, h->pok, reinterpret_cast<unsigned *>(h->pscale + 1), h->pscale, s));
    CKF(launch_block_envelope(h->x, n, h->envst, h->nblk, s));
    CKF(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    CKF(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CKF(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    for (auto &e : h->ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            h->ev_ok = false;
            break;
        } else
            h->ev_ok = true;
    CKF(cudaStreamSynchronize(s));
#undef CKF
    *out = h;
    return DTWS_OK;
}

dtws_status dtws_set_options(dtws_t h, const dtws_options *o) {
    if (!h || !o) return DTWS_EINVAL;
    if (!(o->delta >= 0.0f) || !(o->alpha_per_m >= 0.0f) || o->seed_random < 0 ||
        o->seed_random > 64 || o->seed_proposals < 0 || o->seed_proposals > kPropMax ||
        o->proxy_terms < 1 || o->proxy_terms > 16 || o->wait_limit_ns <= 0 ||
        (o->exact_envelope != 0 && o->exact_envelope != 1) || o->batch_lanes < 1 || o->batch_lanes > 16 ||
        (o->batch_graph != 0 && o->batch_graph != 1) || o->exclusion_zone < 0 ||
        (o->unnormalised != 0 && o->unnormalised != 1) ||
        (o->ordering != DTWS_ORDER_PLAIN && o->ordering != DTWS_ORDER_LEARNED)) {
        set_err("option out of range");
        return DTWS_EINVAL;
    }
    h->opt = *o;
    return DTWS_OK;
}

dtws_status dtws_get_options(dtws_t h, dtws_options *o) {
    if (!h || !o) return DTWS_EINVAL;
    *o = h->opt;
    return DTWS_OK;
}

dtws_status dtws_query(dtws_t h, const float *Q, int32_t m, int32_t r, int32_t k, int64_t *out_idx,
                       float *out_dist, void *stream) {
    dtws_status st = check_query_args(h, Q, m, r, k);
    if (st != DTWS_OK) return st;
    if (!out_idx || !out_dist) { set_err("null output"); return DTWS_EINVAL; }
    // with an exclusion zone z the search finds the K = k(2z+1) best windows
    // (capped at N), among which the greedy answer lies
    // With an exclusion zone z: when k(2z+1) fits the result list, the search
    // finds the K = k(2z+1) best windows (capped at N), among which the greedy
    // answer lies; otherwise the wide form (a threshold from windows more
    // than 2z apart, a candidate buffer, greedy selection at the end).
    const int z = h->opt.exclusion_zone;
    int K = k;
    bool wide = false;
    if (z > 0) {
        const int64_t want = (int64_t)k * (2 * (int64_t)z + 1), N = h->n - m + 1;
        if (want > DTWS_K_MAX) wide = true;
        else K = (int)(want < N ? want : N);
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool qdev = is_device_ptr(Q), idev = is_device_ptr(out_idx), ddev = is_device_ptr(out_dist);
    const size_t qb = (size_t)m * 4, ib = (size_t)k * 8, db = (size_t)k * 4;
    const size_t kib = (size_t)K * 8, kdb = (size_t)K * 4;  // the K-list (exclusion zone only)
    if ((st = ensure_stage(h, 256 + round_up(qb, 256) + round_up(ib, 256) + round_up(db, 256) +
                                  round_up(kib, 256) + round_up(kdb, 256))) != DTWS_OK)
        return st;
    char *sp = (char *)h->stage;
    const float *Qd = Q;
    if (!qdev) {
        CK(cudaMemcpyAsync(sp, Q, qb, cudaMemcpyHostToDevice, s));
        Qd = (const float *)sp;
    }
    int64_t *idx_d = idev ? out_idx : (int64_t *)(sp + round_up(qb, 256));
    float *dist_d = ddev ? out_dist : (float *)(sp + round_up(qb, 256) + round_up(ib, 256));
    if (wide) {
        if ((st = run_query(h, Qd, m, r, k, idx_d, dist_d, s, z)) != DTWS_OK) return st;
    } else if (z > 0) {
        char *kp = sp + round_up(qb, 256) + round_up(ib, 256) + round_up(db, 256);
        int64_t *kidx = (int64_t *)kp;
        float *kdist = (float *)(kp + round_up(kib, 256));
        if ((st = run_query(h, Qd, m, r, K, kidx, kdist, s)) != DTWS_OK) return st;
        CK(launch_exclusion_select(kidx, kdist, K, k, z, idx_d, dist_d, s));
    } else if ((st = run_query(h, Qd, m, r, k, idx_d, dist_d, s)) != DTWS_OK) {
        return st;
    }
    return read_back(h, s, idx_d, dist_d, out_idx, out_dist, ib, db, idev, ddev);
}

dtws_status dtws_query_batch(dtws_t h, const float *Q_cat, const int64_t *q_off, const int32_t *m_arr,
                             const int32_t *r_arr, int32_t nq, int32_t k, int64_t *out_idx,
                             float *out_dist, void *stream) {
    if (!h || !Q_cat || !q_off || !m_arr || !r_arr || !out_idx || !out_dist || nq < 1) {
        set_err("null argument or nq < 1");
        return DTWS_EINVAL;
    }
    if (q_off[0] != 0) { set_err("q_off[0] != 0"); return DTWS_EINVAL; }
    if (h->opt.exclusion_zone > 0) { set_err("exclusion_zone is for dtws_query only"); return DTWS_EINVAL; }
    if (h->opt.unnormalised) { set_err("unnormalised DTW is for dtws_query only"); return DTWS_EINVAL; }
    for (int q = 0; q < nq; ++q) {
        if (q_off[q + 1] - q_off[q] != m_arr[q]) { set_err("q_off/m mismatch at %d", q); return DTWS_EINVAL; }
        dtws_status st = check_query_args(h, Q_cat, m_arr[q], r_arr[q], k);
        if (st != DTWS_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool qdev = is_device_ptr(Q_cat), idev = is_device_ptr(out_idx), ddev = is_device_ptr(out_dist);
    const size_t qb = (size_t)q_off[nq] * 4, ib = (size_t)nq * k * 8, db = (size_t)nq * k * 4;
    dtws_status st = ensure_stage(h, 256 + round_up(qb, 256) + round_up(ib, 256) + round_up(db, 256));
    if (st != DTWS_OK) return st;
    char *sp = (char *)h->stage;
    const float *Qd = Q_cat;
    if (!qdev) {
        CK(cudaMemcpyAsync(sp, Q_cat, qb, cudaMemcpyHostToDevice, s));
        Qd = (const float *)sp;
    }
    int64_t *idx_d = idev ? out_idx : (int64_t *)(sp + round_up(qb, 256));
    float *dist_d = ddev ? out_dist : (float *)(sp + round_up(qb, 256) + round_up(ib, 256));
    st = run_batch(h, Qd, q_off, m_arr, r_arr, nq, k, idx_d, dist_d, s);
    if (st != DTWS_OK) return st;
    return read_back(h, s, idx_d, dist_d, out_idx, out_dist, ib, db, idev, ddev);
}

dtws_status dtws_sync_status(dtws_t h, void *stream) {
    if (!h) return DTWS_EINVAL;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    int flag = 0;
    CK(cudaMemcpy(&flag, h->status, 4, cudaMemcpyDeviceToHost));
    CK(cudaMemset(h->status, 0, 4));
    if (flag & kStNonFinite) return DTWS_ENONFINITE;
    if (flag & kStTimeout) return DTWS_ETIMEOUT;
    if (flag & kStOverflow) return DTWS_EOVERFLOW;
    return DTWS_OK;
}

dtws_status dtws_last_stats(dtws_t h, dtws_query_stats *o) {
    if (!h || !o) return DTWS_EINVAL;
    memset(o, 0, sizeof *o);
    if (!h->have_last) return DTWS_OK;
    CK(cudaStreamSynchronize(h->last_stream));
    QueryState hs;
    CK(cudaMemcpy(&hs, h->last_st ? h->last_st : h->st, sizeof hs, cudaMemcpyDeviceToHost));
    o->windows = h->last_N;
    o->pass_kim = (int64_t)hs.ctr[kCtrKim];
    o->pass_keogh_q = (int64_t)hs.ctr[kCtrKeoghQ];
    o->pass_keogh_s = (int64_t)hs.ctr[kCtrKeoghS];
    o->dtw_started = (int64_t)hs.ctr[kCtrDtwStarted];
    o->dtw_abandoned = (int64_t)hs.ctr[kCtrDtwAbandoned];
    o->dtw_cells = (int64_t)hs.ctr[kCtrCells];
    o->rescored = (int64_t)hs.ctr[kCtrRescored];
    o->kernel_launches = h->last_launches;
    {
        // smallest seed distance: exact DTW seeds or Euclidean seeds (upper bounds)
        unsigned long long key = hs.seed_keys[0] < hs.ed_keys[0] ? hs.seed_keys[0] : hs.ed_keys[0];
        unsigned bits = (unsigned)(key >> 32);
        float f;
        memcpy(&f, &bits, 4);
        o->seed_bsf = key == kEmptyKey ? __builtin_inff() : f;
    }
    if (h->opt.timing && h->ev_ok) {
        // phases: prev event -> this event
        const int order[9] = {8, 6, 7, 0, 1, 2, 3, 4, 5};
        int prev = -1;
        for (int t = 0; t < 9; ++t) {
            int e = order[t];
            if (!h->ev_recorded[e]) continue;
            if (prev >= 0) {
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, h->ev[prev], h->ev[e]);
                if (e < 8) o->phase_ms[e] = ms;
            }
            prev = e;
        }
    }
    return DTWS_OK;
}

dtws_status dtws_clear_cache(dtws_t h) {
    if (!h) return DTWS_EINVAL;
    CK(cudaDeviceSynchronize());
    for (auto &e : h->stats) free_stats(e);
    free_stats(h->ident);
    for (auto &e : h->env) free_env(e);
    for (auto &e : h->learn) free_learn(e);
    drop_graph(h);
    h->stats.clear();
    h->env.clear();
    h->learn.clear();
    return DTWS_OK;
}

dtws_status dtws_debug_lock_selftest(dtws_t h, int64_t wait_ns, void *stream) {
    if (!h || wait_ns < 1 || wait_ns > 10000000000LL) {
        set_err("dtws_debug_lock_selftest: null handle or wait_ns outside [1, 1e10]");
        return DTWS_EINVAL;
    }
    dtws_status st;
    if ((st = ensure_workspace(h)) != DTWS_OK) return st;
    if ((st = ensure_xz(h)) != DTWS_OK) return st;
    QueryBufs b = make_bufs(h, nullptr, nullptr);
    b.wait_ns = wait_ns;
    QueryArgs a = make_args(h, 2, 0, 1);
    a.xz_z = 1;
    CK(launch_lock_selftest(b, a, (cudaStream_t)stream));
    return DTWS_OK;
}

dtws_status dtws_debug_wait_selftest(dtws_t h, int64_t wait_ns, void *stream) {
    if (!h || wait_ns < 1 || wait_ns > 10000000000LL) {
        set_err("dtws_debug_wait_selftest: null handle or wait_ns outside [1, 1e10]");
        return DTWS_EINVAL;
    }
    CK(launch_wait_selftest(h->status, (long long)wait_ns, (cudaStream_t)stream));
    return DTWS_OK;
}

dtws_status dtws_autotune(dtws_t h, const int32_t *m_arr, const int32_t *r_arr, int32_t count, int32_t samples,
                          void *stream) {
    if (!h || !m_arr || !r_arr || count < 1 || samples < 32 || samples > (1 << 20)) {
        set_err("dtws_autotune: null argument, count < 1 or samples out of [32, 2^20]");
        return DTWS_EINVAL;
    }
    for (int i = 0; i < count; ++i)
        if (m_arr[i] < 2 || m_arr[i] > DTWS_M_MAX || (int64_t)m_arr[i] > h->n || r_arr[i] < 0) {
            set_err("dtws_autotune: pair %d out of range", i);
            return DTWS_EINVAL;
        }
    cudaStream_t s = (cudaStream_t)stream;
    dtws_status st;
    if ((st = ensure_workspace(h)) != DTWS_OK) return st;
    CK(cudaStreamSynchronize(s));
    drop_graph(h);  // captured batches may use the old shapes
    const size_t ob = (size_t)samples * 8, fb = (size_t)samples * 4;
    if ((st = ensure_stage(h, ob + 2 * fb + 1024)) != DTWS_OK) return st;
    int64_t *off_d = (int64_t *)h->stage;
    float *ref_d = (float *)((char *)h->stage + round_up(ob, 256));
    float *out_d = (float *)((char *)h->stage + round_up(ob, 256) + round_up(fb, 256));
    std::vector<int64_t> offs(samples);
    std::vector<float> ref(samples), got(samples);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto cleanup = [&](dtws_status r) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return r;
    };
    for (int i = 0; i < count; ++i) {
        const int m = m_arr[i], r = r_arr[i] > m - 1 ? m - 1 : r_arr[i];
        bool seen = false;
        for (int j = 0; j < i; ++j) seen |= m_arr[j] == m && (r_arr[j] > m - 1 ? m - 1 : r_arr[j]) == r;
        if (seen) continue;
        StatsEntry *se;
        bool c;
        if ((st = get_stats(h, m, s, &se, &c)) != DTWS_OK) return cleanup(st);
        const QueryBufs b = make_bufs(h, se, nullptr);
        // shapes are timed on normalised windows whatever the options say
        QueryArgs a = make_args(h, m, r, 1, false);
        a.tune_l = a.tune_k = a.tune_w = 0;
        // the query: a window of the series; the samples: evenly spread windows
        const int64_t N = h->n - m + 1;
        for (int t = 0; t < samples; ++t) offs[t] = (int64_t)((double)t * (double)(N - 1) / samples);
        CK(cudaMemcpyAsync(off_d, offs.data(), ob, cudaMemcpyHostToDevice, s));
        CK(launch_query_reset(b, a, s));
        CK(launch_qprep(h->x + N / 2, b, a, s));
        auto timed = [&](int L, int K, int W, float *out, float *ms) -> cudaError_t {
            float best = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaError_t e = cudaEventRecord(e0, s);
                if (e == cudaSuccess)
                    e = L ? launch_dtw_at_shape(b, a, off_d, samples, out, L, K, W, s)
                          : launch_dtw_at(b, a, off_d, samples, out, s);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) return e;
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                best = t < best ? t : best;
            }
            *ms = best;
            return cudaSuccess;
        };
        // the default is the survivor pass's own shape (DTW at offsets alone
        // takes a four-cell shape for bands of 9 to 64 cells)
        int dL = 0, dK = 0, dW = 0;
        if (!dtw_default_shape(m, r, &dL, &dK, &dW)) dL = dK = dW = 0;
        float ms_def = 0.f;
        CK(timed(dL, dK, dW, ref_d, &ms_def));
        CK(cudaMemcpy(ref.data(), ref_d, fb, cudaMemcpyDeviceToHost));
        TuneEntry best{m, r, 0, 0, 0, ms_def, ms_def};
        const int Ls[6] = {1, 2, 4, 8, 16, 32}, Ks[10] = {0, 1, 2, 3, 4, 6, 8, 10, 12, 16}, Ws[3] = {2, 4, 8};
        for (int L : Ls)
            for (int K : Ks)
                for (int W : Ws) {
                    if (!dtw_shape_valid(m, r, L, K, W)) continue;
                    float ms = 0.f;
                    CK(timed(L, K, W, out_d, &ms));
                    if (!(ms < best.ms_best * 0.97f)) continue;  // keep the default unless clearly faster
                    CK(cudaMemcpy(got.data(), out_d, fb, cudaMemcpyDeviceToHost));
                    if (memcmp(got.data(), ref.data(), fb) != 0) continue;  // must be bit-identical
                    best.L = L;
                    best.K = K;
                    best.warps = W;
                    best.ms_best = ms;
                }
        bool replaced = false;
        for (auto &t : h->tune)
            if (t.m == m && t.r == r) {
                t = best;
                replaced = true;
            }
        if (!replaced) h->tune.push_back(best);
    }
    return cleanup(DTWS_OK);
}

dtws_status dtws_tune_entry(dtws_t h, int32_t m, int32_t r, int32_t *shape, float *ms) {
    if (!h || !shape || !ms) return DTWS_EINVAL;
    const int rr = r > m - 1 ? m - 1 : r;
    for (const auto &t : h->tune)
        if (t.m == m && t.r == rr) {
            shape[0] = t.L;
            shape[1] = t.K;
            shape[2] = t.warps;
            ms[0] = t.ms_default;
            ms[1] = t.ms_best;
            return DTWS_OK;
        }
    set_err("dtws_tune_entry: (m=%d, r=%d) not tuned", m, r);
    return DTWS_EINVAL;
}

dtws_status dtws_set_encoder(dtws_t h, const float *params, int32_t count, void *stream) {
    if (!h || !params || count != kEncParams) {
        set_err("dtws_set_encoder: null argument or count != %d", kEncParams);
        return DTWS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (!h->enc_blob) {
        uint8_t *blob = nullptr;
        if (dalloc(&blob, kEncBlobBytes) != cudaSuccess) {
            cudaGetLastError();
            set_err("dtws_set_encoder: out of device memory");
            return DTWS_ENOMEM;
        }
        h->enc_blob = blob;
    }
    dtws_status st = ensure_stage(h, (size_t)kEncParams * 4 + 256);
    if (st != DTWS_OK) return st;
    CK(cudaStreamSynchronize(s));  // the stage buffer and the blob may be in use by queued work
    float *p = (float *)h->stage;
    CK(cudaMemcpyAsync(p, params, (size_t)kEncParams * 4, cudaMemcpyDefault, s));
    CK(launch_enc_pack(p, nullptr, nullptr, nullptr, h->enc_blob, false, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, s));
    CK(cudaStreamSynchronize(s));
    ++h->enc_version;
    return DTWS_OK;
}

dtws_status dtws_learned_embeddings(dtws_t h, int32_t m, float *out, int64_t rows, void *stream) {
    if (!h || !out || m < 64 || m > DTWS_M_MAX || (int64_t)m > h->n) {
        set_err("dtws_learned_embeddings: null argument or m out of range [64, min(n, %d)]", DTWS_M_MAX);
        return DTWS_EINVAL;
    }
    if (!h->enc_version) { set_err("dtws_learned_embeddings: no encoder installed"); return DTWS_EINVAL; }
    if (rows != enc_rows(h, m)) {
        set_err("dtws_learned_embeddings: rows must be %lld", (long long)enc_rows(h, m));
        return DTWS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    StatsEntry *se;
    LearnEntry *le;
    bool c1, c2;
    dtws_status st;
    if ((st = get_stats(h, m, s, &se, &c1)) != DTWS_OK) return st;
    if ((st = get_learn(h, m, se, s, &le, &c2)) != DTWS_OK) return st;
    if (is_device_ptr(out)) {
        CK(launch_bf16_to_f32(le->E, rows * 64, out, s));
        return DTWS_OK;
    }
    float *tmp = nullptr;
    CK(cudaMalloc(&tmp, (size_t)rows * 64 * 4));
    cudaError_t e1 = launch_bf16_to_f32(le->E, rows * 64, tmp, s);
    cudaError_t e2 = e1 == cudaSuccess ? cudaMemcpyAsync(out, tmp, (size_t)rows * 64 * 4, cudaMemcpyDeviceToHost, s)
                                       : e1;
    cudaError_t e3 = cudaStreamSynchronize(s);
    cudaFree(tmp);
    CK(e2);
    CK(e3);
    return DTWS_OK;
}

dtws_status dtws_window_stats(dtws_t h, int32_t m, float *mu_hi, float *mu_lo, float *inv_sigma,
                              void *stream) {
    if (!h || !mu_hi || !mu_lo || !inv_sigma || m < 2 || m > DTWS_M_MAX || (int64_t)m > h->n) {
        set_err("bad arguments to dtws_window_stats");
        return DTWS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    StatsEntry *se;
    bool c;
    dtws_status st = get_stats(h, m, s, &se, &c);
    if (st != DTWS_OK) return st;
    const size_t bytes = (size_t)(h->n - m + 1) * 4;
    CK(cudaMemcpyAsync(mu_hi, se->mu_hi, bytes, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(mu_lo, se->mu_lo, bytes, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(inv_sigma, se->inv_sigma, bytes, cudaMemcpyDefault, s));
    if (!is_device_ptr(mu_hi) || !is_device_ptr(mu_lo) || !is_device_ptr(inv_sigma))
        CK(cudaStreamSynchronize(s));
    return DTWS_OK;
}

dtws_status dtws_series_envelope(dtws_t h, int32_t r, float *U, float *L, void *stream) {
    if (!h || !U || !L || r < 0 || r >= DTWS_M_MAX) {
        set_err("bad arguments to dtws_series_envelope");
        return DTWS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    EnvEntry *ee;
    bool c;
    dtws_status st = get_env(h, r, s, &ee, &c);
    if (st != DTWS_OK) return st;
    CK(cudaMemcpyAsync(U, ee->U, (size_t)h->n * 4, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(L, ee->L, (size_t)h->n * 4, cudaMemcpyDefault, s));
    if (!is_device_ptr(U) || !is_device_ptr(L)) CK(cudaStreamSynchronize(s));
    return DTWS_OK;
}

// Shared front half of the *_at entry points: validation, staging of Q and
// the offsets, statistics / envelope, query prep.
static dtws_status at_prepare(dtws_t h, const float *Q, int32_t m, int32_t r, const int64_t *offsets,
                              int64_t count, size_t out_bytes, cudaStream_t s, bool need_env,
                              QueryBufs *b, QueryArgs *a, const int64_t **off_d, char **out_stage) {
    dtws_status st = check_query_args(h, Q, m, r, 1);
    if (st != DTWS_OK) return st;
    if (!offsets || count < 0) { set_err("null offsets or count < 0"); return DTWS_EINVAL; }
    const size_t qb = (size_t)m * 4, ob = (size_t)count * 8;
    if ((st = ensure_stage(h, 256 + round_up(qb, 256) + round_up(ob, 256) + round_up(out_bytes, 256))) != DTWS_OK)
        return st;
    char *sp = (char *)h->stage;
    const float *Qd = Q;
    if (!is_device_ptr(Q)) {
        CK(cudaMemcpyAsync(sp, Q, qb, cudaMemcpyHostToDevice, s));
        Qd = (const float *)sp;
    }
    *off_d = offsets;
    if (!is_device_ptr(offsets)) {
        CK(cudaMemcpyAsync(sp + round_up(qb, 256), offsets, ob, cudaMemcpyHostToDevice, s));
        *off_d = (const int64_t *)(sp + round_up(qb, 256));
        // validate offsets on the host (they are host data)
        const int64_t N = h->n - m + 1;
        for (int64_t t = 0; t < count; ++t)
            if (offsets[t] < 0 || offsets[t] >= N) { set_err("offset %lld out of range", (long long)offsets[t]); return DTWS_EINVAL; }
    }
    *out_stage = sp + round_up(qb, 256) + round_up(ob, 256);
    StatsEntry *se;
    EnvEntry *ee = nullptr;
    bool c;
    if ((st = query_stats(h, m, s, &se, &c)) != DTWS_OK) return st;
    const int rr = r > m - 1 ? m - 1 : r;
    if (need_env && (st = get_env(h, rr, s, &ee, &c)) != DTWS_OK) return st;
    if ((st = ensure_workspace(h)) != DTWS_OK) return st;
    *b = make_bufs(h, se, ee);
    *a = make_args(h, m, r, 1);
    a->prescore = 0;
    CK(launch_query_reset(*b, *a, s));
    CK(launch_qprep(Qd, *b, *a, s));
    return DTWS_OK;
}

dtws_status dtws_dtw_at(dtws_t h, const float *Q, int32_t m, int32_t r, const int64_t *offsets,
                        int64_t count, float *out, void *stream) {
    if (!out) return DTWS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    QueryBufs b;
    QueryArgs a;
    const int64_t *off_d;
    char *ostage;
    dtws_status st = at_prepare(h, Q, m, r, offsets, count, (size_t)count * 4, s, false, &b, &a, &off_d, &ostage);
    if (st != DTWS_OK) return st;
    if (count == 0) return DTWS_OK;
    const bool odev = is_device_ptr(out);
    float *od = odev ? out : (float *)ostage;
    CK(launch_dtw_at(b, a, off_d, count, od, s));
    if (!odev) {
        CK(cudaMemcpyAsync(out, od, (size_t)count * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return DTWS_OK;
}

dtws_status dtws_dtw_at_f64(dtws_t h, const float *Q, int32_t m, int32_t r, const int64_t *offsets,
                            int64_t count, double *out, void *stream) {
    if (!out) return DTWS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    QueryBufs b;
    QueryArgs a;
    const int64_t *off_d;
    char *ostage;
    dtws_status st = at_prepare(h, Q, m, r, offsets, count, (size_t)count * 8, s, false, &b, &a, &off_d, &ostage);
    if (st != DTWS_OK) return st;
    if (count == 0) return DTWS_OK;
    const bool odev = is_device_ptr(out);
    double *od = odev ? out : (double *)ostage;
    CK(launch_dtw_at_f64(b, a, off_d, count, od, s));
    if (!odev) {
        CK(cudaMemcpyAsync(out, od, (size_t)count * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return DTWS_OK;
}

dtws_status dtws_lower_bounds_at(dtws_t h, const float *Q, int32_t m, int32_t r, const int64_t *offsets,
                                 int64_t count, float *kim, float *keogh_q, float *keogh_s, void *stream) {
    if (!kim || !keogh_q || !keogh_s) return DTWS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    QueryBufs b;
    QueryArgs a;
    const int64_t *off_d;
    char *ostage;
    const size_t ob = (size_t)count * 4;
    dtws_status st = at_prepare(h, Q, m, r, offsets, count, 3 * round_up(ob, 256), s, true, &b, &a, &off_d, &ostage);
    if (st != DTWS_OK) return st;
    if (count == 0) return DTWS_OK;
    const bool dev = is_device_ptr(kim) && is_device_ptr(keogh_q) && is_device_ptr(keogh_s);
    float *k1 = dev ? kim : (float *)ostage;
    float *k2 = dev ? keogh_q : (float *)(ostage + round_up(ob, 256));
    float *k3 = dev ? keogh_s : (float *)(ostage + 2 * round_up(ob, 256));
    CK(launch_lbs_at(b, a, off_d, count, k1, k2, k3, s));
    if (!dev) {
        CK(cudaMemcpyAsync(kim, k1, ob, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(keogh_q, k2, ob, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(keogh_s, k3, ob, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return DTWS_OK;
}

}  // extern "C"
