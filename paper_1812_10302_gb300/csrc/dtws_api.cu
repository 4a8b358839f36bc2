// dtws_api.cu -- the C ABI of include/dtws.h: handle lifecycle, argument
// validation, device memory, per-series caches and the order in which a
// query's kernels are enqueued on the caller's stream.
#include <cstdarg>
#include <cstdio>
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
    float *smu_hi = nullptr, *smu_lo = nullptr, *sinv_sigma = nullptr;  // every kProxyStride-th window
};
struct EnvEntry {
    int r = 0;
    int64_t used = 0;
    float *U = nullptr, *L = nullptr;
};

constexpr int kCacheSlots = 8;

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
    double *P1 = nullptr, *P2 = nullptr, *T1 = nullptr, *T2 = nullptr, *A = nullptr;
    std::vector<StatsEntry> stats;
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
    // staging of host arrays
    void *stage = nullptr;
    size_t stage_cap = 0;
    dtws_options opt;
    cudaStream_t last_stream = nullptr;
    bool have_last = false;
    int64_t last_N = 0;
    int64_t last_launches = 0;
    cudaEvent_t ev[9] = {};
    bool ev_ok = false;
    bool ev_recorded[9] = {false};
    // side stream for work that overlaps the lower-bound scan
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
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

void free_stats(StatsEntry &e) {
    cudaFree(e.mu_hi);
    cudaFree(e.mu_lo);
    cudaFree(e.inv_sigma);
    cudaFree(e.smu_hi);
    cudaFree(e.smu_lo);
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
    cudaError_t a4 = dalloc(&e.smu_hi, scap), a5 = dalloc(&e.smu_lo, scap), a6 = dalloc(&e.sinv_sigma, scap);
    if (a1 != cudaSuccess || a2 != cudaSuccess || a3 != cudaSuccess || a4 != cudaSuccess ||
        a5 != cudaSuccess || a6 != cudaSuccess) {
        free_stats(e);
        cudaGetLastError();
        set_err("window statistics for m=%d: out of device memory", m);
        return DTWS_ENOMEM;
    }
    CK(cudaMemsetAsync(e.mu_hi, 0, cap * 4, s));
    CK(cudaMemsetAsync(e.mu_lo, 0, cap * 4, s));
    CK(cudaMemsetAsync(e.inv_sigma, 0, cap * 4, s));
    CK(cudaMemsetAsync(e.smu_hi, 0, scap * 4, s));
    CK(cudaMemsetAsync(e.smu_lo, 0, scap * 4, s));
    CK(cudaMemsetAsync(e.sinv_sigma, 0, scap * 4, s));
    CK(launch_window_stats(h->x, h->n, m, h->P1, h->P2, h->T1, h->T2, h->A, e.mu_hi, e.mu_lo,
                           e.inv_sigma, e.smu_hi, e.smu_lo, e.sinv_sigma, s));
    e.used = ++h->clock;
    h->stats.push_back(e);
    *out = &h->stats.back();
    *computed = true;
    return DTWS_OK;
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
    CK(cudaMemsetAsync(e.U, 0, h->n_alloc * 4, s));
    CK(cudaMemsetAsync(e.L, 0, h->n_alloc * 4, s));
    CK(launch_envelope(h->x, h->n, r, e.U, e.L, s));
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
    b.st = h->st;
    b.x = h->x;
    b.mu_hi = se ? se->mu_hi : nullptr;
    b.mu_lo = se ? se->mu_lo : nullptr;
    b.inv_sigma = se ? se->inv_sigma : nullptr;
    b.smu_hi = se ? se->smu_hi : nullptr;
    b.smu_lo = se ? se->smu_lo : nullptr;
    b.sinv_sigma = se ? se->sinv_sigma : nullptr;
    b.U = ee ? ee->U : nullptr;
    b.L = ee ? ee->L : nullptr;
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
    return b;
}

QueryArgs make_args(dtws_t h, int m, int r, int k) {
    QueryArgs a;
    a.N = h->n - m + 1;
    a.m = m;
    a.r = r > m - 1 ? m - 1 : r;
    a.k = k;
    a.list_cap = k + 64 < kListMax ? k + 64 : kListMax;
    a.delta = h->opt.delta;
    a.alpha = h->opt.alpha_per_m * (float)m;
    // largest power of two <= alpha/4 (alpha 0: FP32's smallest normal)
    float g = 1.17549435e-38f;
    while (g * 2.0f <= a.alpha * 0.25f) g *= 2.0f;
    a.qgrid = g;
    a.prescore = a.r <= kDiagRMax ? 1 : 0;
    return a;
}

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
    return DTWS_OK;
}

void record(dtws_t h, int i, cudaStream_t s) {
    if (h->opt.timing && h->ev_ok) {
        cudaEventRecord(h->ev[i], s);
        h->ev_recorded[i] = true;
    }
}

// The device-side query pipeline on device pointers.
dtws_status run_query(dtws_t h, const float *Qd, int m, int r, int k, int64_t *idx_d, float *dist_d,
                      cudaStream_t s) {
    dtws_status st;
    for (bool &v : h->ev_recorded) v = false;
    record(h, 8, s);
    StatsEntry *se;
    EnvEntry *ee;
    bool c1, c2;
    if ((st = get_stats(h, m, s, &se, &c1)) != DTWS_OK) return st;
    record(h, 6, s);
    const int rr = r > m - 1 ? m - 1 : r;
    if ((st = get_env(h, rr, s, &ee, &c2)) != DTWS_OK) return st;
    record(h, 7, s);
    if ((st = ensure_workspace(h)) != DTWS_OK) return st;
    if ((st = ensure_candidates(h)) != DTWS_OK) return st;
    const QueryBufs b = make_bufs(h, se, ee);
    const QueryArgs a = make_args(h, m, r, k);
    const int P = h->opt.seed_proposals, R = h->opt.seed_random;
    int64_t launches = (c1 ? 1 : 0) + (c2 ? 1 : 0);
    CK(launch_query_reset(b, a, s));
    CK(launch_qprep(Qd, b, a, s));
    record(h, 0, s);
    if (P > 0) {
        CK(launch_seed_scan(b, a, P, h->opt.proxy_terms, s));
        ++launches;
    }
    CK(launch_seed_gather(b, a, R, P, h->opt.rng_seed, s));
    CK(launch_seed_ed(b, a, s));
    if (k > 1) {  // exact DTW seeds tighten a k-th bound the Euclidean seeds leave loose
        CK(launch_dtw_seeds(b, a, s));
        ++launches;
    }
    record(h, 1, s);
    // the best Euclidean seed is scored on the side stream during the scan
    if (a.prescore) {
        CK(cudaEventRecord(h->ev_fork, s));
        CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        CK(launch_prescore(b, a, h->side));
        CK(cudaEventRecord(h->ev_join, h->side));
        ++launches;
    }
    CK(launch_lb_scan(b, a, s));
    record(h, 2, s);
    CK(launch_order(b, a, s));
    record(h, 3, s);
    CK(launch_dtw_survivors(b, a, s));
    record(h, 4, s);
    if (a.prescore) CK(cudaStreamWaitEvent(s, h->ev_join, 0));
    CK(launch_finalize(b, a, idx_d, dist_d, s));
    record(h, 5, s);
    launches += 2 + 2 + 1 + 3 + 1 + 3;  // reset, qprep, gather, ED seeds, scan, order x3, DTW, final x3
    h->last_stream = s;
    h->have_last = true;
    h->last_N = a.N;
    h->last_launches = launches;
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

dtws_status dtws_destroy(dtws_t h) {
    if (!h) return DTWS_EINVAL;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (auto &e : h->stats) free_stats(e);
    for (auto &e : h->env) free_env(e);
    void *ptrs[] = {h->x, h->P1, h->P2, h->T1, h->T2, h->A, h->st, h->status, h->qh32, h->Uq,
                    h->Lq, h->sq, h->sU, h->sL, h->qh64, h->ord, h->cand_lb, h->sort_lb,
                    h->cand_idx, h->sort_idx, h->stage};
    for (void *p : ptrs)
        if (p) cudaFree(p);
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
    CKF(dalloc(&h->P1, n));
    CKF(dalloc(&h->P2, n));
    CKF(dalloc(&h->T1, nb));
    CKF(dalloc(&h->T2, nb));
    CKF(dalloc(&h->A, nb));
    CKF(dalloc(&h->status, 1));
    CKF(cudaMemsetAsync(h->x, 0, h->n_alloc * 4, s));
    CKF(cudaMemcpyAsync(h->x, series, n * 4, cudaMemcpyDefault, s));
    CKF(cudaMemsetAsync(h->status, 0, 4, s));
    CKF(launch_check_finite(h->x, n, h->status, s));
    int flag = 0;
    CKF(cudaMemcpyAsync(&flag, h->status, 4, cudaMemcpyDeviceToHost, s));
    CKF(cudaStreamSynchronize(s));
    if (flag) {
        set_err("series contains NaN or Inf");
        return fail(DTWS_ENONFINITE);
    }
    CKF(launch_prefix(h->x, n, h->P1, h->P2, h->T1, h->T2, h->A, s));
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
        (o->ordering != DTWS_ORDER_PLAIN && o->ordering != DTWS_ORDER_LEARNED)) {
        set_err("option out of range");
        return DTWS_EINVAL;
    }
    if (o->ordering == DTWS_ORDER_LEARNED) {
        set_err("learned ordering is not available in this build");
        return DTWS_ENOTIMPL;
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
    cudaStream_t s = (cudaStream_t)stream;
    const bool qdev = is_device_ptr(Q), idev = is_device_ptr(out_idx), ddev = is_device_ptr(out_dist);
    const size_t qb = (size_t)m * 4, ib = (size_t)k * 8, db = (size_t)k * 4;
    if ((st = ensure_stage(h, 256 + round_up(qb, 256) + round_up(ib, 256) + round_up(db, 256))) != DTWS_OK)
        return st;
    char *sp = (char *)h->stage;
    const float *Qd = Q;
    if (!qdev) {
        CK(cudaMemcpyAsync(sp, Q, qb, cudaMemcpyHostToDevice, s));
        Qd = (const float *)sp;
    }
    int64_t *idx_d = idev ? out_idx : (int64_t *)(sp + round_up(qb, 256));
    float *dist_d = ddev ? out_dist : (float *)(sp + round_up(qb, 256) + round_up(ib, 256));
    if ((st = run_query(h, Qd, m, r, k, idx_d, dist_d, s)) != DTWS_OK) return st;
    if (!idev) CK(cudaMemcpyAsync(out_idx, idx_d, ib, cudaMemcpyDeviceToHost, s));
    if (!ddev) CK(cudaMemcpyAsync(out_dist, dist_d, db, cudaMemcpyDeviceToHost, s));
    if (!idev || !ddev) CK(cudaStreamSynchronize(s));
    return DTWS_OK;
}

dtws_status dtws_query_batch(dtws_t h, const float *Q_cat, const int64_t *q_off, const int32_t *m_arr,
                             const int32_t *r_arr, int32_t nq, int32_t k, int64_t *out_idx,
                             float *out_dist, void *stream) {
    if (!h || !Q_cat || !q_off || !m_arr || !r_arr || !out_idx || !out_dist || nq < 1) {
        set_err("null argument or nq < 1");
        return DTWS_EINVAL;
    }
    if (q_off[0] != 0) { set_err("q_off[0] != 0"); return DTWS_EINVAL; }
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
    for (int q = 0; q < nq; ++q) {
        st = run_query(h, Qd + q_off[q], m_arr[q], r_arr[q], k, idx_d + (int64_t)q * k,
                       dist_d + (int64_t)q * k, s);
        if (st != DTWS_OK) return st;
    }
    if (!idev) CK(cudaMemcpyAsync(out_idx, idx_d, ib, cudaMemcpyDeviceToHost, s));
    if (!ddev) CK(cudaMemcpyAsync(out_dist, dist_d, db, cudaMemcpyDeviceToHost, s));
    if (!idev || !ddev) CK(cudaStreamSynchronize(s));
    return DTWS_OK;
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
    CK(cudaMemcpy(&hs, h->st, sizeof hs, cudaMemcpyDeviceToHost));
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
        // k-th seed distance; k is not stored, report the smallest
        unsigned long long key = hs.seed_keys[0];
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
    for (auto &e : h->env) free_env(e);
    h->stats.clear();
    h->env.clear();
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
    if ((st = get_stats(h, m, s, &se, &c)) != DTWS_OK) return st;
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
