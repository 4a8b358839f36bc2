// dtw_pool.cu -- the persistent survivor-DTW stage of dtws_query_batch.
//
// Each query of a batch runs its query preparation, seeding, lower-bound
// scan and survivor ordering on its lane as before; then its ordered
// survivors, with their window statistics, are copied to one pool for the
// whole batch (k_defer_*), so that the lane's statistics slot and survivor
// buffers can serve its next query.  When every lane has done that, one
// persistent launch per kernel shape (k_dtw_pool) runs the survivor DTW of
// all the batch's queries of that shape, query after query, pulling each
// query's survivors from its own cursor; the final stage then runs per query
// on the lanes again.  A query whose survivors do not fit in the pool keeps
// them and runs its survivor pass on its lane, as a single query does.
#include "dtw_kernels.cuh"

namespace dtws {

namespace {

// Reserve the query's run of the pool (one thread): st->deferred = 1 and
// st->pool_off, or 0 when the pool is full (its survivor pass runs on the
// lane then) or nothing is left to score.
__global__ void k_defer_reserve(QueryState *st, unsigned long long *cursor, long long cap) {
    st->deferred = 0;
    const long long n = st->n_cand;
    if (!st->valid || n <= 0) return;
    const unsigned long long off = atomicAdd(cursor, (unsigned long long)n);
    if ((long long)off + n <= cap) {
        st->pool_off = (long long)off;
        st->deferred = 1;
    }
}

// Copy the ordered survivors and gather their statistics into the run.
__global__ void k_defer_copy(QueryBufs b, SurvPool p) {
    const QueryState *st = b.st;
    if (!st->deferred) return;
    const long long n = st->n_cand, off = st->pool_off;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const unsigned idx = b.sort_idx[c];
        const float is = b.inv_sigma[idx];
        p.idx[off + c] = idx;
        p.lb[off + c] = b.sort_lb[c];
        p.mh[off + c] = b.mu_hi[idx];
        p.is[off + c] = is;
        p.ls[off + c] = b.mu_lo[idx] * is;
    }
}

template <int L, int K>
cudaError_t pool_launch(const QueryBufs &base, const PoolQuery *pq, const int *list, int nlist, int m_max, int r_max,
                        cudaStream_t s) {
    DtwPlan p;
    if (!plan_fits<float, L, K>(m_max, r_max, true, &p)) return cudaErrorInvalidValue;
    int per_sm = 0;
    cudaError_t e = cudaFuncSetAttribute(k_dtw_pool<L, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dtw_pool<L, K>, p.warps * 32, p.smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_dtw_pool<L, K><<<base.num_sms * per_sm, p.warps * 32, p.smem, s>>>(base, pq, list, nlist, p.staged);
    return cudaGetLastError();
}

}  // namespace

bool pool_shape(int r, int *L, int *K) {
    if (r > kDiagRMax) return false;
    diag_shape_f32(r, L, K);
    return *K > 0;
}

cudaError_t launch_dtw_pool(const QueryBufs &base_in, const SurvPool &pool, const PoolQuery *pq, const int *list,
                            int nlist, int L, int K, int m_max, int r_max, cudaStream_t s) {
    QueryBufs base = base_in;
    base.sort_idx = pool.idx;
    base.sort_lb = pool.lb;
    base.surv_mh = pool.mh;
    base.surv_is = pool.is;
    base.surv_ls = pool.ls;
#define DTWS_CASE(LL, KK) \
    if (L == LL && K == KK) return pool_launch<LL, KK>(base, pq, list, nlist, m_max, r_max, s);
    DTWS_CASE(1, 1) DTWS_CASE(2, 1) DTWS_CASE(4, 1) DTWS_CASE(8, 1) DTWS_CASE(16, 1)
    DTWS_CASE(4, 2) DTWS_CASE(8, 2) DTWS_CASE(16, 2) DTWS_CASE(8, 4) DTWS_CASE(16, 4)
    DTWS_CASE(32, 1) DTWS_CASE(32, 2) DTWS_CASE(32, 3) DTWS_CASE(32, 4) DTWS_CASE(32, 6) DTWS_CASE(32, 8)
    DTWS_CASE(32, 10) DTWS_CASE(32, 12) DTWS_CASE(32, 16)
#undef DTWS_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_defer(const QueryBufs &b, const SurvPool &pool, cudaStream_t s) {
    k_defer_reserve<<<1, 1, 0, s>>>(b.st, pool.cursor, pool.cap);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_defer_copy<<<b.num_sms * 4, 256, 0, s>>>(b, pool);
    return cudaGetLastError();
}

}  // namespace dtws
