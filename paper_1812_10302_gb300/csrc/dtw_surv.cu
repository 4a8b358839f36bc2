// dtw_surv.cu -- the survivor DTW stage of the search: the k_dtw kernel in
// survivor mode (Eq. 10 pre-check, then the banded DTW with early abandon).
#include "dtw_kernels.cuh"

namespace dtws {

cudaError_t launch_dtw_survivors(const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    return dtw_dispatch<kModeSurv>(b, a, nullptr, 0, nullptr, (int64_t)b.num_sms * 1024, s);
}

}  // namespace dtws
