// dtw_seed.cu -- exact FP32 DTW of the seed windows (k > 1), the k_dtw
// kernel in seed mode.
#include "dtw_kernels.cuh"

namespace dtws {

cudaError_t launch_dtw_seeds(const QueryBufs &b, const QueryArgs &a, cudaStream_t s) {
    return dtw_dispatch<kModeSeed>(b, a, nullptr, 0, nullptr, kSeedMax, s);
}

}  // namespace dtws
