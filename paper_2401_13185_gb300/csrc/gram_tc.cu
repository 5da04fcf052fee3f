// gram_tc.cu -- tcgen05 tensor-core contraction (split FP16 precision).
#include "cvx_internal.cuh"

namespace cvx {

cudaError_t gram_tc(const cv_plan_s *, const void *, int64_t, const void *, int64_t, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace cvx
