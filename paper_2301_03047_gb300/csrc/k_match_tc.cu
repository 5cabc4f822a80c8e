// BF16 tensor-core scorer for glr_match_topk (tcgen05.mma into TMEM, TMA-fed).
#include "glr_kernels.cuh"

namespace glr {

glr_status launch_match_tc(const float*, const glr_images&, const int32_t*, const int32_t*, int, const MatchPlan&,
                           char*, cudaStream_t) {
  return GLR_ENOTSUP;
}

}  // namespace glr
