// Certified FP32 policy (HD_MIXED): not built yet.
#include "hd_bnb.cuh"

namespace hd {
int run_mixed(const RunIO&) { return HD_ERR_INVALID; }
int nearest_points_mixed(const hd_bvh*, const void*, int, int64_t, cudaStream_t, double*, int32_t*, double*,
                         double*) {
  return HD_ERR_INVALID;
}
}  // namespace hd
