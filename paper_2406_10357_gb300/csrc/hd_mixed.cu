// Instantiation of the frontier rounds and point queries for the certified FP32 policy.
#include "hd_bnb.cuh"
#include "hd_mixed.cuh"

namespace hd {

int run_mixed(const RunIO& io) { return run_bnb<PolicyM>(io); }

int nearest_points_mixed(const hd_bvh* B, const void* Pts, int ptype, int64_t n, cudaStream_t s, double* dist,
                         int32_t* idx, double* foot, double* dlo) {
  return nearest_points<PolicyM>(B, Pts, ptype, n, s, dist, idx, foot, dlo);
}

}  // namespace hd
