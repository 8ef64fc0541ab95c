// Instantiation of the frontier rounds and point queries for the certified FP32 policy.
#include "hd_batch.cuh"
#include "hd_bnb.cuh"
#include "hd_mixed.cuh"

namespace hd {

int run_mixed(const RunIO& io) { return run_bnb<PolicyM>(io); }

int run_batch_mixed(const hd_bvh* const* Bs, const hd_mesh* As, int64_t npairs, double tol, const Opts& o,
                    cudaStream_t s, hd_result* outs, std::vector<int64_t>* redo) {
  return run_batch<PolicyM>(Bs, As, npairs, tol, o, s, outs, redo);
}

int nearest_points_mixed(const hd_bvh* B, const void* Pts, int ptype, int64_t n, cudaStream_t s, double* dist,
                         int32_t* idx, double* foot, double* dlo) {
  return nearest_points<PolicyM>(B, Pts, ptype, n, s, dist, idx, foot, dlo);
}

// UpperBound(T, l) in the certified FP32 arithmetic of the rounds, for triangles given in
// double (hd_upper_bounds with HD_MIXED): each vertex becomes a float pair, its distance is
// rounded up, its closest point is kept relative to it with the rounding of that offset as the
// error radius, and every bound of the cascade (u4 included) is evaluated in place.
__global__ void k_upper_bounds_m(BvhDev B, const int* inv, const double* T, const double* Td, const int32_t* TI,
                                 const double* Tq, int64_t n, double l, RunParams rp, double* U, int32_t* code) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  VM t[3];
  double amax = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double* v = T + 9 * i + 3 * k;
    const double* q = Tq + 9 * i + 3 * k;
    const int I = TI[3 * i + k];
    if (I < 0 || I >= B.nF) {  // not a triangle of B: no bound
      U[i] = NAN;
      code[i] = -1;
      return;
    }
    const F3 h = {__double2float_rn(v[0]), __double2float_rn(v[1]), __double2float_rn(v[2])};
    const F3 lo = {__double2float_rn(v[0] - (double)h.x), __double2float_rn(v[1] - (double)h.y),
                   __double2float_rn(v[2] - (double)h.z)};
    // the closest point relative to the float pair, and the rounding of that offset
    const double ox = q[0] - ((double)h.x + (double)lo.x), oy = q[1] - ((double)h.y + (double)lo.y),
                 oz = q[2] - ((double)h.z + (double)lo.z);
    const F3 o = {__double2float_rn(ox), __double2float_rn(oy), __double2float_rn(oz)};
    const double r = sqrt((ox - o.x) * (ox - o.x) + (oy - o.y) * (oy - o.y) + (oz - o.z) * (oz - o.z));
    const double big = fmax(fmax(fabs(q[0]), fabs(q[1])), fmax(fabs(q[2]), fmax(fmax(fabs(v[0]), fabs(v[1])), fabs(v[2]))));
    t[k] = {{h, lo}, __double2float_ru(Td[3 * i + k]), inv[I], o, __double2float_ru(r + 1e-15 * big)};
    amax = fmax(amax, big);
  }
  // the float pairs stand for the vertices within 2^-48 of their magnitude
  rp.slack = ldexp(amax, -40);  // as the rounds take it (PolicyM::slack)
  rp.slack_f = __double2float_ru(rp.slack);
  Counters cnt;
  int c;
  const float u = upper_bound_m(B, t, __double2float_rd(l), rp, c, cnt);
  U[i] = (double)u;
  code[i] = c;
}

int upper_bounds_mixed(const hd_bvh* B, const double* T, const double* Td, const int32_t* TI, const double* Tq,
                       int64_t n, double l, const RunParams& rp, cudaStream_t s, double* U, int32_t* code) {
  k_upper_bounds_m<<<blocks_for(n, 128), 128, 0, s>>>(bvh_dev(B), B->inv, T, Td, TI, Tq, n, l, rp, U, code);
  HD_TRY_LAUNCH();
  return HD_OK;
}

}  // namespace hd
