// Frontier-parallel branch and bound for h(A, B) (Sections 3.1 and 4), templated on the
// arithmetic policy (PolicyD: FP64; PolicyM: certified FP32).
//
// The paper pops one sub-triangle at a time from a priority queue.  Here a round works on
// the whole frontier at once:
//   select   every live item with U > l + eps is split (up to a chunk per round); items with
//            U < l are discarded, items with l <= U <= l + eps are retired (they can never
//            again make u - l exceed eps, so they are not refined; their U is kept in a max);
//   split    three midpoints per split item go to the vertex pool (Section 4: W_A), four
//            children (G_A) are implied by the parent's vertices and the midpoints;
//   query    nearest triangle of B for each new vertex, through the BVH (D, I, C);
//   raise l  atomic max of the new vertex distances (Section 3.1);
//   bound    UpperBound(child, l) for the four children of each split (Section 4) and
//            compaction of the survivors into the next frontier.
// The upper bound of a round is u = max(l, max U of retired items, max U of the frontier);
// the reported u is the minimum over rounds.  The run stops when the frontier is empty,
// i.e. when every item is discarded or retired, which is the paper's (u - l) <= eps.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>

#include "hd_internal.cuh"

namespace hd {

__device__ inline unsigned long long warp_sum(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Flush per-thread counters with one atomic per warp.  Every lane of the warp must call it.
__device__ inline void flush_counters(RunState* st, const Counters& c) {
  unsigned long long e = warp_sum(c.evals), b = warp_sum(c.boxes), lf = warp_sum(c.leaf),
                     x = warp_sum(c.escalations);
  if ((threadIdx.x & 31) == 0) {
    if (e + lf) atomicAdd(&st->evals, e + lf);
    if (lf) atomicAdd(&st->leaf_tests, lf);
    if (b) atomicAdd(&st->box_tests, b);
    if (x) atomicAdd(&st->escalations, x);
  }
  if (c.err) atomicExch(&st->err, 1);
}

// ----------------------------------------------------------------------------- round 0 helpers

// Referenced vertices of A (the paper assumes every vertex is referenced, Section 3; l and
// dA use only referenced ones, Section 5.3) and the validity of F_A.
static __global__ void k_mark_ref(const int32_t* FA, int64_t nFA, int64_t nVA, uint8_t* ref, int* bad) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 3 * nFA) return;
  int32_t v = FA[i];
  if (v < 0 || v >= nVA) atomicExch(bad, 1);
  else ref[v] = 1;
}

__device__ inline unsigned long long double_to_ordered(double d) {
  unsigned long long u = (unsigned long long)__double_as_longlong(d);
  return (u >> 63) ? ~u : (u | (1ull << 63));
}

// Finite coordinates everywhere, and the bounding box of the referenced vertices.
template <typename T>
static __global__ void k_check_bbox(const T* VA, int64_t nVA, const uint8_t* ref, unsigned long long* box, int* bad) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0, 0, 0};
  if (i < nVA) {
    double x = VA[3 * i], y = VA[3 * i + 1], z = VA[3 * i + 2];
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
      atomicExch(bad, 1);
    } else if (ref[i]) {
      lo[0] = hi[0] = double_to_ordered(x);
      lo[1] = hi[1] = double_to_ordered(y);
      lo[2] = hi[2] = double_to_ordered(z);
    }
  }
  // warp reduction first: one atomic per warp and bound instead of one per vertex
  for (int k = 0; k < 3; ++k)
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long a = __shfl_xor_sync(0xffffffffu, lo[k], o), b = __shfl_xor_sync(0xffffffffu, hi[k], o);
      lo[k] = a < lo[k] ? a : lo[k];
      hi[k] = b > hi[k] ? b : hi[k];
    }
  if ((threadIdx.x & 31) == 0 && hi[0] != 0) {
    for (int k = 0; k < 3; ++k) {
      atomicMin(&box[k], lo[k]);
      atomicMax(&box[3 + k], hi[k]);
    }
  }
}

template <class P, typename T>
__global__ void k_init_pool(const T* VA, int64_t nVA, const uint8_t* ref, typename P::Vtx* pool) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nVA) return;
  typename P::Vtx v;
  memset(&v, 0, sizeof v);
  P::set_pos(v, (double)VA[3 * i], (double)VA[3 * i + 1], (double)VA[3 * i + 2]);
  v.tri = ref[i] ? -2 : -1;
  v.hint = -1;
  pool[i] = v;
}

// Nearest-triangle queries for pool vertices [beg, beg + count); count = min(*count_ptr *
// mult, cap) when count_ptr is given (device-side counts), else `cap`.
template <class P>
__global__ void k_query(BvhDev B, typename P::Vtx* pool, int beg, const int* count_ptr, int mult, int cap,
                        RunState* st, double slack) {
  int count = cap;
  if (count_ptr) count = min(*count_ptr * mult, cap);
  Counters c;
  double lmax = 0.0;
  int nq = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;; t += (int64_t)gridDim.x * blockDim.x) {
    bool active = t < count;
    if (__all_sync(0xffffffffu, !active)) break;
    if (active) {
      typename P::Vtx v = pool[beg + t];
      if (v.tri != -1) {
        P::query(B, v, c);
        pool[beg + t] = v;
        lmax = fmax(lmax, P::lower(v) - slack);
        ++nq;
      }
    }
  }
  lmax = warp_max(lmax);
  unsigned long long q = warp_sum((unsigned long long)nq);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&st->l_bits, lmax);
    if (q) atomicAdd(&st->queries, q);
  }
  flush_counters(st, c);
}

// Discard / retire / keep one bounded item (Section 3.1: discard when U < l).
template <class P>
__device__ inline void classify(RunState* st, const typename P::Item& it, double l, double eps, int code,
                                typename P::Item* next, int next_cap) {
  double U = (double)it.U;
  if (U < l) {
    atomicAdd(&st->discards[code], 1ull);
  } else if (U <= __dadd_rd(l, eps)) {
    atomic_max_nonneg(&st->uret_bits, U);
    atomicAdd(&st->retired, 1ull);
  } else {
    int j = atomicAdd(&st->n_next, 1);
    if (j < next_cap) {
      next[j] = it;
      atomic_max_nonneg(&st->umax_bits, U);
    } else {
      atomicExch(&st->overflow, 1);
    }
  }
}

__device__ inline double load_l(const RunState* st) {
  return __longlong_as_double((long long)*(volatile unsigned long long*)&st->l_bits);
}

// Round 0: UpperBound for every face of A.
template <class P>
__global__ void k_bound_faces(BvhDev B, const typename P::Vtx* pool, const int32_t* FA, int64_t nFA, RunState* st,
                              RunParams rp, typename P::Item* next, int next_cap) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double l = load_l(st);
  Counters c;
  if (f < nFA) {
    typename P::Item it;
    it.v[0] = FA[3 * f];
    it.v[1] = FA[3 * f + 1];
    it.v[2] = FA[3 * f + 2];
    int code;
    it.U = P::upper_bound(B, pool[it.v[0]], pool[it.v[1]], pool[it.v[2]], l, rp, code, c);
    classify<P>(st, it, l, rp.eps, code, next, next_cap);
  }
  flush_counters(st, c);
}

// Select the items to split: discard (U < l), retire (U <= l + eps), split up to K of the
// rest (three midpoints each into the pool at mbase), carry the others over.
template <class P>
__global__ void k_select(const typename P::Item* front, int n_front, RunState* st, RunParams rp, int K,
                         int4* split_par, typename P::Vtx* pool, int mbase, typename P::Item* next, int next_cap) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_front) return;
  double l = load_l(st);
  typename P::Item it = front[i];
  double U = (double)it.U;
  if (U < l) {
    atomicAdd(&st->discards[5], 1ull);
    return;
  }
  if (U <= __dadd_rd(l, rp.eps)) {
    atomic_max_nonneg(&st->uret_bits, U);
    atomicAdd(&st->retired, 1ull);
    return;
  }
  int s = atomicAdd(&st->n_split, 1);
  if (s < K) {
    split_par[s] = make_int4(it.v[0], it.v[1], it.v[2], 0);
    typename P::Vtx a = pool[it.v[0]], b = pool[it.v[1]], c = pool[it.v[2]], m;
    P::midpoint(a, b, m);
    pool[mbase + 3 * s] = m;
    P::midpoint(b, c, m);
    pool[mbase + 3 * s + 1] = m;
    P::midpoint(c, a, m);
    pool[mbase + 3 * s + 2] = m;
  } else {
    int j = atomicAdd(&st->n_next, 1);
    if (j < next_cap) {
      next[j] = it;
      atomic_max_nonneg(&st->umax_bits, U);
    } else {
      atomicExch(&st->overflow, 1);
    }
  }
}

// The four children of every split (Section 4, midpoint subdivision):
// (v1, m12, m31), (m12, v2, m23), (m31, m23, v3), (m12, m23, m31).
template <class P>
__global__ void k_bound_children(BvhDev B, const typename P::Vtx* pool, const int4* split_par, int K, int mbase,
                                 RunState* st, RunParams rp, typename P::Item* next, int next_cap) {
  int S = min(*(volatile int*)&st->n_split, K);
  double l = load_l(st);
  Counters c;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;; t += (int64_t)gridDim.x * blockDim.x) {
    bool active = t < 4 * (int64_t)S;
    if (__all_sync(0xffffffffu, !active)) break;
    if (active) {
      int s = (int)(t >> 2), k = (int)(t & 3);
      int4 par = split_par[s];
      int m12 = mbase + 3 * s, m23 = m12 + 1, m31 = m12 + 2;
      typename P::Item it;
      if (k == 0) { it.v[0] = par.x; it.v[1] = m12; it.v[2] = m31; }
      else if (k == 1) { it.v[0] = m12; it.v[1] = par.y; it.v[2] = m23; }
      else if (k == 2) { it.v[0] = m31; it.v[1] = m23; it.v[2] = par.z; }
      else { it.v[0] = m12; it.v[1] = m23; it.v[2] = m31; }
      int code;
      it.U = P::upper_bound(B, pool[it.v[0]], pool[it.v[1]], pool[it.v[2]], l, rp, code, c);
      classify<P>(st, it, l, rp.eps, code, next, next_cap);
    }
  }
  flush_counters(st, c);
}

static __global__ void k_round_reset(RunState* st, int n_front) {
  st->n_front = n_front;
  st->n_next = 0;
  st->n_split = 0;
  st->umax_bits = 0;
  st->overflow = 0;
}

// Nearest queries for external points (hd_nearest): P as double rows.
template <class P>
__global__ void k_query_points(BvhDev B, typename P::Vtx* tmp, int64_t n, RunState* st) {
  Counters c;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;; t += (int64_t)gridDim.x * blockDim.x) {
    bool active = t < n;
    if (__all_sync(0xffffffffu, !active)) break;
    if (active) {
      typename P::Vtx v = tmp[t];
      P::query(B, v, c);
      tmp[t] = v;
    }
  }
  flush_counters(st, c);
}

// ----------------------------------------------------------------------------- host driver

struct RunIO {
  const hd_bvh* B;
  const void* VA;  // device
  int vtype;
  int64_t nVA;
  const int32_t* FA;  // device
  int64_t nFA;
  double tol;
  const Opts* o;
  cudaStream_t s;
  hd_result* out;
};

inline BvhDev bvh_dev(const hd_bvh* B) { return {B->nodes, B->tri32, B->tri64, B->tri_vid, B->nF, B->eta}; }

inline double bits_to_double(unsigned long long b) {
  double d;
  memcpy(&d, &b, 8);
  return d;
}

// Shared part of round 0 (validation, referenced vertices, dA) lives in hd_api.cu.
int prepare_A(const RunIO& io, uint8_t* ref, double* dA, double* amax);

template <class P>
int run_bnb(const RunIO& io) {
  using Vtx = typename P::Vtx;
  using Item = typename P::Item;
  const Opts& o = *io.o;
  cudaStream_t s = io.s;
  hd_result& res = *io.out;
  memset(&res, 0, sizeof res);

  uint8_t* ref = nullptr;
  HD_TRY(cudaMallocAsync((void**)&ref, std::max<int64_t>(io.nVA, 1), s));
  double dA = 0.0;
  double amax = 0.0;
  int rc = prepare_A(io, ref, &dA, &amax);
  if (rc != HD_OK) {
    cudaFreeAsync(ref, s);
    return rc;
  }
  const double eps = o.tol_mode == HD_TOL_REL ? io.tol * dA : io.tol;
  res.stats.dA = dA;
  res.stats.eps_abs = eps;

  // memory: vertex pool, two frontier buffers, split list
  int64_t budget = o.max_frontier_bytes > 0 ? o.max_frontier_bytes : (int64_t)2 << 30;
  int64_t pool_cap = std::max<int64_t>(io.nVA + 3, (int64_t)(0.6 * budget) / (int64_t)sizeof(Vtx));
  int64_t front_cap = std::max<int64_t>(io.nFA + 4, (int64_t)(0.15 * budget) / (int64_t)sizeof(Item));
  pool_cap = std::min<int64_t>(pool_cap, INT32_MAX / 2);
  front_cap = std::min<int64_t>(front_cap, INT32_MAX / 4);
  int64_t chunk = o.frontier_chunk > 0 ? o.frontier_chunk : std::max<int64_t>(front_cap / 4, 1024);
  chunk = std::min<int64_t>(chunk, front_cap);
  Vtx* pool = nullptr;
  Item* front[2] = {nullptr, nullptr};
  int4* split_par = nullptr;
  RunState* st = nullptr;
  HD_TRY(cudaMallocAsync((void**)&pool, sizeof(Vtx) * pool_cap, s));
  HD_TRY(cudaMallocAsync((void**)&front[0], sizeof(Item) * front_cap, s));
  HD_TRY(cudaMallocAsync((void**)&front[1], sizeof(Item) * front_cap, s));
  HD_TRY(cudaMallocAsync((void**)&split_par, sizeof(int4) * chunk, s));
  HD_TRY(cudaMallocAsync((void**)&st, sizeof(RunState), s));
  HD_TRY(cudaMemsetAsync(st, 0, sizeof(RunState), s));
  static thread_local RunState* hst = nullptr;  // pinned read-back buffer, kept for the thread's lifetime
  if (!hst) HD_TRY(cudaMallocHost((void**)&hst, sizeof(RunState)));

  BvhDev B = bvh_dev(io.B);
  RunParams rp;
  rp.eps = eps;
  rp.slack = P::slack(amax);
  memcpy(rp.order, o.order, 4);
  rp.n_bounds = o.n_bounds;
  const int bs = o.block_size;
  int dev_sms = 152;
  {
    int dev;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const unsigned max_grid = (unsigned)dev_sms * 16;

  // round 0: vertices of A, their nearest triangles, l, and the bounds of every face
  {
    TraceScope tr(HD_K_PREP, s);
    if (io.vtype == HD_F64)
      k_init_pool<P, double><<<blocks_for(io.nVA, 256), 256, 0, s>>>((const double*)io.VA, io.nVA, ref, pool);
    else
      k_init_pool<P, float><<<blocks_for(io.nVA, 256), 256, 0, s>>>((const float*)io.VA, io.nVA, ref, pool);
  }
  HD_TRY_LAUNCH();
  {
    TraceScope tr(HD_K_QUERY, s);
    k_query<P><<<std::min(blocks_for(io.nVA, bs), max_grid), bs, 0, s>>>(B, pool, 0, nullptr, 1, (int)io.nVA, st,
                                                                       rp.slack);
  }
  HD_TRY_LAUNCH();
  {
    TraceScope tr(HD_K_BOUND, s);
    k_bound_faces<P><<<blocks_for(io.nFA, bs), bs, 0, s>>>(B, pool, io.FA, io.nFA, st, rp, front[1], (int)front_cap);
  }
  HD_TRY_LAUNCH();
  HD_TRY(cudaMemcpyAsync(hst, st, sizeof(RunState), cudaMemcpyDeviceToHost, s));
  HD_TRY(cudaStreamSynchronize(s));

  int cur = 1;
  int64_t n_front = hst->n_next, n_pool = io.nVA, splits = 0, rounds = 0, peak = n_front;
  double l = bits_to_double(hst->l_bits);
  double u_run = std::max(l, std::max(bits_to_double(hst->uret_bits), n_front ? bits_to_double(hst->umax_bits) : 0.0));
  const double face_cap = o.max_face_factor * (double)io.nFA;
  int status = HD_OK;
  if (hst->overflow) status = HD_ERR_CAPACITY;

  while (status == HD_OK && n_front > 0) {
    if (rounds >= o.max_rounds) {
      status = HD_ERR_TIMEOUT;
      break;
    }
    int64_t K = std::min<int64_t>(chunk, (pool_cap - n_pool) / 3);
    K = std::min<int64_t>(K, (front_cap - n_front) / 3);
    double cap_left = std::floor((face_cap - (double)io.nFA) / 4.0) - (double)splits;
    K = std::min<int64_t>(K, (int64_t)std::max(0.0, std::min(cap_left, 9.0e18)));
    if (K <= 0) {
      status = HD_ERR_CAPACITY;
      break;
    }
    {
      TraceScope tr(HD_K_SELECT, s);
      k_round_reset<<<1, 1, 0, s>>>(st, (int)n_front);
      k_select<P><<<blocks_for(n_front, 256), 256, 0, s>>>(front[cur], (int)n_front, st, rp, (int)K, split_par,
                                                           pool, (int)n_pool, front[cur ^ 1], (int)front_cap);
    }
    {
      TraceScope tr(HD_K_QUERY, s);
      unsigned gq = std::min(blocks_for(3 * K, bs), max_grid);
      k_query<P><<<gq, bs, 0, s>>>(B, pool, (int)n_pool, &st->n_split, 3, (int)(3 * K), st, rp.slack);
    }
    {
      TraceScope tr(HD_K_BOUND, s);
      unsigned gb = std::min(blocks_for(4 * K, bs), max_grid);
      k_bound_children<P><<<gb, bs, 0, s>>>(B, pool, split_par, (int)K, (int)n_pool, st, rp, front[cur ^ 1],
                                            (int)front_cap);
    }
    HD_TRY_LAUNCH();
    HD_TRY(cudaMemcpyAsync(hst, st, sizeof(RunState), cudaMemcpyDeviceToHost, s));
    HD_TRY(cudaStreamSynchronize(s));
    int64_t S = std::min<int64_t>(hst->n_split, K);
    ++rounds;
    splits += S;
    n_pool += 3 * S;
    cur ^= 1;
    n_front = hst->n_next;
    peak = std::max(peak, n_front);
    l = bits_to_double(hst->l_bits);
    double u_round = std::max(l, std::max(bits_to_double(hst->uret_bits), n_front ? bits_to_double(hst->umax_bits) : 0.0));
    u_run = std::min(u_run, u_round);
    if (hst->overflow) status = HD_ERR_CAPACITY;
    if (hst->err) status = HD_ERR_NUMERIC;
  }

  l = bits_to_double(hst->l_bits);
  double uret = bits_to_double(hst->uret_bits);
  if (status == HD_OK) {
    // frontier empty: everything was discarded or retired
    u_run = std::min(u_run, std::max(l, uret));
    if (uret < l && hst->retired == 0 && P::kFp64) status = HD_ERR_NUMERIC;
  }
  res.lower = l;
  res.upper = std::max(l, u_run);
  res.status = status;
  hd_stats& S = res.stats;
  S.rounds = rounds;
  S.splits = splits;
  S.queries = (int64_t)hst->queries;
  S.pointtri_evals = (int64_t)hst->evals;
  S.leaf_tests = (int64_t)hst->leaf_tests;
  S.box_tests = (int64_t)hst->box_tests;
  for (int k = 0; k < 6; ++k) S.discards[k] = (int64_t)hst->discards[k];
  S.retired = (int64_t)hst->retired;
  S.fp64_escalations = (int64_t)hst->escalations;
  S.peak_frontier = peak;
  S.pool_vertices = n_pool;

  cudaFreeAsync(pool, s);
  cudaFreeAsync(front[0], s);
  cudaFreeAsync(front[1], s);
  cudaFreeAsync(split_par, s);
  cudaFreeAsync(st, s);
  cudaFreeAsync(ref, s);
  return HD_OK;
}

// ----------------------------------------------------------------------------- point queries

template <class P, typename T>
__global__ void k_points_in(const T* P_, int64_t n, typename P::Vtx* v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  typename P::Vtx x;
  memset(&x, 0, sizeof x);
  P::set_pos(x, (double)P_[3 * i], (double)P_[3 * i + 1], (double)P_[3 * i + 2]);
  x.tri = -2;
  x.hint = -1;
  v[i] = x;
}

template <class P>
__global__ void k_points_out(const typename P::Vtx* v, int64_t n, const int4* tri_vid, double* dist, int32_t* idx,
                             double* foot, double* dlo) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  typename P::Vtx x = v[i];
  dist[i] = P::out_dist(x);
  idx[i] = x.tri >= 0 ? tri_vid[x.tri].w : -1;
  D3 f = P::out_foot(x);
  foot[3 * i] = f.x;
  foot[3 * i + 1] = f.y;
  foot[3 * i + 2] = f.z;
  if (dlo) dlo[i] = P::out_dlo(x);
}

// hd_nearest: nearest triangle of B for n external points (P as float or double rows).
template <class P>
int nearest_points(const hd_bvh* B, const void* Pts, int ptype, int64_t n, cudaStream_t s, double* dist,
                   int32_t* idx, double* foot, double* dlo) {
  typename P::Vtx* tmp = nullptr;
  RunState* st = nullptr;
  HD_TRY(cudaMallocAsync((void**)&tmp, sizeof(typename P::Vtx) * n, s));
  HD_TRY(cudaMallocAsync((void**)&st, sizeof(RunState), s));
  HD_TRY(cudaMemsetAsync(st, 0, sizeof(RunState), s));
  if (ptype == HD_F64)
    k_points_in<P, double><<<blocks_for(n, 256), 256, 0, s>>>((const double*)Pts, n, tmp);
  else
    k_points_in<P, float><<<blocks_for(n, 256), 256, 0, s>>>((const float*)Pts, n, tmp);
  {
    TraceScope tr(HD_K_QUERY, s);
    k_query_points<P><<<std::min(blocks_for(n, 128), 152u * 16u), 128, 0, s>>>(bvh_dev(B), tmp, n, st);
  }
  k_points_out<P><<<blocks_for(n, 256), 256, 0, s>>>(tmp, n, B->tri_vid, dist, idx, foot, dlo);
  HD_TRY_LAUNCH();
  HD_TRY(cudaFreeAsync(tmp, s));
  HD_TRY(cudaFreeAsync(st, s));
  return HD_OK;
}

}  // namespace hd
