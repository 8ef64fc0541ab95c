// Frontier-parallel branch and bound for h(A, B) (Sections 3.1 and 4), templated on the
// arithmetic policy (PolicyD: FP64; PolicyM: certified FP32).
//
// The paper pops one sub-triangle at a time from a priority queue.  Here a round works on
// the whole frontier at once:
//   select   every live item with U > l + eps is split (up to a chunk per round); items with
//            U < l are discarded, items with l <= U <= l + eps are retired (they can never
//            again make u - l exceed eps, so they are not refined; their U is kept in a max);
//   split    the midpoints of each split item's three edges go to the vertex pool (Section 4:
//            W_A) -- optionally one per edge where two split neighbours share it (a hash
//            table of the round's edges); four children (G_A) are implied by the parent's
//            vertices and the midpoints;
//   query    nearest triangle of B for each new vertex, through the BVH (D, I, C);
//   raise l  atomic max of the new vertex distances (Section 3.1);
//   bound    UpperBound(child, l) for the four children of each split (Section 4) and
//            compaction of the survivors into the next frontier.
// The upper bound of a round is u = max(l, max U of retired items, max U of the frontier);
// the reported u is the minimum over rounds.  The run stops when the frontier is empty,
// i.e. when every item is discarded or retired, which is the paper's (u - l) <= eps.
#pragma once

#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "hd_fp64.cuh"
#include "hd_internal.cuh"

// Register caps of the lane traversal and of the UpperBound kernels (the policy's
// kBoundRegs): more resident warps pay for a few values spilled to L1 in these latency-bound
// kernels.
#ifndef HD_QUERY_REGS
#define HD_QUERY_REGS __maxnreg__(128)
#endif
#ifndef HD_BOUND_REGS
#define HD_BOUND_REGS __maxnreg__((bound_regs<P, kPaper>()))
#endif

namespace hd {

template <class P, bool kPaper>
constexpr int bound_regs() {
  if constexpr (kPaper) return P::kPaperRegs;
  else return P::kBoundRegs;
}

__device__ inline unsigned long long warp_sum(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// The next batch of 32 consecutive items for the calling warp (every lane must call it):
// warps of a persistent grid take batches until `count` is reached, so the grid's last
// wave is not left to a few blocks.
__device__ inline int warp_batch(int* counter) {
  int base = 0;
  if ((threadIdx.x & 31) == 0) base = atomicAdd(counter, 32);
  return __shfl_sync(0xffffffffu, base, 0);
}

// Flush per-thread counters with one atomic per warp.  Every lane of the warp must call it.
// The cooperative traversal (long_pass) also counts its node fetches and leaf tests apart.
__device__ inline void flush_counters(RunState* st, const Counters& c, bool long_pass = false) {
  unsigned long long e = warp_sum((unsigned long long)c.evals), b = warp_sum((unsigned long long)c.boxes),
                     lf = warp_sum((unsigned long long)c.leaf), x = warp_sum((unsigned long long)c.escalations),
                     nd = warp_sum((unsigned long long)c.nodes);
  if ((threadIdx.x & 31) == 0) {
    if (e + lf) atomicAdd(&st->evals, e + lf);
    if (lf) atomicAdd(&st->leaf_tests, lf);
    if (b) atomicAdd(&st->box_tests, b);
    if (x) atomicAdd(&st->escalations, x);
    if (nd) atomicAdd(&st->node_visits, nd);
    if (long_pass && nd) atomicAdd(&st->long_node_visits, nd);
    if (long_pass && lf) atomicAdd(&st->long_leaf_tests, lf);
  }
  if (c.err) atomicExch(&st->err, 1);
}

// ----------------------------------------------------------------------------- round 0 helpers

// Referenced vertices of A (the paper assumes every vertex is referenced, Section 3; l and
// dA use only referenced ones, Section 5.3), the validity of F_A, and the largest squared
// edge length of A's faces (for cut_radius; as the bits of a non-negative double, one
// atomic per block that raises it), with `ev` the longest edge at each vertex.  Entry
// i = 3 f + k is the edge from corner k of face f to corner k + 1.  Launched with 256 threads
// per block on a grid-stride loop (a bounded grid, so that few blocks contend for the edge
// maximum).
template <typename T>
__global__ void k_mark_ref(const int32_t* FA, int64_t nFA, int64_t nVA, uint8_t* ref, int* bad, const T* VA,
                           unsigned long long* e2max_bits, unsigned* ev) {
  grid_dep_wait();
  grid_dep_launch();
  T e2t = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * nFA; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = FA[i];
    if (v < 0 || v >= nVA) {
      atomicExch(bad, 1);
      continue;
    }
    ref[v] = 1;
#if HD_CUT_EDGE
    const int64_t f = i / 3;
    const int k = (int)(i - 3 * f);
    const int32_t w = FA[3 * f + (k == 2 ? 0 : k + 1)], u = FA[3 * f + (k == 0 ? 2 : k - 1)];
    // in the input's precision (FP64 runs at a small fraction of the FP32 rate on GB300):
    // float rounding of a float edge is ~2^-23 relative, covered by the margins k_prep_finish
    // and cut_r add
    const T vx = VA[3 * (int64_t)v], vy = VA[3 * (int64_t)v + 1], vz = VA[3 * (int64_t)v + 2];
    T xw = 0, xu = 0;  // the squared edges at this corner: to the next corner and the previous
    if (w >= 0 && w < nVA) {
      const T dx = VA[3 * (int64_t)w] - vx, dy = VA[3 * (int64_t)w + 1] - vy, dz = VA[3 * (int64_t)w + 2] - vz;
      xw = dx * dx + dy * dy + dz * dz;
      if (xw > e2t) e2t = xw;  // each edge once; NaN (invalid input, flagged elsewhere) is dropped
    }
    if (ev && u >= 0 && u < nVA) {
      const T dx = VA[3 * (int64_t)u] - vx, dy = VA[3 * (int64_t)u + 1] - vy, dz = VA[3 * (int64_t)u + 2] - vz;
      xu = dx * dx + dy * dy + dz * dz;
    }
    const T x = xw > xu ? xw : xu;
    if (ev && x > T(0)) {  // the longest edge at v (float bits: non-negative floats order as unsigned)
      float e;
      if constexpr (std::is_same<T, float>::value)
        e = sqrtf(x);
      else
        e = __double2float_ru(sqrt(x));
      atomicMax(&ev[v], __float_as_uint(e));
    }
#endif
  }
  double e2 = (double)e2t;
  for (int o = 16; o > 0; o >>= 1) e2 = fmax(e2, __shfl_xor_sync(0xffffffffu, e2, o));
  __shared__ double part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = e2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, part[k]);
    const unsigned long long b = (unsigned long long)__double_as_longlong(m);
    if (m > 0.0 && b > *(volatile unsigned long long*)e2max_bits) atomicMax(e2max_bits, b);
  }
}

__device__ inline unsigned long long double_to_ordered(double d) {
  unsigned long long u = (unsigned long long)__double_as_longlong(d);
  return (u >> 63) ? ~u : (u | (1ull << 63));
}

// Finite coordinates everywhere, the bounding box of the referenced vertices, and the pool
// entries of A's vertices (round 0).  The box is kept as six maxima of ordered bits -- the
// minima as complements -- so that a zero-filled block is its starting value; one atomic
// per block and bound.  Launched with 256 threads per block.
template <class P, typename T>
__global__ void k_check_init(const T* VA, int64_t nVA, const uint8_t* ref, unsigned long long* box, int* bad,
                             typename P::Vtx* pool, const unsigned* ev) {
  grid_dep_wait();
  grid_dep_launch();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long m[6] = {0, 0, 0, 0, 0, 0};  // ~lo xyz, hi xyz
  if (i < nVA) {
    T x = VA[3 * i], y = VA[3 * i + 1], z = VA[3 * i + 2];
    const bool used = ref[i] != 0;
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
      atomicExch(bad, 1);
      x = y = z = 0;
    } else if (used) {
      m[3] = double_to_ordered(x);
      m[4] = double_to_ordered(y);
      m[5] = double_to_ordered(z);
      m[0] = ~m[3];
      m[1] = ~m[4];
      m[2] = ~m[5];
    }
    typename P::Vtx v;
    memset(&v, 0, sizeof v);
    if constexpr (std::is_same<T, float>::value)
      P::set_pos_f(v, x, y, z);
    else
      P::set_pos(v, x, y, z);
    v.tri = used ? -2 : -1;
    v.hint = -1;
    if (ev) P::set_edge(v, __uint_as_float(ev[i]));
    pool[i] = v;
  }
  __shared__ unsigned long long part[6][8];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long a = __shfl_xor_sync(0xffffffffu, m[k], o);
      m[k] = a > m[k] ? a : m[k];
    }
    if (lane == 0) part[k][w] = m[k];
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    unsigned long long r = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = part[threadIdx.x][k] > r ? part[threadIdx.x][k] : r;
    if (r) atomicMax(&box[threadIdx.x], r);
  }
}

__device__ inline double ordered_to_double(unsigned long long u) {
  u = (u >> 63) ? (u & ~(1ull << 63)) : ~u;
  return __longlong_as_double((long long)u);
}

// dA, eps and the slack from A's bounding box, on the device (one thread).
static __global__ void k_prep_finish(unsigned long long* box, double tol, int tol_rel, double slack_scale,
                                     DynParams* dyn, RunState* st, double l0, const float* b_meta, int cut) {
  grid_dep_wait();
  grid_dep_launch();
  // B's validity flag (from its build) joins A's in the flag word the host reads with round 0
  if (__float_as_uint(b_meta[1]) != 0u) ((unsigned*)(box + 6))[1] = 1u;
  if (l0 > 0.0) st->l_bits = (unsigned long long)__double_as_longlong(l0);  // warm start of l
  double v[6];
  for (int k = 0; k < 6; ++k) v[k] = ordered_to_double(k < 3 ? ~box[k] : box[k]);
  double dx = v[3] - v[0], dy = v[4] - v[1], dz = v[5] - v[2];
  double dA = sqrt(dx * dx + dy * dy + dz * dz);
  double amax = 0.0;
  for (int k = 0; k < 6; ++k) amax = fmax(amax, fabs(v[k]));
  double slack = slack_scale * amax;
  dyn->dA = dA;
  dyn->eps = tol_rel ? tol * dA : tol;
  dyn->slack = slack;
  dyn->slack_f = __double2float_ru(slack);
  dyn->pad = 0;
  // the longest edge of A, with a relative margin above the rounding of any edge length the
  // cascade computes (sub-triangle edges are about half their parent's)
  dyn->emax = cut && HD_CUT_EDGE ? sqrt(__longlong_as_double((long long)box[7])) * (1.0 + 0x1p-20) : INFINITY;
}

// The round's table of split edges (Section 4's midpoint subdivision, with the midpoint of an
// edge shared by two split sub-triangles made once): open addressing on the key
// (the edge's two pool indices, smaller first, under a set top bit); val = pool slot + 1 once
// published; qhash[slot] = the entry a slot came from (-1: none), so that the query of that
// midpoint clears the entry for the next round.  Key and val are all zero between rounds.
// A null key pointer: midpoints are not shared (three per split, at 3 s + e).
struct MidTable {
  unsigned long long* key;
  int* val;
  int* qhash;
  unsigned mask;  // entries - 1 (a power of two)
};

// A slot in a device-side list for each calling lane: one atomic per warp (the lanes that
// reach the call together share it).
__device__ inline int warp_slot(int* counter) {
  namespace cg = cooperative_groups;
  cg::coalesced_group g = cg::coalesced_threads();
  int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(counter, (int)g.size());
  return g.shfl(base, 0) + (int)g.thread_rank();
}

// The queries a launch of k_query hands to k_query_long: pool indices, with room for as many
// as the launch has queries.  A null list: every lane finishes its own query.  With `sorted`
// and `buckets` (kSortBuckets counters, zero between launches), a list of at least
// kSortMin queries is reordered along a Morton curve of the query points before the
// cooperative pass (k_long_hist, k_long_scan, k_long_scatter), so that queries taken one
// after another share the nodes and triangles near them in L1 and L2.
struct LongList {
  int* idx;
  int cap;
  int* sorted = nullptr;
  unsigned* buckets = nullptr;
};

constexpr int kSortBits = 5;                           // Morton bits per axis of the reordering
constexpr int kSortBuckets = 1 << (3 * kSortBits);     // 32768 cells of B's bounding box
constexpr int kSortMin = 2048;                         // shorter lists keep their order
#ifndef HD_LONG_CHUNK
#define HD_LONG_CHUNK 4
#endif
constexpr int kLongChunk = HD_LONG_CHUNK;              // consecutive sorted queries per warp step
#ifndef HD_LONG_LPT
#define HD_LONG_LPT 1  // with cuts: the costly handed-off queries first, largest distance first (long_cell)
#endif

__device__ inline unsigned spread5(unsigned x) {  // bits 0..4 of x to bits 0, 3, 6, 9, 12
  x &= 31u;
  x = (x | (x << 8)) & 0x0000f00fu;
  x = (x | (x << 4)) & 0x000c30c3u;
  x = (x | (x << 2)) & 0x00249249u;
  return x;
}

// Morton cell of point p in B's bounding box (the union of the root's child boxes).
__device__ inline unsigned long_bucket(const BvhDev& B, float px, float py, float pz) {
  const float4* np = reinterpret_cast<const float4*>(B.nodes);
  const float4 lx = __ldg(np), ly = __ldg(np + 1), lz = __ldg(np + 2);
  const float4 hx = __ldg(np + 3), hy = __ldg(np + 4), hz = __ldg(np + 5);
  const float lo[3] = {fminf(fminf(lx.x, lx.y), fminf(lx.z, lx.w)), fminf(fminf(ly.x, ly.y), fminf(ly.z, ly.w)),
                       fminf(fminf(lz.x, lz.y), fminf(lz.z, lz.w))};
  const float hi[3] = {fmaxf(fmaxf(hx.x, hx.y), fmaxf(hx.z, hx.w)), fmaxf(fmaxf(hy.x, hy.y), fmaxf(hy.z, hy.w)),
                       fmaxf(fmaxf(hz.x, hz.y), fmaxf(hz.z, hz.w))};
  const float p[3] = {px, py, pz};
  unsigned q[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float ext = hi[k] - lo[k];
    const float u = ext > 0.f ? (p[k] - lo[k]) * ((float)(1 << kSortBits) / ext) : 0.f;
    q[k] = (unsigned)fminf(fmaxf(u, 0.f), (float)((1 << kSortBits) - 1));  // NaN -> 0
  }
  return (spread5(q[0]) << 2) | (spread5(q[1]) << 1) | spread5(q[2]);
}

// Nearest-triangle queries for pool vertices [beg, beg + count); count = min(*count_ptr *
// mult, cap) when count_ptr is given (device-side counts), else `cap`.  Warps take batches of
// 32 consecutive vertices, one per lane, each lane traversing on its own (the while-while
// traversal).  With a list, a lane whose traversal tests more than kLongBudget triangles
// stops and hands its query to k_query_long, which runs next and counts it.  Registers are
// capped at 128 (a few spilled to L1), for 8 resident blocks of 64 threads per SM.
#ifndef HD_QUERY_SEGMENTS
#define HD_QUERY_SEGMENTS 8
#endif
constexpr int kQuerySegments = HD_QUERY_SEGMENTS;

template <class P>
__device__ inline void query_body(BvhDev B, typename P::Vtx* pool, int beg, const int* count_ptr, int mult, int cap,
                        RunState* st, double slack_in, const DynParams* dyn, bool round_midpoints, MidTable tab,
                        LongList ll) {
  int count = cap;
  if (round_midpoints) {
    // the midpoints made by this frontier round, from the pool size at its start
    if (st->stop) return;  // the loop ended before this round (uniform over the grid)
    beg = st->n_pool;
    count = st->share_mid ? st->n_mid : 3 * min(st->n_split, st->K);
  } else if (count_ptr) {
    count = min(*count_ptr * mult, cap);
  }
  const double slack = dyn ? dyn->slack : slack_in;
  const bool cutting = HD_CUT_LANE && cut_on(dyn);
  // With cuts, the batches of 32 are taken from kQuerySegments interleaved parts of the
  // list, so that vertices from every part of A (the far ones among them) raise l early and
  // the queries after them cut sooner; each part is still taken in order.
  const int nb = (count + 31) >> 5, segs = cutting ? kQuerySegments : 1, per = (nb + segs - 1) / segs;
  Counters c;
  double lmax = 0.0;
  int nq = 0, ncut = 0;
  for (;;) {
    const int b = warp_batch(&st->q_next) >> 5;
    if (b >= segs * per) break;
    const int base = ((b % segs) * per + b / segs) << 5;
    if (base >= count) continue;
    const double lnow = cutting ? read_lower(st) : 0.0;
    const int t = base + (threadIdx.x & 31);
    bool active = t < count;
    // every lane of the warp enters the query (the MIXED traversal votes across the warp);
    // lanes without a vertex to query take part as already finished
    typename P::Vtx v;
    if (active) {
      v = pool[beg + t];
      if (tab.key) {  // its edge's entry is no longer needed: clear it for the next round
        const int h = tab.qhash[t];
        if (h >= 0) {
          tab.key[h] = 0ull;
          tab.val[h] = 0;
        }
      }
    }
    bool q = active && v.tri != -1;
    bool over = false, was_cut = false;
    const double cut_r = cutting && q ? P::cut_r(lnow, dyn, v) : -1.0;
    P::query(B, v, c, q, ll.idx ? (cut_r > 0.0 ? kLongBudgetCut : P::kLongBudget) : INT_MAX, &over, cut_r, &was_cut);
    if (q) {
      pool[beg + t] = v;
      if (over) {
        const int j = warp_slot(&st->n_long);
        if (j < ll.cap)
          ll.idx[j] = beg + t;
        else
          atomicExch(&st->overflow, 1);  // cannot happen: the list has room for every query
      } else {
        if (!was_cut) lmax = fmax(lmax, P::lower(v) - slack);  // a cut query has no lower bound
        ++nq;
        ncut += was_cut;
      }
    }
    if (cutting) {  // a larger l at once, so that the other warps cut sooner
      const double w = warp_max(lmax);
      if ((threadIdx.x & 31) == 0 && w > lnow) atomic_max_nonneg(&st->l_bits, w);
    }
  }
  lmax = warp_max(lmax);
  unsigned long long q = warp_sum((unsigned long long)nq), qc = warp_sum((unsigned long long)ncut);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&st->l_bits, lmax);
    if (q) atomicAdd(&st->queries, q);
    if (qc) atomicAdd(&st->queries_cut, qc);
  }
  flush_counters(st, c);
}

template <class P>
__global__ void HD_QUERY_REGS k_query(BvhDev B, typename P::Vtx* pool, int beg, const int* count_ptr, int mult, int cap,
                        RunState* st, double slack_in, const DynParams* dyn, bool round_midpoints, MidTable tab,
                        LongList ll) {
  grid_dep_wait();
  grid_dep_launch();
  if (ll.buckets) {  // the cell counters of this launch's reordering (k_long_hist) start at zero
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kSortBuckets; i += gridDim.x * blockDim.x)
      ll.buckets[i] = 0u;
  }
  query_body<P>(B, pool, beg, count_ptr, mult, cap, st, slack_in, dyn, round_midpoints, tab, ll);
}

// The queries k_query handed off, one warp each (traverse_coop, with this warp's stack in
// shared memory), taken one at a time from a counter since their costs vary widely; with
// their contribution to l and to the query counts.
template <class P>
__device__ inline void query_long_body(BvhDev B, typename P::Vtx* pool, LongList ll, RunState* st, double slack_in,
                                       const DynParams* dyn, bool round_midpoints, unsigned* s_code, float* s_e) {
  if (round_midpoints && st->stop) return;  // as k_query (uniform over the grid)
  const int n = min(st->n_long, ll.cap);
  if (n == 0) return;  // uniform over the grid
  const double slack = dyn ? dyn->slack : slack_in;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // a sorted list is taken kLongChunk neighbouring queries at a time
  const bool sorted = ll.sorted && n >= kSortMin;
  const int* list = sorted ? ll.sorted : ll.idx;
  // (ordered by cost with cuts: one at a time, so that the costly ones spread over the warps)
  const int chunk = sorted && !(HD_LONG_LPT && cut_on(dyn)) ? kLongChunk : 1;
  const bool cutting = HD_CUT_LONG && cut_on(dyn);
  Counters c;
  double lmax = 0.0;
  int nq = 0, ncut = 0;
  for (;;) {
    int i0 = 0;
    if (lane == 0) i0 = atomicAdd(&st->long_next, chunk);
    i0 = __shfl_sync(0xffffffffu, i0, 0);
    if (i0 >= n) break;
    for (int i = i0; i < min(i0 + chunk, n); ++i) {
      const int k = list[i];
      typename P::Vtx v = pool[k];
      const bool cut = P::query_coop(B, v, c, s_code + w * kCoopStack, s_e + w * kCoopStack,
                                     cutting ? P::cut_r(read_lower(st), dyn, v) : -1.0);
      if (lane == 0) {
        pool[k] = v;
        const double prev = lmax;
        if (!cut) lmax = fmax(lmax, P::lower(v) - slack);  // a cut query has no lower bound
        ++nq;
        ncut += cut;
        if (cutting && lmax > prev) atomic_max_nonneg(&st->l_bits, lmax);  // other warps cut sooner
      }
    }
  }
  if (lane == 0) {
    atomic_max_nonneg(&st->l_bits, lmax);
    if (nq) {
      atomicAdd(&st->queries, (unsigned long long)nq);
      atomicAdd(&st->long_queries, (unsigned long long)nq);
    }
    if (ncut) atomicAdd(&st->queries_cut, (unsigned long long)ncut);
  }
  flush_counters(st, c, true);
}

template <class P>
__global__ void __launch_bounds__(32 * kCoopWarps, P::kCoopBlocks) k_query_long(BvhDev B, typename P::Vtx* pool, LongList ll,
                                                                RunState* st, double slack_in, const DynParams* dyn,
                                                                bool round_midpoints) {
  __shared__ unsigned s_code[kCoopWarps * kCoopStack];
  __shared__ float s_e[kCoopWarps * kCoopStack];
  grid_dep_wait();
  grid_dep_launch();
  query_long_body<P>(B, pool, ll, st, slack_in, dyn, round_midpoints, s_code, s_e);
}

// The reordering of a long-query list along the Morton curve of its points (a counting sort on
// kSortBuckets cells): per-cell counts, their exclusive scan, then each index to its cell's next
// slot (the order within a cell is arbitrary).  Lists shorter than kSortMin are left as they are
// (every kernel returns at once; uniform over the grid).
//
// The cell of a handed-off query in the reordered list.  Without cuts: its Morton cell.  With
// cuts, the queries whose best triangle so far is not yet within their cut radius (those that
// must traverse) take the first half of the cells, ordered by that triangle's distance r,
// largest first: a far query's search ball holds the most boxes, and starting the costliest
// first keeps the pass from ending on a few warps still working (longest job first).  The
// cheap ones fill in behind in Morton order (the code loses its lowest bit).  l does not
// change between k_long_hist and k_long_scatter, so both find the same cell.
template <class P>
__device__ inline unsigned long_cell(const BvhDev& B, const typename P::Vtx& v, const RunState* st,
                                     const DynParams* dyn) {
  const D3 x = P::exact_pos(v);
  const unsigned m = long_bucket(B, (float)x.x, (float)x.y, (float)x.z);
  if (!cut_on(dyn)) return m;
  const double l = read_lower(st);
  if (P::hint_within(B, v, P::cut_r(l, dyn, v))) return kSortBuckets / 2 + (m >> 1);
  if (!HD_LONG_LPT) return m >> 1;
  // r in [0, 2 l) over the half's cells, larger r first
  constexpr unsigned kHalf = kSortBuckets / 2;
  const double q = l > 0.0 ? P::hint_dist(v) / (2.0 * l) * kHalf : 0.0;
  return kHalf - 1u - (unsigned)fmin(fmax(q, 0.0), (double)(kHalf - 1));
}

template <class P>
__global__ void k_long_hist(BvhDev B, const typename P::Vtx* pool, LongList ll, const RunState* st,
                            bool round_midpoints, const DynParams* dyn) {
  grid_dep_wait();
  grid_dep_launch();
  if (round_midpoints && st->stop) return;
  const int n = min(st->n_long, ll.cap);
  if (n < kSortMin) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicAdd(&ll.buckets[long_cell<P>(B, pool[ll.idx[i]], st, dyn)], 1u);
}

// Exclusive scan of the cell counts: one block of 1024 threads, kSortBuckets / 1024 rows of
// 1024 consecutive counters, each row scanned across the block (coalesced) and carried on.
static __global__ void k_long_scan(LongList ll, const RunState* st, bool round_midpoints) {
  grid_dep_wait();
  grid_dep_launch();
  if (round_midpoints && st->stop) return;
  if (min(st->n_long, ll.cap) < kSortMin) return;
  constexpr int kRows = kSortBuckets / 1024;
  __shared__ unsigned wtot[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned val[kRows];  // every row's counter first: the loads overlap instead of one per row
#pragma unroll
  for (int row = 0; row < kRows; ++row) val[row] = ll.buckets[row * 1024 + threadIdx.x];
  unsigned carry = 0;
#pragma unroll
  for (int row = 0; row < kRows; ++row) {
    const int i = row * 1024 + threadIdx.x;
    const unsigned v = val[row];
    unsigned x = v;  // inclusive warp scan
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wtot[w] = x;
    __syncthreads();
    if (w == 0) {  // the warps' totals, scanned
      unsigned t = wtot[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      wtot[lane] = t;
    }
    __syncthreads();
    ll.buckets[i] = carry + (w ? wtot[w - 1] : 0u) + x - v;
    carry += wtot[31];
    __syncthreads();  // wtot is written again by the next row
  }
}

template <class P>
__global__ void k_long_scatter(BvhDev B, const typename P::Vtx* pool, LongList ll, const RunState* st,
                               bool round_midpoints, const DynParams* dyn) {
  grid_dep_wait();
  grid_dep_launch();
  if (round_midpoints && st->stop) return;
  const int n = min(st->n_long, ll.cap);
  if (n < kSortMin) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k = ll.idx[i];
    const unsigned pos = atomicAdd(&ll.buckets[long_cell<P>(B, pool[k], st, dyn)], 1u);
    ll.sorted[pos] = k;  // pos < n: the cells' counts sum to n
  }
}

// Launches the reordering of the long-query list of the k_query launch queued just before
// (nothing happens on the device for short lists).
template <class P>
void sort_long(const BvhDev& B, const typename P::Vtx* pool, const LongList& ll, const RunState* st,
               bool round_midpoints, int sms, cudaStream_t s, const DynParams* dyn) {
  if (!ll.sorted) return;
  launch_chained(k_long_hist<P>, (unsigned)sms * 4, 256, 0, s, B, pool, ll, st, round_midpoints, dyn);
  launch_chained(k_long_scan, 1, 1024, 0, s, ll, st, round_midpoints);
  launch_chained(k_long_scatter<P>, (unsigned)sms * 4, 256, 0, s, B, pool, ll, st, round_midpoints, dyn);
}

// Per-thread outcome counts and maxima of classified items, flushed once per warp.
template <class P>
struct Tally {
  unsigned d0 = 0, d1 = 0, d2 = 0, d3 = 0, d4 = 0, d5 = 0, retired = 0;
  typename P::UT uret = 0, umax = 0;
  __device__ void discard(int code) {
    d0 += code == 0;
    d1 += code == 1;
    d2 += code == 2;
    d3 += code == 3;
    d4 += code == 4;
    d5 += code == 5;
  }
};

// Every lane of the warp must call it.
template <class P>
__device__ inline void flush_tally(RunState* st, const Tally<P>& t) {
  unsigned long long d[6] = {warp_sum(t.d0), warp_sum(t.d1), warp_sum(t.d2),
                             warp_sum(t.d3), warp_sum(t.d4), warp_sum(t.d5)};
  unsigned long long r = warp_sum(t.retired);
  typename P::UT uret = t.uret, umax = t.umax;
  for (int o = 16; o > 0; o >>= 1) {
    typename P::UT a = __shfl_xor_sync(0xffffffffu, uret, o), b = __shfl_xor_sync(0xffffffffu, umax, o);
    uret = a > uret ? a : uret;
    umax = b > umax ? b : umax;
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (d[k]) atomicAdd(&st->discards[k], d[k]);
    if (r) {
      atomicAdd(&st->retired, r);
      atomic_max_nonneg(&st->uret_bits, (double)uret);
    }
    if (umax > 0) atomic_max_nonneg(&st->umax_bits, (double)umax);
  }
}

// Comparison thresholds in the policy's number type, rounded down so that U < lo implies
// U < l (discard) and U <= hi implies U <= l + eps (retire).
template <class P>
struct Thresholds {
  typename P::UT lo, hi;
  __device__ Thresholds(double l, double eps) : lo(P::ut_down(l)), hi(P::ut_down(add_rd(l, eps))) {}
  struct Raw {};
  __device__ Thresholds(Raw, typename P::UT lo_, typename P::UT hi_) : lo(lo_), hi(hi_) {}
};

// Discard / retire / keep one bounded item (Section 3.1: discard when U < l).  Items whose
// trailing u4 is deferred go to the u4 list instead.
template <class P>
__device__ inline void classify(RunState* st, const typename P::Item& it, const Thresholds<P>& th, int code,
                                typename P::Item* next, int next_cap, typename P::Item* u4list, Tally<P>& ty) {
  if (code == kDeferU4) {
    int j = warp_slot(&st->n_u4);
    if (j < next_cap) u4list[j] = it;
    else atomicExch(&st->overflow, 1);
    return;
  }
  if (it.U < th.lo) {
    ty.discard(code);
  } else if (it.U <= th.hi) {
    ty.uret = ty.uret > it.U ? ty.uret : it.U;
    ++ty.retired;
  } else {
    int j = warp_slot(&st->n_next);
    if (j < next_cap) {
      next[j] = it;
      ty.umax = ty.umax > it.U ? ty.umax : it.U;
    } else {
      atomicExch(&st->overflow, 1);
    }
  }
}

__device__ inline double load_l(const RunState* st) {
  return __longlong_as_double((long long)*(volatile unsigned long long*)&st->l_bits);
}

// l and the comparison thresholds, computed once per block (l does not change while a bound
// or select kernel runs: only the queries raise it) and shared, so that the FP64 conversions
// are not repeated per thread.  Every thread of the block must call it.
template <class P>
struct Level {
  double l;
  float lf;  // l rounded down to float: u < lf implies u < l
  Thresholds<P> th;
};
template <class P>
__device__ inline Level<P> block_level(const RunState* st, double eps) {
  __shared__ double s_l;
  __shared__ float s_lf;
  __shared__ typename P::UT s_lo, s_hi;
  if (threadIdx.x == 0) {
    const double l = load_l(st);
    const Thresholds<P> th(l, eps);
    s_l = l;
    s_lf = __double2float_rd(l);
    s_lo = th.lo;
    s_hi = th.hi;
  }
  __syncthreads();
  return Level<P>{s_l, s_lf, Thresholds<P>(typename Thresholds<P>::Raw{}, s_lo, s_hi)};
}

// UpperBound of one sub-triangle: the cascade in the paper's order with u4 deferred
// (kPaper, straight-line code, MIXED only), or in any order rp gives.
template <class P, bool kPaper>
__device__ inline typename P::UT bound_item(const BvhDev& B, const typename P::Vtx* pool, const typename P::Item& it,
                                            const Level<P>& lv, const RunParams& rp, int& code, Counters& c) {
  if constexpr (kPaper)
    return P::upper_bound_paper(B, pool[it.v[0]], pool[it.v[1]], pool[it.v[2]], lv.l, lv.lf, rp, code, c);
  else
    return P::upper_bound(B, pool[it.v[0]], pool[it.v[1]], pool[it.v[2]], lv.l, lv.lf, rp, code, c);
}

// The paper-order cascade with the items that reach u3 gathered into full warps (MIXED).  The
// exact case, u1 and u2 are cheap and decide many items; u3 costs 4 to 15 point-triangle
// evaluations.  Run item by item, the lanes whose items were decided early idle while the
// others evaluate u3.  Here each warp takes batches of 32 items, runs the cheap part on them,
// and appends the items that still need u3 to its queue in shared memory (64 entries); when 32
// are waiting, every lane takes one and finishes it, so u3 runs on full warps.  The values and
// result codes are those of the item-by-item cascade; only the order of the classification
// changes.  `make(t, it, up)` gives item t (false: no item) and the bound it is clamped to
// (its parent's U, or +inf).
// On for the batched run's kernels (HD_BATCH_REBIN), off for a single run's (HD_REBIN): on the
// 1024-pair batched workload, where 72% of the child items reach u3, it took the UpperBound
// kernels from 168 to 155 ms per call; on the torus pair, where most items are decided by the
// exact case, from 0.091 to 0.098 ms (the queue's traffic costs more than the idle lanes).
#ifndef HD_REBIN
#define HD_REBIN 0
#endif
#ifndef HD_BATCH_REBIN
#define HD_BATCH_REBIN 1
#endif
struct RebinEntry {
  int v[3];
  float u12;  // min(u1, u2)
  float up;   // clamp
};
constexpr int kRebinQueue = 64;  // entries per warp
inline size_t rebin_smem(int block) { return HD_REBIN ? (size_t)(block / 32) * kRebinQueue * sizeof(RebinEntry) : 0; }

template <class P, class Make>
__device__ inline void bound_rebin(const BvhDev& B, const typename P::Vtx* pool, int64_t count, int* counter,
                                   const Level<P>& lv, const RunParams& rp, RunState* st, typename P::Item* next,
                                   int next_cap, typename P::Item* u4list, RebinEntry* q, Counters& c, Tally<P>& ty,
                                   Make make) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int qn = 0;  // entries waiting in this warp's queue (uniform over the warp)
  bool more = true;
  while (more || qn > 0) {
    if (more && qn < 32) {
      const int64_t base = warp_batch(counter);
      if (base >= count) {
        more = false;
      } else {
        const int64_t t = base + lane;
        bool need = false;
        RebinEntry e;
        typename P::Item it;
        float up = INFINITY;
        if (t < count && make(t, it, up)) {
          float U, u12;
          int code;
          if (P::paper_cheap(pool[it.v[0]], pool[it.v[1]], pool[it.v[2]], lv.lf, rp, &U, &code, &u12)) {
            need = true;
            e = RebinEntry{{it.v[0], it.v[1], it.v[2]}, u12, up};
          } else {
            it.U = up < U ? up : U;
            classify<P>(st, it, lv.th, code, next, next_cap, u4list, ty);
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, need);
        if (need) q[qn + __popc(m & lt)] = e;
        qn += __popc(m);
        __syncwarp();
      }
    }
    if (qn >= 32 || (!more && qn > 0)) {
      const int take = min(qn, 32);
      if (lane < take) {
        const RebinEntry e = q[qn - take + lane];
        typename P::Item it;
        it.v[0] = e.v[0];
        it.v[1] = e.v[1];
        it.v[2] = e.v[2];
        int code;
        const float U = P::paper_u3(B, pool[e.v[0]], pool[e.v[1]], pool[e.v[2]], lv.lf, rp, e.u12, code, c);
        it.U = e.up < U ? e.up : U;
        classify<P>(st, it, lv.th, code, next, next_cap, u4list, ty);
      }
      qn -= take;
      __syncwarp();  // the entries taken are read before new ones overwrite them
    }
  }
}

// Round 0: UpperBound for every face of A.
template <class P, bool kPaper = false>
__global__ void HD_BOUND_REGS k_bound_faces(BvhDev B, const typename P::Vtx* pool, const int32_t* FA, int64_t nFA, RunState* st,
                              RunParams rp_in, typename P::Item* next, int next_cap, typename P::Item* u4list,
                              int64_t n_pool_valid) {
  grid_dep_wait();
  grid_dep_launch();
  const RunParams rp = with_dyn(rp_in);
  const Level<P> lv = block_level<P>(st, rp.eps);
  const Thresholds<P>& th = lv.th;
  Counters c;
  Tally<P> ty;
  if constexpr (kPaper && HD_REBIN) {
    extern __shared__ RebinEntry rebin_q[];
    bound_rebin<P>(B, pool, nFA, &st->b_next, lv, rp, st, next, next_cap, u4list, rebin_q + (threadIdx.x >> 5) * kRebinQueue,
                   c, ty, [&](int64_t f, typename P::Item& it, float&) {
                     it.v[0] = FA[3 * f];
                     it.v[1] = FA[3 * f + 1];
                     it.v[2] = FA[3 * f + 2];
                     // A is validated concurrently: skip bad rows
                     return it.v[0] >= 0 && it.v[1] >= 0 && it.v[2] >= 0 && it.v[0] < n_pool_valid &&
                            it.v[1] < n_pool_valid && it.v[2] < n_pool_valid;
                   });
    flush_counters(st, c);
    flush_tally(st, ty);
    return;
  }
  for (;;) {
    const int64_t base = warp_batch(&st->b_next);
    if (base >= nFA) break;
    const int64_t f = base + (threadIdx.x & 31);
    if (f >= nFA) continue;
    typename P::Item it;
    it.v[0] = FA[3 * f];
    it.v[1] = FA[3 * f + 1];
    it.v[2] = FA[3 * f + 2];
    // A is validated concurrently (the host checks the flag with the first round): skip bad rows
    if (!(it.v[0] >= 0 && it.v[1] >= 0 && it.v[2] >= 0 && it.v[0] < n_pool_valid && it.v[1] < n_pool_valid &&
          it.v[2] < n_pool_valid))
      continue;
    int code;
    it.U = bound_item<P, kPaper>(B, pool, it, lv, rp, code, c);
    classify<P>(st, it, th, code, next, next_cap, u4list, ty);
  }
  flush_counters(st, c);
  flush_tally(st, ty);
}

// The u4 pass (MIXED): items whose cascade reached a trailing u4 get it here, in FP64, with
// every lane of a warp on its own item; then discard / retire / keep as usual.
template <class P>
__device__ inline void bound_u4_body(BvhDev B, const typename P::Vtx* pool, const typename P::Item* u4list, int cap,
                           RunState* st, RunParams rp_in, typename P::Item* next, int next_cap) {
  if (st->stop) return;  // the loop ended before this round (uniform over the grid)
  const RunParams rp = with_dyn(rp_in);
  int n = min(*(volatile int*)&st->n_u4, cap);
  const Level<P> lv = block_level<P>(st, rp.eps);
  const Thresholds<P>& th = lv.th;
  Tally<P> ty;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    typename P::Item it = u4list[t];
    typename P::UT u = P::bound_u4(pool[it.v[0]], pool[it.v[1]], pool[it.v[2]], rp, it.U);
    int code = 5;
    if (u < th.lo) {
      code = 4;
      it.U = u;
    } else if (u < it.U) {
      it.U = u;
    }
    classify<P>(st, it, th, code, next, next_cap, nullptr, ty);
  }
  flush_tally(st, ty);
}

template <class P>
__global__ void k_bound_u4(BvhDev B, const typename P::Vtx* pool, const typename P::Item* u4list, int cap,
                           RunState* st, RunParams rp_in, typename P::Item* next, int next_cap) {
  grid_dep_wait();
  grid_dep_launch();
  bound_u4_body<P>(B, pool, u4list, cap, st, rp_in, next, next_cap);
}

__device__ inline unsigned edge_hash(unsigned long long k, unsigned mask) {
  k ^= k >> 31;
  k *= 0x9E3779B97F4A7C15ull;
  return (unsigned)(k >> 32) & mask;
}

// Midpoint of edge e of split s, per active lane; without a table at mbase + 3 s + e.  With
// one, it is called by every lane of the warp: the
// first lane of the round to insert an edge makes its midpoint in a new slot and publishes it;
// the others take that slot, waiting (bounded) for it to be published, and after a timeout
// make a duplicate of their own (a separate pool vertex at the same position: only the
// sharing is lost).  Returns the pool index (mbase + slot), or -1 for inactive lanes.
template <class P>
__device__ inline int mid_slot(bool active, int s, int e, int ia, int ib, const typename P::Vtx& va,
                               const typename P::Vtx& vb, const MidTable& tab, RunState* st, typename P::Vtx* pool,
                               int mbase) {
  if (!tab.key) {  // uniform over the grid
    if (!active) return -1;
    typename P::Vtx m;
    P::midpoint(va, vb, m);
    pool[mbase + 3 * s + e] = m;
    return mbase + 3 * s + e;
  }
  bool win = false, found = false;
  unsigned h = 0;
  if (active) {
    const unsigned long long lo = (unsigned)min(ia, ib), hi = (unsigned)max(ia, ib);
    const unsigned long long key = (1ull << 63) | (lo << 32) | hi;  // never 0 (the empty key)
    h = edge_hash(key, tab.mask);
    for (unsigned p = 0; p <= tab.mask; ++p) {
      const unsigned long long prev = atomicCAS(&tab.key[h], 0ull, key);
      if (prev == 0ull) {
        win = true;
        break;
      }
      if (prev == key) {
        found = true;
        break;
      }
      h = (h + 1) & tab.mask;
    }
  }
  int slot = -1;
  if (win) {
    slot = warp_slot(&st->n_mid);
    typename P::Vtx m;
    P::midpoint(va, vb, m);
    pool[mbase + slot] = m;
    tab.qhash[slot] = (int)h;
    atomicExch(&tab.val[h], slot + 1);
  }
  __syncwarp();  // this warp's new edges are published before its lanes look them up
  if (found) {
    for (int it = 0; it < 4096; ++it) {
      const int v = *(volatile int*)&tab.val[h];
      if (v) {
        slot = v - 1;
        break;
      }
      __nanosleep(32);
    }
  }
  if (active && slot < 0) {  // not published in time (or no free entry): a duplicate
    slot = warp_slot(&st->n_mid);
    typename P::Vtx m;
    P::midpoint(va, vb, m);
    pool[mbase + slot] = m;
    tab.qhash[slot] = -1;
  }
  return active ? mbase + slot : -1;
}

// Select the items to split: discard (U < l), retire (U <= l + eps), split up to K of the
// rest (three midpoints each into the pool at mbase), carry the others over.
template <class P>
__device__ inline void select_body(const typename P::Item* front, RunState* st, RunParams rp_in, int4* split_par,
                         int4* split_mid, MidTable tab, typename P::Vtx* pool, typename P::Item* next, int next_cap,
                         typename P::Item* promo, int promo_cap) {
  if (st->stop) return;  // the loop ended before this round (uniform over the grid)
  const int n_front = st->n_front, K = st->K, mbase = st->n_pool;
  const RunParams rp = with_dyn(rp_in);
  const Level<P> lv = block_level<P>(st, rp.eps);
  const Thresholds<P>& th = lv.th;
  const double l = lv.l;
  Tally<P> ty;
  // warp-uniform loop: the midpoint step below is taken by whole warps
  for (int i = blockIdx.x * blockDim.x + threadIdx.x;; i += gridDim.x * blockDim.x) {
    const bool valid = i < n_front;
    if (__all_sync(0xffffffffu, !valid)) break;
    typename P::Item it;
    typename P::Vtx a, b, c;
    int s = -1;  // split slot of this lane's item
    if (valid) {
      it = front[i];
      const double U = (double)it.U;
      if (it.U < th.lo) {
        ty.discard(5);
      } else if (it.U <= th.hi) {
        ty.uret = ty.uret > it.U ? ty.uret : it.U;
        ++ty.retired;
      } else {
        a = pool[it.v[0]];
        b = pool[it.v[1]];
        c = pool[it.v[2]];
        if (promo && P::promote(a, b, c, U, l)) {  // below the policy's resolution: FP64 phase
          int j = atomicAdd(&st->n_promote, 1);
          if (j < promo_cap) {
            promo[j] = it;
            atomic_max_nonneg(&st->upro_bits, U);
          } else {
            atomicExch(&st->overflow, 1);
          }
        } else {
          s = warp_slot(&st->n_split);
          if (s < K) {
            // the parent's U, rounded up to float, for the children's clamp
            split_par[s] = make_int4(it.v[0], it.v[1], it.v[2], __float_as_int(__double2float_ru(U)));
          } else {
            s = -1;
            int j = warp_slot(&st->n_next);
            if (j < next_cap) {
              next[j] = it;
              ty.umax = ty.umax > it.U ? ty.umax : it.U;
            } else {
              atomicExch(&st->overflow, 1);
            }
          }
        }
      }
    }
    const bool sp = s >= 0;
    const int m01 = mid_slot<P>(sp, s, 0, it.v[0], it.v[1], a, b, tab, st, pool, mbase);
    const int m12 = mid_slot<P>(sp, s, 1, it.v[1], it.v[2], b, c, tab, st, pool, mbase);
    const int m20 = mid_slot<P>(sp, s, 2, it.v[2], it.v[0], c, a, tab, st, pool, mbase);
    if (sp && tab.key) split_mid[s] = make_int4(m01, m12, m20, 0);
  }
  flush_tally(st, ty);
}

template <class P>
__global__ void k_select(const typename P::Item* front, RunState* st, RunParams rp_in, int4* split_par,
                         int4* split_mid, MidTable tab, typename P::Vtx* pool, typename P::Item* next, int next_cap,
                         typename P::Item* promo, int promo_cap) {
  grid_dep_wait();
  grid_dep_launch();
  select_body<P>(front, st, rp_in, split_par, split_mid, tab, pool, next, next_cap, promo, promo_cap);
}

// The four children of every split (Section 4, midpoint subdivision):
// (v1, m12, m31), (m12, v2, m23), (m31, m23, v3), (m12, m23, m31).
template <class P, bool kPaper = false>
__device__ inline void bound_children_body(BvhDev B, const typename P::Vtx* pool, const int4* split_par,
                                 const int4* split_mid, RunState* st, RunParams rp_in, typename P::Item* next, int next_cap, typename P::Item* u4list) {
  if (st->stop) return;  // the loop ended before this round (uniform over the grid)
  const RunParams rp = with_dyn(rp_in);
  const int mbase = st->n_pool, share = st->share_mid;
  int S = min(*(volatile int*)&st->n_split, st->K);
  const Level<P> lv = block_level<P>(st, rp.eps);
  const Thresholds<P>& th = lv.th;
  Counters c;
  Tally<P> ty;
  if constexpr (kPaper && HD_REBIN) {
    extern __shared__ RebinEntry rebin_q[];
    bound_rebin<P>(B, pool, 4 * (int64_t)S, &st->b_next, lv, rp, st, next, next_cap, u4list,
                   rebin_q + (threadIdx.x >> 5) * kRebinQueue, c, ty,
                   [&](int64_t t, typename P::Item& it, float& up) {
                     const int s = (int)(t >> 2), k = (int)(t & 3);
                     const int4 par = split_par[s];
                     const int4 mid = share ? split_mid[s] : make_int4(mbase + 3 * s, mbase + 3 * s + 1, mbase + 3 * s + 2, 0);
                     if (k == 0) { it.v[0] = par.x; it.v[1] = mid.x; it.v[2] = mid.z; }
                     else if (k == 1) { it.v[0] = mid.x; it.v[1] = par.y; it.v[2] = mid.y; }
                     else if (k == 2) { it.v[0] = mid.z; it.v[1] = mid.y; it.v[2] = par.z; }
                     else { it.v[0] = mid.x; it.v[1] = mid.y; it.v[2] = mid.z; }
                     // the child lies inside its parent: h(child, B) <= U(parent)
                     if (rp.parent_clamp) up = __int_as_float(par.w);
                     return true;
                   });
    flush_counters(st, c);
    flush_tally(st, ty);
    return;
  }
  for (;;) {
    const int64_t base = warp_batch(&st->b_next);
    if (base >= 4 * (int64_t)S) break;
    const int64_t t = base + (threadIdx.x & 31);
    if (t < 4 * (int64_t)S) {
      int s = (int)(t >> 2), k = (int)(t & 3);
      const int4 par = split_par[s];
      const int4 mid = share ? split_mid[s] : make_int4(mbase + 3 * s, mbase + 3 * s + 1, mbase + 3 * s + 2, 0);
      const int m12 = mid.x, m23 = mid.y, m31 = mid.z;
      typename P::Item it;
      if (k == 0) { it.v[0] = par.x; it.v[1] = m12; it.v[2] = m31; }
      else if (k == 1) { it.v[0] = m12; it.v[1] = par.y; it.v[2] = m23; }
      else if (k == 2) { it.v[0] = m31; it.v[1] = m23; it.v[2] = par.z; }
      else { it.v[0] = m12; it.v[1] = m23; it.v[2] = m31; }
      int code;
      it.U = bound_item<P, kPaper>(B, pool, it, lv, rp, code, c);
      // the child lies inside its parent: h(child, B) <= U(parent)
      const typename P::UT Up = (typename P::UT)__int_as_float(par.w);
      if (rp.parent_clamp && Up < it.U) it.U = Up;
      classify<P>(st, it, th, code, next, next_cap, u4list, ty);
    }
  }
  flush_counters(st, c);
  flush_tally(st, ty);
}

template <class P, bool kPaper = false>
__global__ void HD_BOUND_REGS k_bound_children(BvhDev B, const typename P::Vtx* pool, const int4* split_par,
                                 const int4* split_mid, RunState* st, RunParams rp_in, typename P::Item* next, int next_cap, typename P::Item* u4list) {
  grid_dep_wait();
  grid_dep_launch();
  bound_children_body<P, kPaper>(B, pool, split_par, split_mid, st, rp_in, next, next_cap, u4list);
}

// Whether the options ask for the paper's cascade (u1, u2, u3, u4) with u4 left to the u4
// pass: then the UpperBound kernels run their straight-line instantiation (kPaper), which
// keeps fewer values live than the loop over rp.order and so needs no spills at its
// register cap.
inline bool paper_cascade(const RunParams& rp) {
  return rp.defer_u4 && rp.n_bounds == 4 && rp.order[0] == 1 && rp.order[1] == 2 && rp.order[2] == 3 &&
         rp.order[3] == 4;
}
template <class P>
auto bound_faces_kernel(bool paper) {
  if constexpr (P::kFp64) return k_bound_faces<P, false>;
  else return paper ? k_bound_faces<P, true> : k_bound_faces<P, false>;
}
template <class P>
auto bound_children_kernel(bool paper) {
  if constexpr (P::kFp64) return k_bound_children<P, false>;
  else return paper ? k_bound_children<P, true> : k_bound_children<P, false>;
}

// Per-loop constants of the round control.
struct RoundCtl {
  long long chunk, pool_cap, front_cap;
  int share;  // midpoints shared through the table
  long long splits_left;  // splits allowed by the face cap m n_A (Section 4) for this loop
  long long rounds_left;  // rounds before HD_ERR_TIMEOUT for this loop
  const unsigned long long* bad;  // A's and B's invalid-input flags
};

__host__ __device__ inline double state_bits_to_double(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, 8);
  return d;
#endif
}
__host__ __device__ inline unsigned long long state_double_to_bits(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(d);
#else
  unsigned long long b;
  memcpy(&b, &d, 8);
  return b;
#endif
}

// The end of a frontier round, on a run state: its splits and pool growth, the new frontier,
// and u as the running minimum of max(l, retired U, frontier U, promoted U).  Returns why the
// loop ends (HD_OK when the frontier is empty, Section 3.1; CAPACITY, TIMEOUT, NUMERIC,
// INVALID), or -1 to go on.  Run by k_round_ctl on the device, and by the host on the last
// state it read when no round was queued after it.
__host__ __device__ inline int close_round(RunState& st, long long rounds_left) {
  if (st.in_round) {
    const int S = st.n_split < st.K ? st.n_split : st.K;
    st.rounds += 1;
    st.splits += S;
    st.n_pool += st.share_mid ? st.n_mid : 3 * S;
    st.in_round = 0;
  }
  const int n_front = st.n_next;
  st.n_front = n_front;
  if (n_front > st.peak) st.peak = n_front;
  double u = fmax(state_bits_to_double(st.l_bits), state_bits_to_double(st.uret_bits));
  if (n_front) u = fmax(u, state_bits_to_double(st.umax_bits));
  if (st.n_promote) u = fmax(u, state_bits_to_double(st.upro_bits));
  if (u < state_bits_to_double(st.urun_bits)) st.urun_bits = state_double_to_bits(u);
  if (st.bad) return HD_ERR_INVALID;
  if (st.err) return HD_ERR_NUMERIC;
  if (st.overflow) return HD_ERR_CAPACITY;
  if (n_front == 0) return HD_OK;
  if (st.rounds >= rounds_left) return HD_ERR_TIMEOUT;
  return -1;
}

// Start of a frontier round, on the device: closes the round before it, decides whether the
// loop goes on, and if so sizes and opens the round.  With init set it first starts the loop
// (pool entries [0, n_pool0), after the bounds of its first items -- the faces of A, or the
// promoted items -- were launched).  Once stopped, later rounds find `stop` set and do
// nothing, so the host may queue a round before it has read the previous one.
// With max_front set, a round over more items than that, or after a round that handed more
// than max_long queries to the cooperative pass, is not opened (the loop goes on with
// in_round cleared, for the normal path to open it).
__device__ inline void round_ctl_body(RunState* st, RoundCtl c, int init, int n_pool0, int max_front = INT_MAX,
                                      int max_long = INT_MAX) {
  if (init) {
    st->stop = 0;
    st->status = HD_OK;
    st->in_round = 0;
    st->rounds = st->splits = st->peak = 0;
    st->urun_bits = (unsigned long long)__double_as_longlong(INFINITY);
    st->n_pool = n_pool0;
    st->share_mid = c.share;
  }
  if (st->stop) return;
  st->bad = *c.bad;
  int status = close_round(*st, c.rounds_left);
  long long K = 0;
  if (status < 0) {
    K = min(c.chunk, (c.pool_cap - (long long)st->n_pool) / 3);
    K = min(K, (c.front_cap - (long long)st->n_front) / 3);
    K = min(K, c.splits_left - st->splits);
    if (K <= 0) status = HD_ERR_CAPACITY;
  }
  if (status >= 0) {
    st->status = status;
    st->stop = 1;
    return;
  }
  if (st->n_front > max_front || st->n_long > max_long) return;
  st->K = (int)K;
  st->n_next = 0;
  st->n_split = 0;
  st->n_u4 = 0;
  st->umax_bits = 0;
  st->overflow = 0;
  st->q_next = 0;
  st->b_next = 0;
  st->n_mid = 0;
  st->n_long = 0;
  st->long_next = 0;
  st->in_round = 1;
}

static __global__ void k_round_ctl(RunState* st, RoundCtl c, int init, int n_pool0) {
  grid_dep_wait();
  grid_dep_launch();
  round_ctl_body(st, c, init, n_pool0);
}

// ----------------------------------------------------------------------------- small rounds

// Rounds over a small frontier (the last rounds of most runs) in one block: each phase of a
// round is a kernel of the normal path, and for a frontier of a few dozen items each is one
// pass of a few warps, so the launches and the host's reading of the round dominate.  Here
// one block runs the same steps (control, select, query, cooperative query, bound, u4) with
// block barriers between them, round after round, until the loop stops, the frontier grows
// past kTailFront, or a round hands more than kTailWarps queries to the cooperative pass (a
// round with many long traversals needs the whole GPU); the normal path then takes over, so
// any frontier is correct.
constexpr int kTailThreads = 256;
constexpr int kTailWarps = kTailThreads / 32;
#ifndef HD_TAIL_LONG
#define HD_TAIL_LONG kTailWarps
#endif
constexpr int kTailLong = HD_TAIL_LONG;  // most long queries a round may hand off and stay in the small-round kernel
constexpr int kTailFront = 64;
constexpr size_t kTailSmem = (sizeof(unsigned) + sizeof(float)) * kTailWarps * kCoopStack;

template <class P>
struct TailBufs {
  typename P::Item* front[2];
  int4* split_par;
  int4* split_mid;
  MidTable tab;
  typename P::Vtx* pool;
  typename P::Item* promo;
  int promo_cap;
  int front_cap;
  typename P::Item* u4list;
  LongList longq;
};

template <class P>
__global__ void __launch_bounds__(kTailThreads) k_tail_rounds(BvhDev B, TailBufs<P> a, RunState* st, RunParams rp,
                                                              RoundCtl c, int init, int n_pool0, int cur) {
  extern __shared__ __align__(16) unsigned char tail_smem[];  // kTailSmem bytes: the warps' cooperative stacks
  unsigned* s_code = reinterpret_cast<unsigned*>(tail_smem);
  float* s_e = reinterpret_cast<float*>(tail_smem + sizeof(unsigned) * kTailWarps * kCoopStack);
  __shared__ int s_go;
  grid_dep_wait();
  grid_dep_launch();
  // a round here hands off at most a few queries: the list keeps its order
  const LongList lq = {a.longq.idx, a.longq.cap, nullptr, nullptr};
  int rounds = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      // the control step of k_round_ctl, refusing to open a round over kTailFront items
      round_ctl_body(st, c, init, n_pool0, kTailFront, kTailLong);
      s_go = !st->stop && st->in_round;
    }
    init = 0;
    __syncthreads();
    if (!s_go) break;
    select_body<P>(a.front[cur], st, rp, a.split_par, a.split_mid, a.tab, a.pool, a.front[cur ^ 1], a.front_cap,
                   a.promo, a.promo_cap);
    __syncthreads();
    query_body<P>(B, a.pool, 0, nullptr, 3, 0, st, rp.slack, rp.dyn, true, a.tab, lq);
    __syncthreads();
    query_long_body<P>(B, a.pool, lq, st, rp.slack, rp.dyn, true, s_code, s_e);
    __syncthreads();
    bound_children_body<P>(B, a.pool, a.split_par, a.split_mid, st, rp, a.front[cur ^ 1], a.front_cap, a.u4list);
    __syncthreads();
    if (a.u4list) bound_u4_body<P>(B, a.pool, a.u4list, a.front_cap, st, rp, a.front[cur ^ 1], a.front_cap);
    __syncthreads();
    cur ^= 1;
    ++rounds;
  }
  if (threadIdx.x == 0) st->tail_rounds = rounds;
}

// Nearest queries for external points (hd_nearest): P as double rows.
template <class P>
__global__ void k_query_points(BvhDev B, typename P::Vtx* tmp, int64_t n, RunState* st) {
  grid_dep_wait();
  grid_dep_launch();
  Counters c;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;; t += (int64_t)gridDim.x * blockDim.x) {
    bool active = t < n;
    if (__all_sync(0xffffffffu, !active)) break;
    typename P::Vtx v;
    if (active) v = tmp[t];
    P::query(B, v, c, active);  // whole warp enters (see k_query)
    if (active) tmp[t] = v;
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
  double l0;  // a known lower bound to start l from (0: none)
};

inline BvhDev bvh_dev(const hd_bvh* B) { return {B->nodes, B->tri32, B->tri64, B->tri_vid, B->nF, B->meta, B->grid}; }

inline double bits_to_double(unsigned long long b) {
  double d;
  memcpy(&d, &b, 8);
  return d;
}

// Queries may be cut (cut_radius) unless exact ones are asked for, and only when u1 is in
// the cascade: u1 is what discards the faces at a cut vertex.
inline bool cut_enabled(const Opts& o) {
  if (o.flags & HD_FLAG_EXACT_QUERIES) return false;
  for (int k = 0; k < o.n_bounds; ++k)
    if (o.order[k] == 1) return true;
  return false;
}

// Shared part of round 0 (validation, referenced vertices, dA) lives in hd_api.cu.
// Enqueues the validation of A, its bounding box and the device-side parameters (no sync).
// Round-0 set-up of A, all on the stream with no host round trip: referenced vertices,
// validation, bounding box and pool entries, then eps / slack (and the warm-start l) on the
// device.  `small` (ref | box | dyn | st) must be zero-filled first.
template <class P>
int prepare_A(const RunIO& io, uint8_t* ref, unsigned long long* box, DynParams* dyn, double slack_scale,
              RunState* st, typename P::Vtx* pool, unsigned* ev) {
  cudaStream_t s = io.s;
  int* bad = (int*)(box + 6);
  TraceScope tr(HD_K_PREP, s);
  const int g_ref = (int)std::min<int64_t>(blocks_for(3 * io.nFA, 256), 16 * 152);
  if (io.vtype == HD_F64) {
    launch_chained(k_mark_ref<double>, g_ref, 256, 0, s, io.FA, io.nFA, io.nVA, ref, bad,
                   (const double*)io.VA, box + 7, ev);
    launch_chained(k_check_init<P, double>, blocks_for(io.nVA, 256), 256, 0, s, (const double*)io.VA, io.nVA, ref, box, bad, pool,
                   (const unsigned*)ev);
  } else {
    launch_chained(k_mark_ref<float>, g_ref, 256, 0, s, io.FA, io.nFA, io.nVA, ref, bad,
                   (const float*)io.VA, box + 7, ev);
    launch_chained(k_check_init<P, float>, blocks_for(io.nVA, 256), 256, 0, s, (const float*)io.VA, io.nVA, ref, box, bad, pool,
                   (const unsigned*)ev);
  }
  launch_chained(k_prep_finish, 1, 1, 0, s, box, io.tol, io.o->tol_mode == HD_TOL_REL ? 1 : 0, slack_scale, dyn, st, io.l0,
                                io.B->meta, cut_enabled(*io.o) ? 1 : 0);
  HD_TRY_LAUNCH();
  return HD_OK;
}

// Buffers of one policy's frontier loop.
template <class P>
struct Rounds {
  char* base = nullptr;  // the single allocation the buffers below are carved from
  typename P::Vtx* pool = nullptr;
  typename P::Item* front[2] = {nullptr, nullptr};
  typename P::Item* promo = nullptr;   // items handed to the FP64 phase (MIXED only)
  typename P::Item* u4list = nullptr;  // items waiting for the u4 pass (MIXED only)
  int4* split_par = nullptr;
  int4* split_mid = nullptr;  // the three midpoint pool indices of every split
  MidTable tab = {nullptr, nullptr, nullptr, 0};
  LongList longq = {nullptr, 0};  // queries handed to k_query_long
  int64_t pool_cap = 0, front_cap = 0, chunk = 0, promo_cap = 0;
  int64_t n_pool = 0, n_front = 0;
  int cur = 1;  // front[cur] holds the current frontier
};

// The largest block the round kernels of policy P launch with (their register use limits it
// below 1024 threads).
template <class P>
int round_block_limit() {
  static std::atomic<int> cached{0};
  int m = cached.load(std::memory_order_relaxed);
  if (!m) {
    m = 1024;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_query<P>) == cudaSuccess) m = std::min(m, fa.maxThreadsPerBlock);
    for (bool paper : {false, true}) {
      if (cudaFuncGetAttributes(&fa, bound_faces_kernel<P>(paper)) == cudaSuccess) m = std::min(m, fa.maxThreadsPerBlock);
      if (cudaFuncGetAttributes(&fa, bound_children_kernel<P>(paper)) == cudaSuccess)
        m = std::min(m, fa.maxThreadsPerBlock);
    }
    if (cudaFuncGetAttributes(&fa, k_bound_u4<P>) == cudaSuccess) m = std::min(m, fa.maxThreadsPerBlock);
    m &= ~31;
    cached.store(m, std::memory_order_relaxed);
  }
  return m;
}

// Blocks of `bs` threads that fill every SM once with `kernel` (at least one per SM): the
// grid of the persistent kernels, whose warps take batches of work (warp_batch).
template <typename K>
unsigned persistent_grid(K kernel, int bs, int sms, size_t smem = 0) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, bs, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
  return (unsigned)(per_sm * sms);
}

// persistent_grid, remembered per block size (32 to 1024 threads, a multiple of 32).
template <typename K>
unsigned persistent_grid_bs(K kernel, int bs, std::atomic<unsigned> (&cache)[33], size_t smem = 0) {
  unsigned g = cache[bs / 32].load(std::memory_order_relaxed);
  if (!g) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g = persistent_grid(kernel, bs, sms, smem);
    cache[bs / 32].store(g, std::memory_order_relaxed);
  }
  return g;
}

// The persistent grids of k_query (per block size) and of k_query_long.
template <class P>
unsigned query_grid(int bs) {
  static std::atomic<unsigned> cache[33];
  return persistent_grid_bs(k_query<P>, bs, cache);
}
template <class P>
unsigned long_grid() {
  static std::atomic<unsigned> cache[33];
  return persistent_grid_bs(k_query_long<P>, 32 * kCoopWarps, cache);
}

struct Totals {
  int64_t rounds = 0, splits = 0, peak = 0;
  int64_t mids = 0;  // midpoints made (shared split edges counted once)
  double u_run = INFINITY;
};

template <class P>
int alloc_rounds(Rounds<P>& R, const Opts& o, int64_t min_pool, int64_t min_front, bool promo, cudaStream_t s) {
  using Vtx = typename P::Vtx;
  using Item = typename P::Item;
  int64_t budget = o.max_frontier_bytes > 0 ? o.max_frontier_bytes : (int64_t)2 << 30;
  R.pool_cap = std::min<int64_t>(std::max<int64_t>(min_pool + 3, (int64_t)(0.6 * budget) / (int64_t)sizeof(Vtx)),
                                 INT32_MAX / 2);
  R.front_cap = std::min<int64_t>(
      std::max<int64_t>(min_front + 4, (int64_t)((promo ? 0.1 : 0.15) * budget) / (int64_t)sizeof(Item)), INT32_MAX / 4);
  R.chunk = o.frontier_chunk > 0 ? o.frontier_chunk : std::max<int64_t>(R.front_cap / 4, 1024);
  R.chunk = std::min<int64_t>(R.chunk, R.front_cap);
  // the midpoint table (shared midpoints only): a power of two of entries, at most half full
  // with the 3 edges of each of a round's splits; the chunk is cut to what it holds (rounds
  // of more splits than the faces of A are rare, and only split over more rounds)
  const bool share = (o.flags & HD_FLAG_SHARE_MIDPOINTS) != 0;
  int64_t n_tab = 0;
  if (share) {
    n_tab = 1 << 12;
    const int64_t want = 6 * std::min<int64_t>(R.chunk, std::max<int64_t>(min_front, 4096));
    while (n_tab < want && n_tab < ((int64_t)1 << 23)) n_tab <<= 1;
    R.chunk = std::max<int64_t>(1, std::min<int64_t>(R.chunk, n_tab / 6));
  }
  R.promo_cap = promo ? R.front_cap : 0;
  // one stream-ordered allocation, carved into the buffers (256-byte aligned)
  auto round_up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_pool = round_up(sizeof(Vtx) * R.pool_cap), b_front = round_up(sizeof(Item) * R.front_cap),
               b_split = round_up(sizeof(int4) * R.chunk), b_promo = promo ? b_front : 0,
               b_key = round_up(sizeof(unsigned long long) * n_tab), b_val = round_up(sizeof(int) * n_tab),
               b_qh = share ? round_up(sizeof(int) * 3 * R.chunk) : 0,
               b_long = round_up(sizeof(int) * std::max<int64_t>(min_pool, 3 * R.chunk));
  // the long-query reordering, where a launch can hand off enough queries for it to matter
  const bool sort = std::max<int64_t>(min_pool, 3 * R.chunk) >= kSortMin;
  const size_t b_sorted = sort ? b_long : 0, b_buckets = sort ? round_up(sizeof(unsigned) * kSortBuckets) : 0;
  char* base = nullptr;
  HD_TRY(cudaMallocAsync((void**)&base, b_pool + 2 * b_front + 2 * b_split + 2 * b_promo + b_key + b_val + b_qh + b_long +
                                            b_sorted + b_buckets,
                         s));
  R.base = base;
  char* p = base;
  auto carve = [&p](size_t b) {
    char* q = p;
    p += b;
    return q;
  };
  R.pool = (Vtx*)carve(b_pool);
  R.front[0] = (Item*)carve(b_front);
  R.front[1] = (Item*)carve(b_front);
  R.split_par = (int4*)carve(b_split);
  R.split_mid = (int4*)carve(b_split);
  R.longq = {(int*)carve(b_long), (int)std::max<int64_t>(min_pool, 3 * R.chunk)};
  if (sort) {
    R.longq.sorted = (int*)carve(b_sorted);
    R.longq.buckets = (unsigned*)carve(b_buckets);
  }
  if (share) {
    R.tab.key = (unsigned long long*)carve(b_key);
    R.tab.val = (int*)carve(b_val);
    R.tab.qhash = (int*)carve(b_qh);
    R.tab.mask = (unsigned)(n_tab - 1);
  }
  if (promo) {
    R.promo = (Item*)carve(b_promo);
    R.u4list = (Item*)carve(b_promo);
  }
  if (share) HD_TRY(cudaMemsetAsync(R.tab.key, 0, b_key + b_val, s));  // key and val are adjacent
  return HD_OK;
}

template <class P>
void free_rounds(Rounds<P>& R, cudaStream_t s) {
  if (R.base) cudaFreeAsync(R.base, s);
  R.base = nullptr;
}

// Pinned host memory the round loop reads into: the final run state and parameters, and a
// ring of two per-round snapshots, with the events that mark them complete.  Kept for the
// thread's lifetime and released when it exits.
struct HostBlock {
  RunState st;
  RunState ring[2];
  DynParams dyn;
};
struct HostRes {
  HostBlock* hb = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ~HostRes() {
    if (hb) cudaFreeHost(hb);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
};
inline int host_res(HostRes*& out) {
  static thread_local HostRes r;
  if (!r.hb) HD_TRY(cudaMallocHost((void**)&r.hb, sizeof(HostBlock)));
  for (cudaEvent_t& e : r.ev)
    if (!e) HD_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  out = &r;
  return HD_OK;
}

#ifndef HD_AHEAD_FROM
#define HD_AHEAD_FROM 2  // rounds read before the host keeps one round queued ahead
#endif

// k_tail_rounds takes more than the default 48 KB of dynamic shared memory: allowed once per
// device.
template <class P>
cudaError_t tail_smem_attr() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_relaxed) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(k_tail_rounds<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_relaxed);
  return e;
}

// Frontier rounds of policy P over the items that the bound kernel before it left in
// R.front[R.cur] (their count in st->n_next), until the frontier is empty, the capacity or
// round limit is reached, or an error is flagged.  Each round starts with k_round_ctl, which
// closes the previous round and sizes this one on the device.  The first two rounds are
// queued one at a time, with grids sized from the frontier the host has just read; from the
// third on (runs with many rounds), the host keeps one round queued ahead of the one it is
// reading, so the GPU does not wait for the host between rounds, with grids sized from a
// bound on the frontier (4 children per item); the round queued after the last one finds
// the loop stopped and does nothing.  On return hr.hb->st and ->dyn hold the final state, T
// is updated and *status says why the loop ended.
template <class P>
int loop_rounds(const RunIO& io, Rounds<P>& R, RunState* st, HostRes& hr, const RunParams& rp, Totals& T,
                int* status, const unsigned long long* bad, int n_pool0, int64_t first_front_bound) {
  const Opts& o = *io.o;
  cudaStream_t s = io.s;
  BvhDev B = bvh_dev(io.B);
  const int bs = o.block_size;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned max_grid = (unsigned)sms * 16;
  RoundCtl c;
  c.chunk = R.chunk;
  c.pool_cap = R.pool_cap;
  c.front_cap = R.front_cap;
  c.share = R.tab.key ? 1 : 0;
  const double cap_splits = std::floor((o.max_face_factor * (double)io.nFA - (double)io.nFA) / 4.0);
  c.splits_left = (long long)std::max(0.0, std::min(cap_splits - (double)T.splits, 9.0e18));
  c.rounds_left = std::max<long long>(0, o.max_rounds - T.rounds);
  c.bad = bad;
  static std::atomic<unsigned> grid_b_cache[2][33];
  const bool paper = paper_cascade(rp);
  const auto k_children = bound_children_kernel<P>(paper);
  const size_t smem_b = rebin_smem(bs);  // the u3 queues of the paper-order kernels
  const unsigned grid_q = query_grid<P>(bs),
                 grid_b = persistent_grid_bs(k_children, bs, grid_b_cache[paper ? 1 : 0], smem_b);
  const unsigned grid_long = long_grid<P>();
  int64_t front_bound = first_front_bound;  // the first round is queued without a wait
  int cur = R.cur;
  bool init = true;
  // the run state and parameters after the work queued so far, into ring slot `slot`
  auto snapshot = [&](int slot) -> int {
    HD_TRY(cudaMemcpyAsync(&hr.hb->ring[slot], st, sizeof(RunState), cudaMemcpyDeviceToHost, s));
    HD_TRY(cudaMemcpyAsync(&hr.hb->dyn, rp.dyn, sizeof(DynParams), cudaMemcpyDeviceToHost, s));
    g_d2h_bytes += sizeof(RunState) + sizeof(DynParams);
    HD_TRY(cudaEventRecord(hr.ev[slot], s));
    return HD_OK;
  };
  auto issue = [&](int slot, int64_t nf) -> int {
    // grids for a frontier of at most nf items (grid-stride kernels: any size is correct)
    const int64_t k = std::max<int64_t>(1, std::min<int64_t>(nf, R.chunk));
    const unsigned g_sel = std::min(blocks_for(std::max<int64_t>(nf, 1), 256), (unsigned)sms * 8);
    const unsigned g_q = std::min(blocks_for(3 * k, bs), grid_q), g_b = std::min(blocks_for(4 * k, bs), grid_b);
    const unsigned g_u4 = std::min(blocks_for(4 * k, bs), max_grid);
    {
      TraceScope tr(HD_K_SELECT, s);
      launch_chained(k_round_ctl, 1, 1, 0, s, st, c, init ? 1 : 0, n_pool0);
      init = false;
      launch_chained(k_select<P>, g_sel, 256, 0, s, R.front[cur], st, rp, R.split_par, R.split_mid, R.tab, R.pool,
                                        R.front[cur ^ 1],
                                        (int)R.front_cap, R.promo, (int)R.promo_cap);
    }
    {
      TraceScope tr(HD_K_QUERY, s);
      launch_chained(k_query<P>, g_q, bs, 0, s, B, R.pool, 0, nullptr, 3, 0, st, rp.slack, rp.dyn, true, R.tab, R.longq);
    }
    {
      TraceScope tr(HD_K_LONG, s);
      sort_long<P>(B, R.pool, R.longq, st, true, sms, s, rp.dyn);
      launch_chained(k_query_long<P>, grid_long, 32 * kCoopWarps, 0, s, B, R.pool, R.longq, st, rp.slack, rp.dyn, true);
    }
    {
      TraceScope tr(HD_K_BOUND, s);
      launch_chained(k_children, g_b, bs, smem_b, s, B, R.pool, R.split_par, R.split_mid, st, rp, R.front[cur ^ 1],
                     (int)R.front_cap, R.u4list);
      if (R.u4list)
        launch_chained(k_bound_u4<P>, g_u4, bs, 0, s, B, R.pool, R.u4list, (int)R.front_cap, st, rp, R.front[cur ^ 1],
                                          (int)R.front_cap);
    }
    HD_TRY_LAUNCH();
    cur ^= 1;
    return snapshot(slot);
  };
  // the small-round kernel, for a frontier of at most kTailFront items; it may run any number
  // of rounds, so nothing is queued after it until its snapshot has been read
  const TailBufs<P> tb = {{R.front[0], R.front[1]}, R.split_par, R.split_mid, R.tab, R.pool, R.promo, (int)R.promo_cap,
                          (int)R.front_cap, R.u4list, R.longq};
  auto issue_tail = [&](int slot) -> int {
    HD_TRY(tail_smem_attr<P>());
    {
      TraceScope tr(HD_K_SMALL, s);
      launch_chained(k_tail_rounds<P>, 1, kTailThreads, kTailSmem, s, B, tb, st, rp, c, init ? 1 : 0, n_pool0, cur);
      init = false;
    }
    HD_TRY_LAUNCH();
    return snapshot(slot);
  };
  long long issued = 0, seen = 0, tail_at = -1;  // tail_at: the snapshot of the small-round kernel in flight
  int last_long = 0;  // long queries of the last round read
  for (;;) {
    const long long ahead = seen >= HD_AHEAD_FROM ? 2 : 1;  // rounds in flight, the one being read included
    while (issued < seen + ahead && tail_at < 0) {
      int rc;
      if (front_bound <= kTailFront && last_long <= kTailLong && !(o.flags & HD_FLAG_NO_SMALL_ROUNDS)) {
        rc = issue_tail((int)(issued & 1));
        tail_at = issued;
      } else {
        rc = issue((int)(issued & 1), front_bound);
      }
      if (rc != HD_OK) return rc;
      ++issued;
      front_bound = std::min<int64_t>(4 * front_bound, R.front_cap);  // for a round queued ahead
    }
    HD_TRY(cudaEventSynchronize(hr.ev[seen & 1]));
    const RunState& h = hr.hb->ring[seen & 1];
    if (seen == tail_at) {  // the small-round kernel's rounds each swapped the frontier buffers
      if (h.tail_rounds & 1) cur ^= 1;
      tail_at = -1;
    }
    last_long = h.n_long;
    ++seen;
    // the next round's frontier is h.n_next; one more round ahead may have up to 4x as many
    front_bound = issued == seen ? (int64_t)h.n_next : std::min<int64_t>(4 * (int64_t)h.n_next, R.front_cap);
    // over once a round stopped, or when the next round's control will stop it
    const bool done = h.stop || h.n_next == 0 || h.overflow || h.err || h.bad ||
                      h.rounds + (h.in_round ? 1 : 0) >= c.rounds_left;
    if (done) break;
  }
  if (issued == seen) {
    // nothing queued after the last round read: that state is final once the round is closed
    // (the same closing step k_round_ctl would take); the parameters were read with it
    hr.hb->st = hr.hb->ring[(seen - 1) & 1];
    RunState& f = hr.hb->st;
    if (!f.stop) {
      const int r = close_round(f, c.rounds_left);
      f.status = r >= 0 ? r : HD_ERR_CAPACITY;  // -1 cannot happen here: the loop was done
      f.stop = 1;
    }
  } else {
    HD_TRY(cudaMemcpyAsync(&hr.hb->st, st, sizeof(RunState), cudaMemcpyDeviceToHost, s));
    HD_TRY(cudaMemcpyAsync(&hr.hb->dyn, rp.dyn, sizeof(DynParams), cudaMemcpyDeviceToHost, s));
    g_d2h_bytes += sizeof(RunState) + sizeof(DynParams);
    HD_TRY(cudaStreamSynchronize(s));
  }
  const RunState& f = hr.hb->st;
  T.rounds += f.rounds;
  T.splits += f.splits;
  T.mids += f.n_pool - n_pool0;
  T.peak = std::max<int64_t>(T.peak, f.peak);
  T.u_run = std::min(T.u_run, bits_to_double(f.urun_bits));
  R.n_pool = f.n_pool;
  R.n_front = f.n_front;
  *status = f.status;
  return HD_OK;
}

// Promoted MIXED items: their vertices at exact positions in an FP64 pool, and index triples.
template <class P>
__global__ void k_promote_init(const typename P::Item* promo, int n, const typename P::Vtx* pool, VtxD* poolD,
                               int32_t* tris) {
  grid_dep_wait();
  grid_dep_launch();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  typename P::Item it = promo[i];
  for (int k = 0; k < 3; ++k) {
    typename P::Vtx v = pool[it.v[k]];
    D3 x = P::exact_pos(v);
    VtxD d;
    memset(&d, 0, sizeof d);
    d.x = x.x;
    d.y = x.y;
    d.z = x.z;
    d.tri = -2;
    d.hint = v.tri;
    poolD[3 * i + k] = d;
    tris[3 * i + k] = 3 * i + k;
  }
}

// Final certification (a7): sub-triangles whose gap the FP32 error radius cannot resolve are
// re-queried and bounded in FP64 (with the same slack margin) and refined to the end there.
// Start of the FP64 phase: an empty next frontier and no promotions.
static __global__ void k_phase_reset(RunState* st) {
  grid_dep_wait();
  grid_dep_launch();
  st->q_next = 0;
  st->b_next = 0;
  st->n_next = 0;
  st->n_split = 0;
  st->n_u4 = 0;
  st->umax_bits = 0;
  st->overflow = 0;
  st->upro_bits = 0;
  st->n_promote = 0;
  st->n_mid = 0;
  st->n_long = 0;
  st->long_next = 0;
}

template <class P>
int finish_in_fp64(const RunIO& io, Rounds<P>& RM, int64_t n_pro, RunState* st, HostRes& hr, const RunParams& rp,
                   Totals& T, int* status, const unsigned long long* bad) {
  cudaStream_t s = io.s;
  const Opts& o = *io.o;
  BvhDev B = bvh_dev(io.B);
  Rounds<PolicyD> D;
  int rc = alloc_rounds<PolicyD>(D, o, 3 * n_pro, n_pro, false, s);
  if (rc != HD_OK) return rc;
  int32_t* tris = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&tris, sizeof(int32_t) * 3 * n_pro, s);
  if (e != cudaSuccess) {
    free_rounds(D, s);
    return set_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
  }
  {
    TraceScope tr(HD_K_PREP, s);
    launch_chained(k_promote_init<P>, blocks_for(n_pro, 256), 256, 0, s, RM.promo, (int)n_pro, RM.pool, D.pool, tris);
    launch_chained(k_phase_reset, 1, 1, 0, s, st);
  }
  HD_TRY_LAUNCH();
  {
    TraceScope tr(HD_K_QUERY, s);
    launch_chained(k_query<PolicyD>, blocks_for(3 * n_pro, o.block_size), o.block_size, 0, s,
        B, D.pool, 0, nullptr, 1, (int)(3 * n_pro), st, rp.slack, rp.dyn, false, MidTable{nullptr, nullptr, nullptr, 0},
        D.longq);
  }
  {
    TraceScope tr(HD_K_LONG, s);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sort_long<PolicyD>(B, D.pool, D.longq, st, false, sms, s, rp.dyn);
    launch_chained(k_query_long<PolicyD>, long_grid<PolicyD>(), 32 * kCoopWarps, 0, s, B, D.pool, D.longq, st, rp.slack,
                   rp.dyn, false);
  }
  {
    TraceScope tr(HD_K_BOUND, s);
    RunParams rpd = rp;
    rpd.defer_u4 = 0;
    launch_chained(k_bound_faces<PolicyD>, blocks_for(n_pro, o.block_size), o.block_size, 0, s, B, D.pool, tris, n_pro, st, rpd,
                                                                                   D.front[1], (int)D.front_cap,
                                                                                   nullptr, 3 * n_pro);
  }
  HD_TRY_LAUNCH();
  D.cur = 1;
  rc = loop_rounds<PolicyD>(io, D, st, hr, rp, T, status, bad, (int)(3 * n_pro), n_pro);
  cudaFreeAsync(tris, s);
  free_rounds(D, s);
  return rc;
}

template <class P>
int run_bnb(const RunIO& io) {
  const Opts& o = *io.o;
  cudaStream_t s = io.s;
  hd_result& res = *io.out;
  memset(&res, 0, sizeof res);
  // a block the round kernels cannot launch with (MIXED also runs the FP64 ones)
  if (o.block_size > round_block_limit<P>() || (!P::kFp64 && o.block_size > round_block_limit<PolicyD>()))
    return HD_ERR_INVALID;
  const long long launches0 = g_launches, d2h0 = g_d2h_bytes;

  HostRes* hr = nullptr;
  {
    const int rh = host_res(hr);
    if (rh != HD_OK) return rh;
  }

  // small per-call device block: referenced-vertex flags, A's bbox + invalid flag, the
  // device-side parameters, and the run state
  // device-side parameters, and the run state; with cuts, the longest edge at each vertex
  const size_t ref_bytes = ((size_t)std::max<int64_t>(io.nVA, 1) + 255) & ~(size_t)255;
  const size_t st_bytes = (sizeof(RunState) + 255) & ~(size_t)255;
  const size_t ev_bytes = cut_enabled(o) && P::kEdgePerVertex ? sizeof(unsigned) * (size_t)std::max<int64_t>(io.nVA, 1) : 0;
  unsigned char* small = nullptr;
  HD_TRY(cudaMallocAsync((void**)&small, ref_bytes + 512 + st_bytes + ev_bytes, s));
  uint8_t* ref = small;
  unsigned long long* box = (unsigned long long*)(small + ref_bytes);  // [0..5] bbox, [6] invalid flags, [7] A's longest edge squared
  DynParams* dyn = (DynParams*)(small + ref_bytes + 256);
  RunState* st = (RunState*)(small + ref_bytes + 512);
  unsigned* ev = ev_bytes ? (unsigned*)(small + ref_bytes + 512 + st_bytes) : nullptr;
  HD_TRY(cudaMemsetAsync(small, 0, ref_bytes + 512 + st_bytes + ev_bytes, s));

  Rounds<P> R;
  int rc = alloc_rounds<P>(R, o, io.nVA, io.nFA, !P::kFp64, s);
  if (rc != HD_OK) {
    cudaFreeAsync(small, s);
    return rc;
  }
  // validation of A, its bbox and the pool entries of its vertices run asynchronously; the
  // host reads the result with round 0
  rc = prepare_A<P>(io, ref, box, dyn, P::slack(1.0), st, R.pool, ev);
  if (rc != HD_OK) {
    free_rounds(R, s);
    cudaFreeAsync(small, s);
    return rc;
  }

  BvhDev B = bvh_dev(io.B);
  RunParams rp;
  rp.eps = 0.0;  // taken from dyn on the device
  rp.slack = 0.0;
  rp.slack_f = 0.f;
  rp.dyn = dyn;
  rp.defer_u4 = P::kFp64 ? 0 : 1;
  rp.parent_clamp = (o.flags & HD_FLAG_NO_PARENT_CLAMP) ? 0 : 1;
  memcpy(rp.order, o.order, 4);
  rp.n_bounds = o.n_bounds;
  const int bs = o.block_size;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned max_grid = (unsigned)sms * 16;

  // round 0: vertices of A, their nearest triangles, l, and the bounds of every face
  {
    TraceScope tr(HD_K_QUERY, s);
    launch_chained(k_query<P>, std::min(blocks_for(io.nVA, bs), query_grid<P>(bs)), bs, 0, s,
        B, R.pool, 0, nullptr, 1, (int)io.nVA, st, rp.slack, rp.dyn, false, MidTable{nullptr, nullptr, nullptr, 0},
        R.longq);
  }
  {
    TraceScope tr(HD_K_LONG, s);
    sort_long<P>(B, R.pool, R.longq, st, false, sms, s, rp.dyn);
    launch_chained(k_query_long<P>, long_grid<P>(), 32 * kCoopWarps, 0, s, B, R.pool, R.longq, st, rp.slack, rp.dyn, false);
  }
  HD_TRY_LAUNCH();
  {
    TraceScope tr(HD_K_BOUND, s);
    const auto k_faces = bound_faces_kernel<P>(paper_cascade(rp));
    launch_chained(k_faces, std::min(blocks_for(io.nFA, bs), persistent_grid(k_faces, bs, sms, rebin_smem(bs))), bs,
                   rebin_smem(bs), s, 
        B, R.pool, io.FA, io.nFA, st, rp, R.front[1],
                                                           (int)R.front_cap, R.u4list, io.nVA);
    if (R.u4list)
      launch_chained(k_bound_u4<P>, max_grid, bs, 0, s, B, R.pool, R.u4list, (int)R.front_cap, st, rp, R.front[1],
                                            (int)R.front_cap);
  }
  HD_TRY_LAUNCH();

  // frontier rounds; A's and B's validity is read with the first of them (their results are
  // not used when either is invalid)
  const unsigned long long* bad = box + 6;
  Totals T;
  R.cur = 1;
  int status = HD_OK;
  rc = loop_rounds<P>(io, R, st, *hr, rp, T, &status, bad, (int)io.nVA, io.nFA);
  if (rc == HD_OK && status == HD_ERR_INVALID) rc = HD_ERR_INVALID;
  const int64_t n_pro = hr->hb->st.n_promote;
  if (rc == HD_OK && status == HD_OK && n_pro > 0)
    rc = finish_in_fp64<P>(io, R, std::min<int64_t>(n_pro, R.promo_cap), st, *hr, rp, T, &status, bad);
  if (rc != HD_OK) {
    free_rounds(R, s);
    cudaFreeAsync(small, s);
    return rc;
  }
  const RunState* hst = &hr->hb->st;
  res.stats.dA = hr->hb->dyn.dA;
  res.stats.eps_abs = hr->hb->dyn.eps;

  double l = bits_to_double(hst->l_bits);
  double uret = bits_to_double(hst->uret_bits);
  if (status == HD_OK) {
    // frontier empty: everything was discarded or retired
    T.u_run = std::min(T.u_run, std::max(l, uret));
    // in exact arithmetic the sub-triangle holding the farthest point of A is never
    // discarded, so some retired U is >= h >= l -- unless l was warm-started above h
    if (P::kFp64 && uret < l && !(io.l0 > 0.0)) status = HD_ERR_NUMERIC;
  }
  res.lower = l;
  res.upper = std::max(l, T.u_run);
  res.status = status;
  hd_stats& S = res.stats;
  S.rounds = T.rounds;
  S.splits = T.splits;
  S.queries = (int64_t)hst->queries;
  S.long_queries = (int64_t)hst->long_queries;
  S.kernel_launches = g_launches - launches0;
  S.d2h_bytes = g_d2h_bytes - d2h0;
  S.pointtri_evals = (int64_t)hst->evals;
  S.leaf_tests = (int64_t)hst->leaf_tests;
  S.box_tests = (int64_t)hst->box_tests;
  for (int k = 0; k < 6; ++k) S.discards[k] = (int64_t)hst->discards[k];
  S.retired = (int64_t)hst->retired;
  S.fp64_escalations = (int64_t)hst->escalations;
  S.promoted = n_pro;
  S.node_visits = (int64_t)hst->node_visits;
  S.long_node_visits = (int64_t)hst->long_node_visits;
  S.long_leaf_tests = (int64_t)hst->long_leaf_tests;
  S.queries_cut = (int64_t)hst->queries_cut;
  S.peak_frontier = T.peak;
  S.pool_vertices = io.nVA + T.mids;

  free_rounds(R, s);
  cudaFreeAsync(small, s);
  return HD_OK;
}

// ----------------------------------------------------------------------------- point queries

template <class P, typename T>
__global__ void k_points_in(const T* P_, int64_t n, typename P::Vtx* v) {
  grid_dep_wait();
  grid_dep_launch();
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
  grid_dep_wait();
  grid_dep_launch();
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

// Nearest queries of n point records (k_points_in) on stream s.  With a list of n ints (and
// n below 2^30), the lane traversal hands long queries to k_query_long as in the rounds;
// without one, every lane finishes its own query.  `st` must be zeroed.
template <class P>
void query_points(const BvhDev& B, typename P::Vtx* rec, int64_t n, RunState* st, int* list, cudaStream_t s,
                  int* sorted = nullptr, unsigned* buckets = nullptr) {
  if (list && n <= INT32_MAX / 2) {
    const LongList ll = {list, (int)n, sorted, buckets};
    launch_chained(k_query<P>, std::min(blocks_for(n, 128), query_grid<P>(128)), 128, 0, s, B, rec, 0, nullptr, 1,
                   (int)n, st, 0.0, nullptr, false, MidTable{nullptr, nullptr, nullptr, 0}, ll);
    if (sorted) {
      int dev = 0, sms = 1;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      sort_long<P>(B, rec, ll, st, false, sms, s, nullptr);
    }
    launch_chained(k_query_long<P>, long_grid<P>(), 32 * kCoopWarps, 0, s, B, rec, ll, st, 0.0, nullptr, false);
  } else {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    launch_chained(k_query_points<P>, std::min(blocks_for(n, 128), (unsigned)sms * 16u), 128, 0, s, B, rec, n, st);
  }
}

// hd_nearest: nearest triangle of B for n external points (P as float or double rows).
template <class P>
int nearest_points(const hd_bvh* B, const void* Pts, int ptype, int64_t n, cudaStream_t s, double* dist,
                   int32_t* idx, double* foot, double* dlo) {
  typename P::Vtx* tmp = nullptr;
  RunState* st = nullptr;
  int* list = nullptr;
  int* sorted = nullptr;
  unsigned* buckets = nullptr;
  const bool two_phase = n <= INT32_MAX / 2;  // k_query counts in int
  HD_TRY(cudaMallocAsync((void**)&tmp, sizeof(typename P::Vtx) * n, s));
  HD_TRY(cudaMallocAsync((void**)&st, sizeof(RunState), s));
  if (two_phase) HD_TRY(cudaMallocAsync((void**)&list, sizeof(int) * n, s));
  if (two_phase && n >= kSortMin) {
    HD_TRY(cudaMallocAsync((void**)&sorted, sizeof(int) * n, s));
    HD_TRY(cudaMallocAsync((void**)&buckets, sizeof(unsigned) * kSortBuckets, s));
  }
  HD_TRY(cudaMemsetAsync(st, 0, sizeof(RunState), s));
  if (ptype == HD_F64)
    launch_chained(k_points_in<P, double>, blocks_for(n, 256), 256, 0, s, (const double*)Pts, n, tmp);
  else
    launch_chained(k_points_in<P, float>, blocks_for(n, 256), 256, 0, s, (const float*)Pts, n, tmp);
  {
    TraceScope tr(HD_K_QUERY, s);
    query_points<P>(bvh_dev(B), tmp, n, st, list, s, sorted, buckets);
  }
  launch_chained(k_points_out<P>, blocks_for(n, 256), 256, 0, s, tmp, n, B->tri_vid, dist, idx, foot, dlo);
  HD_TRY_LAUNCH();
  HD_TRY(cudaFreeAsync(tmp, s));
  HD_TRY(cudaFreeAsync(st, s));
  if (list) HD_TRY(cudaFreeAsync(list, s));
  if (sorted) HD_TRY(cudaFreeAsync(sorted, s));
  if (buckets) HD_TRY(cudaFreeAsync(buckets, s));
  return HD_OK;
}

}  // namespace hd
