// Many independent pairs (A_i, B_i) in one frontier-parallel branch and bound (Sections 3.1
// and 4 for every pair at once): the same steps as the single-pair rounds of hd_bnb.cuh, but
// every launch works on the items of all pairs together, so a batch of small pairs is not
// bound by launches and host waits.
//
//  * Work queue.  Every phase kernel is a persistent grid whose warps take batches of 32
//    consecutive work items (vertices, faces, frontier items, split slots) from one
//    device-side counter; an item carries its pair, whose BVH, tolerance, lower bound l and
//    statistics it works with.  Items of one pair are mostly contiguous, so a batch of 32
//    usually belongs to one pair: per-pair counts and maxima are then combined across the
//    warp into one atomic, and lane by lane only when the batch straddles pairs.
//  * Storage.  One vertex pool, two frontier buffers, a split list, the u4 and promotion lists
//    (MIXED) for all pairs, each with a parallel array of pair indices; A's vertices of pair p
//    occupy pool slots [vbase_p, vbase_p + nV_p), midpoints are appended for all pairs.
//  * Per pair, in device memory: its l, the retired / frontier / promoted maxima of U, the
//    running minimum of the round upper bounds, its counts, status and stop flag (a RunState
//    each), and its eps / slack (a DynParams each).  A pair retires on its own: when its
//    frontier is empty (u - l <= eps, Section 3.1), its face cap m n_A is reached (CAPACITY)
//    or its round limit (TIMEOUT); its items are then dropped by the next select.
//  * Round control on the device (k_batch_ctl, one block): closes every pair's round with the
//    same close_round step as the single-pair loop, then sizes the next round for the whole
//    batch (a split budget from the free pool and frontier room); the host only reads a
//    snapshot per round, one round behind the one it queues.
//  * MIXED: items whose gap is below FP32 resolution are promoted as in a single run and
//    finished afterwards by the same batched machinery in FP64 (a7).
#pragma once

#include <vector>

#include "hd_bnb.cuh"

namespace hd {

// One pair of a batch, as the kernels see it.
struct PairDev {
  BvhDev B;
  const void* VA;     // device, nVA x 3, element type vtype
  const int32_t* FA;  // device, nFA x 3 (indices into this pair's vertices)
  int vtype;
  int nVA, nFA;
  int vbase;  // pool slot of this pair's first vertex
  long long splits_cap;  // splits the face cap m n_A allows this pair (Section 4)
};

// Batch-wide round state.
struct BatchState {
  int n_front;    // items in the current frontier (all pairs)
  int n_next;     // items appended to the next frontier
  int n_split;    // split slots taken this round
  int n_u4;       // items in the u4 list (MIXED)
  int n_promote;  // items handed to the FP64 phase (MIXED)
  int n_long;     // queries handed to the cooperative traversal by the last query launch
  int q_next, b_next, long_next;  // work counters of the query, bound and cooperative kernels
  int K;          // split slots this round
  int n_pool;     // pool vertices before this round's midpoints
  int overflow;   // a list ran out of room (cannot happen with the sizes chosen on the host)
  int stop;       // every pair is done
  int in_round;   // a round has been opened
  int active;     // pairs still running
  int pad0;
  long long rounds;
};

// Per-launch constants of the batched kernels.
struct BatchCtx {
  const PairDev* pd;
  RunState* sts;
  DynParams* dyn;
  BatchState* bs;
  const int* vbase;  // npairs + 1 prefix sums of the pairs' vertex counts (pool slots)
  const int* fbase;  // npairs + 1 prefix sums of the pairs' face counts
  int npairs;
  int nV, nF;        // totals
  RunParams rp;      // order, n_bounds, defer_u4, parent_clamp (eps and slack come per pair)
};

// The pair whose range [base[p], base[p + 1]) holds g (base ascending, base[0] = 0).
__device__ inline int find_pair(const int* base, int np, int g) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The pair all lanes with a pair (>= 0) share, -1 if no lane has one, -2 if they differ.
// Every lane of the warp must call it.
__device__ inline int warp_pair(int pair) {
  const int key = pair >= 0 ? pair : INT_MAX;
  int m = key;
  for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (m == INT_MAX) return -1;
  return __all_sync(0xffffffffu, pair < 0 || pair == m) ? m : -2;
}

// The parameters of pair p: RunParams with its eps and slack, and its l and thresholds.
template <class P>
struct PairLevel {
  RunParams rp;
  Level<P> lv;
};
template <class P>
__device__ inline PairLevel<P> pair_level(const BatchCtx& x, int p) {
  RunParams rp = x.rp;
  rp.dyn = x.dyn + p;
  rp = with_dyn(rp);
  const double l = load_l(x.sts + p);
  return PairLevel<P>{rp, Level<P>{l, __double2float_rd(l), Thresholds<P>(l, rp.eps)}};
}

// Work counters of one lane for pair `pair` (-1: none), flushed per batch of 32.  Every lane
// of the warp must call it.
__device__ inline void flush_counters_pair(RunState* sts, int pair, const Counters& c, bool long_pass = false) {
  const int u = warp_pair(pair);
  if (u >= 0) {
    flush_counters(sts + u, c, long_pass);
    return;
  }
  if (u == -1 || pair < 0) return;
  RunState* st = sts + pair;
  if (c.evals + c.leaf) atomicAdd(&st->evals, (unsigned long long)(c.evals + c.leaf));
  if (c.leaf) atomicAdd(&st->leaf_tests, (unsigned long long)c.leaf);
  if (c.boxes) atomicAdd(&st->box_tests, (unsigned long long)c.boxes);
  if (c.escalations) atomicAdd(&st->escalations, (unsigned long long)c.escalations);
  if (c.nodes) atomicAdd(&st->node_visits, (unsigned long long)c.nodes);
  if (long_pass && c.nodes) atomicAdd(&st->long_node_visits, (unsigned long long)c.nodes);
  if (long_pass && c.leaf) atomicAdd(&st->long_leaf_tests, (unsigned long long)c.leaf);
  if (c.err) atomicExch(&st->err, 1);
}

// Lower bound and query count of one lane for its pair.  Every lane must call it.  l stays
// non-negative (a certified vertex distance less its slack can be below 0), which the atomic
// maximum on its bits needs.
__device__ inline void flush_lower_pair(RunState* sts, int pair, double lmax, int nq, bool long_pass) {
  lmax = fmax(lmax, 0.0);
  const int u = warp_pair(pair);
  if (u >= 0) {
    const double m = warp_max(pair >= 0 ? lmax : 0.0);
    const unsigned long long q = warp_sum((unsigned long long)(pair >= 0 ? nq : 0));
    if ((threadIdx.x & 31) == 0) {
      atomic_max_nonneg(&sts[u].l_bits, m);
      if (q) atomicAdd(&sts[u].queries, q);
      if (q && long_pass) atomicAdd(&sts[u].long_queries, q);
    }
    return;
  }
  if (u == -1 || pair < 0) return;
  atomic_max_nonneg(&sts[pair].l_bits, lmax);
  if (nq) atomicAdd(&sts[pair].queries, (unsigned long long)nq);
  if (nq && long_pass) atomicAdd(&sts[pair].long_queries, (unsigned long long)nq);
}

// Outcome of one lane's item for its pair (the Tally of a single run, one item at a time,
// plus the pair's frontier count), flushed per batch of 32.  Every lane must call it.
template <class P>
struct PairTally {
  int discard = -1;  // deciding bound of a discard (0..5), -1 none
  int retired = 0, kept = 0;
  typename P::UT uret = 0, umax = 0;
};
template <class P>
__device__ inline void flush_tally_pair(RunState* sts, int pair, const PairTally<P>& t) {
  const int u = warp_pair(pair);
  if (u >= 0) {
    Tally<P> w;
    const bool on = pair >= 0;
    w.d0 = on && t.discard == 0;
    w.d1 = on && t.discard == 1;
    w.d2 = on && t.discard == 2;
    w.d3 = on && t.discard == 3;
    w.d4 = on && t.discard == 4;
    w.d5 = on && t.discard == 5;
    w.retired = on ? t.retired : 0;
    w.uret = on ? t.uret : 0;
    w.umax = on ? t.umax : 0;
    flush_tally(sts + u, w);
    const unsigned long long k = warp_sum((unsigned long long)(on ? t.kept : 0));
    if ((threadIdx.x & 31) == 0 && k) atomicAdd(&sts[u].n_next, (int)k);
    return;
  }
  if (u == -1 || pair < 0) return;
  RunState* st = sts + pair;
  if (t.discard >= 0) atomicAdd(&st->discards[t.discard], 1ull);
  if (t.retired) {
    atomicAdd(&st->retired, 1ull);
    atomic_max_nonneg(&st->uret_bits, (double)t.uret);
  }
  if (t.kept) {
    atomicAdd(&st->n_next, 1);
    atomic_max_nonneg(&st->umax_bits, (double)t.umax);
  }
}

// Discard / retire / keep one bounded item of pair p (Section 3.1: discard when U < l); a
// trailing u4 goes to the u4 list (MIXED).
template <class P>
__device__ inline void classify_pair(BatchState* bs, const typename P::Item& it, int p, const Thresholds<P>& th,
                                     int code, typename P::Item* next, int* next_pair, int next_cap,
                                     typename P::Item* u4list, int* u4_pair, PairTally<P>& ty) {
  if (code == kDeferU4) {
    const int j = warp_slot(&bs->n_u4);
    if (j < next_cap) {
      u4list[j] = it;
      u4_pair[j] = p;
    } else {
      atomicExch(&bs->overflow, 1);
    }
    return;
  }
  if (it.U < th.lo) {
    ty.discard = code;
  } else if (it.U <= th.hi) {
    ty.retired = 1;
    ty.uret = it.U;
  } else {
    const int j = warp_slot(&bs->n_next);
    if (j < next_cap) {
      next[j] = it;
      next_pair[j] = p;
      ty.kept = 1;
      ty.umax = it.U;
    } else {
      atomicExch(&bs->overflow, 1);
    }
  }
}

// ----------------------------------------------------------------------------- round 0

// Referenced vertices and the validity of every pair's faces (one thread per face corner).
static __global__ void k_batch_mark_ref(BatchCtx x, uint8_t* ref, unsigned long long* boxes) {
  grid_dep_wait();
  grid_dep_launch();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 3 * (int64_t)x.nF) return;
  const int g = (int)(i / 3);
  const int p = find_pair(x.fbase, x.npairs, g);
  const PairDev& d = x.pd[p];
  const int v = d.FA[3 * (int64_t)(g - x.fbase[p]) + (int)(i % 3)];
  if (v < 0 || v >= d.nVA) atomicOr(&boxes[8 * p + 6], 1ull);
  else ref[d.vbase + v] = 1;
}

// Finite coordinates, each pair's bounding box of referenced vertices (ordered bits, as
// k_check_init) and the pool entries of every pair's vertices.
template <class P>
__global__ void k_batch_check_init(BatchCtx x, const uint8_t* ref, unsigned long long* boxes, typename P::Vtx* pool,
                                   int* vpair) {
  grid_dep_wait();
  grid_dep_launch();
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < x.nV; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = base + threadIdx.x;
    int p = -1;
    unsigned long long m[6] = {0, 0, 0, 0, 0, 0};
    if (g < x.nV) {
      p = find_pair(x.vbase, x.npairs, (int)g);
      const PairDev& d = x.pd[p];
      const int64_t k = g - d.vbase;
      double X, Y, Z;
      if (d.vtype == HD_F64) {
        const double* V = (const double*)d.VA;
        X = V[3 * k], Y = V[3 * k + 1], Z = V[3 * k + 2];
      } else {
        const float* V = (const float*)d.VA;
        X = V[3 * k], Y = V[3 * k + 1], Z = V[3 * k + 2];
      }
      const bool used = ref[g] != 0;
      if (!(isfinite(X) && isfinite(Y) && isfinite(Z))) {
        atomicOr(&boxes[8 * p + 6], 1ull);
        X = Y = Z = 0.0;
      } else if (used) {
        m[3] = double_to_ordered(X);
        m[4] = double_to_ordered(Y);
        m[5] = double_to_ordered(Z);
        m[0] = ~m[3];
        m[1] = ~m[4];
        m[2] = ~m[5];
      }
      typename P::Vtx v;
      memset(&v, 0, sizeof v);
      P::set_pos(v, X, Y, Z);
      v.tri = used ? -2 : -1;
      v.hint = -1;
      pool[g] = v;
      vpair[g] = p;
    }
    // the box maxima: one atomic per warp and bound when the warp's vertices are one pair's
    const int u = warp_pair(p);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      if (u >= 0) {
        unsigned long long r = m[k];
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long a = __shfl_xor_sync(0xffffffffu, r, o);
          r = a > r ? a : r;
        }
        if ((threadIdx.x & 31) == 0 && r) atomicMax(&boxes[8 * u + k], r);
      } else if (p >= 0 && m[k]) {
        atomicMax(&boxes[8 * p + k], m[k]);
      }
    }
  }
}

// eps, dA and slack of every pair from its box (the step k_prep_finish takes for one run),
// and B's validity flag next to A's.
static __global__ void k_batch_prep_finish(BatchCtx x, unsigned long long* boxes, double tol, int tol_rel,
                                           double slack_scale) {
  grid_dep_wait();
  grid_dep_launch();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= x.npairs) return;
  unsigned long long* box = boxes + 8 * p;
  if (__float_as_uint(x.pd[p].B.meta[1]) != 0u) box[6] |= 1ull << 32;
  double v[6];
  for (int k = 0; k < 6; ++k) v[k] = ordered_to_double(k < 3 ? ~box[k] : box[k]);
  const double dx = v[3] - v[0], dy = v[4] - v[1], dz = v[5] - v[2];
  const double dA = sqrt(dx * dx + dy * dy + dz * dz);
  double amax = 0.0;
  for (int k = 0; k < 6; ++k) amax = fmax(amax, fabs(v[k]));
  const double slack = slack_scale * amax;
  DynParams& d = x.dyn[p];
  d.dA = dA;
  d.eps = tol_rel ? tol * dA : tol;
  d.slack = slack;
  d.slack_f = __double2float_ru(slack);
  d.pad = 0;
  d.emax = INFINITY;  // the batched queries are never cut
}

// ----------------------------------------------------------------------------- queries

// Nearest-triangle queries of pool vertices: round 0 (every vertex of every pair, [0, nV)) or
// the midpoints of a round ([n_pool, n_pool + 3 K')).  As query_body, with each lane on its
// own pair's BVH; a lane past the budget hands its query to k_batch_query_long.
template <class P>
__global__ void HD_QUERY_REGS k_batch_query(BatchCtx x, typename P::Vtx* pool, const int* vpair, LongList ll,
                                            bool round_midpoints) {
  grid_dep_wait();
  grid_dep_launch();
  BatchState* bs = x.bs;
  int beg = 0, count = x.nV;
  if (round_midpoints) {
    if (bs->stop) return;  // uniform over the grid
    beg = bs->n_pool;
    count = 3 * min(bs->n_split, bs->K);
  }
  for (;;) {
    const int base = warp_batch(&bs->q_next);
    if (base >= count) break;
    const int t = base + (threadIdx.x & 31);
    const bool active = t < count;
    typename P::Vtx v;
    int p = -1;
    if (active) {
      v = pool[beg + t];
      p = vpair[beg + t];
    }
    const bool q = active && p >= 0 && v.tri != -1;
    Counters c;
    bool over = false;
    const BvhDev B = x.pd[q ? p : 0].B;
    P::query(B, v, c, q, ll.idx ? P::kLongBudget : INT_MAX, &over);
    double lmax = 0.0;
    int nq = 0;
    if (q) {
      pool[beg + t] = v;
      if (over) {
        const int j = warp_slot(&bs->n_long);
        if (j < ll.cap) ll.idx[j] = beg + t;
        else atomicExch(&bs->overflow, 1);
      } else {
        lmax = P::lower(v) - x.dyn[p].slack;
        nq = 1;
      }
    }
    const int fp = q ? p : -1;
    flush_lower_pair(x.sts, fp, lmax, nq, false);
    flush_counters_pair(x.sts, fp, c);
  }
}

// The handed-off queries, one warp each (traverse_coop), with their pair's BVH.
template <class P>
__global__ void __launch_bounds__(32 * kCoopWarps, P::kCoopBlocks)
    k_batch_query_long(BatchCtx x, typename P::Vtx* pool, const int* vpair, LongList ll, bool round_midpoints) {
  __shared__ unsigned s_code[kCoopWarps * kCoopStack];
  __shared__ float s_e[kCoopWarps * kCoopStack];
  grid_dep_wait();
  grid_dep_launch();
  BatchState* bs = x.bs;
  if (round_midpoints && bs->stop) return;
  const int n = min(bs->n_long, ll.cap);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    int i = 0;
    if (lane == 0) i = atomicAdd(&bs->long_next, 1);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= n) break;
    const int k = ll.idx[i];
    const int p = vpair[k];
    typename P::Vtx v = pool[k];
    Counters c;
    P::query_coop(x.pd[p].B, v, c, s_code + w * kCoopStack, s_e + w * kCoopStack);
    if (lane == 0) pool[k] = v;
    flush_lower_pair(x.sts, lane == 0 ? p : -1, P::lower(v) - x.dyn[p].slack, 1, true);
    flush_counters_pair(x.sts, p, c, true);
  }
}

// ----------------------------------------------------------------------------- bounds

// The paper-order cascade with the items that reach u3 gathered into full warps, as
// bound_rebin of a single run, each item with its pair.  `make(t, it, up)` gives item t's
// vertices and clamp and returns its pair (-1: no item).
struct BatchRebinEntry {
  int v[3];
  float u12;
  float up;
  int pair;
};
inline size_t batch_rebin_smem(int block) {
  return HD_BATCH_REBIN ? (size_t)(block / 32) * kRebinQueue * sizeof(BatchRebinEntry) : 0;
}

template <class P, class Make>
__device__ inline void batch_bound_rebin(const BatchCtx& x, const typename P::Vtx* pool, int64_t count, int* counter,
                                         typename P::Item* next, int* next_pair, int next_cap, typename P::Item* u4list,
                                         int* u4_pair, BatchRebinEntry* q, Make make) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int qn = 0;
  bool more = true;
  while (more || qn > 0) {
    if (more && qn < 32) {
      const int64_t base = warp_batch(counter);
      if (base >= count) {
        more = false;
      } else {
        const int64_t t = base + lane;
        bool need = false;
        BatchRebinEntry e;
        typename P::Item it;
        float up = INFINITY;
        int p = -1;
        PairTally<P> ty;
        if (t < count) p = make(t, it, up);
        if (p >= 0) {
          const PairLevel<P> pl = pair_level<P>(x, p);
          float U, u12;
          int code;
          if (P::paper_cheap(pool[it.v[0]], pool[it.v[1]], pool[it.v[2]], pl.lv.lf, pl.rp, &U, &code, &u12)) {
            need = true;
            e = BatchRebinEntry{{it.v[0], it.v[1], it.v[2]}, u12, up, p};
          } else {
            it.U = up < U ? up : U;
            classify_pair<P>(x.bs, it, p, pl.lv.th, code, next, next_pair, next_cap, u4list, u4_pair, ty);
          }
        }
        flush_tally_pair<P>(x.sts, need ? -1 : p, ty);
        const unsigned m = __ballot_sync(0xffffffffu, need);
        if (need) q[qn + __popc(m & lt)] = e;
        qn += __popc(m);
        __syncwarp();
      }
    }
    if (qn >= 32 || (!more && qn > 0)) {
      const int take = min(qn, 32);
      int p = -1;
      Counters cnt;
      PairTally<P> ty;
      if (lane < take) {
        const BatchRebinEntry e = q[qn - take + lane];
        p = e.pair;
        typename P::Item it;
        it.v[0] = e.v[0];
        it.v[1] = e.v[1];
        it.v[2] = e.v[2];
        const PairLevel<P> pl = pair_level<P>(x, p);
        int code;
        const float U =
            P::paper_u3(x.pd[p].B, pool[e.v[0]], pool[e.v[1]], pool[e.v[2]], pl.lv.lf, pl.rp, e.u12, code, cnt);
        it.U = e.up < U ? e.up : U;
        classify_pair<P>(x.bs, it, p, pl.lv.th, code, next, next_pair, next_cap, u4list, u4_pair, ty);
      }
      qn -= take;
      __syncwarp();  // the entries taken are read before new ones overwrite them
      flush_counters_pair(x.sts, p, cnt);
      flush_tally_pair<P>(x.sts, p, ty);
    }
  }
}

// UpperBound of the round-0 items: every face of every pair (tri == nullptr), or n given
// index triples with their pairs (the promoted items of the FP64 phase).
template <class P, bool kPaper = false>
__global__ void HD_BOUND_REGS k_batch_bound_faces(BatchCtx x, const typename P::Vtx* pool, const int32_t* tri,
                                                  const int* tri_pair, int n, typename P::Item* next, int* next_pair,
                                                  int next_cap, typename P::Item* u4list, int* u4_pair) {
  grid_dep_wait();
  grid_dep_launch();
  BatchState* bs = x.bs;
  const int count = tri ? n : x.nF;
  if constexpr (kPaper && HD_BATCH_REBIN) {
    extern __shared__ BatchRebinEntry batch_rebin_q[];
    batch_bound_rebin<P>(x, pool, count, &bs->b_next, next, next_pair, next_cap, u4list, u4_pair,
                         batch_rebin_q + (threadIdx.x >> 5) * kRebinQueue,
                         [&](int64_t f, typename P::Item& it, float&) -> int {
                           if (tri) {
                             it.v[0] = tri[3 * f];
                             it.v[1] = tri[3 * f + 1];
                             it.v[2] = tri[3 * f + 2];
                             return tri_pair[f];
                           }
                           const int p = find_pair(x.fbase, x.npairs, (int)f);
                           const PairDev& d = x.pd[p];
                           const int32_t* F = d.FA + 3 * (int64_t)(f - x.fbase[p]);
                           const int a = F[0], b = F[1], c = F[2];
                           if (!(a >= 0 && b >= 0 && c >= 0 && a < d.nVA && b < d.nVA && c < d.nVA)) return -1;
                           it.v[0] = d.vbase + a;
                           it.v[1] = d.vbase + b;
                           it.v[2] = d.vbase + c;
                           return p;
                         });
    return;
  }
  for (;;) {
    const int base = warp_batch(&bs->b_next);
    if (base >= count) break;
    const int f = base + (threadIdx.x & 31);
    int p = -1;
    typename P::Item it;
    if (f < count) {
      if (tri) {
        p = tri_pair[f];
        it.v[0] = tri[3 * f];
        it.v[1] = tri[3 * f + 1];
        it.v[2] = tri[3 * f + 2];
      } else {
        p = find_pair(x.fbase, x.npairs, f);
        const PairDev& d = x.pd[p];
        const int32_t* F = d.FA + 3 * (int64_t)(f - x.fbase[p]);
        const int a = F[0], b = F[1], c = F[2];
        // the validation runs concurrently (the host reads the flags with the first round):
        // a bad row is skipped
        if (a >= 0 && b >= 0 && c >= 0 && a < d.nVA && b < d.nVA && c < d.nVA) {
          it.v[0] = d.vbase + a;
          it.v[1] = d.vbase + b;
          it.v[2] = d.vbase + c;
        } else {
          p = -1;
        }
      }
    }
    Counters cnt;
    PairTally<P> ty;
    if (p >= 0) {
      const PairLevel<P> pl = pair_level<P>(x, p);
      int code;
      it.U = bound_item<P, kPaper>(x.pd[p].B, pool, it, pl.lv, pl.rp, code, cnt);
      classify_pair<P>(bs, it, p, pl.lv.th, code, next, next_pair, next_cap, u4list, u4_pair, ty);
    }
    flush_counters_pair(x.sts, p, cnt);
    flush_tally_pair<P>(x.sts, p, ty);
  }
}

// The u4 pass (MIXED): items whose cascade reached a trailing u4, with full warps.
template <class P>
__global__ void k_batch_bound_u4(BatchCtx x, const typename P::Vtx* pool, const typename P::Item* u4list,
                                 const int* u4_pair, int cap, typename P::Item* next, int* next_pair, int next_cap,
                                 bool round_midpoints) {
  grid_dep_wait();
  grid_dep_launch();
  BatchState* bs = x.bs;
  if (round_midpoints && bs->stop) return;
  const int n = min(*(volatile int*)&bs->n_u4, cap);
  // warp-uniform loop: each warp takes 32 consecutive items per step
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = base + (threadIdx.x & 31);
    int p = -1;
    PairTally<P> ty;
    if (t < n) {
      p = u4_pair[t];
      typename P::Item it = u4list[t];
      const PairLevel<P> pl = pair_level<P>(x, p);
      const typename P::UT u = P::bound_u4(pool[it.v[0]], pool[it.v[1]], pool[it.v[2]], pl.rp, it.U);
      int code = 5;
      if (u < pl.lv.th.lo) {
        code = 4;
        it.U = u;
      } else if (u < it.U) {
        it.U = u;
      }
      classify_pair<P>(bs, it, p, pl.lv.th, code, next, next_pair, next_cap, nullptr, nullptr, ty);
    }
    flush_tally_pair<P>(x.sts, p, ty);
  }
}

// Select (Section 3.1 / 4): every item of a running pair with U > l + eps is split while the
// round's split slots last and its pair's face cap allows; the others are discarded (U < l),
// retired (U <= l + eps), promoted to the FP64 phase (MIXED, gap below FP32 resolution) or
// carried over.  Items of a stopped pair are dropped.  A split slot whose pair turns out to
// be at its face cap is left empty (its pair index -1): its midpoints are made as unreferenced
// vertices and its children are not bounded.
template <class P>
__global__ void k_batch_select(BatchCtx x, const typename P::Item* front, const int* front_pair, int4* split_par,
                               int* split_pair, typename P::Vtx* pool, int* vpair, typename P::Item* next,
                               int* next_pair, int next_cap, typename P::Item* promo, int* promo_pair, int promo_cap) {
  grid_dep_wait();
  grid_dep_launch();
  BatchState* bs = x.bs;
  if (bs->stop) return;
  const int n_front = bs->n_front, K = bs->K, mbase = bs->n_pool;
  // warp-uniform loop: each warp takes 32 consecutive items per step
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < n_front;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + (threadIdx.x & 31);
    int p = -1;
    PairTally<P> ty;
    if (i < n_front) {
      p = front_pair[i];
      if (x.sts[p].stop) p = -1;  // the pair is done: its items go
    }
    if (p >= 0) {
      typename P::Item it = front[i];
      const PairLevel<P> pl = pair_level<P>(x, p);
      const Thresholds<P>& th = pl.lv.th;
      if (it.U < th.lo) {
        ty.discard = 5;
      } else if (it.U <= th.hi) {
        ty.retired = 1;
        ty.uret = it.U;
      } else {
        const typename P::Vtx a = pool[it.v[0]], b = pool[it.v[1]], c = pool[it.v[2]];
        const double U = (double)it.U;
        bool carry = false;
        if (promo && P::promote(a, b, c, U, pl.lv.l)) {  // below the policy's resolution: FP64 phase
          const int j = atomicAdd(&bs->n_promote, 1);
          if (j < promo_cap) {
            promo[j] = it;
            promo_pair[j] = p;
            atomicAdd(&x.sts[p].n_promote, 1);
            atomic_max_nonneg(&x.sts[p].upro_bits, U);
          } else {
            atomicExch(&bs->overflow, 1);
          }
        } else {
          const int s = warp_slot(&bs->n_split);
          if (s < K) {
            // the pair's face cap: splits of earlier rounds plus this round's so far
            const int k = atomicAdd(&x.sts[p].n_split, 1);
            const bool ok = x.sts[p].splits + k < x.pd[p].splits_cap;
            if (!ok) {
              atomicSub(&x.sts[p].n_split, 1);
              atomicExch(&x.sts[p].overflow, 1);  // the pair stops with CAPACITY
            }
            split_par[s] = make_int4(it.v[0], it.v[1], it.v[2], __float_as_int(__double2float_ru(U)));
            split_pair[s] = ok ? p : -1;
            typename P::Vtx m;
            P::midpoint(a, b, m);
            if (!ok) m.tri = -1;
            pool[mbase + 3 * s] = m;
            vpair[mbase + 3 * s] = ok ? p : -1;
            P::midpoint(b, c, m);
            if (!ok) m.tri = -1;
            pool[mbase + 3 * s + 1] = m;
            vpair[mbase + 3 * s + 1] = ok ? p : -1;
            P::midpoint(c, a, m);
            if (!ok) m.tri = -1;
            pool[mbase + 3 * s + 2] = m;
            vpair[mbase + 3 * s + 2] = ok ? p : -1;
            carry = !ok;
          } else {
            carry = true;
          }
        }
        if (carry) {
          const int j = warp_slot(&bs->n_next);
          if (j < next_cap) {
            next[j] = it;
            next_pair[j] = p;
            ty.kept = 1;
            ty.umax = it.U;
          } else {
            atomicExch(&bs->overflow, 1);
          }
        }
      }
    }
    flush_tally_pair<P>(x.sts, p, ty);
  }
}

// The four children of every split (Section 4, midpoint subdivision), bounded with their
// pair's l and clamped to their parent's U.
template <class P, bool kPaper = false>
__global__ void HD_BOUND_REGS k_batch_bound_children(BatchCtx x, const typename P::Vtx* pool, const int4* split_par,
                                                     const int* split_pair, typename P::Item* next, int* next_pair,
                                                     int next_cap, typename P::Item* u4list, int* u4_pair) {
  grid_dep_wait();
  grid_dep_launch();
  BatchState* bs = x.bs;
  if (bs->stop) return;
  const int mbase = bs->n_pool;
  const int S = min(*(volatile int*)&bs->n_split, bs->K);
  if constexpr (kPaper && HD_BATCH_REBIN) {
    extern __shared__ BatchRebinEntry batch_rebin_q[];
    batch_bound_rebin<P>(x, pool, 4 * (int64_t)S, &bs->b_next, next, next_pair, next_cap, u4list, u4_pair,
                         batch_rebin_q + (threadIdx.x >> 5) * kRebinQueue,
                         [&](int64_t t, typename P::Item& it, float& up) -> int {
                           const int s = (int)(t >> 2), k = (int)(t & 3);
                           const int p = split_pair[s];
                           if (p < 0) return -1;
                           const int4 par = split_par[s];
                           const int m12 = mbase + 3 * s, m23 = m12 + 1, m31 = m12 + 2;
                           if (k == 0) { it.v[0] = par.x; it.v[1] = m12; it.v[2] = m31; }
                           else if (k == 1) { it.v[0] = m12; it.v[1] = par.y; it.v[2] = m23; }
                           else if (k == 2) { it.v[0] = m31; it.v[1] = m23; it.v[2] = par.z; }
                           else { it.v[0] = m12; it.v[1] = m23; it.v[2] = m31; }
                           if (x.rp.parent_clamp) up = __int_as_float(par.w);
                           return p;
                         });
    return;
  }
  for (;;) {
    const int64_t base = warp_batch(&bs->b_next);
    if (base >= 4 * (int64_t)S) break;
    const int64_t t = base + (threadIdx.x & 31);
    int p = -1;
    int s = 0, k = 0;
    if (t < 4 * (int64_t)S) {
      s = (int)(t >> 2);
      k = (int)(t & 3);
      p = split_pair[s];
    }
    Counters cnt;
    PairTally<P> ty;
    if (p >= 0) {
      const int4 par = split_par[s];
      const int m12 = mbase + 3 * s, m23 = m12 + 1, m31 = m12 + 2;
      typename P::Item it;
      if (k == 0) { it.v[0] = par.x; it.v[1] = m12; it.v[2] = m31; }
      else if (k == 1) { it.v[0] = m12; it.v[1] = par.y; it.v[2] = m23; }
      else if (k == 2) { it.v[0] = m31; it.v[1] = m23; it.v[2] = par.z; }
      else { it.v[0] = m12; it.v[1] = m23; it.v[2] = m31; }
      const PairLevel<P> pl = pair_level<P>(x, p);
      int code;
      it.U = bound_item<P, kPaper>(x.pd[p].B, pool, it, pl.lv, pl.rp, code, cnt);
      // the child lies inside its parent: h(child, B) <= U(parent)
      const typename P::UT Up = (typename P::UT)__int_as_float(par.w);
      if (pl.rp.parent_clamp && Up < it.U) it.U = Up;
      classify_pair<P>(bs, it, p, pl.lv.th, code, next, next_pair, next_cap, u4list, u4_pair, ty);
    }
    flush_counters_pair(x.sts, p, cnt);
    flush_tally_pair<P>(x.sts, p, ty);
  }
}

// The UpperBound kernels of policy P: the straight-line paper-order instantiation (MIXED only)
// or the general one.
template <class P>
auto batch_faces_kernel(bool paper) {
  if constexpr (P::kFp64) return k_batch_bound_faces<P, false>;
  else return paper ? k_batch_bound_faces<P, true> : k_batch_bound_faces<P, false>;
}
template <class P>
auto batch_children_kernel(bool paper) {
  if constexpr (P::kFp64) return k_batch_bound_children<P, false>;
  else return paper ? k_batch_bound_children<P, true> : k_batch_bound_children<P, false>;
}

// ----------------------------------------------------------------------------- round control

// Per-batch constants of the round control.
struct BatchCtl {
  long long chunk, pool_cap, front_cap;
  long long rounds_left;  // rounds before HD_ERR_TIMEOUT, per pair
  const unsigned long long* boxes;  // per pair: [6] = invalid-input flags of A (low word) and B (high word);
                                    // null: the flags were read already (FP64 phase)
};

// One block: closes the round of every running pair (close_round, as the single-pair loop),
// then the batch's round, and opens the next one unless every pair is done.  With init set it
// first starts every pair's loop (`only`: pairs whose own status is OK and that promoted items,
// for the FP64 phase; null: every pair).
static __global__ void k_batch_ctl(BatchCtx x, BatchCtl c, int init, int n_pool0, const int* only) {
  grid_dep_wait();
  grid_dep_launch();
  __shared__ int s_active;
  BatchState* bs = x.bs;
  if (threadIdx.x == 0) s_active = 0;
  __syncthreads();
  if (!bs->stop || init) {
    for (int p = threadIdx.x; p < x.npairs; p += blockDim.x) {
      RunState& st = x.sts[p];
      if (init) {
        const bool run = !only || only[p];
        st.stop = run ? 0 : 1;
        if (run) {
          st.status = HD_OK;
          st.in_round = 0;
          st.rounds = st.splits = st.peak = 0;
          st.urun_bits = (unsigned long long)__double_as_longlong(INFINITY);
          st.K = INT_MAX;
          st.share_mid = 0;
        }
      }
      if (st.stop) continue;
      if (c.boxes) st.bad = c.boxes[8 * p + 6];
      int status = close_round(st, c.rounds_left);
      if (status >= 0) {
        st.status = status;
        st.stop = 1;
        continue;
      }
      st.n_next = 0;
      st.n_split = 0;
      st.umax_bits = 0;
      st.in_round = 1;
      atomicAdd(&s_active, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (init) {
    bs->stop = 0;
    bs->in_round = 0;
    bs->n_pool = n_pool0;
    bs->rounds = 0;
  }
  if (bs->stop) return;
  if (bs->in_round) {
    bs->n_pool += 3 * min(bs->n_split, bs->K);
    bs->rounds += 1;
    bs->in_round = 0;
  }
  bs->n_front = bs->n_next;
  bs->active = s_active;
  long long K = min(c.chunk, (c.pool_cap - (long long)bs->n_pool) / 3);
  K = min(K, (c.front_cap - (long long)bs->n_front) / 3);
  if (s_active == 0 || K <= 0 || bs->overflow) {
    // done, or out of room: the pairs still running stop with CAPACITY (their bracket is the
    // valid one of the last round), marked so that the host can finish them on their own
    if (s_active > 0) {
      for (int p = 0; p < x.npairs; ++p) {
        RunState& st = x.sts[p];
        if (!st.stop) {
          st.in_round = 0;
          st.status = HD_ERR_CAPACITY;
          st.stop = 1;
          st.batch_capacity = 1;
        }
      }
    }
    bs->stop = 1;
    return;
  }
  bs->K = (int)K;
  bs->n_next = 0;
  bs->n_split = 0;
  bs->n_u4 = 0;
  bs->n_long = 0;
  bs->q_next = 0;
  bs->b_next = 0;
  bs->long_next = 0;
  bs->in_round = 1;
}

// Promoted MIXED items of the batch: their vertices at exact positions in an FP64 pool, index
// triples and pairs.
template <class P>
__global__ void k_batch_promote_init(const typename P::Item* promo, const int* promo_pair, int n,
                                     const typename P::Vtx* pool, VtxD* poolD, int* vpairD, int32_t* tris,
                                     int* tri_pair) {
  grid_dep_wait();
  grid_dep_launch();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const typename P::Item it = promo[i];
  const int p = promo_pair[i];
  for (int k = 0; k < 3; ++k) {
    const typename P::Vtx v = pool[it.v[k]];
    const D3 X = P::exact_pos(v);
    VtxD d;
    memset(&d, 0, sizeof d);
    d.x = X.x;
    d.y = X.y;
    d.z = X.z;
    d.tri = -2;
    d.hint = v.tri;
    poolD[3 * i + k] = d;
    vpairD[3 * i + k] = p;
    tris[3 * i + k] = 3 * i + k;
  }
  tri_pair[i] = p;
}

// Start of a phase: the batch-wide counters the round-0 kernels use.
static __global__ void k_batch_phase_reset(BatchState* bs) {
  grid_dep_wait();
  grid_dep_launch();
  bs->n_next = 0;
  bs->n_split = 0;
  bs->n_u4 = 0;
  bs->n_promote = 0;
  bs->n_long = 0;
  bs->q_next = 0;
  bs->b_next = 0;
  bs->long_next = 0;
  bs->overflow = 0;
}

// Start of the FP64 phase of one pair (as k_phase_reset for a single run).
static __global__ void k_batch_pair_reset(BatchCtx x) {
  grid_dep_wait();
  grid_dep_launch();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= x.npairs) return;
  RunState& st = x.sts[p];
  st.n_next = 0;
  st.n_split = 0;
  st.umax_bits = 0;
  st.overflow = 0;
  st.upro_bits = 0;
  st.n_promote = 0;
}

}  // namespace hd

// ----------------------------------------------------------------------------- host driver

namespace hd {

// Buffers of one policy's batched loop, carved from one allocation.
template <class P>
struct BatchBufs {
  char* base = nullptr;
  typename P::Vtx* pool = nullptr;
  int* vpair = nullptr;
  typename P::Item* front[2] = {nullptr, nullptr};
  int* front_pair[2] = {nullptr, nullptr};
  int4* split_par = nullptr;
  int* split_pair = nullptr;
  typename P::Item* u4list = nullptr;  // MIXED only
  int* u4_pair = nullptr;
  typename P::Item* promo = nullptr;   // MIXED only
  int* promo_pair = nullptr;
  LongList longq = {nullptr, 0};
  int64_t pool_cap = 0, front_cap = 0, chunk = 0;
};

template <class P>
int alloc_batch(BatchBufs<P>& R, const Opts& o, int64_t min_pool, int64_t min_front, bool mixed, cudaStream_t s) {
  using Vtx = typename P::Vtx;
  using Item = typename P::Item;
  const int64_t per_v = sizeof(Vtx) + 4, per_i = sizeof(Item) + 4;
  // All pairs' frontiers and midpoints share these buffers (the pool is not recycled between
  // rounds), so the automatic budget is many times what A's vertices and faces alone need
  // (at least 2 GiB), but at most half the device memory that is free.
  int64_t want = std::max<int64_t>((int64_t)2 << 30, 48 * (min_pool * per_v + min_front * per_i));
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && free_b > 0)
    want = std::min<int64_t>(want, std::max<int64_t>((int64_t)(free_b / 2), (int64_t)2 << 30));
  const int64_t budget = o.max_frontier_bytes > 0 ? o.max_frontier_bytes : want;
  R.pool_cap = std::min<int64_t>(std::max<int64_t>(min_pool + 3, (int64_t)(0.6 * budget) / per_v), INT32_MAX / 2);
  R.front_cap = std::min<int64_t>(std::max<int64_t>(min_front + 4, (int64_t)((mixed ? 0.08 : 0.15) * budget) / per_i),
                                  INT32_MAX / 4);
  R.chunk = o.frontier_chunk > 0 ? o.frontier_chunk : std::max<int64_t>(R.front_cap / 4, 1024);
  R.chunk = std::min<int64_t>(R.chunk, R.front_cap);
  const int64_t n_long = std::max<int64_t>(min_pool, 3 * R.chunk);
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_pool = up(sizeof(Vtx) * R.pool_cap), b_vp = up(4 * R.pool_cap), b_front = up(sizeof(Item) * R.front_cap),
               b_fp = up(4 * R.front_cap), b_split = up(sizeof(int4) * R.chunk), b_sp = up(4 * R.chunk),
               b_long = up(4 * n_long);
  const size_t total = b_pool + b_vp + 2 * (b_front + b_fp) + b_split + b_sp + b_long + (mixed ? 2 * (b_front + b_fp) : 0);
  char* base = nullptr;
  HD_TRY(cudaMallocAsync((void**)&base, total, s));
  R.base = base;
  char* p = base;
  auto carve = [&p](size_t b) {
    char* q = p;
    p += b;
    return q;
  };
  R.pool = (Vtx*)carve(b_pool);
  R.vpair = (int*)carve(b_vp);
  for (int k = 0; k < 2; ++k) {
    R.front[k] = (Item*)carve(b_front);
    R.front_pair[k] = (int*)carve(b_fp);
  }
  R.split_par = (int4*)carve(b_split);
  R.split_pair = (int*)carve(b_sp);
  R.longq = {(int*)carve(b_long), (int)n_long};
  if (mixed) {
    R.u4list = (Item*)carve(b_front);
    R.u4_pair = (int*)carve(b_fp);
    R.promo = (Item*)carve(b_front);
    R.promo_pair = (int*)carve(b_fp);
  }
  return HD_OK;
}

// Pinned host memory for the round snapshots of a batched run (per host thread).
struct BatchHost {
  BatchState ring[2];
};
struct BatchHostRes {
  BatchHost* hb = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ~BatchHostRes() {
    if (hb) cudaFreeHost(hb);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
};
inline int batch_host_res(BatchHostRes*& out) {
  static thread_local BatchHostRes r;
  if (!r.hb) HD_TRY(cudaMallocHost((void**)&r.hb, sizeof(BatchHost)));
  for (cudaEvent_t& e : r.ev)
    if (!e) HD_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  out = &r;
  return HD_OK;
}

// Persistent grid of a kernel at block size bs (cached per kernel and block size).
template <typename K>
unsigned batch_grid(K kernel, int bs, int sms, size_t smem = 0) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, bs, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
  return (unsigned)(per_sm * sms);
}

// Frontier rounds of the batch (all pairs) until every pair is done; `cur` is the frontier
// buffer round 0 filled.  Returns HD_OK or a CUDA error; per-pair outcomes are in x.sts.
template <class P>
int batch_rounds(const BatchCtx& x, BatchBufs<P>& R, const BatchCtl& c, int n_pool0, const int* only, int bs_,
                 cudaStream_t s, long long* rounds_out) {
  int dev = 0, sms = 1;
  HD_TRY(cudaGetDevice(&dev));
  HD_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BatchHostRes* hr = nullptr;
  {
    const int rh = batch_host_res(hr);
    if (rh != HD_OK) return rh;
  }
  const bool paper = !P::kFp64 && paper_cascade(x.rp);
  auto k_children = batch_children_kernel<P>(paper);
  const size_t smem_b = batch_rebin_smem(bs_);  // the u3 queues of the paper-order kernels
  const unsigned g_q = batch_grid(k_batch_query<P>, bs_, sms), g_b = batch_grid(k_children, bs_, sms, smem_b);
  const unsigned g_long = batch_grid(k_batch_query_long<P>, 32 * kCoopWarps, sms);
  const unsigned g_sel = (unsigned)sms * 8, g_u4 = (unsigned)sms * 8;
  int cur = 1;
  bool init = true;
  auto issue = [&](int slot) -> int {
    {
      TraceScope tr(HD_K_SELECT, s);
      launch_chained(k_batch_ctl, 1, 1024, 0, s, x, c, init ? 1 : 0, n_pool0, only);
      init = false;
      launch_chained(k_batch_select<P>, g_sel, 256, 0, s, x, R.front[cur], R.front_pair[cur], R.split_par, R.split_pair,
                     R.pool, R.vpair, R.front[cur ^ 1], R.front_pair[cur ^ 1], (int)R.front_cap, R.promo, R.promo_pair,
                     R.promo ? (int)R.front_cap : 0);
    }
    {
      TraceScope tr(HD_K_QUERY, s);
      launch_chained(k_batch_query<P>, g_q, bs_, 0, s, x, R.pool, (const int*)R.vpair, R.longq, true);
    }
    {
      TraceScope tr(HD_K_LONG, s);
      launch_chained(k_batch_query_long<P>, g_long, 32 * kCoopWarps, 0, s, x, R.pool, (const int*)R.vpair, R.longq, true);
    }
    {
      TraceScope tr(HD_K_BOUND, s);
      launch_chained(k_children, g_b, bs_, smem_b, s, x, R.pool, R.split_par, (const int*)R.split_pair, R.front[cur ^ 1],
                     R.front_pair[cur ^ 1], (int)R.front_cap, R.u4list, R.u4_pair);
      if (R.u4list)
        launch_chained(k_batch_bound_u4<P>, g_u4, bs_, 0, s, x, R.pool, R.u4list, (const int*)R.u4_pair, (int)R.front_cap,
                       R.front[cur ^ 1], R.front_pair[cur ^ 1], (int)R.front_cap, true);
    }
    HD_TRY_LAUNCH();
    cur ^= 1;
    HD_TRY(cudaMemcpyAsync(&hr->hb->ring[slot], x.bs, sizeof(BatchState), cudaMemcpyDeviceToHost, s));
    g_d2h_bytes += sizeof(BatchState);
    HD_TRY(cudaEventRecord(hr->ev[slot], s));
    return HD_OK;
  };
  long long issued = 0, seen = 0;
  for (;;) {
    while (issued < seen + 2) {  // one round queued ahead of the one being read
      const int rc = issue((int)(issued & 1));
      if (rc != HD_OK) return rc;
      ++issued;
    }
    HD_TRY(cudaEventSynchronize(hr->ev[seen & 1]));
    const BatchState& h = hr->hb->ring[seen & 1];
    ++seen;
    if (h.stop) break;
  }
  HD_TRY(cudaStreamSynchronize(s));  // the round queued after the last one finds the loop stopped
  *rounds_out = seen;
  return HD_OK;
}

// a7 for the batch (as finish_in_fp64 for one run): the promoted items of the pairs flagged in
// `only` are rebuilt in an FP64 pool at their exact positions, re-queried and bounded in FP64
// with each pair's slack, and refined to the end there; every pair keeps its l and retired
// maximum, and its running upper bound restarts.
template <class P>
int batch_finish_fp64(const BatchCtx& xm, BatchBufs<P>& RM, int64_t n_pro, const std::vector<int>& only, int* d_only,
                      const Opts& o, int bsz, cudaStream_t s) {
  int dev = 0, sms = 1;
  HD_TRY(cudaGetDevice(&dev));
  HD_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BatchBufs<PolicyD> D;
  int rc = alloc_batch<PolicyD>(D, o, 3 * n_pro, n_pro, false, s);
  if (rc != HD_OK) return rc;
  int32_t* tris = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&tris, sizeof(int32_t) * 4 * n_pro, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(D.base, s);
    return set_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
  }
  int* tri_pair = tris + 3 * n_pro;
  BatchCtx x = xm;
  x.nV = (int)(3 * n_pro);
  x.nF = (int)n_pro;
  x.rp.defer_u4 = 0;
  auto fail = [&](cudaError_t err, const char* what) {
    cudaFreeAsync(tris, s);
    cudaFreeAsync(D.base, s);
    return set_cuda_error(err, what, __FILE__, __LINE__);
  };
  e = cudaMemcpyAsync(d_only, only.data(), sizeof(int) * only.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(e, "cudaMemcpyAsync");
  {
    TraceScope tr(HD_K_PREP, s);
    launch_chained(k_batch_promote_init<P>, blocks_for(n_pro, 256), 256, 0, s, (const typename P::Item*)RM.promo,
                   (const int*)RM.promo_pair, (int)n_pro, (const typename P::Vtx*)RM.pool, D.pool, D.vpair, tris,
                   tri_pair);
    launch_chained(k_batch_phase_reset, 1, 1, 0, s, x.bs);
    launch_chained(k_batch_pair_reset, blocks_for(x.npairs, 128), 128, 0, s, x);
  }
  {
    TraceScope tr(HD_K_QUERY, s);
    launch_chained(k_batch_query<PolicyD>, std::min(blocks_for(3 * n_pro, bsz), batch_grid(k_batch_query<PolicyD>, bsz, sms)),
                   bsz, 0, s, x, D.pool, (const int*)D.vpair, D.longq, false);
  }
  {
    TraceScope tr(HD_K_LONG, s);
    launch_chained(k_batch_query_long<PolicyD>, batch_grid(k_batch_query_long<PolicyD>, 32 * kCoopWarps, sms),
                   32 * kCoopWarps, 0, s, x, D.pool, (const int*)D.vpair, D.longq, false);
  }
  {
    TraceScope tr(HD_K_BOUND, s);
    launch_chained(k_batch_bound_faces<PolicyD, false>, blocks_for(n_pro, bsz), bsz, 0, s, x,
                   (const VtxD*)D.pool, (const int32_t*)tris, (const int*)tri_pair, (int)n_pro, D.front[1],
                   D.front_pair[1], (int)D.front_cap, (ItemD*)nullptr, (int*)nullptr);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(e, "launch");
  BatchCtl c;
  c.chunk = D.chunk;
  c.pool_cap = D.pool_cap;
  c.front_cap = D.front_cap;
  c.rounds_left = o.max_rounds;
  c.boxes = nullptr;
  long long rounds = 0;
  rc = batch_rounds<PolicyD>(x, D, c, (int)(3 * n_pro), d_only, bsz, s, &rounds);
  cudaFreeAsync(tris, s);
  cudaFreeAsync(D.base, s);
  return rc;
}

// npairs independent problems in one batched run of policy P (hd_hausdorff_batched).
// Pairs stopped because the batch's shared buffers ran out (not by their own limits) are
// listed in *redo, with a valid bracket and status CAPACITY in outs.
template <class P>
int run_batch(const hd_bvh* const* Bs, const hd_mesh* As, int64_t npairs, double tol, const Opts& o, cudaStream_t s,
              hd_result* outs, std::vector<int64_t>* redo) {
  const int np = (int)npairs;
  const long long launches0 = g_launches, d2h0 = g_d2h_bytes;
  if (o.block_size > round_block_limit<P>() || (!P::kFp64 && o.block_size > round_block_limit<PolicyD>()))
    return HD_ERR_INVALID;
  // pairs, prefix sums, and A's arrays on the device (host arrays copied into one block)
  std::vector<PairDev> pd(np);
  std::vector<int> vbase(np + 1), fbase(np + 1);
  int64_t nV = 0, nF = 0, host_bytes = 0;
  for (int i = 0; i < np; ++i) {
    vbase[i] = (int)nV;
    fbase[i] = (int)nF;
    nV += As[i].nV;
    nF += As[i].nF;
    if (!As[i].on_device)
      host_bytes += ((As[i].nV * 3 * (As[i].vtype == HD_F64 ? 8 : 4) + 15) & ~15ll) + ((As[i].nF * 12 + 15) & ~15ll);
  }
  vbase[np] = (int)nV;
  fbase[np] = (int)nF;
  char* staging = nullptr;
  if (host_bytes) HD_TRY(cudaMallocAsync((void**)&staging, host_bytes, s));
  int64_t off = 0;
  for (int i = 0; i < np; ++i) {
    const hd_mesh& A = As[i];
    PairDev& d = pd[i];
    d.B = bvh_dev(Bs[i]);
    d.vtype = A.vtype;
    d.nVA = (int)A.nV;
    d.nFA = (int)A.nF;
    d.vbase = vbase[i];
    const double cap = std::floor((o.max_face_factor * (double)A.nF - (double)A.nF) / 4.0);
    d.splits_cap = (long long)std::max(0.0, std::min(cap, 9.0e18));
    if (A.on_device) {
      d.VA = A.V;
      d.FA = A.F;
    } else {
      const size_t vb = A.nV * 3 * (A.vtype == HD_F64 ? 8 : 4), fb = A.nF * 12;
      HD_TRY(cudaMemcpyAsync(staging + off, A.V, vb, cudaMemcpyHostToDevice, s));
      d.VA = staging + off;
      off += (vb + 15) & ~(size_t)15;
      HD_TRY(cudaMemcpyAsync(staging + off, A.F, fb, cudaMemcpyHostToDevice, s));
      d.FA = (const int32_t*)(staging + off);
      off += (fb + 15) & ~(size_t)15;
    }
  }
  // the per-pair and batch-wide state: pairs, prefix sums, run states, parameters, boxes,
  // referenced flags and the FP64-phase selection, in one zeroed block
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_pd = up(sizeof(PairDev) * np), b_pref = up(4 * (np + 1)), b_st = up(sizeof(RunState) * np),
               b_dyn = up(sizeof(DynParams) * np), b_box = up(64 * (size_t)np), b_bs = up(sizeof(BatchState)),
               b_ref = up(nV), b_only = up(4 * (size_t)np);
  const size_t small_bytes = b_pd + 2 * b_pref + b_st + b_dyn + b_box + b_bs + b_ref + b_only;
  char* small = nullptr;
  HD_TRY(cudaMallocAsync((void**)&small, small_bytes, s));
  HD_TRY(cudaMemsetAsync(small, 0, small_bytes, s));
  char* q = small;
  auto carve = [&q](size_t b) {
    char* r = q;
    q += b;
    return r;
  };
  PairDev* d_pd = (PairDev*)carve(b_pd);
  int* d_vbase = (int*)carve(b_pref);
  int* d_fbase = (int*)carve(b_pref);
  RunState* d_st = (RunState*)carve(b_st);
  DynParams* d_dyn = (DynParams*)carve(b_dyn);
  unsigned long long* d_box = (unsigned long long*)carve(b_box);
  BatchState* d_bs = (BatchState*)carve(b_bs);
  uint8_t* d_ref = (uint8_t*)carve(b_ref);
  int* d_only = (int*)carve(b_only);
  // pageable host sources: the copies complete before cudaMemcpyAsync returns
  HD_TRY(cudaMemcpyAsync(d_pd, pd.data(), sizeof(PairDev) * np, cudaMemcpyHostToDevice, s));
  HD_TRY(cudaMemcpyAsync(d_vbase, vbase.data(), 4 * (np + 1), cudaMemcpyHostToDevice, s));
  HD_TRY(cudaMemcpyAsync(d_fbase, fbase.data(), 4 * (np + 1), cudaMemcpyHostToDevice, s));

  BatchCtx x;
  x.pd = d_pd;
  x.sts = d_st;
  x.dyn = d_dyn;
  x.bs = d_bs;
  x.vbase = d_vbase;
  x.fbase = d_fbase;
  x.npairs = np;
  x.nV = (int)nV;
  x.nF = (int)nF;
  RunParams& rp = x.rp;
  rp.eps = 0.0;
  rp.slack = 0.0;
  rp.slack_f = 0.f;
  rp.dyn = nullptr;
  rp.defer_u4 = P::kFp64 ? 0 : 1;
  rp.parent_clamp = (o.flags & HD_FLAG_NO_PARENT_CLAMP) ? 0 : 1;
  memcpy(rp.order, o.order, 4);
  rp.n_bounds = o.n_bounds;

  BatchBufs<P> R;
  int rc = alloc_batch<P>(R, o, nV, nF, !P::kFp64, s);
  auto release = [&]() {
    if (R.base) cudaFreeAsync(R.base, s);
    cudaFreeAsync(small, s);
    if (staging) cudaFreeAsync(staging, s);
  };
  if (rc != HD_OK) {
    release();
    return rc;
  }
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int bsz = o.block_size;
  const bool paper = !P::kFp64 && paper_cascade(rp);
  // round 0 of every pair: validation, boxes, pool entries, eps; vertex queries; face bounds
  {
    TraceScope tr(HD_K_PREP, s);
    launch_chained(k_batch_mark_ref, blocks_for(3 * nF, 256), 256, 0, s, x, d_ref, d_box);
    launch_chained(k_batch_check_init<P>, std::min(blocks_for(nV, 256), (unsigned)sms * 16), 256, 0, s, x,
                   (const uint8_t*)d_ref, d_box, R.pool, R.vpair);
    launch_chained(k_batch_prep_finish, blocks_for(np, 128), 128, 0, s, x, d_box, tol, o.tol_mode == HD_TOL_REL ? 1 : 0,
                   P::slack(1.0));
  }
  {
    TraceScope tr(HD_K_QUERY, s);
    launch_chained(k_batch_query<P>, std::min(blocks_for(nV, bsz), batch_grid(k_batch_query<P>, bsz, sms)), bsz, 0, s,
                   x, R.pool, (const int*)R.vpair, R.longq, false);
  }
  {
    TraceScope tr(HD_K_LONG, s);
    launch_chained(k_batch_query_long<P>, batch_grid(k_batch_query_long<P>, 32 * kCoopWarps, sms), 32 * kCoopWarps, 0,
                   s, x, R.pool, (const int*)R.vpair, R.longq, false);
  }
  {
    TraceScope tr(HD_K_BOUND, s);
    auto k_faces = batch_faces_kernel<P>(paper);
    launch_chained(k_faces, std::min(blocks_for(nF, bsz), batch_grid(k_faces, bsz, sms, batch_rebin_smem(bsz))), bsz,
                   batch_rebin_smem(bsz), s, x,
                   (const typename P::Vtx*)R.pool, (const int32_t*)nullptr, (const int*)nullptr, 0, R.front[1],
                   R.front_pair[1], (int)R.front_cap, R.u4list, R.u4_pair);
    if (R.u4list)
      launch_chained(k_batch_bound_u4<P>, (unsigned)sms * 8, bsz, 0, s, x, (const typename P::Vtx*)R.pool,
                     (const typename P::Item*)R.u4list, (const int*)R.u4_pair, (int)R.front_cap, R.front[1],
                     R.front_pair[1], (int)R.front_cap, false);
  }
  HD_TRY_LAUNCH();
  BatchCtl c;
  c.chunk = R.chunk;
  c.pool_cap = R.pool_cap;
  c.front_cap = R.front_cap;
  c.rounds_left = o.max_rounds;
  c.boxes = d_box;
  long long rounds = 0;
  rc = batch_rounds<P>(x, R, c, (int)nV, nullptr, bsz, s, &rounds);
  std::vector<RunState> hs(np);
  std::vector<DynParams> hdyn(np);
  if (rc == HD_OK) {
    HD_TRY(cudaMemcpy(hs.data(), d_st, sizeof(RunState) * np, cudaMemcpyDeviceToHost));
    HD_TRY(cudaMemcpy(hdyn.data(), d_dyn, sizeof(DynParams) * np, cudaMemcpyDeviceToHost));
    g_d2h_bytes += (sizeof(RunState) + sizeof(DynParams)) * np;
  }
  // a7 for the batch: the promoted items of every pair that finished OK, in FP64
  std::vector<double> urun0(np, INFINITY);
  std::vector<long long> rounds0(np, 0), splits0(np, 0), peak0(np, 0), promoted0(np, 0);
  int64_t n_pro = 0;
  std::vector<int> only(np, 0);
  for (int i = 0; i < np && rc == HD_OK; ++i) {
    urun0[i] = bits_to_double(hs[i].urun_bits);
    rounds0[i] = hs[i].rounds;
    splits0[i] = hs[i].splits;
    peak0[i] = hs[i].peak;
    promoted0[i] = hs[i].n_promote;
    if (hs[i].status == HD_OK && hs[i].n_promote > 0) {
      only[i] = 1;
      n_pro += hs[i].n_promote;
    }
  }
  if (rc == HD_OK && n_pro > 0 && !P::kFp64) {
    n_pro = std::min<int64_t>(n_pro, R.front_cap);
    rc = batch_finish_fp64<P>(x, R, n_pro, only, d_only, o, bsz, s);
    if (rc == HD_OK) {
      HD_TRY(cudaMemcpy(hs.data(), d_st, sizeof(RunState) * np, cudaMemcpyDeviceToHost));
      g_d2h_bytes += sizeof(RunState) * np;
    }
  }
  release();
  if (rc != HD_OK) return rc;
  int result = HD_OK;
  for (int i = 0; i < np; ++i) {
    const RunState& h = hs[i];
    hd_result& r = outs[i];
    memset(&r, 0, sizeof r);
    double u_run = urun0[i];
    long long nr = rounds0[i], ns = splits0[i], pk = peak0[i];
    if (only[i] && !P::kFp64) {  // the FP64 phase ran for this pair
      u_run = std::min(u_run, bits_to_double(h.urun_bits));
      nr += h.rounds;
      ns += h.splits;
      pk = std::max(pk, h.peak);
    }
    int status = h.status;
    const double l = bits_to_double(h.l_bits), uret = bits_to_double(h.uret_bits);
    if (status == HD_OK) {
      u_run = std::min(u_run, std::max(l, uret));
      if (P::kFp64 && uret < l) status = HD_ERR_NUMERIC;
    }
    if (status == HD_ERR_INVALID) result = HD_ERR_INVALID;
    if (h.batch_capacity && redo) redo->push_back(i);
    r.lower = l;
    r.upper = std::max(l, u_run);
    r.status = status;
    hd_stats& S = r.stats;
    S.rounds = nr;
    S.splits = ns;
    S.queries = (int64_t)h.queries;
    S.long_queries = (int64_t)h.long_queries;
    S.pointtri_evals = (int64_t)h.evals;
    S.leaf_tests = (int64_t)h.leaf_tests;
    S.box_tests = (int64_t)h.box_tests;
    for (int k = 0; k < 6; ++k) S.discards[k] = (int64_t)h.discards[k];
    S.retired = (int64_t)h.retired;
    S.fp64_escalations = (int64_t)h.escalations;
    S.promoted = promoted0[i];
    S.peak_frontier = pk;
    S.pool_vertices = As[i].nV + 3 * ns;
    S.eps_abs = hdyn[i].eps;
    S.dA = hdyn[i].dA;
    S.node_visits = (int64_t)h.node_visits;
    S.long_node_visits = (int64_t)h.long_node_visits;
    S.long_leaf_tests = (int64_t)h.long_leaf_tests;
    S.queries_cut = (int64_t)h.queries_cut;
    // the batch's launches and read-backs are shared by its pairs: each result holds the totals
    S.kernel_launches = g_launches - launches0;
    S.d2h_bytes = g_d2h_bytes - d2h0;
  }
  return result;
}

}  // namespace hd
