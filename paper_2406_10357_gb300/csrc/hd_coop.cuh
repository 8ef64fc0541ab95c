// Warp-cooperative nearest-triangle traversal, for the queries that a lane's own traversal
// does not finish within a budget of triangle tests.
//
// A query point far from B (a sub-triangle vertex deep inside a closed surface, say) has many
// BVH boxes within its nearest distance, and a one-lane depth-first traversal visits them one
// dependent node fetch at a time while the other lanes of its warp wait.  Here the whole warp
// works on one query: every step pops up to eight inner nodes from a stack in shared memory,
// each group of four lanes fetches one node (the four lanes read the four child boxes of the
// same 128-byte node), each lane bounds one child box, tests a leaf child's triangles at once,
// and the inner children still within the warp's radius are pushed back (ballot compaction).
// Pruning is order-independent: a subtree is dropped only when its box bound exceeds the
// smallest triangle distance bound found so far by any lane, which is what the lane
// traversal also guarantees, so the result (the nearest triangle, and the certified lower
// bound) has the same meaning.
#pragma once

#include "hd_internal.cuh"

namespace hd {

// Build-time tunables (measured on GB300: the sliver, large-soup and benchmark workloads).
#ifndef HD_LONG_BUDGET
#define HD_LONG_BUDGET 6
#endif
#ifndef HD_COOP_STACK
#define HD_COOP_STACK 320
#endif
#ifndef HD_COOP_SORT
#define HD_COOP_SORT 0
#endif
// Leaf tests gathered per warp (0: each lane tests its leaf children at once).  A popped node's
// leaf children go to a per-warp queue, and up to 32 wait until the queue holds HD_COOP_LEAFQ
// of them: the certified point-triangle tests then run on full warps instead of on the few
// lanes whose child was a leaf, at the price of a radius that shrinks a step later.  On the
// large soup's long queries: 1.71 ms per call item by item, 1.12 / 1.13 / 1.19 / 1.31 ms with
// thresholds 32 / 24 / 16 / 8.
#ifndef HD_COOP_LEAFQ
#define HD_COOP_LEAFQ 32
#endif
static_assert(HD_COOP_LEAFQ >= 0 && HD_COOP_LEAFQ <= 32, "the leaf queue holds 64 entries: at most 31 + 32");
constexpr int kCoopStack = HD_COOP_STACK;  // stack entries per warp (8 bytes each, shared memory)
constexpr int kCoopWarps = 4;              // warps per block of k_query_long
#ifndef HD_COOP_MIN_BLOCKS
#define HD_COOP_MIN_BLOCKS 12
#endif
// resident blocks per SM asked of the compiler: 12 blocks of 4 warps (<= 40 registers, a few
// values spilled to L1; 10 KB of stacks each).  The traversal waits on dependent node fetches,
// so warps in flight pay: on the large soup's long queries, blocks x stack entries of 6 x 768,
// 8 x 512, 10 x 384, 12 x 320 and 16 x 256 took 2.03, 1.86, 1.70, 1.67 and 1.80 ms per call.
constexpr int kCoopMinBlocks = HD_COOP_MIN_BLOCKS;
// The FP64 policy's cooperative traversal keeps doubles in flight (its query point, the best
// squared distance and closest point, the triangle being tested): at 40 registers it spills
// heavily, so it asks for fewer blocks per SM, and its lanes keep their queries longer.
#ifndef HD_COOP_MIN_BLOCKS_D
#define HD_COOP_MIN_BLOCKS_D 6
#endif
#ifndef HD_LONG_BUDGET_D
#define HD_LONG_BUDGET_D 10
#endif
// Triangles a lane's traversal tests before it hands its query to a warp.  The hand-off
// restarts the traversal from the root with the best triangle found so far as the radius,
// so a small budget wastes little; most queries finish well within it (a point near B tests
// a few triangles).  6 against 10 on the large soup: lane pass 0.64 -> 0.55 ms, cooperative
// pass 1.67 -> 1.72 ms (8% more queries handed off).
constexpr int kLongBudget = HD_LONG_BUDGET;
// The budget of a query that may be cut (cut_radius > 0).  On the large soup 6, 10, 16 and 32
// tests took 1.49, 1.54, 1.68 and 1.97 ms per call: the queries that do not cut within a few
// tests are the far ones, cheaper in a warp; so the default is the budget without cuts.
#ifndef HD_LONG_BUDGET_CUT
#define HD_LONG_BUDGET_CUT HD_LONG_BUDGET
#endif
constexpr int kLongBudgetCut = HD_LONG_BUDGET_CUT;

__device__ inline float warp_min_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Must be called by all 32 lanes of the warp with the same query.  `t` is each lane's own
// nearest state (test1 / range over triangle indices; r2(): its squared radius rounded up to
// float); `box(lx, ly, lz, hx, hy, hz)` returns a lower bound of the squared distance from the
// query point to a box, rounded down to float.  s_code / s_e: this warp's kCoopStack entries
// (node index, box bound).  With kCut, the traversal stops early, returning true, once the
// warp's squared radius is below cut2 (cut_radius).  The two forms are separate
// instantiations, chosen per query: the loop without the checks is compiled as if they did
// not exist (on the large soup the checks alone cost 20% in the queries that never cut).
template <bool kCut, class Near, class Box>
__device__ inline bool traverse_coop(const BvhDev& B, Near& t, const Box& box, unsigned* s_code, float* s_e,
                                     Counters& c, float cut2) {
  const int lane = threadIdx.x & 31, g = lane >> 2, ch = lane & 3;
  if (lane == 0) {
    s_code[0] = 0u;  // the root, an inner node
    s_e[0] = 0.f;
  }
  int sp = 1;
  float r2 = warp_min_f(t.coop_r2());
  if constexpr (kCut) {
    if (r2 < cut2) return true;  // the triangle the lane traversal found is close enough
  }
#if HD_COOP_LEAFQ
  // leaf children wait in a queue (the top kLeafQ entries of the stack array) until
  // HD_COOP_LEAFQ of them are there, then up to 32 are tested at once, one per lane
  constexpr int kLeafQ = 64;
  constexpr int cap = kCoopStack - kLeafQ;
  unsigned* lq_code = s_code + cap;
  int lq = 0;
  __syncwarp();
  while (sp > 0 || lq > 0) {
    if (sp > 0) {
#else
  constexpr int cap = kCoopStack;
  __syncwarp();
  while (sp > 0) {
    {
#endif
    // pop up to 8 nodes, leaving room for their 4 children each (sp - P + 4 P <= capacity)
    int P = min(sp, 8);
    const int room = (cap - sp) / 3;
    if (P > room) P = max(room, 1);
    int node = -1;
    if (g < P) {
      const int k = sp - 1 - g;
      if (s_e[k] <= r2) node = (int)s_code[k];
    }
    __syncwarp();  // the popped entries are read before the pushes below overwrite them
    sp -= P;
    unsigned code = kNoChild;
    float e = INFINITY;
    if (node >= 0) {
      const float* nf = reinterpret_cast<const float*>(B.nodes + node);
      c.nodes += ch == 0;  // one fetch of the node by its four lanes
      code = __ldg(reinterpret_cast<const unsigned*>(nf) + 24 + ch);
      if (code != kNoChild) {
        ++c.boxes;
        e = box(__ldg(nf + ch), __ldg(nf + 4 + ch), __ldg(nf + 8 + ch), __ldg(nf + 12 + ch), __ldg(nf + 16 + ch),
                __ldg(nf + 20 + ch));
      }
    }
    const bool hit = code != kNoChild && e <= r2;
#if HD_COOP_LEAFQ
    {
      const bool leaf = hit && code_count(code) > 0;
      const unsigned lm = __ballot_sync(0xffffffffu, leaf);
      if (leaf) lq_code[lq + __popc(lm & ((1u << lane) - 1u))] = code;  // lq < HD_COOP_LEAFQ <= 32 here
      lq += __popc(lm);
    }
#else
    if (hit && code_count(code) > 0) t.range(code_ref(code), code_count(code));
    r2 = warp_min_f(t.coop_r2());
    if constexpr (kCut) {
      if (r2 < cut2) return true;
    }
#endif
    const bool push = hit && code_count(code) == 0 && e <= r2;
    const unsigned m = __ballot_sync(0xffffffffu, push);
#if HD_COOP_SORT
    // the pushed children farthest first, so that the nearest end on top of the stack and are
    // popped next (closer to a best-first order: the radius shrinks sooner, more boxes are
    // pruned): a bitonic sort of the 32 lanes by box bound, descending, lanes that push nothing
    // last
    {
      float key = push ? e : -INFINITY;
      unsigned cd = (unsigned)code_ref(code);
#pragma unroll
      for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
          const float ok = __shfl_xor_sync(0xffffffffu, key, j);
          const unsigned oc = __shfl_xor_sync(0xffffffffu, cd, j);
          const bool desc = (lane & k) == 0 || k == 32;  // this run sorts descending
          const bool low = (lane & j) == 0;              // the lower lane of the pair
          const bool take = (low == desc) ? ok > key : ok < key;
          if (take) {
            key = ok;
            cd = oc;
          }
        }
      }
      const int cnt = __popc(m);
      if (lane < cnt) {
        const int k = sp + lane;
        if (k < cap) {
          s_code[k] = cd;
          s_e[k] = key;
        } else {
          c.err = 1;  // stack overflow: the subtree is skipped and the error reported
        }
      }
    }
#else
    if (push) {
      const int k = sp + __popc(m & ((1u << lane) - 1u));
      if (k < cap) {
        s_code[k] = (unsigned)code_ref(code);
        s_e[k] = e;
      } else {
        c.err = 1;  // stack overflow: the subtree is skipped and the error reported
      }
    }
#endif
    sp = min(sp + __popc(m), cap);
    __syncwarp();
    }
#if HD_COOP_LEAFQ
    if (lq >= HD_COOP_LEAFQ || (sp == 0 && lq > 0)) {
      const int take = min(lq, 32);
      if (lane < take) {
        const unsigned code = lq_code[lq - take + lane];
        t.range(code_ref(code), code_count(code));
      }
      lq -= take;
      __syncwarp();  // the entries taken are read before new ones overwrite them
      r2 = warp_min_f(t.coop_r2());
      if constexpr (kCut) {
        if (r2 < cut2) return true;
      }
    }
#endif
  }
  return false;
}

}  // namespace hd
