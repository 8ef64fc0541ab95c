// Internal types and device helpers shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "hd.h"

namespace hd {

// ----------------------------------------------------------------------------- errors

int set_cuda_error(cudaError_t e, const char* what, const char* file, int line);

#define HD_TRY(call)                                                                  \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return ::hd::set_cuda_error(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define HD_TRY_LAUNCH() HD_TRY(cudaGetLastError())

// ----------------------------------------------------------------------------- BVH layout

// One traversal node, 128 bytes, with up to four children (a node of the binary radix tree
// together with its children's children, so a traversal takes half as many dependent node
// fetches): the children's boxes stored by component (lo.x of children 0..3, then lo.y, ...),
// and per child a code, count << 27 | index -- an inner node (count 0), a leaf range
// [index, index + count) of sorted triangles (count > 0), or no child (kNoChild, with an
// empty box: lo = +inf, hi = -inf).  `rep` lets a cut query (cut_radius) stop at a child
// whose whole box lies within the cut radius: any triangle inside is then close enough.
struct __align__(16) BvhNode {
  float4 lox, loy, loz, hix, hiy, hiz;
  uint4 code;
  uint4 rep;  // per child, one of its triangles (the first of its range; 0 for no child)
};
static_assert(sizeof(BvhNode) == 128, "node is 128 B");
constexpr unsigned kNoChild = 0xffffffffu;
__host__ __device__ inline unsigned node_code(int ref, int cnt) { return ((unsigned)cnt << 27) | (unsigned)ref; }
__host__ __device__ inline int code_count(unsigned code) { return (int)(code >> 27); }
__host__ __device__ inline int code_ref(unsigned code) { return (int)(code & 0x07ffffffu); }

}  // namespace hd

// The handle behind hd_bvh*.  Triangles are stored in BVH (Morton) order.
struct hd_bvh {
  int device;
  int64_t nF;
  int leaf_size;
  int input_f64;
  int64_t n_nodes;
  void* block;         // one stream-ordered allocation; the arrays below are carved from it
  hd::BvhNode* nodes;  // n_nodes
  float4* tri32;       // 3 per triangle: a.xyz|orig-index-bits, b.xyz|0, c.xyz|0 (RN of input)
  double* tri64;       // 9 per triangle: a, b, c (exact input values); null for float32 input,
                       // whose values tri32 holds exactly
  int4* tri_vid;       // per triangle: the F_B row (vertex indices) and the original face index
  int* inv;            // original face index -> sorted position
  float eta;           // max distance between a float vertex of tri32 and its input value (0 for f32
                       // input); the host copy, valid once the build has been waited for
  float* meta;         // device: [0] eta as above, [1] nonzero if B was invalid (as bits), [4..9] the
                       // centroid box of the Morton codes (lo xyz, hi xyz), [10] bits per axis,
                       // [11] bits per axis of the hint grid (as int bits)
  int* grid;           // hint grid: per coarse Morton cell, one triangle whose centroid lies in it
                       // (the first in BVH order), or -1
  int grid_bits;       // bits per axis of the hint grid (8^grid_bits cells)
};

namespace hd {

// ----------------------------------------------------------------------------- pool and frontier

// A vertex of A or of a sub-triangle of A, with its nearest-triangle data (D, I, C of
// Section 4).  Positions are double: midpoints of float or double inputs stay exact for
// about 29 levels of subdivision.
struct __align__(16) VtxD {  // HD_FP64
  double x, y, z;
  double d;           // |p - q|
  double qx, qy, qz;  // closest point q on B
  int tri;            // nearest triangle (sorted index); -1 = not referenced
  int hint;           // triangle tried first by the query (warm start), -1 = none
};
static_assert(sizeof(VtxD) == 64, "VtxD is 64 B");

struct __align__(16) VtxM {  // HD_MIXED
  float hx, hy, hz;  // position p = h + l: h the nearest float, l the float residual
  float lx, ly, lz;
  float qx, qy, qz;  // closest point q relative to p
  float qerr;        // a point of triangle `tri` lies within qerr of p + (qx,qy,qz)
  float dhi;         // >= d(p, S_tri) (certified)
  float dlo;         // <= d(p, B) (certified)
  int tri;
  int hint;
  float pad0, pad1;
};
static_assert(sizeof(VtxM) == 64, "VtxM is 64 B");

struct ItemD {
  int v[3];
  int pad;
  double U;
};
struct ItemM {
  int v[3];
  float U;
};

// Device-side state of one hd_hausdorff run.  All counters are updated with atomics.
struct RunState {
  unsigned long long l_bits;     // lower bound l (double bits; non-negative so ordered as uint64)
  unsigned long long uret_bits;  // max U of retired sub-triangles (double bits)
  unsigned long long umax_bits;  // max U over the next frontier (double bits)
  int n_front;                   // items in the current frontier
  int n_next;                    // items appended to the next frontier
  int n_split;                   // items split this round
  int n_pool;                    // vertices in the pool
  int overflow;                  // next frontier or split list ran out of room
  int err;                       // traversal stack overflow and similar
  int n_promote;                 // MIXED items handed to the FP64 phase
  int n_u4;                      // MIXED items whose u4 is evaluated in the separate u4 pass
  unsigned long long upro_bits;  // max U of those items (double bits)
  unsigned long long evals, box_tests, queries, retired, escalations, leaf_tests;
  unsigned long long discards[6];
  // round control on the device (k_round_ctl), so that the host can queue a round before it
  // has read the previous one
  int K;                         // items that may be split this round
  int stop;                      // set when the loop is over; later rounds do nothing
  int status;                    // HD_OK, or why the loop stopped (CAPACITY, TIMEOUT, NUMERIC)
  int in_round;                  // a frontier round has been opened (its splits are counted)
  long long rounds, splits, peak;  // of this loop
  unsigned long long urun_bits;  // running minimum of the round upper bounds (double bits)
  unsigned long long bad;        // invalid-input flags of A (low word) and B (high word)
  int q_next, b_next;            // work counters of the query and bound kernels (warps take
                                 // batches of 32 items until none are left)
  int n_mid;                     // midpoints made this round, when shared (else 3 per split)
  int share_mid;                 // split edges share midpoints (HD_FLAG_SHARE_MIDPOINTS)
  int n_long;                    // queries handed to k_query_long by the last query launch
  int long_next;                 // work counter of k_query_long
  unsigned long long long_queries;  // queries finished by a whole warp (traverse_coop)
  int tail_rounds;               // rounds the last k_tail_rounds launch ran
  int batch_capacity;            // batched run: stopped because the batch's shared buffers ran out
  unsigned long long node_visits;  // BVH nodes fetched by the traversals (128 bytes each)
  unsigned long long long_node_visits, long_leaf_tests;  // ... of which by k_query_long, and its leaf tests
  unsigned long long queries_cut;  // queries stopped once their vertex could no longer keep a face (cut_radius)
};

// Device view of hd_bvh, passed to kernels by value.
struct BvhDev {
  const BvhNode* nodes;
  const float4* tri32;
  const double* tri64;  // null for float32 input (tri32 is exact then)
  const int4* tri_vid;
  int64_t nF;
  const float* meta;  // [0] eta: max distance between a float vertex of tri32 and its input
  const int* grid;    // the hint grid (hd_bvh::grid), or null
};

// 10 bits -> every third bit of 30 (the Morton interleave of the build's codes)
__device__ inline unsigned spread10(unsigned v) {
  unsigned x = v & 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

// A triangle of B near p to start a query from, when it has no hint of its own: the grid
// cell of p in the quantisation of the build's Morton codes, coarsened to the hint grid's
// bits (every index stays in range: the cell coordinates are clamped to the grid).  -1: none.
__device__ inline int grid_hint(const BvhDev& B, float px, float py, float pz) {
  if (B.grid == nullptr) return -1;
  const float4 m1 = __ldg(reinterpret_cast<const float4*>(B.meta) + 1);  // lo xyz, hi x
  const float4 m2 = __ldg(reinterpret_cast<const float4*>(B.meta) + 2);  // hi yz, bits, grid bits
  const int bits = __float_as_int(m2.z), gbits = __float_as_int(m2.w);
  const float cells = (float)(1u << bits);
  const float lo[3] = {m1.x, m1.y, m1.z}, hi[3] = {m1.w, m2.x, m2.y}, p[3] = {px, py, pz};
  unsigned q[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float ext = hi[k] - lo[k];
    const float u = ext > 0.f ? (p[k] - lo[k]) * (cells / ext) : 0.5f * cells;
    q[k] = ((unsigned)fminf(fmaxf(u, 0.f), cells - 1.f)) >> (bits - gbits);  // NaN -> 0
  }
  return __ldg(B.grid + ((spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2])));
}

// Per-run values that are only known on the device (they depend on A's bounding box):
// written by k_prep_finish, read by every round kernel, so that no host round trip is needed
// between validating A and round 0.
struct DynParams {
  double eps;     // absolute tolerance
  double slack;   // see RunParams
  double dA;      // bbox diagonal of A's referenced vertices
  float slack_f;  // slack rounded up to float
  int pad;
  double emax;    // above every edge length of A's faces (cut_radius); +inf: queries are never cut
};

// Early end of a vertex query.  Bound u1 (Eq. u1) of a face containing vertex v is at most
// (longest edge at v) + d(v, B), so once a query has found a triangle of B within
// l - e_v of v (l the running lower bound, e_v above every edge at v of a face or
// sub-triangle: the longest edge at v in A, or for a midpoint the larger bound of its edge's
// ends; emax, above every edge of A, where the policy keeps no e_v), every face (and
// sub-triangle) at v is discarded by u1, whatever v's exact distance: the nearest triangle
// is no longer needed.  The vertex then keeps the triangle found (its upper bounds stay
// valid, since every bound of Section 3.2 holds for any point of B in place of q_i) and a
// lower bound of 0, so it never raises l; l itself can only have been larger than d(v, B).
// The discarded faces, hence the splits, rounds and the final bracket, are those of exact
// queries.  Returns the radius below which a query may stop (negative: never), before the
// policy's own rounding margins, for the lower bound l read from the run state (a smaller,
// older l only cuts less).
#ifndef HD_CUT_EDGE
#define HD_CUT_EDGE 1  // 0: no cut at all (A's longest edge is not measured)
#endif
#ifndef HD_CUT_LANE
#define HD_CUT_LANE 1  // 0: the lane traversal never cuts
#endif
#ifndef HD_CUT_LONG
#define HD_CUT_LONG 1  // 0: the cooperative traversal never cuts
#endif
__device__ inline bool cut_on(const DynParams* dyn) { return dyn != nullptr && dyn->emax < INFINITY; }
__device__ inline double read_lower(const RunState* st) {
  return __longlong_as_double((long long)*(const volatile unsigned long long*)&st->l_bits);
}
__device__ inline double cut_radius(double l, double e) {
  return l * (1.0 - 0x1p-12) - e;  // the margin covers the rounding of the FP32 bounds
}

// Per-run constants of the round kernels.
struct RunParams {
  double eps;    // absolute tolerance
  double slack;  // added to upper bounds, subtracted from lower bounds (MIXED: representation
                 // error of subdivided vertices as float pairs; 0 in FP64)
  uint8_t order[4];
  int n_bounds;
  float slack_f;  // slack rounded up to float
  int defer_u4;   // MIXED: a trailing u4 is evaluated in the separate u4 pass
  int parent_clamp;  // children's U is clamped to their parent's U
  const DynParams* dyn;  // if set, eps / slack / slack_f are taken from here on the device
};

__device__ inline RunParams with_dyn(RunParams rp) {
  if (rp.dyn) {
    rp.eps = rp.dyn->eps;
    rp.slack = rp.dyn->slack;
    rp.slack_f = rp.dyn->slack_f;
  }
  return rp;
}

// UpperBound result code: u4 still to be evaluated by the u4 pass (MIXED)
constexpr int kDeferU4 = 6;

// Per-thread statistics, flushed with one atomic per warp.
// Per-thread work counters, summed over the warp and flushed with 64-bit atomics; 32 bits
// per thread are ample (a thread handles a few thousand items at most).
struct Counters {
  unsigned evals = 0, boxes = 0, escalations = 0, leaf = 0, nodes = 0;
  int err = 0;
};

// ----------------------------------------------------------------------------- launch chaining

// Programmatic dependent launch: a kernel launched with the programmatic-serialization
// attribute (launch_chained) may be scheduled while the kernel before it in the stream is
// still running.  Every such kernel calls grid_dep_wait() first, which returns once the kernel
// before it has completed and its writes are visible, so only the launch latency overlaps;
// grid_dep_launch() lets the next kernel be scheduled as soon as every block of this one has
// started.  Both are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Kernels this host thread has launched through launch_chained, and bytes it has read back
// from the device in runs (the library's own counts).
inline thread_local long long g_launches = 0;
inline thread_local long long g_d2h_bytes = 0;

// Launches kernel<<<grid, block, smem, s>>>(args...) chained to the kernel before it in the
// stream (see grid_dep_wait).  Errors are left for cudaGetLastError (HD_TRY_LAUNCH).
template <typename... KArgs, typename... Args>
inline void launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                           Args&&... args) {
  ++g_launches;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ----------------------------------------------------------------------------- small math

struct D3 {
  double x, y, z;
};
__host__ __device__ inline D3 d3(double x, double y, double z) { return {x, y, z}; }
__host__ __device__ inline D3 operator+(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__host__ __device__ inline D3 operator-(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__host__ __device__ inline D3 operator*(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
__host__ __device__ inline double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ inline D3 cross(D3 a, D3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__host__ __device__ inline double len(D3 a) { return sqrt(dot(a, a)); }

__device__ inline unsigned float_to_ordered(float f) {
  unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ inline float ordered_to_float(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__device__ inline double add_rd(double a, double b) { return __dadd_rd(a, b); }

__device__ inline void atomic_max_nonneg(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// Closest point of triangle (a, b, c) to p by Voronoi-region classification on the
// barycentric dot products (Ericson, Real-Time Collision Detection, 2005, Sect. 5.1.5).
// Divisions are guarded: a triangle whose face region has a non-positive denominator
// (zero area) is handled as its three edges.
__device__ inline D3 closest_on_segment(D3 p, D3 a, D3 b) {
  D3 e = b - a;
  double ee = dot(e, e);
  double t = ee > 0.0 ? fmin(1.0, fmax(0.0, dot(p - a, e) / ee)) : 0.0;
  return a + t * e;
}

__device__ inline D3 closest_on_edges(D3 p, D3 a, D3 b, D3 c) {
  D3 q0 = closest_on_segment(p, a, b), q1 = closest_on_segment(p, b, c), q2 = closest_on_segment(p, c, a);
  double e0 = dot(p - q0, p - q0), e1 = dot(p - q1, p - q1), e2 = dot(p - q2, p - q2);
  D3 q = q0;
  if (e1 < e0) { q = q1; e0 = e1; }
  if (e2 < e0) q = q2;
  return q;
}

__device__ inline D3 closest_on_triangle(D3 p, D3 a, D3 b, D3 c) {
  D3 ab = b - a, ac = c - a, ap = p - a;
  // Degenerate (coincident or collinear vertices) and extreme slivers first: the region tests
  // below assume a proper triangle (with a zero-length edge the edge test can fire spuriously),
  // and such a triangle is, to rounding, its three edges.
  double aa = dot(ab, ab), cc = dot(ac, ac), bc = dot(ab, ac);
  if (!(aa * cc - bc * bc > 1e-10 * aa * cc)) return closest_on_edges(p, a, b, c);
  double d1 = dot(ab, ap), d2 = dot(ac, ap);
  if (d1 <= 0.0 && d2 <= 0.0) return a;
  D3 bp = p - b;
  double d3v = dot(ab, bp), d4 = dot(ac, bp);
  if (d3v >= 0.0 && d4 <= d3v) return b;
  double vc = d1 * d4 - d3v * d2;
  if (vc <= 0.0 && d1 >= 0.0 && d3v <= 0.0) {
    double den = d1 - d3v;
    return a + (den > 0.0 ? d1 / den : 0.0) * ab;
  }
  D3 cp = p - c;
  double d5 = dot(ab, cp), d6 = dot(ac, cp);
  if (d6 >= 0.0 && d5 <= d6) return c;
  double vb = d5 * d2 - d1 * d6;
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
    double den = d2 - d6;
    return a + (den > 0.0 ? d2 / den : 0.0) * ac;
  }
  double va = d3v * d6 - d5 * d4;
  if (va <= 0.0 && (d4 - d3v) >= 0.0 && (d5 - d6) >= 0.0) {
    double den = (d4 - d3v) + (d5 - d6);
    return b + (den > 0.0 ? (d4 - d3v) / den : 0.0) * (c - b);
  }
  // face region; den = |ab x ac|^2 (Lagrange), so den / (|ab|^2 |ac|^2) = sin^2 of the angle at a
  double den = va + vb + vc;
  D3 q = a;
  double e = INFINITY;
  if (den > 0.0) {
    double v = fmin(fmax(vb / den, 0.0), 1.0);
    double w = fmin(fmax(vc / den, 0.0), 1.0 - v);
    q = a + v * ab + w * ac;  // a point of the triangle even when the weights were rounded badly
    if (den > 1e-10 * dot(ab, ab) * dot(ac, ac)) return q;
    e = dot(p - q, p - q);
  }
  // ill-conditioned face weights: compare with the three edges (all candidates are on the triangle)
  D3 qe = closest_on_edges(p, a, b, c);
  return dot(p - qe, p - qe) < e ? qe : q;
}

// Triangle i of B in double: the exact input values (tri64, float64 input) or, for float32
// input, which tri32 holds exactly, its float vertices widened (tri64 is not kept then).
__device__ inline void load_tri_d(const double* tri64, const float4* tri32, int i, D3& a, D3& b, D3& c) {
  if (tri64) {
    const double* t = tri64 + 9 * (size_t)i;
    a = {t[0], t[1], t[2]};
    b = {t[3], t[4], t[5]};
    c = {t[6], t[7], t[8]};
    return;
  }
  const float4* t = tri32 + 3 * (size_t)i;
  const float4 x = __ldg(t), y = __ldg(t + 1), z = __ldg(t + 2);
  a = {x.x, x.y, x.z};
  b = {y.x, y.y, y.z};
  c = {z.x, z.y, z.z};
}

// Squared distance from p to an axis-aligned box (0 inside).
__device__ inline double box_dist2(D3 p, float lx, float ly, float lz, float hx, float hy, float hz) {
  double dx = fmax(fmax((double)lx - p.x, p.x - (double)hx), 0.0);
  double dy = fmax(fmax((double)ly - p.y, p.y - (double)hy), 0.0);
  double dz = fmax(fmax((double)lz - p.z, p.z - (double)hz), 0.0);
  return dx * dx + dy * dy + dz * dz;
}

// Squared distance from p to the farthest point of the box: every triangle inside lies within
// it.  A cut query tests one triangle of a child box within its cut radius (BvhNode::rep),
// and stops if that triangle's own distance is below the cut radius: the box bound only
// picks the moment, so it needs no directed rounding.
__device__ inline float box_far2(float px, float py, float pz, float lx, float ly, float lz, float hx, float hy,
                                float hz) {
  const float dx = fmaxf(px - lx, hx - px), dy = fmaxf(py - ly, hy - py), dz = fmaxf(pz - lz, hz - pz);
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// ----------------------------------------------------------------------------- launch helpers

inline unsigned blocks_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : b);
}

// Options after defaults and validation.
struct Opts {
  int tol_mode, precision, leaf_size, block_size, n_bounds, flags;
  double max_face_factor;
  int64_t frontier_chunk, max_rounds, max_frontier_bytes;
  uint8_t order[4];
};
int resolve_options(const hd_options* in, Opts* out);

// Kernel timing trace (hd_trace_enable): an event pair around a launch when enabled.
struct TraceScope {
  TraceScope(int kind, cudaStream_t s);
  ~TraceScope();
  int kind;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
};

// Build-time helpers implemented in hd_lbvh.cu.
int build_bvh(const hd_mesh* B, const Opts& o, cudaStream_t s, hd_bvh** out);

}  // namespace hd
