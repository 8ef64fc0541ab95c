// FP64 policy: every distance and bound in IEEE double with round-to-nearest, the
// arithmetic of the paper's implementation (Section 4).
#pragma once

#include "hd_coop.cuh"
#include "hd_internal.cuh"

namespace hd {

constexpr int kStack = 96;  // up to 3 pushes per 4-wide node

// Nearest triangle of B to p by ordered depth-first traversal of the BVH: both child
// boxes come with one node fetch, leaf children are tested at once, the nearer internal
// child is entered and the farther one pushed with its box distance, which is re-checked
// when popped.  `Test` gets a triangle range and may shrink the pruning radius it holds.
// Returns kTravOver once `test` has tested more than `budget` triangles, and kTravCut once
// its squared radius is below test.cut2 (cut_radius), with the traversal unfinished (what
// `test` holds is then the best triangle found so far); kTravDone when it finished.
constexpr int kTravDone = 0, kTravOver = 1, kTravCut = 2;
template <bool kCut, class Test>
__device__ inline int traverse(const BvhDev& B, D3 p, Test& test, Counters& c, int budget = INT_MAX) {
  int stack_node[kStack];
  double stack_d[kStack];
  int sp = 0;
  int node = 0;
  for (;;) {
    if ((int)test.evals > budget) return kTravOver;
    if constexpr (kCut) {
      if (test.radius2() < test.cut2) return kTravCut;
    }
    const float4* np = reinterpret_cast<const float4*>(B.nodes + node);
    const float4 lx = __ldg(np), ly = __ldg(np + 1), lz = __ldg(np + 2);
    const float4 hx = __ldg(np + 3), hy = __ldg(np + 4), hz = __ldg(np + 5);
    const uint4 cd = __ldg(reinterpret_cast<const uint4*>(np + 6));
    ++c.nodes;
    double e[4] = {box_dist2(p, lx.x, ly.x, lz.x, hx.x, hy.x, hz.x), box_dist2(p, lx.y, ly.y, lz.y, hx.y, hy.y, hz.y),
                   box_dist2(p, lx.z, ly.z, lz.z, hx.z, hy.z, hz.z), box_dist2(p, lx.w, ly.w, lz.w, hx.w, hy.w, hz.w)};
    unsigned k[4] = {cd.x, cd.y, cd.z, cd.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      c.boxes += k[j] != kNoChild;
      if (k[j] == kNoChild) e[j] = INFINITY;
    }
    // nearest first (sorting network on four)
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int a = q == 0 ? 0 : q == 1 ? 2 : q == 2 ? 0 : q == 3 ? 1 : 1;
      const int b = q == 0 ? 1 : q == 1 ? 3 : q == 2 ? 2 : q == 3 ? 3 : 2;
      if (e[b] < e[a]) {
        double te = e[a];
        e[a] = e[b];
        e[b] = te;
        unsigned tk = k[a];
        k[a] = k[b];
        k[b] = tk;
      }
    }
    if constexpr (kCut) {
      // a child box wholly within the cut radius: one of its triangles is close enough
      const uint4 rp = __ldg(reinterpret_cast<const uint4*>(np + 7));
      const float px = (float)p.x, py = (float)p.y, pz = (float)p.z;
      const float c2 = (float)test.cut2;
      int pick = -1;
      if (cd.w != kNoChild && box_far2(px, py, pz, lx.w, ly.w, lz.w, hx.w, hy.w, hz.w) < c2) pick = (int)rp.w;
      if (cd.z != kNoChild && box_far2(px, py, pz, lx.z, ly.z, lz.z, hx.z, hy.z, hz.z) < c2) pick = (int)rp.z;
      if (cd.y != kNoChild && box_far2(px, py, pz, lx.y, ly.y, lz.y, hx.y, hy.y, hz.y) < c2) pick = (int)rp.y;
      if (cd.x != kNoChild && box_far2(px, py, pz, lx.x, ly.x, lz.x, hx.x, hy.x, hz.x) < c2) pick = (int)rp.x;
      if (pick >= 0) {
        test.range(pick, 1);
        if (test.radius2() < test.cut2) return kTravCut;
      }
    }
    // leaf ranges first, nearest first, so that the radius shrinks before the inner
    // children are kept or dropped
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (k[j] != kNoChild && code_count(k[j]) > 0 && e[j] < test.radius2()) test.range(code_ref(k[j]), code_count(k[j]));
    const double r2 = test.radius2();
    int next = -1;
    double next_d = 0.0;
#pragma unroll
    for (int j = 3; j >= 0; --j) {  // farthest inner children pushed first; the nearest is taken
      if (k[j] == kNoChild || code_count(k[j]) > 0 || !(e[j] < r2)) continue;
      if (next >= 0) {
        if (sp < kStack) {
          stack_node[sp] = next;
          stack_d[sp] = next_d;
          ++sp;
        } else {
          c.err = 1;  // stack overflow: the subtree is skipped and the error reported
        }
      }
      next = code_ref(k[j]);
      next_d = e[j];
    }
    if (next >= 0) {
      node = next;
      continue;
    }
    bool found = false;
    while (sp > 0) {
      --sp;
      if (stack_d[sp] < test.radius2()) {
        node = stack_node[sp];
        found = true;
        break;
      }
    }
    if (!found) break;
  }
  return kTravDone;
}

struct NearestD {
  D3 p;
  const double* tri64;
  const float4* tri32;
  double best2 = INFINITY;
  double cut2 = -1.0;  // the traversal may stop once best2 < cut2 (cut_radius)
  int best = -1;
  D3 q = {0, 0, 0};
  unsigned evals = 0;
  __device__ double radius2() const { return best2; }
  __device__ float coop_r2() const { return __double2float_ru(best2); }
  __device__ void test1(int j) {
    D3 a, b, c;
    load_tri_d(tri64, tri32, j, a, b, c);
    D3 x = closest_on_triangle(p, a, b, c);
    D3 e = p - x;
    double d2 = dot(e, e);
    ++evals;
    if (d2 < best2) {
      best2 = d2;
      best = j;
      q = x;
    }
  }
  __device__ void range(int first, int count) {
    for (int j = first; j < first + count; ++j) test1(j);
  }
};

__device__ inline double dist_to_tri64(const BvhDev& B, int j, D3 x) {
  D3 a, b, c;
  load_tri_d(B.tri64, B.tri32, j, a, b, c);
  return len(x - closest_on_triangle(x, a, b, c));
}

// ----------------------------------------------------------------------------- bounds (Section 3.2)

struct VI {
  D3 v;
  double d;
  int I;
  D3 q;
};

// Eq. (uexact): the three vertices are nearest to one triangle S; h(T,S) = max_i |v_i - q_i|.
__device__ inline double ub_exact(const VI t[3]) { return fmax(t[0].d, fmax(t[1].d, t[2].d)); }

// Eq. (u1)
__device__ inline double ub_u1(const VI t[3]) {
  double u = INFINITY;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double e1 = len(t[i].v - t[(i + 1) % 3].v), e2 = len(t[i].v - t[(i + 2) % 3].v);
    u = fmin(u, fmax(e1, e2) + t[i].d);
  }
  return u;
}

// Eq. (u2): g + max_i d_i with g = R if s - r > 2R, else half the longest edge.
__device__ inline double ub_u2(const VI t[3]) {
  double e1 = len(t[1].v - t[2].v), e2 = len(t[2].v - t[0].v), e3 = len(t[0].v - t[1].v);
  double area = 0.5 * len(cross(t[1].v - t[0].v, t[2].v - t[0].v));
  double g = 0.5 * fmax(e1, fmax(e2, e3));
  if (area > 0.0) {
    double R = e1 * e2 * e3 / (4.0 * area);
    double s = 0.5 * (e1 + e2 + e3);
    double r = area / s;
    if (s - r > 2.0 * R) g = R;
  }
  return g + fmax(t[0].d, fmax(t[1].d, t[2].d));
}

// Shared edge of triangles f, g of B (equal vertex indices of their F_B rows): returns
// true with the slots of the two shared vertices in f and the opposite slots in f and g.
__device__ inline bool shared_edge(const BvhDev& B, int f, int g, int& fs0, int& fs1, int& fo, int& go) {
  int4 a = __ldg(B.tri_vid + f), b = __ldg(B.tri_vid + g);
  int av[3] = {a.x, a.y, a.z}, bv[3] = {b.x, b.y, b.z};
  bool ash[3];
  int nsh = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) ash[i] = (av[i] == bv[0] || av[i] == bv[1] || av[i] == bv[2]);
  // distinct shared vertex indices of f
  int sl[3], ns = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (!ash[i]) continue;
    bool dup = false;
    for (int k = 0; k < ns; ++k) dup |= av[sl[k]] == av[i];
    if (!dup) sl[ns++] = i;
  }
  nsh = ns;
  if (nsh != 2) return false;
  fs0 = sl[0];
  fs1 = sl[1];
  fo = go = -1;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (av[i] != av[fs0] && av[i] != av[fs1]) fo = i;
    if (bv[i] != av[fs0] && bv[i] != av[fs1]) go = i;
  }
  return fo >= 0 && go >= 0;
}

__device__ inline D3 tri_vertex(const BvhDev& B, int j, int slot) {
  if (B.tri64) {
    const double* t = B.tri64 + 9 * (size_t)j + 3 * slot;
    return {t[0], t[1], t[2]};
  }
  const float4 v = __ldg(B.tri32 + 3 * (size_t)j + slot);
  return {v.x, v.y, v.z};
}

// Kang et al. 2018 bound, Eqs. (Kang2018_case1) and (Kang2018_case2).
__device__ inline double ub_u3(const BvhDev& B, const VI t[3], unsigned& evals) {
  int lone = -1;
  if (!(t[0].I == t[1].I && t[1].I == t[2].I)) {
    if (t[1].I == t[2].I) lone = 0;
    else if (t[0].I == t[2].I) lone = 1;
    else if (t[0].I == t[1].I) lone = 2;
  }
  int fs0, fs1, fo, go;
  // v1 is the vertex alone on its triangle (selected by branches: no runtime array index)
  VI v1 = t[0], v2 = t[1], v3 = t[2];
  if (lone == 1) { v1 = t[1]; v2 = t[2]; v3 = t[0]; }
  else if (lone == 2) { v1 = t[2]; v2 = t[0]; v3 = t[1]; }
  if (lone >= 0 && shared_edge(B, v1.I, v2.I, fs0, fs1, fo, go)) {
    int S1 = v1.I, S2 = v2.I;
    D3 p0 = tri_vertex(B, S1, fs0), e = tri_vertex(B, S1, fs1) - p0;
    D3 b1 = 0.5 * (v1.v + v2.v), b2 = 0.5 * (v1.v + v3.v);
    double el = len(e);
    if (el > 0.0) {
      D3 eh = (1.0 / el) * e;
      D3 a1 = tri_vertex(B, S1, fo) - p0, a2 = tri_vertex(B, S2, go) - p0;
      D3 w1 = a1 - dot(a1, eh) * eh, w2 = a2 - dot(a2, eh) * eh;
      double n1 = len(w1), n2 = len(w2);
      if (n1 > 0.0 && n2 > 0.0) {
        D3 nb = (1.0 / n1) * w1 - (1.0 / n2) * w2;
        double s1 = dot(nb, v1.v - p0), s2 = dot(nb, v2.v - p0), s3 = dot(nb, v3.v - p0);
        if (s1 >= 0.0 && s2 <= 0.0 && s3 <= 0.0 && s1 - s2 > 0.0 && s1 - s3 > 0.0) {
          b1 = v1.v + (s1 / (s1 - s2)) * (v2.v - v1.v);
          b2 = v1.v + (s1 / (s1 - s3)) * (v3.v - v1.v);
        }
      }
    }
    evals += 7;
    double hR = fmax(dist_to_tri64(B, S1, v1.v), fmax(dist_to_tri64(B, S1, b1), dist_to_tri64(B, S1, b2)));
    double hQ = fmax(fmax(dist_to_tri64(B, S2, v3.v), dist_to_tri64(B, S2, b2)),
                     fmax(dist_to_tri64(B, S2, b1), dist_to_tri64(B, S2, v2.v)));
    return fmax(hR, hQ);
  }
  D3 m[3], bc = (1.0 / 3.0) * (t[0].v + t[1].v + t[2].v);
#pragma unroll
  for (int i = 0; i < 3; ++i) m[i] = 0.5 * (t[i].v + t[(i + 1) % 3].v);
  double ut = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    int S = t[i].I;
    double h = fmax(fmax(dist_to_tri64(B, S, t[i].v), dist_to_tri64(B, S, m[i])),
                    fmax(dist_to_tri64(B, S, bc), dist_to_tri64(B, S, m[(i + 2) % 3])));
    ut = fmax(ut, h);
  }
  double best = INFINITY;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double h = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) h = fmax(h, dist_to_tri64(B, t[i].I, t[j].v));
    best = fmin(best, h);
  }
  evals += 21;
  return fmin(ut, best);
}

// Squared max over T of d(., {a, b}), attained at a vertex of T or where an edge of T crosses
// the bisector plane of a and b (Section 3.2.4).  Squared distances throughout: the one square
// root is taken by ub_u4 (FP64 square roots are costly on GB300, whose FP64 rate is low).
__device__ inline double h2_two_points(const VI t[3], D3 a, D3 b) {
  double h2 = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    D3 ea = t[i].v - a, eb = t[i].v - b;
    h2 = fmax(h2, fmin(dot(ea, ea), dot(eb, eb)));
  }
  D3 n = b - a;
  if (dot(n, n) == 0.0) return h2;
  D3 mid = 0.5 * (a + b);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    D3 x0 = t[i].v, x1 = t[(i + 1) % 3].v;
    double c0 = dot(n, x0 - mid), c1 = dot(n, x1 - mid);
    if (((c0 <= 0.0 && c1 >= 0.0) || (c0 >= 0.0 && c1 <= 0.0)) && c0 != c1) {
      D3 x = x0 + (c0 / (c0 - c1)) * (x1 - x0);
      D3 ea = x - a, eb = x - b;
      h2 = fmax(h2, fmin(dot(ea, ea), dot(eb, eb)));
    }
  }
  return h2;
}

// Eq. (bound_u4)
__device__ inline double ub_u4(const VI t[3]) {
  D3 e0 = t[0].v - t[1].v, e1 = t[1].v - t[2].v, e2 = t[2].v - t[0].v;
  double l0 = dot(e0, e0), l1 = dot(e1, e1), l2 = dot(e2, e2);
  int k = 0;
  double m = l0;
  if (l1 < m) { k = 1; m = l1; }
  if (l2 < m) k = 2;
  D3 q2 = t[0].q, q3 = t[1].q, q1 = t[2].q;  // shortest edge v1v2 (k = 0)
  if (k == 1) { q2 = t[1].q; q3 = t[2].q; q1 = t[0].q; }
  else if (k == 2) { q2 = t[2].q; q3 = t[0].q; q1 = t[1].q; }
  return sqrt(fmin(h2_two_points(t, q1, q2), h2_two_points(t, q1, q3)));
}

// UpperBound(T, l) of Section 4.
__device__ inline double upper_bound_d(const BvhDev& B, const VI t[3], double l, const uint8_t* order, int nb,
                                       int& code, unsigned& evals) {
  if (t[0].I == t[1].I && t[1].I == t[2].I) {
    code = 0;
    return ub_exact(t);
  }
  double U = INFINITY;
  for (int k = 0; k < nb; ++k) {
    double u;
    switch (order[k]) {
      case 1: u = ub_u1(t); break;
      case 2: u = ub_u2(t); break;
      case 3: u = ub_u3(B, t, evals); break;
      default: u = ub_u4(t); break;
    }
    if (u < l) {
      code = order[k];
      return u;
    }
    U = fmin(U, u);
  }
  code = 5;
  return U;
}

// ----------------------------------------------------------------------------- the policy

#ifndef HD_FP64_BOUND_REGS
#define HD_FP64_BOUND_REGS 128
#endif

struct PolicyD {
  using Vtx = VtxD;
  using Item = ItemD;
  using UT = double;
  static constexpr bool kFp64 = true;
  static constexpr int kCoopBlocks = HD_COOP_MIN_BLOCKS_D;  // resident blocks per SM of the cooperative traversal
  static constexpr int kLongBudget = HD_LONG_BUDGET_D;      // triangle tests of a lane before the hand-off
  static constexpr int kBoundRegs = HD_FP64_BOUND_REGS;  // register cap of the UpperBound kernels

  // Nearest triangle of v.  With `over` given, a traversal that tests more than `budget`
  // triangles stops, sets *over and leaves its best triangle so far in v (hint, d = its
  // squared distance, q) for query_coop to finish.
  // With cut_r >= 0 (cut_radius), the query may stop at a triangle within cut_r of v: it
  // then sets *was_cut and keeps that triangle and its distance (not a lower bound then).
  __device__ static void query(const BvhDev& B, Vtx& v, Counters& c, bool active, int budget = INT_MAX,
                               bool* over = nullptr, double cut_r = -1.0, bool* was_cut = nullptr) {
    if (!active) return;  // no warp-collective operations below
    NearestD t;
    t.p = {v.x, v.y, v.z};
    t.tri64 = B.tri64;
    t.tri32 = B.tri32;
    if (cut_r > 0.0) t.cut2 = cut_r * cut_r;
    // start from the hint, or from a triangle of the point's grid cell (a first radius)
    const int h0 = v.hint >= 0 ? v.hint : grid_hint(B, (float)v.x, (float)v.y, (float)v.z);
    if (h0 >= 0) t.test1(h0);
    if (v.hint < 0 && h0 >= 0 && budget < INT_MAX) ++budget;  // the grid's triangle is not the traversal's
    const int how = cut_r > 0.0 ? traverse<true>(B, t.p, t, c, budget) : traverse<false>(B, t.p, t, c, budget);
    c.leaf += t.evals;
    if (how == kTravCut && was_cut) *was_cut = true;
    if (how == kTravOver) {
      *over = true;
      v.hint = t.best;
      v.d = t.best2;
      v.qx = t.q.x;
      v.qy = t.q.y;
      v.qz = t.q.z;
      return;
    }
    v.tri = t.best;
    v.d = sqrt(t.best2);
    v.qx = t.q.x;
    v.qy = t.q.y;
    v.qz = t.q.z;
  }
  // query() of a vertex that a lane's traversal handed off, by the whole warp (every lane
  // passes the same v; lane 0 returns the result in it).
  // With cut_r >= 0 the traversal may stop as query() does (the same for the whole warp);
  // returns true if it did.
  __device__ static bool query_coop(const BvhDev& B, Vtx& v, Counters& c, unsigned* s_code, float* s_e,
                                    double cut_r = -1.0) {
    const int lane = threadIdx.x & 31;
    NearestD t;
    t.p = {v.x, v.y, v.z};
    t.tri64 = B.tri64;
    t.tri32 = B.tri32;
    if (lane == 0 && v.hint >= 0) {  // the lane traversal's best so far
      t.best = v.hint;
      t.best2 = v.d;
      t.q = {v.qx, v.qy, v.qz};
    }
    const D3 p = t.p;
    auto box = [p](float lx, float ly, float lz, float hx, float hy, float hz) {
      return __double2float_rd(box_dist2(p, lx, ly, lz, hx, hy, hz));
    };
    const float cut2 = cut_r > 0.0 ? __double2float_rd(cut_r * cut_r) : 0.f;
    const bool cut = cut2 > 0.f ? traverse_coop<true>(B, t, box, s_code, s_e, c, cut2)
                                : traverse_coop<false>(B, t, box, s_code, s_e, c, 0.f);
    c.leaf += t.evals;
    double m = t.best2;
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int src = __ffs(__ballot_sync(0xffffffffu, t.best2 == m)) - 1;
    const int best = __shfl_sync(0xffffffffu, t.best, src);
    const double qx = __shfl_sync(0xffffffffu, t.q.x, src), qy = __shfl_sync(0xffffffffu, t.q.y, src),
                 qz = __shfl_sync(0xffffffffu, t.q.z, src);
    v.tri = best;
    v.d = sqrt(m);
    v.qx = qx;
    v.qy = qy;
    v.qz = qz;
    return cut;
  }
  __device__ static double lower(const Vtx& v) { return v.d; }
  __device__ static double out_dist(const Vtx& v) { return v.d; }
  __device__ static double out_dlo(const Vtx& v) { return v.d; }
  __device__ static D3 out_foot(const Vtx& v) { return {v.qx, v.qy, v.qz}; }
  static double slack(double) { return 0.0; }
  __device__ static double ut_down(double x) { return x; }
  __device__ static double bound_u4(const Vtx&, const Vtx&, const Vtx&, const RunParams&, double) { return INFINITY; }
  __device__ static D3 exact_pos(const Vtx& v) { return {v.x, v.y, v.z}; }
  __device__ static bool promote(const Vtx&, const Vtx&, const Vtx&, double, double) { return false; }
  __device__ static void set_pos_f(Vtx& v, float x, float y, float z) { set_pos(v, x, y, z); }
  // the distance of a handed-off query's best triangle so far (d holds its square then)
  __device__ static double hint_dist(const Vtx& v) { return sqrt(v.d); }
  // whether a handed-off query's best triangle so far (hint, d = its squared distance) is
  // already within the cut radius cut_r
  __device__ static bool hint_within(const BvhDev&, const Vtx& v, double cut_r) {
    return v.hint >= 0 && cut_r > 0.0 && v.d < cut_r * cut_r;
  }
  // no room in the vertex for its own edge bound: the longest edge of A for every vertex
  static constexpr bool kEdgePerVertex = false;
  __device__ static void set_edge(Vtx&, float) {}
  __device__ static double cut_r(double l, const DynParams* dyn, const Vtx&) { return cut_radius(l, dyn->emax); }
  __device__ static void set_pos(Vtx& v, double x, double y, double z) {
    v.x = x;
    v.y = y;
    v.z = z;
  }
  __device__ static void midpoint(const Vtx& a, const Vtx& b, Vtx& m) {
    m.x = 0.5 * (a.x + b.x);
    m.y = 0.5 * (a.y + b.y);
    m.z = 0.5 * (a.z + b.z);
    m.d = 0.0;
    m.qx = m.qy = m.qz = 0.0;
    m.tri = -2;
    m.hint = a.tri;
  }
  __device__ static UT upper_bound(const BvhDev& B, const Vtx& a, const Vtx& b, const Vtx& c, double l, float,
                                   const RunParams& rp, int& code, Counters& cnt) {
    VI t[3] = {{{a.x, a.y, a.z}, a.d, a.tri, {a.qx, a.qy, a.qz}},
               {{b.x, b.y, b.z}, b.d, b.tri, {b.qx, b.qy, b.qz}},
               {{c.x, c.y, c.z}, c.d, c.tri, {c.qx, c.qy, c.qz}}};
    // slack is 0 in a pure FP64 run; in the certification phase of a MIXED run it is the
    // margin that covers the double rounding
    double U = upper_bound_d(B, t, l - rp.slack, rp.order, rp.n_bounds, code, cnt.evals);
    return U + rp.slack;
  }
};

}  // namespace hd
