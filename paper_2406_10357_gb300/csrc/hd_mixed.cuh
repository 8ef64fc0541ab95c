// Certified FP32 policy (HD_MIXED).
//
// Distances and bounds run in float with directed rounding where a bound needs it, so that
// every lower bound stays below and every upper bound above the exact value:
//
//  * Positions of sub-triangle vertices are pairs of floats h + l (l holds the rounding
//    residual of the exact midpoint), and every geometric difference is taken locally,
//    (x - h) - l, so rounding errors scale with local sizes (distances, triangle sizes),
//    not with the coordinates.
//  * Point-triangle distance: the closest point is found on the local triangle by
//    Voronoi-region classification (Ericson 2005) with barycentric weights clamped into
//    the simplex, so it is a point of the triangle up to a few units of rounding; its
//    length plus an a-priori error term (48 u M, M the local magnitude, u = 2^-24) is an
//    upper bound.  The lower bound is a support-function certificate: for any n with
//    |n| <= 1, d(p, S) >= min over the vertices X of S of n.(X - p), evaluated with
//    downward rounding; n is chosen by the closest point's region (the plane normal for
//    the face, the closest-point direction less its along-edge component for an edge, the
//    direction itself for a vertex), which makes it tight whenever the classification was
//    right.  If the certificate is loose (near-degenerate sliver, where the barycentric
//    test is ill-conditioned), the test is redone in FP64.
//  * Terms of u3 need only upper bounds, and any point of the triangle gives one: there
//    the closest point is found without branches (plane projection if inside, else the
//    nearest edge projection) with the same margin.
//  * Box distances for pruning are lower bounds (downward rounding); pruning compares
//    them with the best certified upper bound, so the minimum of the tested lower bounds
//    is a lower bound of d(p, B).
//  * Bounds of Section 3.2 take certified vertex distances (upper bounds), edge lengths
//    rounded up, the circumradius only with the area rounded down, and the split points of
//    u3 with their representation error added.  u4 is certified in FP32 too: the vertex and
//    footpoint differences are float pairs formed with error-free sums, and each remaining
//    rounded dot product or norm is raised by a bound on its error (ubm_u4).
#pragma once

#include "hd_fp64.cuh"
#include "hd_internal.cuh"

namespace hd {

constexpr float kU = 5.9604644775390625e-08f;  // 2^-24

struct F3 {
  float x, y, z;
};
__device__ inline F3 f3(float x, float y, float z) { return {x, y, z}; }
__device__ inline F3 operator+(F3 a, F3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ inline F3 operator-(F3 a, F3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ inline float dotf(F3 a, F3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ inline float amax3(F3 a) { return fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))); }
// Square root and quotient with outward rounding: the correctly rounded (round-to-nearest)
// result is within half an ulp, so one multiplication by 1 +- 2^-23, rounded outward, bounds
// the exact value.
// Square roots rounded up / down, from x * rsqrtf(x): rsqrtf is within 2 ulp (4u relative,
// the CUDA math library's documented bound) and the product adds u, so the result is within
// 5u of sqrt(x); one multiplication by 1 +- 8u in the matching direction covers that.  Tiny
// and infinite arguments take the safe branch (the product would be 0 * inf there).
__device__ inline float sqrt_up(float x) {
  if (!(x >= 1e-30f && x < INFINITY)) return x < 1e-30f ? 1e-15f : x;
  return __fmul_ru(x * rsqrtf(x), 1.f + 8.f * kU);
}
__device__ inline float sqrt_dn(float x) {
  if (!(x >= 1e-30f && x < INFINITY)) return x < 1e-30f ? 0.f : x;
  return __fmul_rd(x * rsqrtf(x), 1.f - 8.f * kU);
}
__device__ inline float div_up(float a, float b) { return __fmul_ru(__fdiv_rn(a, b), 1.f + 2.f * kU); }
__device__ inline float div_dn(float a, float b) { return __fmul_rz(__fdiv_rn(a, b), 1.f - 2.f * kU); }
__device__ inline float norm_ru(F3 a) { return sqrt_up(__fmaf_ru(a.x, a.x, __fmaf_ru(a.y, a.y, __fmul_ru(a.z, a.z)))); }
__device__ inline float norm_rd(F3 a) { return sqrt_dn(__fmaf_rd(a.x, a.x, __fmaf_rd(a.y, a.y, __fmul_rd(a.z, a.z)))); }

// A point as the unevaluated sum h + l of two float triples.
struct FFP {
  F3 h, l;
};

// x - p for a float point x, taken locally: (x - h) - l.
__device__ inline F3 local_off(float4 x, const FFP& p) {
  return {(x.x - p.h.x) - p.l.x, (x.y - p.h.y) - p.l.y, (x.z - p.h.z) - p.l.z};
}

// Barycentric weights (v, w) of the point of triangle (A, B, C) closest to the origin,
// Voronoi-region classification, clamped so that v, w >= 0 and v + w <= 1 exactly.
// Returns the region: 0 face, 1 edge AB, 2 edge AC, 3 edge BC, 4 vertex (A, B or C).
// Degenerate triangles and extreme slivers (|AB x AC|^2 below 1e-5 |AB|^2 |AC|^2, where the
// region tests are ill-conditioned or, with a zero-length edge, wrong) take the nearest of
// the three edges.
__device__ inline int closest_edge_bary(F3 A, F3 B, F3 C, float& v, float& w) {
  F3 e[3] = {B - A, C - B, A - C};
  F3 o[3] = {A, B, C};
  float best = INFINITY;
  int region = 1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float ee = dotf(e[k], e[k]);
    float t = ee > 0.f ? fminf(fmaxf(-dotf(o[k], e[k]) / ee, 0.f), 1.f) : 0.f;
    F3 q = {fmaf(t, e[k].x, o[k].x), fmaf(t, e[k].y, o[k].y), fmaf(t, e[k].z, o[k].z)};
    float dq = dotf(q, q);
    if (dq < best) {
      best = dq;
      int r = (t == 0.f || t == 1.f) ? 4 : (k == 0 ? 1 : (k == 1 ? 3 : 2));
      region = r;
      if (k == 0) { v = t; w = 0.f; }
      else if (k == 1) { v = __fsub_rd(1.f, t); w = t; }
      else { v = 0.f; w = __fsub_rd(1.f, t); }
    }
  }
  return region;
}

__device__ inline int closest_bary(F3 A, F3 B, F3 C, float& v, float& w) {
  F3 ab = B - A, ac = C - A;
  v = 0.f;
  w = 0.f;
  float aa = dotf(ab, ab), cc = dotf(ac, ac), bc = dotf(ab, ac);
  if (!(aa * cc - bc * bc > 1e-5f * aa * cc)) return closest_edge_bary(A, B, C, v, w);
  float d1 = -dotf(ab, A), d2 = -dotf(ac, A);
  if (d1 <= 0.f && d2 <= 0.f) return 4;
  float d3 = -dotf(ab, B), d4 = -dotf(ac, B);
  if (d3 >= 0.f && d4 <= d3) {
    v = 1.f;
    return 4;
  }
  float vc = d1 * d4 - d3 * d2;
  if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
    float den = d1 - d3;
    v = den > 0.f ? fminf(fmaxf(d1 / den, 0.f), 1.f) : 0.f;
    return 1;
  }
  float d5 = -dotf(ab, C), d6 = -dotf(ac, C);
  if (d6 >= 0.f && d5 <= d6) {
    w = 1.f;
    return 4;
  }
  float vb = d5 * d2 - d1 * d6;
  if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
    float den = d2 - d6;
    w = den > 0.f ? fminf(fmaxf(d2 / den, 0.f), 1.f) : 0.f;
    return 2;
  }
  float va = d3 * d6 - d5 * d4;
  if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
    float den = (d4 - d3) + (d5 - d6);
    float t = den > 0.f ? fminf(fmaxf((d4 - d3) / den, 0.f), 1.f) : 0.f;
    v = __fsub_rd(1.f, t);
    w = t;
    return 3;
  }
  float den = va + vb + vc;
  if (!(den > 0.f)) return closest_edge_bary(A, B, C, v, w);
  float inv = 1.f / den;
  v = fminf(fmaxf(vb * inv, 0.f), 1.f);
  w = fminf(fmaxf(vc * inv, 0.f), __fsub_rd(1.f, v));
  return 0;
}

struct PtOut {
  float hi;    // >= d(p, S)
  float lo;    // <= d(p, S)
  F3 q;        // closest point relative to p
  float qerr;  // a point of S lies within qerr of p + q
  bool esc;    // redone in FP64
};

// min over the vertices of n . X, rounded down, for |n| <= 1 (support-function lower bound)
__device__ inline float support_rd(F3 n, F3 A, F3 B, F3 C) {
  float da = __fmaf_rd(n.x, A.x, __fmaf_rd(n.y, A.y, __fmul_rd(n.z, A.z)));
  float db = __fmaf_rd(n.x, B.x, __fmaf_rd(n.y, B.y, __fmul_rd(n.z, B.z)));
  float dc = __fmaf_rd(n.x, C.x, __fmaf_rd(n.y, C.y, __fmul_rd(n.z, C.z)));
  return fminf(da, fminf(db, dc));
}

// n scaled so that |n| <= 1 (rounded toward zero); false if n is zero
__device__ inline bool unit_rz(F3& n) {
  float l = norm_ru(n);
  if (!(l > 0.f)) return false;
  float s = div_dn(1.f, l);
  n = {__fmul_rz(n.x, s), __fmul_rz(n.y, s), __fmul_rz(n.z, s)};
  return true;
}

// The FP64 redo of pt_cert for ill-conditioned cases (rare): not inlined, so that its
// double-precision temporaries do not add to the register budget of the traversal.
static __device__ __noinline__ void pt_escalate(FFP P, float4 a4, float4 b4, float4 c4, float M, PtOut& o) {
  D3 p = {(double)P.h.x + (double)P.l.x, (double)P.h.y + (double)P.l.y, (double)P.h.z + (double)P.l.z};
  D3 a = {a4.x, a4.y, a4.z}, b = {b4.x, b4.y, b4.z}, c = {c4.x, c4.y, c4.z};
  D3 q = closest_on_triangle(p, a, b, c) - p;  // a point of the triangle, relative to p
  double d = len(q);
  // covers the double rounding of these few operations, done in absolute coordinates
  double m = 1e-12 * ((double)M + d + fmax(fabs(p.x), fmax(fabs(p.y), fabs(p.z)))) + 1e-30;
  // support-function lower bounds along the closest-point direction and both plane normals:
  // the first is tight when the nearest point is on an edge or vertex, the others when it
  // is inside the face
  D3 Ad = a - p, Bv = b - p, Cv = c - p;
  auto support = [&](D3 nn) {
    double s = len(nn);
    if (!(s > 0.0)) return 0.0;
    nn = (1.0 / (s * (1.0 + 1e-15))) * nn;
    return fmin(dot(nn, Ad), fmin(dot(nn, Bv), dot(nn, Cv)));
  };
  D3 N = cross(Bv - Ad, Cv - Ad);
  double lo64 = fmax(support(q), fmax(support(N), support((-1.0) * N))) - m;
  o.esc = true;
  o.lo = fmaxf(o.lo, __double2float_rd(fmax(lo64, 0.0)));
  float hi64 = __double2float_ru(d + m);
  if (hi64 < o.hi) {
    o.hi = hi64;
    o.q = {(float)q.x, (float)q.y, (float)q.z};
    // float rounding of q plus the double margin
    o.qerr = __double2float_ru(3e-7 * (fabs(q.x) + fabs(q.y) + fabs(q.z)) + m);
  }
}

// Certified distance from p = h + l to the float triangle (a, b, c).
__device__ inline void pt_cert(const FFP& P, float4 a4, float4 b4, float4 c4, bool want_lo, PtOut& o) {
  F3 A = local_off(a4, P), B = local_off(b4, P), C = local_off(c4, P);
  float M = fmaxf(fmaxf(amax3(A), amax3(B)), fmaxf(amax3(C), amax3(P.l)));
  float v, w;
  int region = closest_bary(A, B, C, v, w);
  F3 E1 = B - A, E2 = C - A;
  F3 Q = {fmaf(w, E2.x, fmaf(v, E1.x, A.x)), fmaf(w, E2.y, fmaf(v, E1.y, A.y)), fmaf(w, E2.z, fmaf(v, E1.z, A.z))};
  float nq = norm_ru(Q);
  o.hi = __fadd_ru(nq, __fmul_ru(48.f * kU, M));
  o.q = Q;
  o.qerr = __fmul_ru(40.f * kU, M);
  o.esc = false;
  o.lo = 0.f;
  if (!want_lo) return;
  // Support direction by region, so that the certificate stays tight when the triangle is
  // much larger than the distance (the direction of Q alone carries an error of about u M / d):
  // face -> the plane normal; edge -> Q with its component along the edge removed;
  // vertex -> Q, which is then the vertex itself.
  F3 n = Q;
  if (region == 0) {
    F3 np = {E1.y * E2.z - E1.z * E2.y, E1.z * E2.x - E1.x * E2.z, E1.x * E2.y - E1.y * E2.x};
    n = dotf(np, Q) >= 0.f ? np : F3{-np.x, -np.y, -np.z};
  } else if (region != 4) {
    F3 e = region == 1 ? E1 : (region == 2 ? E2 : C - B);
    float ee = dotf(e, e), qe = dotf(Q, e);
    if (ee > 0.f) n = {Q.x * ee - e.x * qe, Q.y * ee - e.y * qe, Q.z * ee - e.z * qe};
  }
  float lo = 0.f;
  if (unit_rz(n)) lo = fmaxf(__fsub_rd(support_rd(n, A, B, C), __fmul_ru(6.f * kU, M)), 0.f);
  o.lo = lo;
  // a loose certificate means the classification was ill-conditioned: redo in FP64
  if (__fsub_rd(nq, lo) > __fmul_ru(256.f * kU, M)) pt_escalate(P, a4, b4, c4, M, o);
}

// Lower bound of |p - box|^2 (downward rounding), with p given by an enclosure
// [plo, phi] of the float pair h + l on each axis (h + l rounded down and up).
__device__ inline float box_lo2(F3 plo, F3 phi, float lx, float ly, float lz, float hx, float hy, float hz) {
  float gx = fmaxf(fmaxf(__fsub_rd(lx, phi.x), __fsub_rd(plo.x, hx)), 0.f);
  float gy = fmaxf(fmaxf(__fsub_rd(ly, phi.y), __fsub_rd(plo.y, hy)), 0.f);
  float gz = fmaxf(fmaxf(__fsub_rd(lz, phi.z), __fsub_rd(plo.z, hz)), 0.f);
  return __fmaf_rd(gx, gx, __fmaf_rd(gy, gy, __fmul_rd(gz, gz)));
}

struct NearestM {
  FFP P;
  const float4* tri32;
  float best_hi = INFINITY;
  float dlo = INFINITY;
  float cut = -1.f;   // the traversal may stop once best_hi < cut (cut_radius)
  float cut2 = -1.f;  // cut squared, for the farthest-point box test
  int best = -1;
  F3 q = {0.f, 0.f, 0.f};
  float qerr = 0.f;
  unsigned evals = 0, esc = 0;
  __device__ float radius2() const { return __fmul_ru(best_hi, best_hi); }
  __device__ float coop_r2() const { return radius2(); }
  __device__ void test1(int j) {
    const float4* t = tri32 + 3 * (size_t)j;
    PtOut o;
    pt_cert(P, __ldg(t), __ldg(t + 1), __ldg(t + 2), true, o);
    ++evals;
    esc += o.esc;
    dlo = fminf(dlo, o.lo);
    if (o.hi < best_hi) {
      best_hi = o.hi;
      best = j;
      q = o.q;
      qerr = o.qerr;
    }
  }
  __device__ void range(int first, int count) {
    for (int j = first; j < first + count; ++j) test1(j);
  }
};

// Ordered depth-first traversal with certified float box bounds, in the "while-while" form
// of Aila and Laine (HPG 2009): each lane expands inner nodes until it holds a pending leaf
// range, then the lanes that hold one test one triangle each, together.  The expensive
// certified point-triangle test thus runs with most lanes of the warp active, and the cheap
// node steps absorb the divergence.  Stack entries pack a node index (count 0) or a leaf
// range (first, count) into 32 bits: count in bits 27..31, index below (n_B < 2^27).
// Compare-exchange of (distance, code) pairs, smaller distance first.
__device__ inline void sort2(float& ea, unsigned& ca, float& eb, unsigned& cb) {
  if (eb < ea) {
    float e = ea;
    ea = eb;
    eb = e;
    unsigned c = ca;
    ca = cb;
    cb = c;
  }
}

// Push a child found within the radius (distance < +inf) onto the traversal stack.
__device__ inline void push_code(unsigned* stack_code, float* stack_d, int& sp, unsigned code, float d,
                                 Counters& c) {
  if (!(d < INFINITY)) return;
  if (sp < kStack) {
    stack_code[sp] = code;
    stack_d[sp] = d;
    ++sp;
  } else {
    c.err = 1;  // stack overflow: the subtree is skipped and the error reported
  }
}

// Must be called by all 32 lanes of the warp; inactive lanes start finished.  A lane that
// has tested more than `budget` triangles stops unfinished before its next stack pop and sets
// `over` (t then holds its best so far); one whose best distance bound fell below t.cut stops
// there too and sets `cut` (kCut only: the traversal without the check is a separate
// instantiation, as in traverse_coop).
template <bool kCut>
__device__ inline void traverse_m(const BvhDev& B, NearestM& t, Counters& c, bool active, int budget,
                                  bool& over, bool& cut) {
  unsigned stack_code[kStack];
  float stack_d[kStack];
  int sp = 0;
  int node = active ? 0 : -1;  // inner node to expand next, -1 = none
  int lfirst = 0, lcount = 0;
  bool done = !active;
  // an enclosure of the query point h + l, for the box bounds
  const F3 plo = {__fadd_rd(t.P.h.x, t.P.l.x), __fadd_rd(t.P.h.y, t.P.l.y), __fadd_rd(t.P.h.z, t.P.l.z)};
  const F3 phi = {__fadd_ru(t.P.h.x, t.P.l.x), __fadd_ru(t.P.h.y, t.P.l.y), __fadd_ru(t.P.h.z, t.P.l.z)};
  for (;;) {
    while (!done && lcount == 0) {
      if (node < 0) {
        if constexpr (kCut) {
          if (t.best_hi < t.cut) {
            cut = done = true;
            continue;
          }
        }
        bool found = false;
        while (sp > 0) {
          --sp;
          if (stack_d[sp] <= t.radius2()) {
            unsigned code = stack_code[sp];
            int cnt = (int)(code >> 27), ref = (int)(code & 0x07ffffffu);
            if (cnt > 0) { lfirst = ref; lcount = cnt; }
            else node = ref;
            found = true;
            break;
          }
        }
        if (!found) done = true;
        if (!done && (int)t.evals > budget) over = done = true;  // hand the query off
        continue;
      }
      const float4* np = reinterpret_cast<const float4*>(B.nodes + node);
      const float4 lx = __ldg(np), ly = __ldg(np + 1), lz = __ldg(np + 2);
      const float4 hx = __ldg(np + 3), hy = __ldg(np + 4), hz = __ldg(np + 5);
      const uint4 cd = __ldg(reinterpret_cast<const uint4*>(np + 6));
      ++c.nodes;
      const float r2 = t.radius2();
      // children within the current radius (the others at +inf), nearest first
      float e0 = box_lo2(plo, phi, lx.x, ly.x, lz.x, hx.x, hy.x, hz.x);
      float e1 = box_lo2(plo, phi, lx.y, ly.y, lz.y, hx.y, hy.y, hz.y);
      float e2 = box_lo2(plo, phi, lx.z, ly.z, lz.z, hx.z, hy.z, hz.z);
      float e3 = box_lo2(plo, phi, lx.w, ly.w, lz.w, hx.w, hy.w, hz.w);
      unsigned c0 = cd.x, c1 = cd.y, c2 = cd.z, c3 = cd.w;
      c.boxes += (c0 != kNoChild) + (c1 != kNoChild) + (c2 != kNoChild) + (c3 != kNoChild);
      int pick = -1;  // kCut: a triangle of a child whose whole box lies within the cut radius
      if constexpr (kCut) {
        const float px = t.P.h.x, py = t.P.h.y, pz = t.P.h.z;
        const uint4 rp = __ldg(reinterpret_cast<const uint4*>(np + 7));
        if (c3 != kNoChild && box_far2(px, py, pz, lx.w, ly.w, lz.w, hx.w, hy.w, hz.w) < t.cut2) pick = (int)rp.w;
        if (c2 != kNoChild && box_far2(px, py, pz, lx.z, ly.z, lz.z, hx.z, hy.z, hz.z) < t.cut2) pick = (int)rp.z;
        if (c1 != kNoChild && box_far2(px, py, pz, lx.y, ly.y, lz.y, hx.y, hy.y, hz.y) < t.cut2) pick = (int)rp.y;
        if (c0 != kNoChild && box_far2(px, py, pz, lx.x, ly.x, lz.x, hx.x, hy.x, hz.x) < t.cut2) pick = (int)rp.x;
      }
      if (!(e0 <= r2) || c0 == kNoChild) e0 = INFINITY;
      if (!(e1 <= r2) || c1 == kNoChild) e1 = INFINITY;
      if (!(e2 <= r2) || c2 == kNoChild) e2 = INFINITY;
      if (!(e3 <= r2) || c3 == kNoChild) e3 = INFINITY;
      sort2(e0, c0, e1, c1);
      sort2(e2, c2, e3, c3);
      sort2(e0, c0, e2, c2);
      sort2(e1, c1, e3, c3);
      sort2(e1, c1, e2, c2);
      // the farther hits go on the stack (farthest first, so the nearest of them is popped
      // first); the nearest is taken now
      push_code(stack_code, stack_d, sp, c3, e3, c);
      push_code(stack_code, stack_d, sp, c2, e2, c);
      push_code(stack_code, stack_d, sp, c1, e1, c);
      if constexpr (kCut) {
        if (pick >= 0) {
          // test that one triangle; the check before the next pop then stops the query (should
          // its certified distance miss the cut by a rounding, the children are all pushed)
          push_code(stack_code, stack_d, sp, c0, e0, c);
          lfirst = pick;
          lcount = 1;
          node = -1;
          continue;
        }
      }
      if (e0 < INFINITY) {
        const int cnt = code_count(c0), ref = code_ref(c0);
        if (cnt > 0) {
          lfirst = ref;
          lcount = cnt;
          node = -1;
        } else {
          node = ref;
        }
      } else {
        node = -1;
      }
    }
    if (__all_sync(0xffffffffu, lcount == 0)) break;
    if (lcount > 0) {
      t.test1(lfirst);
      ++lfirst;
      --lcount;
    }
  }
}

// ----------------------------------------------------------------------------- bounds

struct VM {  // one vertex of T in the cascade
  FFP p;
  float dhi;
  int I;
  F3 q;  // closest point relative to p
  float qerr;
};

// Certified edge vector p_j - p_i (components carry a relative error of about 2u).
__device__ inline F3 edge(const VM& a, const VM& b) { return (b.p.h - a.p.h) + (b.p.l - a.p.l); }
__device__ inline float len_hi(F3 e) { return __fmul_ru(norm_ru(e), 1.f + 4.f * kU); }
__device__ inline float len_lo(F3 e) { return __fmul_rd(norm_rd(e), 1.f - 4.f * kU); }

// The edges of T, e[i] opposite vertex i (v2 - v1, v0 - v2, v1 - v0), and their lengths
// rounded up: computed once per item for u1 and u2.
struct EdgesM {
  F3 e[3];
  float hi[3];
  __device__ explicit EdgesM(const VM t[3]) {
    e[0] = edge(t[1], t[2]);
    e[1] = edge(t[2], t[0]);
    e[2] = edge(t[0], t[1]);
#pragma unroll
    for (int i = 0; i < 3; ++i) hi[i] = len_hi(e[i]);
  }
};

// u1, Eq. (u1), with edge lengths rounded up: vertex i's two edges are the two not opposite it
__device__ inline float ubm_u1(const VM t[3], const EdgesM& E) {
  const float u0 = __fadd_ru(fmaxf(E.hi[1], E.hi[2]), t[0].dhi);
  const float u1 = __fadd_ru(fmaxf(E.hi[2], E.hi[0]), t[1].dhi);
  const float u2 = __fadd_ru(fmaxf(E.hi[0], E.hi[1]), t[2].dhi);
  return fminf(u0, fminf(u1, u2));
}

// u2, Eq. (u2): g is half the longest edge when T is certainly obtuse (longest edge squared,
// rounded down, above the sum of the other two squared, rounded up), else the circumradius
// with the area rounded down.  Acute <=> s - r > 2R, so this is the paper's g wherever the
// sign of the test is certain, and the circumradius (always a valid g) elsewhere.
__device__ inline float ubm_u2(const VM t[3], const EdgesM& E) {
  // the longest edge k and the other two, selected by branches (no runtime array index, so
  // the edges stay in registers)
  F3 ek = E.e[0];
  float hk = E.hi[0], h1 = E.hi[1], h2 = E.hi[2];
  if (E.hi[1] > hk && E.hi[1] >= E.hi[2]) {
    ek = E.e[1];
    hk = E.hi[1];
    h1 = E.hi[2];
    h2 = E.hi[0];
  } else if (E.hi[2] > hk && E.hi[2] > E.hi[1]) {
    ek = E.e[2];
    hk = E.hi[2];
    h1 = E.hi[0];
    h2 = E.hi[1];
  }
  const float lok = len_lo(ek);
  float g;
  if (__fmul_rd(lok, lok) > __fmaf_ru(h1, h1, __fmul_ru(h2, h2))) {
    g = __fmul_ru(0.5f, hk);
  } else {
    F3 a = E.e[2], b = {-E.e[1].x, -E.e[1].y, -E.e[1].z};  // v1 - v0 and v2 - v0
    F3 cr = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
    float err = __fmul_ru(__fmul_ru(32.f * kU, amax3(a)), amax3(b));
    float c2 = __fsub_rd(norm_rd(cr), err);  // lower bound of 2|T|
    g = c2 > 0.f ? div_up(__fmul_ru(__fmul_ru(E.hi[0], E.hi[1]), E.hi[2]), __fmul_rd(2.f, c2)) : INFINITY;
  }
  return __fadd_ru(g, fmaxf(t[0].dhi, fmaxf(t[1].dhi, t[2].dhi)));
}

// Upper bound of d(x, S) for the float triangle S = (a4, b4, c4), x = h + l, computed without
// branches: the distance to the projection of x onto the plane of S when it falls inside S
// (well-conditioned triangles only), else to the nearest of the three edge projections.  Any
// point of S gives an upper bound, so the parameters need not be exact; they only have to lie
// in [0, 1] (the face point: v, w >= 0, v + w <= 1), and the point built from a vertex, the
// parameters and the edge vectors carries the same rounding as in pt_cert, covered by the
// same 48 u M margin.
__device__ inline float pt_hi(const FFP& P, float4 a4, float4 b4, float4 c4) {
  F3 A = local_off(a4, P), B = local_off(b4, P), C = local_off(c4, P);
  float M = fmaxf(fmaxf(amax3(A), amax3(B)), fmaxf(amax3(C), amax3(P.l)));
  F3 E1 = B - A, E2 = C - A, E3 = C - B;
  float d00 = dotf(E1, E1), d01 = dotf(E1, E2), d11 = dotf(E2, E2);
  float a1 = -dotf(A, E1), a2 = -dotf(A, E2);
  // edge parameters; a zero-length edge gives 0/0 = NaN, which saturates to 0
  float t1 = __saturatef(__fdividef(a1, d00)), t2 = __saturatef(__fdividef(a2, d11));
  float t3 = __saturatef(__fdividef(-dotf(B, E3), dotf(E3, E3)));
  F3 Q = {fmaf(t1, E1.x, A.x), fmaf(t1, E1.y, A.y), fmaf(t1, E1.z, A.z)};
  F3 Q2 = {fmaf(t2, E2.x, A.x), fmaf(t2, E2.y, A.y), fmaf(t2, E2.z, A.z)};
  F3 Q3 = {fmaf(t3, E3.x, B.x), fmaf(t3, E3.y, B.y), fmaf(t3, E3.z, B.z)};
  float n = dotf(Q, Q), n2 = dotf(Q2, Q2), n3 = dotf(Q3, Q3);
  if (n2 < n) { Q = Q2; n = n2; }
  if (n3 < n) Q = Q3;
  float den = d00 * d11 - d01 * d01;
  if (den > 1e-5f * d00 * d11) {
    float r = __fdividef(1.f, den);
    float v = (d11 * a1 - d01 * a2) * r, w = (d00 * a2 - d01 * a1) * r;
    if (v >= 0.f && w >= 0.f && v + w <= 1.f) {
      w = fminf(w, __fsub_rd(1.f, v));  // v + w <= 1 exactly
      Q = {fmaf(w, E2.x, fmaf(v, E1.x, A.x)), fmaf(w, E2.y, fmaf(v, E1.y, A.y)), fmaf(w, E2.z, fmaf(v, E1.z, A.z))};
    }
  }
  return __fadd_ru(norm_ru(Q), __fmul_ru(48.f * kU, M));
}

__device__ inline float dist_hi(const BvhDev& B, int j, const FFP& x, float beta) {
  const float4* t = B.tri32 + 3 * (size_t)j;
  return __fadd_ru(pt_hi(x, __ldg(t), __ldg(t + 1), __ldg(t + 2)), beta);
}

// Point base + s * e (s in [0, 1]) as a float pair, with its representation error.
__device__ inline FFP along(const VM& base, F3 e, float s, float& beta) {
  FFP x;
  x.h = base.p.h;
  x.l = {fmaf(s, e.x, base.p.l.x), fmaf(s, e.y, base.p.l.y), fmaf(s, e.z, base.p.l.z)};
  beta = __fmul_ru(8.f * kU, fmaxf(amax3(e), amax3(base.p.l)));
  return x;
}

// u3 (Kang et al. 2018), Eqs. (Kang2018_case1) and (Kang2018_case2).  Both cases start with
// point-triangle distances that are laid out as six evaluation slots, so that the lanes of a
// warp run the same code whichever case each item is in: case 1 fills four slots, (b1, S1),
// (b2, S1), (b1, S2), (b2, S2); case 2 fills all six with (v_j, S_i), j != i.
__device__ inline float ubm_u3(const BvhDev& B, const VM t[3], float l, unsigned& evals) {
  int lone = -1;
  if (!(t[0].I == t[1].I && t[1].I == t[2].I)) {
    if (t[1].I == t[2].I) lone = 0;
    else if (t[0].I == t[2].I) lone = 1;
    else if (t[0].I == t[1].I) lone = 2;
  }
  int fs0, fs1, fo, go;
  // v1 is the vertex alone on its triangle; selected by branches (no runtime array index, so
  // the three vertices stay in registers)
  VM v1 = t[0], v2 = t[1], v3 = t[2];
  if (lone == 1) { v1 = t[1]; v2 = t[2]; v3 = t[0]; }
  else if (lone == 2) { v1 = t[2]; v2 = t[0]; v3 = t[1]; }
  const bool c1 = lone >= 0 && shared_edge(B, v1.I, v2.I, fs0, fs1, fo, go);
  const int S1 = v1.I, S2 = v2.I;
  FFP b1 = v1.p, b2 = v1.p;
  float be1 = 0.f, be2 = 0.f;
  if (c1) {
    F3 e12 = edge(v1, v2), e13 = edge(v1, v3);
    // split parameters: the bisecting plane of the two supporting half-planes (any value
    // in [0, 1] gives a valid split; this choice only affects tightness)
    float s2 = 0.5f, s3 = 0.5f;
    const float4* T1 = B.tri32 + 3 * (size_t)S1;
    const float4* T2 = B.tri32 + 3 * (size_t)S2;
    float4 P0 = __ldg(T1 + fs0), P1 = __ldg(T1 + fs1), O1 = __ldg(T1 + fo), O2 = __ldg(T2 + go);
    F3 p0 = {P0.x, P0.y, P0.z}, ed = F3{P1.x, P1.y, P1.z} - p0;
    // (plain fast arithmetic: any split parameter in [0, 1] gives a valid bound)
    const float ee = dotf(ed, ed);
    if (ee > 0.f) {
      const float ie = rsqrtf(ee);
      F3 eh = {ed.x * ie, ed.y * ie, ed.z * ie};
      F3 a1 = F3{O1.x, O1.y, O1.z} - p0, a2 = F3{O2.x, O2.y, O2.z} - p0;
      float k1 = dotf(a1, eh), k2 = dotf(a2, eh);
      F3 w1 = {a1.x - k1 * eh.x, a1.y - k1 * eh.y, a1.z - k1 * eh.z};
      F3 w2 = {a2.x - k2 * eh.x, a2.y - k2 * eh.y, a2.z - k2 * eh.z};
      const float q1 = dotf(w1, w1), q2 = dotf(w2, w2);
      if (q1 > 0.f && q2 > 0.f) {
        const float i1 = rsqrtf(q1), i2 = rsqrtf(q2);
        F3 nb = {w1.x * i1 - w2.x * i2, w1.y * i1 - w2.y * i2, w1.z * i1 - w2.z * i2};
        F3 r1 = (v1.p.h - p0) + v1.p.l;
        float sv1 = dotf(nb, r1), sv2 = sv1 + dotf(nb, e12), sv3 = sv1 + dotf(nb, e13);
        if (sv1 >= 0.f && sv2 <= 0.f && sv3 <= 0.f && sv1 - sv2 > 0.f && sv1 - sv3 > 0.f) {
          s2 = __saturatef(__fdividef(sv1, sv1 - sv2));
          s3 = __saturatef(__fdividef(sv1, sv1 - sv3));
        }
      }
    }
    b1 = along(v1, e12, s2, be1);
    b2 = along(v1, e13, s3, be2);
  }
  float d[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    // case 2 slot k: triangle of vertex k / 2, and the next or the other vertex
    const int i = k >> 1, j = (k == 0 || k == 5) ? 1 : ((k == 1 || k == 3) ? 2 : 0);
    FFP x = c1 ? ((k & 1) ? b2 : b1) : t[j].p;
    float be = c1 ? ((k & 1) ? be2 : be1) : 0.f;
    int S = c1 ? (k < 2 ? S1 : S2) : t[i].I;
    d[k] = (c1 && k >= 4) ? 0.f : dist_hi(B, S, x, be);
  }
  const float dmax = fmaxf(t[0].dhi, fmaxf(t[1].dhi, t[2].dhi));
  if (c1) {
    evals += 4;
    return fmaxf(dmax, fmaxf(fmaxf(d[0], d[1]), fmaxf(d[2], d[3])));
  }
  // case 2: u3 = min(u3~, min_i h(T, S_i)).  The second term comes from the slots: once it is
  // below l the item is discarded whatever u3~ is (U of a discarded item is not used
  // further), and the quadrilateral maximum u3~ is abandoned as soon as it reaches the
  // current minimum, since it can then no longer lower it.
  float best = fminf(fmaxf(t[0].dhi, fmaxf(d[0], d[1])),
                     fminf(fmaxf(t[1].dhi, fmaxf(d[2], d[3])), fmaxf(t[2].dhi, fmaxf(d[4], d[5]))));
  evals += 6;
  if (best < l) return best;
  // quadrilaterals (v_i, m_i, b, m_{i-1}) against S_i
  F3 e01 = edge(t[0], t[1]), e02 = edge(t[0], t[2]), e12 = edge(t[1], t[2]);
  float bm[3];
  FFP m[3];
  m[0] = along(t[0], e01, 0.5f, bm[0]);
  m[1] = along(t[1], e12, 0.5f, bm[1]);
  m[2] = along(t[0], e02, 0.5f, bm[2]);  // m3 on v3v1
  F3 sum = e01 + e02;
  float bb;
  FFP bc = along(t[0], sum, 1.f / 3.f, bb);
  bb = __fmul_ru(16.f * kU, fmaxf(amax3(e01), fmaxf(amax3(e02), amax3(t[0].p.l))));
  float ut = dmax;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (ut >= best) break;
    int S = t[i].I;
    ut = fmaxf(ut, dist_hi(B, S, m[i], bm[i]));
    ut = fmaxf(ut, dist_hi(B, S, bc, bb));
    ut = fmaxf(ut, dist_hi(B, S, m[(i + 2) % 3], bm[(i + 2) % 3]));
    evals += 3;
  }
  return fminf(ut, best);
}

// ---- u4 in certified FP32.  Differences of vertices and footpoints are formed as float pairs
// (h + l) with error-free sums: each such difference is within T = 64u (L + uM) of the exact
// one per component, where L bounds the vertices' low parts and M every coordinate involved
// (u = 2^-24; each pair operation adds at most 2u times the low parts it combines, which grow
// to a few L + uM along the chain).  Only the final dot products and norms round, and each is
// raised by a bound on its error.

// a + b as s + e exactly (Knuth's two-sum; intrinsics, so that nothing is contracted or
// reassociated).
__device__ inline void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ inline FFP pair_sub(const FFP& a, const FFP& b) {
  FFP r;
  two_sum(a.h.x, -b.h.x, r.h.x, r.l.x);
  two_sum(a.h.y, -b.h.y, r.h.y, r.l.y);
  two_sum(a.h.z, -b.h.z, r.h.z, r.l.z);
  r.l = {__fadd_rn(r.l.x, __fsub_rn(a.l.x, b.l.x)), __fadd_rn(r.l.y, __fsub_rn(a.l.y, b.l.y)),
         __fadd_rn(r.l.z, __fsub_rn(a.l.z, b.l.z))};
  return r;
}
__device__ inline FFP pair_add(const FFP& a, const FFP& b) {
  FFP r;
  two_sum(a.h.x, b.h.x, r.h.x, r.l.x);
  two_sum(a.h.y, b.h.y, r.h.y, r.l.y);
  two_sum(a.h.z, b.h.z, r.h.z, r.l.z);
  r.l = {__fadd_rn(r.l.x, __fadd_rn(a.l.x, b.l.x)), __fadd_rn(r.l.y, __fadd_rn(a.l.y, b.l.y)),
         __fadd_rn(r.l.z, __fadd_rn(a.l.z, b.l.z))};
  return r;
}
__device__ inline F3 pair_f(const FFP& a) {  // h + l rounded: within u |h + l| per component
  return {__fadd_rn(a.h.x, a.l.x), __fadd_rn(a.h.y, a.l.y), __fadd_rn(a.h.z, a.l.z)};
}
__device__ inline float sum1(F3 a) { return __fadd_ru(__fadd_ru(fabsf(a.x), fabsf(a.y)), fabsf(a.z)); }

// Upper bound of the length of the exact vector whose float-pair form rounds to d: each
// component of d is within u |d_c| + 3T of it (two differences of pairs and one more pair
// operation), so the exact length is at most |d| (1 + u) + 6T; tiny >= 12T covers it.
__device__ inline float len_cert(F3 d, float tiny) { return __fadd_ru(__fmul_ru(norm_ru(d), 1.f + 4.f * kU), tiny); }

// H(a, b) of Eq. (bound_u4), the largest distance from a point of T to the nearer of a and b,
// certified.  It is attained at a vertex of T or where an edge crosses the bisector plane of a
// and b.  X are T's vertices and a, b the footpoints, as float pairs relative to T's first
// vertex.  For an edge x0 x1 with c_j = n . (x_j - mid) (n = b - a, mid = (a + b) / 2),
// computed as dot products of rounded vectors with |error| <= E_j = 8u |n|_1 |w_j|_1 +
// 4T (|n|_1 + |w_j|_1), the edge is skipped only when both c_j lie beyond E_j on the same
// side (it certainly does not cross).  Otherwise its term is the distance from a to the
// farther endpoint (|x - a| is convex along the edge, so this bounds the crossing's distance
// wherever it is) or, when |c0 - c1| > 4 (E0 + E1), the smaller of that and the distance at
// the computed crossing x0 + tau (x1 - x0) plus tau's error, (2 E0 + E1) / |c0 - c1| + 3u,
// times the edge length.  Every term bounds its exact counterpart from above, and extra terms
// only raise the maximum, so the result bounds H(a, b).
__device__ inline float u4_h_cert(const FFP X[3], const FFP& a, const FFP& b, float T) {
  const float tiny = __fmul_ru(16.f, T);
  F3 dA[3];
  float h = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dA[i] = pair_f(pair_sub(X[i], a));
    const F3 db = pair_f(pair_sub(X[i], b));
    h = fmaxf(h, fminf(len_cert(dA[i], tiny), len_cert(db, tiny)));
  }
  const F3 n = pair_f(pair_sub(b, a));
  FFP mid = pair_add(a, b);
  mid.h = {0.5f * mid.h.x, 0.5f * mid.h.y, 0.5f * mid.h.z};
  mid.l = {0.5f * mid.l.x, 0.5f * mid.l.y, 0.5f * mid.l.z};
  const float n1 = sum1(n), m2 = __fmul_ru(4.f, T);
  float c[3], E[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const F3 w = pair_f(pair_sub(X[i], mid));
    const float w1 = sum1(w);
    c[i] = dotf(n, w);
    E[i] = __fadd_ru(__fmul_ru(__fmul_ru(8.f * kU, n1), w1), __fmul_ru(m2, __fadd_ru(n1, w1)));
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int k = (i + 1) % 3;
    const float c0 = c[i], c1 = c[k], E0 = E[i], E1 = E[k];
    if ((c0 > E0 && c1 > E1) || (c0 < -E0 && c1 < -E1)) continue;
    float term = fmaxf(len_cert(dA[i], tiny), len_cert(dA[k], tiny));
    const float D = fabsf(__fsub_rn(c0, c1));
    if (D > __fmul_ru(4.f, __fadd_ru(E0, E1))) {
      const float tau = __saturatef(__fdiv_rn(c0, __fsub_rn(c0, c1)));
      const F3 e = pair_f(pair_sub(X[k], X[i]));
      // x - a = (x0 - a) + tau e, each component within u (|x0 - a| + |e| + |x - a|) + 6T
      const F3 r = {fmaf(tau, e.x, dA[i].x), fmaf(tau, e.y, dA[i].y), fmaf(tau, e.z, dA[i].z)};
      const float slop = __fadd_ru(__fmul_ru(2.f * kU, __fadd_ru(__fadd_ru(amax3(dA[i]), amax3(e)), amax3(r))), tiny);
      const float errt = __fadd_ru(__fdiv_ru(__fadd_ru(__fmul_ru(2.f, E0), E1), D), 3.f * kU);
      const float at = __fadd_ru(__fadd_ru(norm_ru(r), slop), __fmul_ru(errt, len_cert(e, tiny)));
      term = fminf(term, at);
    }
    h = fmaxf(h, term);
  }
  return h;
}

// u4, Eq. (bound_u4), certified in FP32: the footpoints q1 of the vertex opposite T's shortest
// edge and q2, q3 of its ends, u4 = min(H(q1, q2), H(q1, q3)), plus the footpoints' error
// radii (the points of B they stand for are within qerr) and twice the vertices'
// representation error.
__device__ inline float ubm_u4(const VM t[3], float slack_f) {
  const FFP zero = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  const FFP X[3] = {zero, pair_sub(t[1].p, t[0].p), pair_sub(t[2].p, t[0].p)};
  FFP Q[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Q[i] = pair_add(X[i], FFP{t[i].q, {0.f, 0.f, 0.f}});
  float M = 0.f, L = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    M = fmaxf(M, fmaxf(amax3(X[i].h), amax3(Q[i].h)));
    L = fmaxf(L, amax3(t[i].p.l));
  }
  M = __fmul_ru(M, 2.f);  // also bounds midpoints and differences of two of these
  const float T = __fmul_ru(64.f * kU, __fadd_ru(L, __fmul_ru(kU, M)));
  const F3 x1 = pair_f(X[1]), x2 = pair_f(X[2]), e12 = x2 - x1;
  const float l0 = dotf(x1, x1), l1 = dotf(e12, e12), l2 = dotf(x2, x2);
  // shortest edge v1v2 with footpoints q1 (the opposite vertex's), q2, q3 (any choice is
  // valid; this one is the paper's)
  FFP q2 = Q[0], q3 = Q[1], q1 = Q[2];
  if (l1 < l0 && l1 <= l2) { q2 = Q[1]; q3 = Q[2]; q1 = Q[0]; }
  else if (l2 < l0 && l2 < l1) { q2 = Q[2]; q3 = Q[0]; q1 = Q[1]; }
  const float h = fminf(u4_h_cert(X, q1, q2, T), u4_h_cert(X, q1, q3, T));
  const float qe = fmaxf(t[0].qerr, fmaxf(t[1].qerr, t[2].qerr));
  return __fadd_ru(__fadd_ru(h, qe), __fmul_ru(2.f, slack_f));
}

// lf is l rounded down to float: comparisons against it in float are safe, u < lf => u < l
__device__ inline float upper_bound_m(const BvhDev& B, const VM t[3], float lf, const RunParams& rp, int& code,
                                      Counters& c) {
  float U;
  if (t[0].I == t[1].I && t[1].I == t[2].I) {
    code = 0;
    U = fmaxf(t[0].dhi, fmaxf(t[1].dhi, t[2].dhi));
  } else {
    U = INFINITY;
    code = 5;
    const EdgesM E(t);  // shared by u1 and u2
    for (int k = 0; k < rp.n_bounds; ++k) {
      if (rp.order[k] == 4 && k == rp.n_bounds - 1 && rp.defer_u4) {
        // u4 (FP64) is evaluated for all such items together in the u4 pass, with full
        // warps, instead of by scattered lanes here; U so far is a valid upper bound
        code = kDeferU4;
        break;
      }
      float u;
      switch (rp.order[k]) {
        case 1: u = ubm_u1(t, E); break;
        case 2: u = ubm_u2(t, E); break;
        case 3: u = ubm_u3(B, t, lf, c.evals); break;
        default: u = ubm_u4(t, rp.slack_f); break;
      }
      U = fminf(U, u);
      if (u < lf) {
        code = rp.order[k];
        U = u;
        break;
      }
    }
  }
  return __fadd_ru(U, rp.slack_f);
}

// The cascade in the paper's order (u1, u2, u3, then u4, which the u4 pass evaluates) as
// straight-line code: the same values and result codes as upper_bound_m's loop over
// rp.order, but the edges are dead once u2 is known and the footpoints are not needed at all,
// so that fewer values are live across u3, the heaviest bound.
__device__ inline float upper_bound_m_paper(const BvhDev& B, const VM t[3], float lf, const RunParams& rp, int& code,
                                            Counters& c) {
  float U;
  if (t[0].I == t[1].I && t[1].I == t[2].I) {
    code = 0;
    U = fmaxf(t[0].dhi, fmaxf(t[1].dhi, t[2].dhi));
  } else {
    const EdgesM E(t);
    const float u1 = ubm_u1(t, E);
    if (u1 < lf) {
      code = 1;
      U = u1;
    } else {
      const float u2 = ubm_u2(t, E);
      if (u2 < lf) {
        code = 2;
        U = u2;
      } else {
        const float u3 = ubm_u3(B, t, lf, c.evals);
        if (u3 < lf) {
          code = 3;
          U = u3;
        } else {
          code = kDeferU4;
          U = fminf(fminf(u1, u2), u3);
        }
      }
    }
  }
  return __fadd_ru(U, rp.slack_f);
}

// ----------------------------------------------------------------------------- the policy

#ifndef HD_MIXED_BOUND_REGS
#define HD_MIXED_BOUND_REGS 96
#endif
#ifndef HD_MIXED_PAPER_REGS
#define HD_MIXED_PAPER_REGS 96
#endif

struct PolicyM {
  using Vtx = VtxM;
  using Item = ItemM;
  using UT = float;
  static constexpr bool kFp64 = false;
  static constexpr int kCoopBlocks = kCoopMinBlocks;  // resident blocks per SM of the cooperative traversal
  static constexpr int kLongBudget = ::hd::kLongBudget;  // triangle tests of a lane before the hand-off
  static constexpr int kBoundRegs = HD_MIXED_BOUND_REGS;  // register cap of the UpperBound kernels
  static constexpr int kPaperRegs = HD_MIXED_PAPER_REGS;  // ... of their paper-order instantiation

  // 2^-40 of the largest coordinate: covers the float-pair representation of subdivided
  // vertices (2^-48 relative per level, at most 60 levels) and the double rounding of u4
  static double slack(double amax) { return ldexp(amax, -40); }
  __device__ static float ut_down(double x) { return __double2float_rd(x); }
  // the u4 pass: Eq. (bound_u4) for one item (certified FP32), plus the slack.  The item's
  // bound so far (the last argument) is not needed.
  __device__ static float bound_u4(const Vtx& a, const Vtx& b, const Vtx& c, const RunParams& rp, float) {
    const VM t[3] = {{pos(a), a.dhi, a.tri, {a.qx, a.qy, a.qz}, a.qerr},
                     {pos(b), b.dhi, b.tri, {b.qx, b.qy, b.qz}, b.qerr},
                     {pos(c), c.dhi, c.tri, {c.qx, c.qy, c.qz}, c.qerr}};
    return __fadd_ru(ubm_u4(t, rp.slack_f), rp.slack_f);
  }

  __device__ static FFP pos(const Vtx& v) { return {{v.hx, v.hy, v.hz}, {v.lx, v.ly, v.lz}}; }
  __device__ static D3 exact_pos(const Vtx& v) {
    return {(double)v.hx + (double)v.lx, (double)v.hy + (double)v.ly, (double)v.hz + (double)v.lz};
  }
  // Split further in FP32 only while the gap U - l is well above the FP32 error width of the
  // vertex distances; below that, refinement cannot make progress and the item is finished
  // in the FP64 phase.
  __device__ static bool promote(const Vtx& a, const Vtx& b, const Vtx& c, double U, double l) {
    float err = fmaxf(fmaxf(a.dhi - a.dlo, b.dhi - b.dlo), c.dhi - c.dlo);
    return U - l <= 4.0 * (double)err + ldexp(U, -18);
  }

  // a float input vertex is its own float pair (residual 0), with no FP64 arithmetic
  __device__ static void set_pos_f(Vtx& v, float x, float y, float z) {
    v.hx = x;
    v.hy = y;
    v.hz = z;
    v.lx = v.ly = v.lz = 0.f;
  }
  // the longest edge at the vertex (cut_radius) lives in pad0
  static constexpr bool kEdgePerVertex = true;
  __device__ static void set_edge(Vtx& v, float e) { v.pad0 = e; }
  __device__ static double cut_r(double l, const DynParams*, const Vtx& v) {
    return cut_radius(l, (double)v.pad0 * (1.0 + 0x1p-20));
  }
  __device__ static void set_pos(Vtx& v, double x, double y, double z) {
    v.hx = (float)x;
    v.hy = (float)y;
    v.hz = (float)z;
    v.lx = (float)(x - (double)v.hx);
    v.ly = (float)(y - (double)v.hy);
    v.lz = (float)(z - (double)v.hz);
  }

  // Called by every lane of the warp (the traversal votes with __all_sync over the full
  // warp); lanes with active == false only vote and leave v untouched.
  // Nearest triangle of v, certified.  With `over` given, a traversal that tests more than
  // `budget` triangles stops, sets *over and leaves its best triangle so far in v (hint, dhi =
  // its distance bound without eta, q, qerr) for query_coop to finish.
  // With cut_r >= 0 (cut_radius), the query may stop at a triangle within cut_r of v: it
  // then sets *was_cut and keeps that triangle with a lower bound of 0.
  __device__ static void query(const BvhDev& B, Vtx& v, Counters& c, bool active, int budget = INT_MAX,
                               bool* over = nullptr, double cut_r = -1.0, bool* was_cut = nullptr) {
    NearestM t;
    t.tri32 = B.tri32;
    if (active) {
      t.P = pos(v);
      // start from the hint, or from a triangle of the point's grid cell: a first radius
      // (often already within the cut radius)
      const int h0 = v.hint >= 0 ? v.hint : grid_hint(B, t.P.h.x, t.P.h.y, t.P.h.z);
      if (h0 >= 0) t.test1(h0);
      if (v.hint < 0 && h0 >= 0 && budget < INT_MAX) ++budget;  // the grid's triangle is not the traversal's
      t.cut = cut_bound(B, cut_r);
      if (t.cut > 0.f) t.cut2 = __fmul_rd(t.cut, t.cut);
    } else {
      t.P = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    }
    bool unfinished = false, cut = active && t.best_hi < t.cut;  // the hint may be close enough
    if (__any_sync(0xffffffffu, t.cut > 0.f))  // one instantiation for the whole warp
      traverse_m<true>(B, t, c, active && !cut, budget, unfinished, cut);
    else
      traverse_m<false>(B, t, c, active, budget, unfinished, cut);
    if (!active) return;
    c.leaf += t.evals;
    c.escalations += t.esc;
    if (cut) {
      finish(B, v, t.best, t.best_hi, 0.f, t.q, t.qerr);
      if (was_cut) *was_cut = true;
      return;
    }
    if (unfinished) {
      *over = true;
      v.hint = t.best;
      v.dhi = t.best_hi;
      v.qx = t.q.x;
      v.qy = t.q.y;
      v.qz = t.q.z;
      v.qerr = t.qerr;
      return;
    }
    finish(B, v, t.best, t.best_hi, t.dlo, t.q, t.qerr);
  }
  // The distance bound of a handed-off query's best triangle so far.
  __device__ static double hint_dist(const Vtx& v) { return v.dhi; }
  // Whether a handed-off query's best triangle so far (hint, dhi without eta) is already
  // within the cut radius cut_r.
  __device__ static bool hint_within(const BvhDev& B, const Vtx& v, double cut_r) {
    return v.hint >= 0 && v.dhi < cut_bound(B, cut_r);
  }
  // The bound on best_hi (the certified distance to B's float triangles, before eta) below
  // which a query stops: best_hi + eta < cut_r, rounded so that it holds in exact arithmetic.
  __device__ static float cut_bound(const BvhDev& B, double cut_r) {
    if (!(cut_r > 0.0)) return -1.f;
    return __fsub_rd(__double2float_rd(cut_r), __ldg(B.meta));
  }
  // The query's result in v: eta (the distance between B's float triangles and its input)
  // widens both bounds.
  __device__ static void finish(const BvhDev& B, Vtx& v, int best, float best_hi, float dlo, F3 q, float qerr) {
    const float eta = __ldg(B.meta);
    v.tri = best;
    v.dhi = __fadd_ru(best_hi, eta);
    v.dlo = fmaxf(__fsub_rd(fminf(dlo, best_hi), eta), 0.f);
    v.qx = q.x;
    v.qy = q.y;
    v.qz = q.z;
    v.qerr = __fadd_ru(qerr, eta);
  }
  // query() of a vertex that a lane's traversal handed off, by the whole warp (every lane
  // passes the same v; lane 0 returns the result in it).  The certified lower bound is the
  // smallest lower bound over the triangles tested and the final best upper bound (every
  // pruned box lies beyond the radius of the moment, which is at least that).
  // With cut_r >= 0 the traversal may stop as query() does (the same for the whole warp);
  // returns true if it did.
  __device__ static bool query_coop(const BvhDev& B, Vtx& v, Counters& c, unsigned* s_code, float* s_e,
                                    double cut_r = -1.0) {
    const int lane = threadIdx.x & 31;
    NearestM t;
    t.tri32 = B.tri32;
    t.P = pos(v);
    if (lane == 0 && v.hint >= 0) {  // the lane traversal's best so far
      t.best = v.hint;
      t.best_hi = v.dhi;
      t.q = {v.qx, v.qy, v.qz};
      t.qerr = v.qerr;
    }
    const F3 plo = {__fadd_rd(t.P.h.x, t.P.l.x), __fadd_rd(t.P.h.y, t.P.l.y), __fadd_rd(t.P.h.z, t.P.l.z)};
    const F3 phi = {__fadd_ru(t.P.h.x, t.P.l.x), __fadd_ru(t.P.h.y, t.P.l.y), __fadd_ru(t.P.h.z, t.P.l.z)};
    auto box = [plo, phi](float lx, float ly, float lz, float hx, float hy, float hz) {
      return box_lo2(plo, phi, lx, ly, lz, hx, hy, hz);
    };
    const float cb = cut_bound(B, cut_r);
    const bool cut = cb > 0.f ? traverse_coop<true>(B, t, box, s_code, s_e, c, __fmul_rd(cb, cb))
                              : traverse_coop<false>(B, t, box, s_code, s_e, c, 0.f);
    c.leaf += t.evals;
    c.escalations += t.esc;
    const float m = warp_min_f(t.best_hi), dlo = cut ? 0.f : warp_min_f(t.dlo);
    const int src = __ffs(__ballot_sync(0xffffffffu, t.best_hi == m)) - 1;
    const int best = __shfl_sync(0xffffffffu, t.best, src);
    const F3 q = {__shfl_sync(0xffffffffu, t.q.x, src), __shfl_sync(0xffffffffu, t.q.y, src),
                  __shfl_sync(0xffffffffu, t.q.z, src)};
    const float qerr = __shfl_sync(0xffffffffu, t.qerr, src);
    finish(B, v, best, m, dlo, q, qerr);
    return cut;
  }
  __device__ static double lower(const Vtx& v) { return v.dlo; }
  __device__ static double out_dist(const Vtx& v) { return v.dhi; }
  __device__ static double out_dlo(const Vtx& v) { return v.dlo; }
  __device__ static D3 out_foot(const Vtx& v) {
    return {(double)v.hx + (double)v.lx + (double)v.qx, (double)v.hy + (double)v.ly + (double)v.qy,
            (double)v.hz + (double)v.lz + (double)v.qz};
  }
  __device__ static void midpoint(const Vtx& a, const Vtx& b, Vtx& m) {
    double x = 0.5 * (((double)a.hx + (double)a.lx) + ((double)b.hx + (double)b.lx));
    double y = 0.5 * (((double)a.hy + (double)a.ly) + ((double)b.hy + (double)b.ly));
    double z = 0.5 * (((double)a.hz + (double)a.lz) + ((double)b.hz + (double)b.lz));
    set_pos(m, x, y, z);
    m.qx = m.qy = m.qz = 0.f;
    m.qerr = m.dhi = m.dlo = 0.f;
    m.tri = -2;
    m.hint = a.tri;
    // every edge of a sub-triangle at m is at most the longest edge at a or at b (each edge
    // of the parent touches a or b)
    m.pad0 = fmaxf(a.pad0, b.pad0);
    m.pad1 = 0.f;
  }
  // upper_bound for the paper's cascade order with u4 deferred (only valid for those
  // options; the kernels pick it on the host): u4 comes later, so the footpoints are not read
  __device__ static UT upper_bound_paper(const BvhDev& B, const Vtx& a, const Vtx& b, const Vtx& c, double,
                                         float lf, const RunParams& rp, int& code, Counters& cnt) {
    const VM t[3] = {{pos(a), a.dhi, a.tri, {0.f, 0.f, 0.f}, 0.f},
                     {pos(b), b.dhi, b.tri, {0.f, 0.f, 0.f}, 0.f},
                     {pos(c), c.dhi, c.tri, {0.f, 0.f, 0.f}, 0.f}};
    return upper_bound_m_paper(B, t, lf, rp, code, cnt);
  }
  // The paper-order cascade in two parts, for kernels that gather the items reaching u3 into
  // full warps: paper_cheap runs the exact case, u1 and u2; it returns true when u3 is still
  // needed (U so far in *u12), else the result in *U and *code as upper_bound_paper.
  // paper_u3 then finishes such an item; together they give upper_bound_paper's values.
  __device__ static bool paper_cheap(const Vtx& a, const Vtx& b, const Vtx& c, float lf, const RunParams& rp,
                                     float* U, int* code, float* u12) {
    const VM t[3] = {{pos(a), a.dhi, a.tri, {0.f, 0.f, 0.f}, 0.f},
                     {pos(b), b.dhi, b.tri, {0.f, 0.f, 0.f}, 0.f},
                     {pos(c), c.dhi, c.tri, {0.f, 0.f, 0.f}, 0.f}};
    if (t[0].I == t[1].I && t[1].I == t[2].I) {
      *code = 0;
      *U = __fadd_ru(fmaxf(t[0].dhi, fmaxf(t[1].dhi, t[2].dhi)), rp.slack_f);
      return false;
    }
    const EdgesM E(t);
    const float u1 = ubm_u1(t, E);
    if (u1 < lf) {
      *code = 1;
      *U = __fadd_ru(u1, rp.slack_f);
      return false;
    }
    const float u2 = ubm_u2(t, E);
    if (u2 < lf) {
      *code = 2;
      *U = __fadd_ru(u2, rp.slack_f);
      return false;
    }
    *u12 = fminf(u1, u2);
    return true;
  }
  __device__ static UT paper_u3(const BvhDev& B, const Vtx& a, const Vtx& b, const Vtx& c, float lf, const RunParams& rp,
                                float u12, int& code, Counters& cnt) {
    const VM t[3] = {{pos(a), a.dhi, a.tri, {0.f, 0.f, 0.f}, 0.f},
                     {pos(b), b.dhi, b.tri, {0.f, 0.f, 0.f}, 0.f},
                     {pos(c), c.dhi, c.tri, {0.f, 0.f, 0.f}, 0.f}};
    const float u3 = ubm_u3(B, t, lf, cnt.evals);
    float U;
    if (u3 < lf) {
      code = 3;
      U = u3;
    } else {
      code = kDeferU4;
      U = fminf(u12, u3);
    }
    return __fadd_ru(U, rp.slack_f);
  }
  __device__ static UT upper_bound(const BvhDev& B, const Vtx& a, const Vtx& b, const Vtx& c, double,
                                   float lf, const RunParams& rp, int& code, Counters& cnt) {
    VM t[3] = {{pos(a), a.dhi, a.tri, {a.qx, a.qy, a.qz}, a.qerr},
               {pos(b), b.dhi, b.tri, {b.qx, b.qy, b.qz}, b.qerr},
               {pos(c), c.dhi, c.tri, {c.qx, c.qy, c.qz}, c.qerr}};
    return upper_bound_m(B, t, lf, rp, code, cnt);
  }
};

}  // namespace hd
