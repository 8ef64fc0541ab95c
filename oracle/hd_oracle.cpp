// Plain FP64 CPU oracle for the one-sided Pompeiu-Hausdorff distance h(A,B) between two
// triangle soups, following Sacht & Jacobson, "Cascading upper bounds for triangle soup
// Pompeiu-Hausdorff distance" (SGP 2024).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that the
// CUDA path is checked against.  Only the tests, the package smoke check and the
// benchmark's CPU-baseline leg may load it; the library's product path never does.  It
// shares no code, header or constant with the CUDA sources.
//
// What it does, in the paper's order (Section 3.1 and Section 4):
//   * distances D_A, nearest triangles I_A and closest points C_A of the vertices of A
//     to B -- by brute force over every triangle of B (no hierarchy);
//   * lower bound l = max of the vertex distances (Section 3.1);
//   * UpperBound(T, l): exact case (Eq. uexact), then u1 (Eq. u1), u2 (Eq. u2),
//     u3 (Eqs. Kang2018_case1 / Kang2018_case2), u4 (Eq. bound_u4), stopping at the
//     first bound below l, else the minimum of the four (Section 3.2, Section 4);
//   * a best-first priority queue over sub-triangles, midpoint 1->4 subdivision, the
//     running upper bound, the face cap m * n_A (Section 4) and the stopping rule
//     (u - l) <= eps (Section 3.1).
// All arithmetic is IEEE double with round-to-nearest, as in the paper's Section 4.
//
// Readings of points the paper leaves open (each also listed in the design notes):
//   * stop when u - l <= eps (Section 3.1 loop text), eps absolute or relative to the
//     bounding-box diagonal of A's referenced vertices;
//   * discard strictly when U < l; U >= l is kept (Section 4);
//   * the running upper bound is the minimum over iterations of max(l, top of queue);
//   * "same triangle" = equal nearest-triangle indices, ties in the brute-force nearest
//     search go to the lowest triangle index;
//   * u3 case 1 "share an edge" = the two face rows of B share exactly two vertex
//     indices; the bisecting plane contains the shared edge and has normal w1 - w2,
//     w_i the unit in-plane direction perpendicular to the edge pointing into S_i; the
//     split points are used only when the lone vertex lies on S1's side and both other
//     vertices on S2's side, otherwise the edge midpoints;
//   * u4: the shortest edge is the first minimum among (v1v2, v2v3, v3v1); edge/plane
//     crossings with parameter t in [0,1] count; equal footpoints use vertices only;
//   * u2: the acute test is the paper's s - r > 2R; a zero-area triangle takes the
//     half-longest-edge branch.
//
// Parity status: point_triangle, nearest, every bound and the full loop are pinned by
// the CPU tests (closed forms, brute-force sampling, convexity cases, invariants).
// What stays unpinned is only how tight u - l gets per iteration.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <queue>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// status codes (numeric values chosen to be the same as the library's, by convention)
constexpr int ST_OK = 0;
constexpr int ST_INVALID = 1;
constexpr int ST_CAPACITY = 2;
constexpr int ST_NUMERIC = 3;

struct P3 {
  double x, y, z;
};
inline P3 operator+(P3 a, P3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline P3 operator-(P3 a, P3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline P3 operator*(double s, P3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(P3 a, P3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline P3 cross(P3 a, P3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(P3 a) { return std::sqrt(dot(a, a)); }

// ------------------------------------------------------------------ point-triangle distance
// The paper takes these from libigl/CGAL and does not print a formula (Section 4).  The
// oracle uses the plain definition by feature enumeration: the closest point of a triangle
// is the orthogonal projection onto its plane when that projection lies inside the
// triangle, and otherwise lies on one of the three edges.

struct Foot {
  double d;
  P3 q;
};

Foot point_segment(P3 p, P3 s0, P3 s1) {
  P3 e = s1 - s0;
  double ee = dot(e, e);
  double t = 0.0;
  if (ee > 0.0) t = std::min(1.0, std::max(0.0, dot(p - s0, e) / ee));
  P3 q = s0 + t * e;
  return {norm(p - q), q};
}

Foot point_triangle(P3 p, P3 a, P3 b, P3 c) {
  P3 n = cross(b - a, c - a);
  double nn = dot(n, n);
  if (nn > 0.0) {
    double s = dot(p - a, n) / nn;
    P3 x = p - s * n;  // orthogonal projection of p onto the plane of the triangle
    // signed areas (scaled by |n|) of the three sub-triangles around x
    double wa = dot(cross(b - x, c - x), n);
    double wb = dot(cross(c - x, a - x), n);
    double wc = dot(cross(a - x, b - x), n);
    if (wa >= 0.0 && wb >= 0.0 && wc >= 0.0) return {std::fabs(s) * std::sqrt(nn), x};
  }
  Foot best = point_segment(p, a, b);
  Foot f = point_segment(p, b, c);
  if (f.d < best.d) best = f;
  f = point_segment(p, c, a);
  if (f.d < best.d) best = f;
  return best;
}

// ------------------------------------------------------------------ meshes and nearest queries

struct Mesh {
  std::vector<P3> V;
  const int32_t* F;
  int64_t nF;
  P3 vert(int64_t f, int k) const { return V[F[3 * f + k]]; }
};

struct Near {
  double d;
  int32_t idx;
  P3 q;
};

// d(p, B) by brute force; ties go to the lowest triangle index.
Near nearest(const Mesh& B, P3 p) {
  Near best{INFINITY, -1, {0, 0, 0}};
  for (int64_t f = 0; f < B.nF; ++f) {
    Foot r = point_triangle(p, B.vert(f, 0), B.vert(f, 1), B.vert(f, 2));
    if (r.d < best.d) best = {r.d, (int32_t)f, r.q};
  }
  return best;
}

// Same, parallel over the triangles of B (used for the few midpoint queries per split).
Near nearest_par(const Mesh& B, P3 p) {
#ifdef _OPENMP
  if (B.nF >= 4096) {
    int nt = omp_get_max_threads();
    std::vector<Near> part(nt, Near{INFINITY, -1, {0, 0, 0}});
#pragma omp parallel
    {
      int t = omp_get_thread_num();
      Near best{INFINITY, -1, {0, 0, 0}};
#pragma omp for schedule(static)
      for (int64_t f = 0; f < B.nF; ++f) {
        Foot r = point_triangle(p, B.vert(f, 0), B.vert(f, 1), B.vert(f, 2));
        if (r.d < best.d) best = {r.d, (int32_t)f, r.q};
      }
      part[t] = best;
    }
    Near best = part[0];
    for (int t = 1; t < nt; ++t)  // static chunks are in index order, so the first strict min wins
      if (part[t].d < best.d) best = part[t];
    return best;
  }
#endif
  return nearest(B, p);
}

// ------------------------------------------------------------------ upper bounds (Section 3.2)

// Everything the bounds need to know about one vertex of T: its position v, distance d to
// B, nearest triangle index I and closest point q (the paper's D_A, I_A, C_A).
struct VInfo {
  P3 v;
  double d;
  int32_t I;
  P3 q;
};

enum { B_EXACT = 0, B_U1 = 1, B_U2 = 2, B_U3 = 3, B_U4 = 4, B_KEPT = 5 };

struct Counter {
  int64_t evals = 0;
};

// Exact case, Eq. (uexact): all three vertices have the same nearest triangle S, and then
// h(T, B) <= h(T, S) = max_i |v_i - q_i|.
double bound_exact(const VInfo t[3]) { return std::max(t[0].d, std::max(t[1].d, t[2].d)); }

// First bound, Eq. (u1): min_i [ max(|v_i - v_{i+1}|, |v_i - v_{i+2}|) + |v_i - q_i| ].
double bound_u1(const VInfo t[3]) {
  double u = INFINITY;
  for (int i = 0; i < 3; ++i) {
    const VInfo& a = t[i];
    const VInfo& b = t[(i + 1) % 3];
    const VInfo& c = t[(i + 2) % 3];
    u = std::min(u, std::max(norm(a.v - b.v), norm(a.v - c.v)) + a.d);
  }
  return u;
}

// g of Eq. (u2): circumradius R when s - r > 2R (acute), else half the longest edge.
double bound_g(const VInfo t[3]) {
  double e1 = norm(t[1].v - t[2].v), e2 = norm(t[2].v - t[0].v), e3 = norm(t[0].v - t[1].v);
  double area = 0.5 * norm(cross(t[1].v - t[0].v, t[2].v - t[0].v));
  double emax = std::max(e1, std::max(e2, e3));
  if (area > 0.0) {
    double R = e1 * e2 * e3 / (4.0 * area);
    double s = 0.5 * (e1 + e2 + e3);
    double r = area / s;
    if (s - r > 2.0 * R) return R;
  }
  return 0.5 * emax;
}

// Second bound, Eq. (u2): g + max_i |v_i - q_i|.
double bound_u2(const VInfo t[3]) { return bound_g(t) + std::max(t[0].d, std::max(t[1].d, t[2].d)); }

double dist_to_face(const Mesh& B, int32_t f, P3 x, Counter& cnt) {
  ++cnt.evals;
  return point_triangle(x, B.vert(f, 0), B.vert(f, 1), B.vert(f, 2)).d;
}

// Do faces f and g of B share an edge, i.e. exactly two vertex indices?  Returns the two
// shared indices in s0, s1 and the opposite vertex of each face in of, og.
bool share_edge(const Mesh& B, int32_t f, int32_t g, int32_t& s0, int32_t& s1, int32_t& of, int32_t& og) {
  int shared[3], ns = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (B.F[3 * f + a] == B.F[3 * g + b]) {
        bool dup = false;
        for (int k = 0; k < ns; ++k) dup |= shared[k] == B.F[3 * f + a];
        if (!dup) shared[ns++] = B.F[3 * f + a];
      }
  if (ns != 2) return false;
  s0 = shared[0];
  s1 = shared[1];
  of = og = -1;
  for (int a = 0; a < 3; ++a) {
    int32_t vf = B.F[3 * f + a], vg = B.F[3 * g + a];
    if (vf != s0 && vf != s1) of = vf;
    if (vg != s0 && vg != s1) og = vg;
  }
  return of >= 0 && og >= 0;
}

// Third bound (Kang et al. 2018), Eqs. (Kang2018_case1) and (Kang2018_case2).
double bound_u3(const Mesh& B, const VInfo t[3], Counter& cnt) {
  // case 1: exactly two distinct nearest triangles, and they share an edge
  int lone = -1;
  if (t[0].I != t[1].I || t[1].I != t[2].I) {
    if (t[1].I == t[2].I) lone = 0;
    else if (t[0].I == t[2].I) lone = 1;
    else if (t[0].I == t[1].I) lone = 2;
  }
  int32_t s0, s1, o1, o2;
  if (lone >= 0 && share_edge(B, t[lone].I, t[(lone + 1) % 3].I, s0, s1, o1, o2)) {
    const VInfo& v1 = t[lone];          // the vertex alone on S1
    const VInfo& v2 = t[(lone + 1) % 3];  // v2, v3 on S2
    const VInfo& v3 = t[(lone + 2) % 3];
    int32_t S1 = v1.I, S2 = v2.I;
    // bisecting plane of the two supporting half-planes through the shared edge
    P3 p0 = B.V[s0], e = B.V[s1] - B.V[s0];
    P3 b1 = 0.5 * (v1.v + v2.v), b2 = 0.5 * (v1.v + v3.v);  // fallback: edge midpoints
    double el = norm(e);
    if (el > 0.0) {
      P3 eh = (1.0 / el) * e;
      P3 a1 = B.V[o1] - p0, a2 = B.V[o2] - p0;
      P3 w1 = a1 - dot(a1, eh) * eh, w2 = a2 - dot(a2, eh) * eh;
      double n1 = norm(w1), n2 = norm(w2);
      if (n1 > 0.0 && n2 > 0.0) {
        P3 nb = (1.0 / n1) * w1 - (1.0 / n2) * w2;
        double sv1 = dot(nb, v1.v - p0), sv2 = dot(nb, v2.v - p0), sv3 = dot(nb, v3.v - p0);
        if (sv1 >= 0.0 && sv2 <= 0.0 && sv3 <= 0.0 && sv1 - sv2 > 0.0 && sv1 - sv3 > 0.0) {
          b1 = v1.v + (sv1 / (sv1 - sv2)) * (v2.v - v1.v);
          b2 = v1.v + (sv1 / (sv1 - sv3)) * (v3.v - v1.v);
        }
      }
    }
    // R = (v1, b1, b2) against S1, Q = (v3, b2, b1, v2) against S2; the distance from a
    // convex polygon to a triangle is attained at one of the polygon's vertices.
    double hR = std::max(dist_to_face(B, S1, v1.v, cnt),
                         std::max(dist_to_face(B, S1, b1, cnt), dist_to_face(B, S1, b2, cnt)));
    double hQ = std::max(std::max(dist_to_face(B, S2, v3.v, cnt), dist_to_face(B, S2, b2, cnt)),
                         std::max(dist_to_face(B, S2, b1, cnt), dist_to_face(B, S2, v2.v, cnt)));
    return std::max(hR, hQ);
  }
  // case 2: three quadrilaterals Q_i = (v_i, m_i, b, m_{i-1}) each against S_i
  P3 m[3], bc = (1.0 / 3.0) * (t[0].v + t[1].v + t[2].v);
  for (int i = 0; i < 3; ++i) m[i] = 0.5 * (t[i].v + t[(i + 1) % 3].v);  // m1 on v1v2, m2 on v2v3, m3 on v3v1
  double ut = 0.0;
  for (int i = 0; i < 3; ++i) {
    int32_t S = t[i].I;
    double h = std::max(std::max(dist_to_face(B, S, t[i].v, cnt), dist_to_face(B, S, m[i], cnt)),
                        std::max(dist_to_face(B, S, bc, cnt), dist_to_face(B, S, m[(i + 2) % 3], cnt)));
    ut = std::max(ut, h);
  }
  // min_i h(T, S_i), each the maximum of T's vertex distances to S_i
  double best = INFINITY;
  for (int i = 0; i < 3; ++i) {
    double h = 0.0;
    for (int j = 0; j < 3; ++j) h = std::max(h, dist_to_face(B, t[i].I, t[j].v, cnt));
    best = std::min(best, h);
  }
  return std::min(ut, best);
}

// max over T of d(., {a, b}): attained at a vertex of T or where an edge of T crosses the
// bisector plane of a and b (Bartoň et al. 2010, as used in Section 3.2.4).
double h_tri_two_points(const VInfo t[3], P3 a, P3 b) {
  auto f = [&](P3 x) { return std::min(norm(x - a), norm(x - b)); };
  double h = std::max(f(t[0].v), std::max(f(t[1].v), f(t[2].v)));
  P3 n = b - a;
  if (dot(n, n) == 0.0) return h;
  P3 mid = 0.5 * (a + b);
  for (int i = 0; i < 3; ++i) {
    P3 x0 = t[i].v, x1 = t[(i + 1) % 3].v;
    double c0 = dot(n, x0 - mid), c1 = dot(n, x1 - mid);
    if (((c0 <= 0.0 && c1 >= 0.0) || (c0 >= 0.0 && c1 <= 0.0)) && c0 != c1) {
      double s = c0 / (c0 - c1);
      h = std::max(h, f(x0 + s * (x1 - x0)));
    }
  }
  return h;
}

// Fourth bound, Eq. (bound_u4): q2, q3 are the footpoints of the shortest edge's
// vertices, q1 that of the other vertex; u4 = min(h(T,{q1,q2}), h(T,{q1,q3})).
double bound_u4(const VInfo t[3]) {
  double len[3];
  for (int i = 0; i < 3; ++i) len[i] = norm(t[i].v - t[(i + 1) % 3].v);  // v1v2, v2v3, v3v1
  int k = 0;
  if (len[1] < len[k]) k = 1;
  if (len[2] < len[k]) k = 2;
  P3 q2 = t[k].q, q3 = t[(k + 1) % 3].q, q1 = t[(k + 2) % 3].q;
  return std::min(h_tri_two_points(t, q1, q2), h_tri_two_points(t, q1, q3));
}

struct UB {
  double U;
  int code;  // B_EXACT..B_U4 = the bound that decided (discarded if U < l), B_KEPT = none did
};

// UpperBound(T, l) of Section 4: exact case first, then the bounds in `order`, stopping at
// the first one below l; otherwise the minimum of those computed.
UB upper_bound(const Mesh& B, const VInfo t[3], double l, const uint8_t* order, int n_bounds, Counter& cnt) {
  if (t[0].I == t[1].I && t[1].I == t[2].I) return {bound_exact(t), B_EXACT};
  double U = INFINITY;
  for (int k = 0; k < n_bounds; ++k) {
    double u = 0.0;
    switch (order[k]) {
      case 1: u = bound_u1(t); break;
      case 2: u = bound_u2(t); break;
      case 3: u = bound_u3(B, t, cnt); break;
      case 4: u = bound_u4(t); break;
      default: u = INFINITY;
    }
    if (u < l) return {u, (int)order[k]};
    U = std::min(U, u);
  }
  return {U, B_KEPT};
}

struct Item {
  double U;
  int32_t v[3];
  bool operator<(const Item& o) const { return U < o.U; }  // max-heap on U
};

Mesh make_mesh(const double* V, int64_t nV, const int32_t* F, int64_t nF) {
  Mesh m;
  m.V.resize(nV);
  for (int64_t i = 0; i < nV; ++i) m.V[i] = {V[3 * i], V[3 * i + 1], V[3 * i + 2]};
  m.F = F;
  m.nF = nF;
  return m;
}

bool valid_mesh(const double* V, int64_t nV, const int32_t* F, int64_t nF) {
  if (nV <= 0 || nF <= 0) return false;
  for (int64_t i = 0; i < 3 * nV; ++i)
    if (!std::isfinite(V[i])) return false;
  for (int64_t i = 0; i < 3 * nF; ++i)
    if (F[i] < 0 || F[i] >= nV) return false;
  return true;
}

}  // namespace

// ============================================================================ C interface

extern "C" {

struct or_stats {
  int64_t splits;
  int64_t pointtri_evals;
  int64_t discards[6];  // by deciding bound: exact, u1, u2, u3, u4, (kept)
  int64_t max_queue;
  int64_t iterations;
};

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_point_triangle(const double* p, const double* a, const double* b, const double* c, double* d,
                       double* q) {
  Foot f = point_triangle({p[0], p[1], p[2]}, {a[0], a[1], a[2]}, {b[0], b[1], b[2]}, {c[0], c[1], c[2]});
  *d = f.d;
  q[0] = f.q.x;
  q[1] = f.q.y;
  q[2] = f.q.z;
}

// Brute-force nearest triangle of B for nP points (parallel over the points).
void or_nearest(const double* P, int64_t nP, const double* VB, int64_t nVB, const int32_t* FB, int64_t nFB,
                double* d, int32_t* idx, double* q) {
  Mesh B = make_mesh(VB, nVB, FB, nFB);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nP; ++i) {
    Near r = nearest(B, {P[3 * i], P[3 * i + 1], P[3 * i + 2]});
    d[i] = r.d;
    idx[i] = r.idx;
    q[3 * i] = r.q.x;
    q[3 * i + 1] = r.q.y;
    q[3 * i + 2] = r.q.z;
  }
}

// Every bound of one triangle T (tv = 3x3 vertex rows) whose vertices have distances td,
// nearest triangles tI and closest points tq (3x3).  out = {exact (NaN unless all three
// tI agree), u1, u2, u3, u4, g}.
void or_bounds_all(const double* tv, const double* td, const int32_t* tI, const double* tq, const double* VB,
                   int64_t nVB, const int32_t* FB, int64_t nFB, double* out) {
  Mesh B = make_mesh(VB, nVB, FB, nFB);
  VInfo t[3];
  for (int i = 0; i < 3; ++i)
    t[i] = {{tv[3 * i], tv[3 * i + 1], tv[3 * i + 2]}, td[i], tI[i], {tq[3 * i], tq[3 * i + 1], tq[3 * i + 2]}};
  Counter c;
  out[0] = (t[0].I == t[1].I && t[1].I == t[2].I) ? bound_exact(t) : NAN;
  out[1] = bound_u1(t);
  out[2] = bound_u2(t);
  out[3] = bound_u3(B, t, c);
  out[4] = bound_u4(t);
  out[5] = bound_g(t);
}

// UpperBound(T, l) for one triangle, as above; returns U and the deciding bound code.
double or_upper_bound(const double* tv, const double* td, const int32_t* tI, const double* tq, const double* VB,
                      int64_t nVB, const int32_t* FB, int64_t nFB, double l, const uint8_t* order, int n_bounds,
                      int* code) {
  Mesh B = make_mesh(VB, nVB, FB, nFB);
  VInfo t[3];
  for (int i = 0; i < 3; ++i)
    t[i] = {{tv[3 * i], tv[3 * i + 1], tv[3 * i + 2]}, td[i], tI[i], {tq[3 * i], tq[3 * i + 1], tq[3 * i + 2]}};
  Counter c;
  UB r = upper_bound(B, t, l, order, n_bounds, c);
  *code = r.code;
  return r.U;
}

// The branch-and-bound of Sections 3.1 and 4.  tol_mode 0: eps = tol; 1: eps = tol * dA.
// trace (optional, may be NULL): per iteration the pair (l, u_running), at most max_trace.
int or_hausdorff(const double* VA, int64_t nVA, const int32_t* FA, int64_t nFA, const double* VB, int64_t nVB,
                 const int32_t* FB, int64_t nFB, double tol, int tol_mode, double max_face_factor,
                 const uint8_t* order, int n_bounds, double* lower, double* upper, or_stats* stats, double* trace,
                 int64_t max_trace, int64_t* n_trace) {
  or_stats st;
  std::memset(&st, 0, sizeof st);
  if (n_trace) *n_trace = 0;
  if (!(tol > 0.0) || !valid_mesh(VA, nVA, FA, nFA) || !valid_mesh(VB, nVB, FB, nFB) || n_bounds < 0 ||
      n_bounds > 4) {
    if (stats) *stats = st;
    return ST_INVALID;
  }
  Mesh B = make_mesh(VB, nVB, FB, nFB);
  Counter cnt;

  // referenced vertices of A: l and dA use only these (the paper assumes no others exist)
  std::vector<char> ref(nVA, 0);
  for (int64_t i = 0; i < 3 * nFA; ++i) ref[FA[i]] = 1;
  P3 lo{INFINITY, INFINITY, INFINITY}, hi{-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < nVA; ++i)
    if (ref[i]) {
      lo = {std::min(lo.x, VA[3 * i]), std::min(lo.y, VA[3 * i + 1]), std::min(lo.z, VA[3 * i + 2])};
      hi = {std::max(hi.x, VA[3 * i]), std::max(hi.y, VA[3 * i + 1]), std::max(hi.z, VA[3 * i + 2])};
    }
  double dA = norm(hi - lo);
  double eps = tol_mode == 1 ? tol * dA : tol;

  // D_A, I_A, C_A for the vertices (Section 4)
  std::vector<VInfo> X(nVA);
  for (int64_t i = 0; i < nVA; ++i) X[i] = {{VA[3 * i], VA[3 * i + 1], VA[3 * i + 2]}, 0.0, -1, {0, 0, 0}};
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nVA; ++i)
    if (ref[i]) {
      Near r = nearest(B, X[i].v);
      X[i].d = r.d;
      X[i].I = r.idx;
      X[i].q = r.q;
    }
  cnt.evals += (int64_t)std::count(ref.begin(), ref.end(), 1) * nFB;

  // initial lower bound: maximum vertex distance (Section 3.1)
  double l = 0.0;
  for (int64_t i = 0; i < nVA; ++i)
    if (ref[i]) l = std::max(l, X[i].d);

  // upper bounds of every face, global upper bound, queue of the faces with U >= l
  std::priority_queue<Item> Q;
  double u_run = l;
  for (int64_t f = 0; f < nFA; ++f) {
    VInfo t[3] = {X[FA[3 * f]], X[FA[3 * f + 1]], X[FA[3 * f + 2]]};
    UB r = upper_bound(B, t, l, order, n_bounds, cnt);
    u_run = std::max(u_run, r.U);
    if (r.U >= l) Q.push({r.U, {FA[3 * f], FA[3 * f + 1], FA[3 * f + 2]}});
    else ++st.discards[r.code];
  }
  const double m_f = max_face_factor * (double)nFA;
  double c_f = (double)nFA;
  int status = ST_OK;

  for (;;) {
    ++st.iterations;
    st.max_queue = std::max<int64_t>(st.max_queue, (int64_t)Q.size());
    double u_now = Q.empty() ? l : std::max(l, Q.top().U);
    u_run = std::min(u_run, u_now);
    if (trace && n_trace && *n_trace < max_trace) {
      trace[2 * *n_trace] = l;
      trace[2 * *n_trace + 1] = u_run;
      ++*n_trace;
    }
    if (Q.empty()) {  // every sub-triangle was discarded: only rounding can do this (Section 5.3)
      status = ST_NUMERIC;
      break;
    }
    if (u_run - l <= eps) break;
    Item it = Q.top();
    Q.pop();
    if (it.U < l) continue;
    // midpoint subdivision: three new vertices W_A, four new faces G_A
    int32_t v1 = it.v[0], v2 = it.v[1], v3 = it.v[2];
    int32_t m12 = (int32_t)X.size(), m23 = m12 + 1, m31 = m12 + 2;
    P3 mp[3] = {0.5 * (X[v1].v + X[v2].v), 0.5 * (X[v2].v + X[v3].v), 0.5 * (X[v3].v + X[v1].v)};
    for (int k = 0; k < 3; ++k) {
      Near r = nearest_par(B, mp[k]);
      X.push_back({mp[k], r.d, r.idx, r.q});
      l = std::max(l, r.d);
    }
    cnt.evals += 3 * nFB;
    ++st.splits;
    const int32_t kids[4][3] = {{v1, m12, m31}, {m12, v2, m23}, {m31, m23, v3}, {m12, m23, m31}};
    for (const auto& k : kids) {
      VInfo t[3] = {X[k[0]], X[k[1]], X[k[2]]};
      UB r = upper_bound(B, t, l, order, n_bounds, cnt);
      if (r.U >= l) Q.push({r.U, {k[0], k[1], k[2]}});
      else ++st.discards[r.code];
    }
    c_f += 4.0;
    if (c_f > m_f) {
      u_run = std::min(u_run, Q.empty() ? l : std::max(l, Q.top().U));
      status = ST_CAPACITY;
      break;
    }
  }
  st.pointtri_evals = cnt.evals;
  *lower = l;
  *upper = std::max(l, u_run);
  if (stats) *stats = st;
  return status;
}

// Sampling bracket (Section 2, sampling methods, plus 1-Lipschitz continuity of d(., B)):
// every face of A gets the barycentric grid {(i/k, j/k)}; lo = max sampled distance is a
// lower bound of h, and since each point of a face lies within (longest edge)/k of a
// sample of that face, hi = max over faces of (max sampled distance + longest edge / k)
// is an upper bound.
void or_sampling_bracket(const double* VA, int64_t nVA, const int32_t* FA, int64_t nFA, const double* VB,
                         int64_t nVB, const int32_t* FB, int64_t nFB, int k, double* lo, double* hi) {
  Mesh A = make_mesh(VA, nVA, FA, nFA), B = make_mesh(VB, nVB, FB, nFB);
  double L = 0.0, H = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(max : L, H)
  for (int64_t f = 0; f < nFA; ++f) {
    P3 a = A.vert(f, 0), b = A.vert(f, 1), c = A.vert(f, 2);
    double m = 0.0;
    for (int i = 0; i <= k; ++i)
      for (int j = 0; i + j <= k; ++j) {
        double wb = (double)i / k, wc = (double)j / k;
        P3 s = (1.0 - wb - wc) * a + wb * b + wc * c;
        m = std::max(m, nearest(B, s).d);
      }
    double emax = std::max(norm(b - a), std::max(norm(c - b), norm(a - c)));
    L = std::max(L, m);
    H = std::max(H, m + emax / k);
  }
  *lo = L;
  *hi = H;
}

}  // extern "C"
