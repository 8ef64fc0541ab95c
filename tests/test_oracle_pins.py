"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself.

Each test states what it pins.  Independent references used here:
  * closed forms of h derived by hand (tests/golden/closed_forms.json);
  * a second closest-point-on-triangle algorithm (Voronoi-region tests on barycentric
    dot products, as in Ericson's "Real-Time Collision Detection" Sect. 5.1.5), written
    below and unrelated to the oracle's feature enumeration;
  * dense barycentric sampling, using that d(., B) is 1-Lipschitz;
  * convexity: for a convex B the maximum of d(., B) over a triangle is at a vertex;
  * invariants of the branch and bound (l non-decreasing, running u non-increasing).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import meshgen as mg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


# ----------------------------------------------------------------------------- independent helpers


def closest_point_regions(p, a, b, c):
    """Closest point on triangle abc by classifying p against the vertex/edge/face Voronoi regions."""
    ab, ac, ap = b - a, c - a, p - a
    d1, d2 = ab @ ap, ac @ ap
    if d1 <= 0 and d2 <= 0:
        return a
    bp = p - b
    d3, d4 = ab @ bp, ac @ bp
    if d3 >= 0 and d4 <= d3:
        return b
    vc = d1 * d4 - d3 * d2
    if vc <= 0 and d1 >= 0 and d3 <= 0:
        return a + d1 / (d1 - d3) * ab
    cp = p - c
    d5, d6 = ab @ cp, ac @ cp
    if d6 >= 0 and d5 <= d6:
        return c
    vb = d5 * d2 - d1 * d6
    if vb <= 0 and d2 >= 0 and d6 <= 0:
        return a + d2 / (d2 - d6) * ac
    va = d3 * d6 - d5 * d4
    if va <= 0 and (d4 - d3) >= 0 and (d5 - d6) >= 0:
        return b + (d4 - d3) / ((d4 - d3) + (d5 - d6)) * (c - b)
    den = 1.0 / (va + vb + vc)
    return a + ab * (vb * den) + ac * (vc * den)


def dist_regions(p, a, b, c):
    return float(np.linalg.norm(p - closest_point_regions(p, a, b, c)))


def dist_mesh_regions(p, V, F):
    return min(dist_regions(p, V[f[0]], V[f[1]], V[f[2]]) for f in F)


def bary_grid(k):
    return np.array([(1 - i / k - j / k, i / k, j / k) for i in range(k + 1) for j in range(k + 1 - i)])


def random_triangle(rng, kind):
    if kind == "sliver":
        a = rng.normal(size=3)
        d = rng.normal(size=3)
        return np.stack([a, a + d, a + 0.5 * d + 1e-4 * rng.normal(size=3)])
    if kind == "tiny":
        a = rng.normal(size=3)
        return np.stack([a, a + 1e-3 * rng.normal(size=3), a + 1e-3 * rng.normal(size=3)])
    return rng.normal(size=(3, 3))


# ----------------------------------------------------------------------------- P8: point-triangle


def test_point_triangle_textbook_cases(orc):
    a, b, c = np.array([0.0, 0, 0]), np.array([2.0, 0, 0]), np.array([0.0, 2, 0])
    # interior projection: distance to the plane
    d, q = orc.point_triangle(np.array([0.5, 0.5, -3.0]), a, b, c)
    assert d == pytest.approx(3.0, abs=1e-15) and np.allclose(q, [0.5, 0.5, 0])
    # vertex region
    d, q = orc.point_triangle(np.array([-1.0, -1.0, 1.0]), a, b, c)
    assert d == pytest.approx(math.sqrt(3.0), rel=1e-15) and np.allclose(q, a)
    # edge region (hypotenuse x + y = 2): foot (1.5, 0.5, 0)
    d, q = orc.point_triangle(np.array([2.0, 1.0, 0.0]), a, b, c)
    assert d == pytest.approx(math.sqrt(0.5), rel=1e-15) and np.allclose(q, [1.5, 0.5, 0])
    # degenerate triangles fall back to segments
    d, _ = orc.point_triangle(np.array([1.0, 1.0, 0.0]), a, b, 0.5 * (a + b))
    assert d == pytest.approx(1.0, rel=1e-15)
    d, _ = orc.point_triangle(np.array([1.0, 1.0, 1.0]), a, a, a)
    assert d == pytest.approx(math.sqrt(3.0), rel=1e-15)


@pytest.mark.parametrize("kind", ["generic", "sliver", "tiny"])
def test_point_triangle_matches_region_method(orc, kind):
    rng = np.random.default_rng(7)
    for _ in range(400):
        a, b, c = random_triangle(rng, kind)
        p = rng.normal(size=3) * (3 if kind == "generic" else 1)
        d, q = orc.point_triangle(p, a, b, c)
        ref = dist_regions(p, a, b, c)
        assert abs(d - ref) <= 1e-9 * max(1.0, ref)
        assert abs(np.linalg.norm(p - q) - d) <= 1e-12 * max(1.0, d)


def test_point_triangle_against_dense_grid(orc):
    rng = np.random.default_rng(11)
    k = 60
    W = bary_grid(k)
    for _ in range(60):
        T = rng.normal(size=(3, 3))
        p = rng.normal(size=3) * 2
        d, _ = orc.point_triangle(p, *T)
        S = W @ T
        gmin = np.min(np.linalg.norm(S - p, axis=1))
        diam = max(np.linalg.norm(T[0] - T[1]), np.linalg.norm(T[1] - T[2]), np.linalg.norm(T[2] - T[0]))
        assert d <= gmin + 1e-12
        assert gmin <= d + diam / k + 1e-12


def test_nearest_brute_force_matches_region_method(orc):
    p = mg.workload(1)
    rng = np.random.default_rng(3)
    P = rng.normal(size=(200, 3)) * 1.2
    d, idx, q = orc.nearest(P, p.VB, p.FB)
    for i in range(len(P)):
        ref = dist_mesh_regions(P[i], p.VB, p.FB)
        assert abs(d[i] - ref) <= 1e-12 * max(1, ref)
        f = p.FB[idx[i]]
        assert abs(dist_regions(P[i], *p.VB[f]) - d[i]) <= 1e-12 * max(1, ref)


# ----------------------------------------------------------------------------- P6/P7: bounds


def _infos(orc, T, VB, FB):
    d, I, q = orc.nearest(T, VB, FB)
    return d, I, q


def test_g_is_a_covering_radius(orc):
    """P7: g of Eq. (u2) bounds max_{p in T} min_i |p - v_i| (sampled), and hits the textbook values."""
    rng = np.random.default_rng(5)
    W = bary_grid(40)
    VB = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]])
    FB = np.array([[0, 1, 2]])
    for kind in ["generic"] * 150 + ["sliver"] * 50:
        T = random_triangle(rng, kind)
        d, I, q = _infos(orc, T, VB, FB)
        g = orc.bounds_all(T, d, I, q, VB, FB)[5]
        S = W @ T
        cover = np.max(np.min(np.linalg.norm(S[:, None, :] - T[None], axis=2), axis=1))
        assert cover <= g * (1 + 1e-12) + 1e-15
    # equilateral (acute): circumradius e / sqrt(3)
    T = np.array([[0.0, 0, 0], [1, 0, 0], [0.5, math.sqrt(3) / 2, 0]])
    d, I, q = _infos(orc, T, VB, FB)
    assert orc.bounds_all(T, d, I, q, VB, FB)[5] == pytest.approx(1 / math.sqrt(3), rel=1e-12)
    # obtuse: half the longest edge
    T = np.array([[0.0, 0, 0], [4, 0, 0], [1, 0.5, 0]])
    d, I, q = _infos(orc, T, VB, FB)
    assert orc.bounds_all(T, d, I, q, VB, FB)[5] == pytest.approx(2.0, rel=1e-12)
    # zero area: half the longest edge
    T = np.array([[0.0, 0, 0], [4, 0, 0], [1, 0, 0]])
    d, I, q = _infos(orc, T, VB, FB)
    assert orc.bounds_all(T, d, I, q, VB, FB)[5] == pytest.approx(2.0, rel=1e-12)


def test_bounds_closed_form_right_triangle(orc):
    """Right isosceles T at height 1 over a large triangle of z=0: every bound by hand.
    exact = 1, u1 = 2 (Eq. u1), g = sqrt(2)/2 and u2 = 1 + sqrt(2)/2 (Eq. u2),
    u3 = 1 (case 2 with S1=S2=S3), u4 = sqrt(2) (Eq. bound_u4, shortest edge v1v2)."""
    VB = np.array([[-10.0, -10, 0], [10, -10, 0], [0, 10, 0]])
    FB = np.array([[0, 1, 2]])
    T = np.array([[0.0, 0, 1], [1, 0, 1], [0, 1, 1]])
    d, I, q = _infos(orc, T, VB, FB)
    ex, u1, u2, u3, u4, g = orc.bounds_all(T, d, I, q, VB, FB)
    assert ex == pytest.approx(1.0, abs=1e-15)
    assert u1 == pytest.approx(2.0, rel=1e-15)
    assert g == pytest.approx(math.sqrt(2) / 2, rel=1e-14)
    assert u2 == pytest.approx(1 + math.sqrt(2) / 2, rel=1e-14)
    assert u3 == pytest.approx(1.0, rel=1e-15)
    assert u4 == pytest.approx(math.sqrt(2), rel=1e-14)


def test_u3_case1_uses_the_bisecting_plane(orc):
    """u3 case 1 (Eq. Kang2018_case1) over a unit square split on its anti-diagonal: with the
    bisecting plane x + y = 1 both pieces stay above their own triangle, so u3 = 1 exactly; the
    midpoint fallback would give more than 1 here."""
    VB = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]])
    FB = np.array([[0, 1, 2], [1, 3, 2]])
    T = np.array([[0.1, 0.1, 1.0], [0.9, 0.6, 1.0], [0.6, 0.9, 1.0]])
    d, I, q = _infos(orc, T, VB, FB)
    assert list(I) == [0, 1, 1]
    u3 = orc.bounds_all(T, d, I, q, VB, FB)[3]
    assert u3 == pytest.approx(1.0, rel=1e-14)


def _fan(height_apex):
    """Three triangles of B around the origin, bounded by the rays through the edge midpoints of
    the equilateral T used below; apex at z = -height_apex, outer vertices at z = 0."""
    ang = np.radians([90.0, 210.0, 330.0])
    T = np.stack([np.cos(ang), np.sin(ang), np.ones(3)], 1)
    mids = [0.5 * (T[i] + T[(i + 1) % 3]) for i in range(3)]  # m1 (v1v2), m2 (v2v3), m3 (v3v1)
    rays = [10 * m[:2] / np.linalg.norm(m[:2]) for m in mids]
    VB = np.array([[0, 0, -height_apex]] + [[r[0], r[1], 0.0] for r in rays])
    FB = np.array([[0, 3, 1], [0, 1, 2], [0, 2, 3]], np.int32)  # S1: m3..m1, S2: m1..m2, S3: m2..m3
    return T, VB, FB


def test_u3_case2_flat_fan(orc):
    """u3 case 2 (Eq. Kang2018_case2): T at height 1 over a flat fan whose sector boundaries pass
    under T's edge midpoints and barycentre; each quadrilateral Q_i lies over its own S_i, so
    the partial bound is exactly 1 while every h(T, S_i) exceeds 1: u3 = 1."""
    T, VB, FB = _fan(0.0)
    d, I, q = _infos(orc, T, VB, FB)
    assert list(I) == [0, 1, 2]
    u3 = orc.bounds_all(T, d, I, q, VB, FB)[3]
    assert u3 == pytest.approx(1.0, rel=1e-13)


def test_u3_case2_cone_barycentre_matters(orc):
    """Same fan folded into a cone (apex below the barycentre): the farthest point of each Q_i
    from S_i is the barycentre, so u3 must still bound the sampled maximum of d(., B)."""
    T, VB, FB = _fan(0.5)
    d, I, q = _infos(orc, T, VB, FB)
    assert len(set(I)) == 3
    u3 = orc.bounds_all(T, d, I, q, VB, FB)[3]
    ds, _, _ = orc.nearest(bary_grid(60) @ T, VB, FB)
    assert ds.max() <= u3 * (1 + 1e-13)
    assert u3 <= ds.max() + 0.05  # and it is the tight bound here, not min_i h(T, S_i)


def test_u4_closed_form_bridge(orc):
    """u4 (Eq. bound_u4) on the thin bridge of the golden pair: the shortest edge is v2v3, so
    q1 = foot of v1 = (0,0.4,0), q2 = (2,0.4,0), q3 = (2,0.6,0).  By hand h(T,{q1,q2}) =
    sqrt(2.01) (edge v3v1 meets the bisector x = 1 at (1,0.5,1)) and h(T,{q1,q3}) =
    sqrt(2.0201) (edge v1v2 meets its bisector at x = 1.01): u4 = sqrt(2.01)."""
    VB = np.array([[0.0, 0, 0], [0, 1, 0], [-1, 0, 0], [2, 0, 0], [3, 0, 0], [2, 1, 0]])
    FB = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    T = np.array([[0.0, 0.4, 1], [2, 0.4, 1], [2, 0.6, 1]])
    d, I, q = _infos(orc, T, VB, FB)
    assert list(I) == [0, 1, 1]
    u4 = orc.bounds_all(T, d, I, q, VB, FB)[4]
    assert u4 == pytest.approx(math.sqrt(2.01), rel=1e-14)


def test_u4_is_the_sampled_two_point_radius(orc):
    """u4 (Eq. bound_u4) written from its definition, for arbitrary footpoints: with q2, q3 the
    footpoints of the shortest edge's ends (edges v1v2, v2v3, v3v1, ties to the first) and q1
    that of the opposite vertex, u4 = min(H(q1, q2), H(q1, q3)), where H(a, b) is the largest
    min(|p - a|, |p - b|) over p in T.  That is a maximum of a 1-Lipschitz function over T, so
    a barycentric grid with k steps brackets it: sampled <= H <= sampled + longest edge / k
    (the grid's covering radius).  This pins the oracle's vertex-and-bisector evaluation and its
    footpoint labels without using either."""
    rng = np.random.default_rng(41)
    VB = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]])
    FB = np.array([[0, 1, 2]], np.int32)
    k = 150
    W = bary_grid(k)
    for t in range(120):
        T = random_triangle(rng, "generic" if t % 4 else "sliver")
        q = T + rng.normal(size=(3, 3)) * rng.choice([0.05, 0.5, 2.0])
        d = np.linalg.norm(q - T, axis=1)
        I = np.zeros(3, np.int32)
        u4 = orc.bounds_all(T, d, I, q, VB, FB)[4]
        e = [np.linalg.norm(T[0] - T[1]), np.linalg.norm(T[1] - T[2]), np.linalg.norm(T[2] - T[0])]
        s = int(np.argmin(e))
        q1, q2, q3 = q[(s + 2) % 3], q[s], q[(s + 1) % 3]
        P = W @ T

        def H(a, b):
            return np.max(np.minimum(np.linalg.norm(P - a, axis=1), np.linalg.norm(P - b, axis=1)))

        us = min(H(q1, q2), H(q1, q3))
        assert us - 1e-12 <= u4 <= us + max(e) / k + 1e-12, (t, u4, us, max(e) / k)


def test_bounds_closed_form_unequal_heights(orc):
    """T = (0,0,1), (1,0,2), (0,1,3) over a large triangle of z=0, so d = (1, 2, 3) and all
    three project to one triangle.  By hand: exact = 3; u1 = 1 + sqrt(5) (vertex v1, longest
    edge v1v3 = sqrt(5)); T is right-angled at v1, so g = sqrt(5)/2 and u2 = 3 + sqrt(5)/2."""
    VB = np.array([[-10.0, -10, 0], [10, -10, 0], [0, 10, 0]])
    FB = np.array([[0, 1, 2]])
    T = np.array([[0.0, 0, 1], [1, 0, 2], [0, 1, 3]])
    d, I, q = _infos(orc, T, VB, FB)
    ex, u1, u2, u3, u4, g = orc.bounds_all(T, d, I, q, VB, FB)
    assert ex == pytest.approx(3.0, rel=1e-15)
    assert u1 == pytest.approx(1 + math.sqrt(5), rel=1e-15)
    assert u2 == pytest.approx(3 + math.sqrt(5) / 2, rel=1e-14)


def _random_small_mesh(rng, n):
    V = rng.normal(size=(3 * n, 3)) * 0.6
    return V, np.arange(3 * n, dtype=np.int32).reshape(n, 3)


@pytest.mark.parametrize("seed", range(6))
def test_every_bound_is_an_upper_bound(orc, seed):
    """P6: d(p, B) <= u_k(T, B) for dense samples p of T, for the exact case and u1..u4."""
    rng = np.random.default_rng(100 + seed)
    if seed % 2 == 0:
        VB, FB = _random_small_mesh(rng, 12)
    else:  # a closed, connected B so that u3 case 1 (shared edges) occurs
        VB, FB = mg.icosphere(1)
        VB = VB * 0.8
    W = bary_grid(24)
    seen_case1 = False
    for t in range(60):
        kind = ["generic", "sliver", "tiny"][t % 3]
        T = random_triangle(rng, kind) * (0.5 if kind == "generic" else 1.0)
        if seed % 2 == 1:
            T = T * 0.3 + rng.normal(size=3) * 0.6
        d, I, q = _infos(orc, T, VB, FB)
        b = orc.bounds_all(T, d, I, q, VB, FB)
        ds, _, _ = orc.nearest(W @ T, VB, FB)
        h = ds.max()
        for k, name in enumerate(["exact", "u1", "u2", "u3", "u4"]):
            if not np.isnan(b[k]):
                assert h <= b[k] * (1 + 1e-12) + 1e-12, (name, h, b[k])
        assert max(d) <= h + 1e-15  # vertices are samples too
        if len(set(I)) == 2:
            seen_case1 = True
    if seed % 2 == 1:
        assert seen_case1


@pytest.mark.parametrize("seed", range(4))
def test_bounds_hold_for_any_points_of_B(orc, seed):
    """The proofs of Section 3.2 (exact case, u1..u4) use each vertex's footpoint q_i only as a
    point of B, so every bound stays an upper bound of h(T, B) when q_i is the closest point of
    any triangle S_i of B instead of the nearest one.  That reading is what lets a vertex
    query stop at a triangle that is merely close enough (cut queries).  Sampled h against
    each bound, with S_i drawn at random (one S for all three vertices in a third of the cases,
    so that the exact case applies), on a soup and on a closed mesh; and u1 at most the
    longest edge at any vertex plus that vertex's distance, the inequality the cut relies on."""
    rng = np.random.default_rng(300 + seed)
    if seed % 2 == 0:
        VB, FB = _random_small_mesh(rng, 12)
    else:
        VB, FB = mg.icosphere(1)
        VB = VB * 0.8
    W = bary_grid(24)
    exact_seen = 0
    for t in range(60):
        kind = ["generic", "sliver", "tiny"][t % 3]
        T = random_triangle(rng, kind) * (0.5 if kind == "generic" else 1.0)
        if seed % 2 == 1:
            T = T * 0.3 + rng.normal(size=3) * 0.6
        I = np.full(3, rng.integers(len(FB))) if t % 3 == 0 else rng.integers(len(FB), size=3)
        I = I.astype(np.int32)
        d, q = np.zeros(3), np.zeros((3, 3))
        for i in range(3):
            a, b, c = (np.asarray(VB, float)[j] for j in FB[I[i]])
            d[i], q[i] = orc.point_triangle(T[i], a, b, c)
        bnd = orc.bounds_all(T, d, I, q, VB, FB)
        ds, _, _ = orc.nearest(W @ T, VB, FB)
        h = ds.max()
        for k, name in enumerate(["exact", "u1", "u2", "u3", "u4"]):
            if not np.isnan(bnd[k]):
                assert h <= bnd[k] * (1 + 1e-12) + 1e-12, (name, t, h, bnd[k])
        exact_seen += not np.isnan(bnd[0])
        e = [np.linalg.norm(T[(i + 1) % 3] - T[i]) for i in range(3)]  # e[i]: edge from vertex i to i + 1
        for i in range(3):
            assert bnd[1] <= (max(e[i], e[(i + 2) % 3]) + d[i]) * (1 + 1e-12) + 1e-15
    assert exact_seen >= 10


# ----------------------------------------------------------------------------- full loop pins


def _load_golden():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _load_golden(), ids=lambda c: c["name"])
def test_closed_form_pairs(orc, case):
    """Hand-derived h of tiny pairs: the bracket must contain it and be within tol."""
    VA, FA = np.array(case["VA"], float), np.array(case["FA"], np.int32)
    VB, FB = np.array(case["VB"], float), np.array(case["FB"], np.int32)
    r = orc.hausdorff(VA, FA, VB, FB, case["tol"], 0)
    assert r["status"] == orc.OK
    assert r["lower"] <= case["h"] + 1e-12 and case["h"] <= r["upper"] + 1e-12
    assert r["upper"] - r["lower"] <= case["tol"]


def test_single_triangle_B_maximiser_at_a_vertex(orc):
    """P3: with B one triangle, d(., B) is convex, so h = max over A's vertices of d(v, B)
    (computed with the independent region method)."""
    VA, FA = mg.icosphere(1)
    VA = VA * 0.7 + np.array([0.3, -0.2, 0.9])
    VB = np.array([[-0.5, -0.4, 0.1], [0.8, -0.3, -0.2], [0.1, 0.9, 0.3]])
    FB = np.array([[0, 1, 2]], np.int32)
    h = max(dist_regions(v, *VB) for v in VA)
    r = orc.hausdorff(VA, FA, VB, FB, 1e-7, 0)
    assert r["status"] == orc.OK
    assert r["lower"] <= h + 1e-12 <= r["upper"] + 2e-12 and r["upper"] - r["lower"] <= 1e-7


def test_outside_convex_polyhedron(orc):
    """P4: A outside a closed convex B: h = max over A's vertices of the distance to the solid,
    which for outside points is the distance to the surface (region method, brute force)."""
    VB, FB = mg.icosphere(0)  # icosahedron, circumradius 1
    VA, FA = mg.icosphere(1)
    VA = VA * 1.6 + np.array([0.4, 0.1, -0.2])
    assert np.min(np.linalg.norm(VA, axis=1)) > 1.05
    h = max(dist_mesh_regions(v, VB, FB) for v in VA)
    r = orc.hausdorff(VA, FA, VB, FB, 1e-7, 0)
    assert r["status"] == orc.OK
    assert r["lower"] <= h + 1e-12 <= r["upper"] + 2e-12 and r["upper"] - r["lower"] <= 1e-7


@pytest.mark.parametrize("k", [1, 2])
def test_identical_meshes(orc, k):
    """P1: h(A, A) = 0."""
    if k == 1:
        V, F = mg.icosphere(2)
    else:
        p = mg.workload(2, 0.002)
        V, F = p.VA.astype(float), p.FA
    # h(A, A) is the paper's hardest (near-zero) case, Section 5.3; a loose tol keeps it fast
    r = orc.hausdorff(V, F, V, F, 1e-3, 0)
    assert r["status"] == orc.OK
    assert 0 <= r["lower"] <= 1e-12 and r["upper"] <= 1e-3


def test_sampling_bracket_agrees_workload1(orc):
    """P5: the Lipschitz sampling bracket and the branch-and-bound bracket both contain h."""
    p = mg.workload(1)
    lo, hi = orc.sampling_bracket(p.VA, p.FA, p.VB, p.FB, 12)
    r = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, p.tol_mode)
    assert max(lo, r["lower"]) <= min(hi, r["upper"]) + 1e-15
    assert r["upper"] - r["lower"] <= p.tol


@pytest.mark.parametrize("k", [4, 5, 10, 11, 40, 41])
def test_sampling_bracket_thin_bridge_closed_form(orc, k):
    """P5 pinned to a closed form: on the thin bridge (tests/golden/closed_forms.json, h = sqrt(2)
    at x = 1, interior to A) the sampling bracket holds h for every k.  With one face its width
    is the covering radius emax / k (emax = A's longest edge), so it shrinks like 1/k.  An even
    k puts a sample on x = 1, so lo = h; an odd k's nearest samples are 1/k away in x, so
    h - lo ~ 0.71 / k: a covering radius below that (a quarter of the true one, say) would
    leave hi < h there."""
    c = [c for c in _load_golden() if c["name"] == "thin_bridge_interior_maximiser"][0]
    VA, FA = np.array(c["VA"], float), np.array(c["FA"], np.int32)
    VB, FB = np.array(c["VB"], float), np.array(c["FB"], np.int32)
    h = math.sqrt(2.0)
    lo, hi = orc.sampling_bracket(VA, FA, VB, FB, k)
    emax = max(np.linalg.norm(VA[1] - VA[0]), np.linalg.norm(VA[2] - VA[1]), np.linalg.norm(VA[0] - VA[2]))
    assert lo <= h + 1e-12 and h <= hi + 1e-12, (k, lo, hi)
    assert abs((hi - lo) - emax / k) <= 1e-12
    if k % 2 == 0:
        assert abs(lo - h) <= 1e-12
    else:
        assert 0.5 / k <= h - lo <= 1.0 / k, (k, h - lo)


@pytest.mark.parametrize("seed", range(4))
def test_sampling_bracket_random_soups(orc, seed):
    """P5 on random soups where the maximiser is usually interior."""
    rng = np.random.default_rng(900 + seed)
    VA, FA = _random_small_mesh(rng, 3)
    VB, FB = _random_small_mesh(rng, 6)
    lo, hi = orc.sampling_bracket(VA, FA, VB, FB, 400)
    r = orc.hausdorff(VA, FA, VB, FB, 1e-6, 0)
    assert r["status"] == orc.OK
    assert max(lo, r["lower"]) <= min(hi, r["upper"]) + 1e-15
    assert r["lower"] >= lo - 1e-12  # l is a max over vertices and midpoints, at least the vertex samples


def test_invariants_trace(orc):
    """P9: l non-decreasing, running u non-increasing, l <= u, final gap <= eps."""
    p = mg.workload(2, 0.01)
    r = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, p.tol_mode, trace=True)
    tr = r["trace"]
    assert r["status"] == orc.OK and len(tr) > 10
    assert np.all(np.diff(tr[:, 0]) >= 0)
    assert np.all(np.diff(tr[:, 1]) <= 0)
    assert np.all(tr[:, 0] <= tr[:, 1])
    VA = p.VA.astype(float)
    dA = np.linalg.norm(VA.max(0) - VA.min(0))
    assert r["upper"] - r["lower"] <= p.tol * dA


def test_tight_run_nests(orc):
    """A run at eps/100 brackets h too, so the two brackets intersect and the tight one is narrower."""
    p = mg.workload(1)
    r1 = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, 0)
    r2 = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol / 100, 0)
    assert max(r1["lower"], r2["lower"]) <= min(r1["upper"], r2["upper"])
    assert r2["upper"] - r2["lower"] <= p.tol / 100


def test_all_64_bound_orders_bracket_h(orc):
    """Section 5 tests all 64 ordered subsets of {u1..u4}; each must still bracket h."""
    p = mg.workload(1)
    ref = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, 1e-6, 0)
    orders = [o for k in range(1, 5) for o in itertools.permutations((1, 2, 3, 4), k)]
    assert len(orders) == 64
    for o in orders:
        r = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, 1e-4, 0, order=o, max_face_factor=2000)
        assert r["status"] in (orc.OK, orc.CAPACITY)
        assert max(r["lower"], ref["lower"]) <= min(r["upper"], ref["upper"]) + 1e-15, o


def test_capacity_keeps_a_valid_bracket(orc):
    p = mg.workload(1)
    ref = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, 1e-6, 0)
    r = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, 1e-6, 0, max_face_factor=1.5)
    assert r["status"] == orc.CAPACITY
    assert r["lower"] <= ref["upper"] and ref["lower"] <= r["upper"]


def test_invalid_inputs(orc):
    V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]])
    F = np.array([[0, 1, 2]], np.int32)
    assert orc.hausdorff(V, F, V, F, 0.0, 0)["status"] == orc.INVALID
    assert orc.hausdorff(V, np.array([[0, 1, 3]], np.int32), V, F, 1e-3, 0)["status"] == orc.INVALID
    Vn = V.copy()
    Vn[1, 1] = np.nan
    assert orc.hausdorff(V, F, Vn, F, 1e-3, 0)["status"] == orc.INVALID


def test_unreferenced_vertices_are_ignored(orc):
    """Section 5.3: an unreferenced vertex must not raise l (reading: l and dA use referenced ones)."""
    V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [50, 50, 50]])
    F = np.array([[0, 1, 2]], np.int32)
    VB = np.array([[0.0, 0, 0.5], [1, 0, 0.5], [0, 1, 0.5]])
    r = orc.hausdorff(V, F, VB, F, 1e-6, 0)
    assert r["status"] == orc.OK and r["lower"] == pytest.approx(0.5) and r["upper"] <= 0.5 + 1e-6
    # relative tolerance: dA is the diagonal of the referenced vertices only (sqrt(2) here)
    r = orc.hausdorff(V, F, VB, F, 1e-6, 1)
    assert r["status"] == orc.OK and r["upper"] - r["lower"] <= 1e-6 * math.sqrt(2)
    # workload 1 plus one far unreferenced vertex: the relative gap must use A's referenced
    # diagonal (2 sqrt(3)), not the far vertex's
    p = mg.workload(1)
    VA = np.concatenate([p.VA, [[50.0, 50.0, 50.0]]])
    r = orc.hausdorff(VA, p.FA, p.VB, p.FB, 1e-4, 1)
    assert r["status"] == orc.OK and r["upper"] - r["lower"] <= 1e-4 * 2 * math.sqrt(3)
