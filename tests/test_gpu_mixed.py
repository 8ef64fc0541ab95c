"""The certified FP32 path (HD_MIXED) against the FP64 oracle, through the C ABI.

Certification: for every query the returned interval [dist_lo, dist] must contain the
oracle's distance (which is exact to ~1e-16 relative; 1e-12 relative is allowed for it),
and every MIXED bracket [l, u] must contain h (closed forms) or intersect the oracle's.
Tightness: the intervals must be narrow (the bound is a few float roundings of the local
magnitude, far below the workloads' tolerances).
"""
import json
import os

import numpy as np
import pytest

import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")
ORACLE_REL = 1e-12


@pytest.fixture(scope="module")
def hd():
    from paper_2406_10357_gb300 import build

    build.build()
    import paper_2406_10357_gb300 as hd

    return hd


def _dA(V, F):
    R = np.asarray(V, float)[np.unique(np.asarray(F).ravel())]
    return float(np.linalg.norm(R.max(0) - R.min(0)))


def _check_certified(hd, orc, VB, FB, P, tight_rel=None, floor=None):
    """Certification is exact (the oracle's distance lies in every interval).  Tightness: the
    width may be a few hundred float roundings of the local magnitude M <= d + the diameter of
    B's largest triangle (the FP64 redo takes over above 256 roundings)."""
    bvh = hd.hd_build_B(VB, FB)
    Pt = torch.from_numpy(np.ascontiguousarray(P)).cuda()
    hi, idx, foot, lo = (x.cpu().numpy() for x in hd.hd_nearest(bvh, Pt, hd.HD_MIXED))
    do, _, _ = orc.nearest(np.asarray(P, float), np.asarray(VB, float), FB)
    slack = ORACLE_REL * np.maximum(1.0, do)
    assert np.all(lo <= do + slack), np.max(lo - do)
    assert np.all(hi >= do - slack), np.max(do - hi)
    assert np.all(idx >= 0)
    gap = hi - lo
    T = np.asarray(VB, float)[FB]
    diam = max(np.max(np.linalg.norm(T[:, 0] - T[:, 1], axis=1)), np.max(np.linalg.norm(T[:, 1] - T[:, 2], axis=1)),
               np.max(np.linalg.norm(T[:, 2] - T[:, 0], axis=1)))
    lim = 400 * 2.0**-24 * (do + diam) + 1e-12
    assert np.all(gap <= lim), (np.max(gap / lim), np.argmax(gap / lim), gap[np.argmax(gap / lim)])
    # the returned triangle realises the upper bound
    VBd = np.asarray(VB, float)
    for i in np.random.default_rng(1).choice(len(P), size=min(40, len(P)), replace=False):
        d_idx, _ = orc.point_triangle(np.asarray(P[i], float), *VBd[FB[idx[i]]])
        assert d_idx <= hi[i] + slack[i]
    return gap


@pytest.mark.parametrize("k,scale", [(1, 1.0), (2, 0.05), (3, 0.02), (5, 0.01)])
def test_nearest_mixed_is_certified(hd, orc, k, scale):
    p = mg.workload(k, scale)
    rng = np.random.default_rng(10 + k)
    V = np.asarray(p.VA, float)
    P = np.concatenate([V[rng.choice(len(V), size=min(3000, len(V)), replace=False)],
                        V.mean(0) + rng.normal(size=(500, 3)) * V.std(0) * 1.5]).astype(np.float32)
    _check_certified(hd, orc, p.VB, p.FB, P, tight_rel=2e-5)


@pytest.mark.parametrize("scale", [0.02, 0.2])
def test_nearest_mixed_deep_interior_points(hd, orc, scale):
    """Points deep inside workload 3's superquadric have much of B within their distance:
    their lane traversals pass the budget and whole warps finish them (k_query_long).  The
    intervals stay certified and tight."""
    p = mg.workload(3, scale)
    rng = np.random.default_rng(31)
    u = rng.normal(size=(1500, 3))
    P = (u / np.linalg.norm(u, axis=1, keepdims=True) * rng.uniform(0, 0.7, size=(1500, 1))).astype(np.float32)
    _check_certified(hd, orc, p.VB, p.FB, P)


def test_nearest_mixed_full_size_workload2_sampled(hd, orc):
    p = mg.workload(2)
    rng = np.random.default_rng(21)
    P = p.VA[rng.choice(len(p.VA), size=3000, replace=False)]
    gap = _check_certified(hd, orc, p.VB, p.FB, P, tight_rel=1e-5, floor=0.01)
    assert np.median(gap) < 1e-7


@pytest.mark.parametrize("aspect", [1e2, 1e4, 1e6])
def test_nearest_mixed_slivers_and_degenerate(hd, orc, aspect):
    """Slivers, zero-area and repeated-vertex triangles in B; points near their edges."""
    rng = np.random.default_rng(int(aspect))
    n = 400
    a = rng.normal(size=(n, 3))
    d = rng.normal(size=(n, 3))
    side = np.cross(d, rng.normal(size=(n, 3)))
    side /= np.linalg.norm(side, axis=1, keepdims=True)
    L = np.linalg.norm(d, axis=1, keepdims=True)
    c = a + 0.37 * d + side * L / aspect
    T = np.stack([a, a + d, c], 1)
    T[::17, 2] = T[::17, 0]          # repeated vertex
    T[::23, 2] = 0.5 * (T[::23, 0] + T[::23, 1])  # collinear
    VB = T.reshape(-1, 3).astype(np.float32)
    FB = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    P = np.concatenate([
        (VB[0::3] + 0.5 * (VB[1::3] - VB[0::3]) + rng.normal(size=(n, 3)) * 1e-3),
        (VB[2::3] + rng.normal(size=(n, 3)) * 1e-4),
        rng.normal(size=(n, 3)) * 2,
    ]).astype(np.float32)
    gap = _check_certified(hd, orc, VB, FB, P, tight_rel=2e-5)
    assert np.median(gap) < 1e-5


def test_nearest_mixed_double_input_B(hd, orc):
    """B given in float64 (not representable in float): the float copy's error is covered."""
    p = mg.workload(1)
    VB = np.asarray(p.VB, float) * (1 + 1e-9) + 1e-9
    rng = np.random.default_rng(3)
    P = rng.normal(size=(2000, 3)) * 1.1
    _check_certified(hd, orc, VB, p.FB, P, tight_rel=2e-5)


def _load_golden():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _load_golden(), ids=lambda c: c["name"])
def test_closed_form_pairs_mixed(hd, case):
    VA, FA = np.array(case["VA"], float), np.array(case["FA"], np.int32)
    VB, FB = np.array(case["VB"], float), np.array(case["FB"], np.int32)
    bvh = hd.hd_build_B(VB, FB)
    r = hd.hd_hausdorff(bvh, VA, FA, case["tol"], hd.hd_options_default(precision=hd.HD_MIXED))
    assert r["status"] == hd.HD_OK, r
    assert r["lower"] <= case["h"] and case["h"] <= r["upper"]
    assert r["upper"] - r["lower"] <= case["tol"]


@pytest.mark.parametrize("k,scale", [(1, 1.0), (2, 0.02), (2, 0.1), (3, 0.01), (5, 0.005)])
def test_bracket_mixed_vs_oracle(hd, orc, k, scale):
    p = mg.workload(k, scale)
    bvh = hd.hd_build_B(p.VB, p.FB)
    r = hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol, hd.hd_options_default(tol_mode=p.tol_mode, precision=hd.HD_MIXED))
    ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, p.tol_mode)
    eps = p.tol * (_dA(p.VA, p.FA) if p.tol_mode else 1.0)
    assert r["status"] == hd.HD_OK, r
    assert r["upper"] - r["lower"] <= eps
    assert max(r["lower"], ro["lower"]) <= min(r["upper"], ro["upper"]) + ORACLE_REL * ro["upper"]
    if k != 3:
        # the oracle at eps / 100 brackets h within a hundredth of eps: a MIXED bracket that
        # missed h would miss this narrow one, even where it meets the wide one above
        rt = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol / 100, p.tol_mode)
        assert rt["status"] == orc.OK
        assert r["lower"] <= rt["upper"] + ORACLE_REL * rt["upper"] and rt["lower"] <= r["upper"] + ORACLE_REL * rt["upper"]
    # MIXED and FP64 GPU brackets intersect too
    r64 = hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol, hd.hd_options_default(tol_mode=p.tol_mode))
    assert max(r["lower"], r64["lower"]) <= min(r["upper"], r64["upper"]) + ORACLE_REL * r64["upper"]


@pytest.mark.parametrize("order", [(4,), (1, 4), (4, 3), (1, 2, 3, 4)])
@pytest.mark.parametrize("k,scale", [(1, 1.0), (2, 0.02)])
def test_bracket_mixed_bound_orders(hd, orc, order, k, scale):
    """MIXED runs whose cascades lean on u4 (alone, first, or last as in the paper): the
    bracket intersects the oracle's, so every discard u4 made was valid."""
    p = mg.workload(k, scale)
    bvh = hd.hd_build_B(p.VB, p.FB)
    o = hd.hd_options_default(tol_mode=p.tol_mode, precision=hd.HD_MIXED, bound_order=order, max_face_factor=2000)
    r = hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol, o)
    ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, p.tol_mode)
    assert r["status"] in (hd.HD_OK, hd.HD_ERR_CAPACITY), (order, r)
    assert max(r["lower"], ro["lower"]) <= min(r["upper"], ro["upper"]) + ORACLE_REL * ro["upper"], order
    if r["status"] == hd.HD_OK:
        eps = p.tol * (_dA(p.VA, p.FA) if p.tol_mode else 1.0)
        assert r["upper"] - r["lower"] <= eps


def test_full_size_workload2_mixed_properties(hd, orc):
    p = mg.workload(2)
    bvh = hd.hd_build_B(p.VB, p.FB)
    r = hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol, hd.hd_options_default(tol_mode=p.tol_mode, precision=hd.HD_MIXED))
    eps = p.tol * _dA(p.VA, p.FA)
    assert r["status"] == hd.HD_OK and r["upper"] - r["lower"] <= eps
    rng = np.random.default_rng(19)
    P = np.asarray(p.VA, float)[rng.choice(len(p.VA), size=3000, replace=False)]
    do, _, _ = orc.nearest(P, p.VB, p.FB)
    assert do.max() <= r["upper"]
    r64 = hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol, hd.hd_options_default(tol_mode=p.tol_mode))
    assert max(r["lower"], r64["lower"]) <= min(r["upper"], r64["upper"])


def test_identical_meshes_mixed(hd):
    V, F = mg.icosphere(2)
    bvh = hd.hd_build_B(V, F)
    r = hd.hd_hausdorff(bvh, V, F, 1e-3, hd.hd_options_default(precision=hd.HD_MIXED))
    assert r["status"] == hd.HD_OK and 0 <= r["lower"] <= 1e-6 and r["upper"] <= 1e-3 + 1e-6


def _bary_grid(k):
    """Barycentric weights of a regular grid with k steps per edge (vertices included)."""
    return np.array([(i / k, j / k, (k - i - j) / k) for i in range(k + 1) for j in range(k + 1 - i)])


@pytest.mark.parametrize("order", [(1, 2, 3, 4), (1,), (2,), (3,), (4,)])
def test_upper_bounds_mixed_certified(hd, orc, order):
    """UpperBound(T, l) in the certified FP32 arithmetic (hd_upper_bounds with HD_MIXED), each
    bound alone and the paper's cascade, for random sub-triangles of A's faces with the
    oracle's nearest data.  Validity: every value is at least max d(p, B) over a dense sample of
    T, since d(p, B) <= h(T, B) <= any of the paper's bounds.  Tightness: for a single bound the
    value is within a few float roundings of the local magnitude of the oracle's FP64 value of
    the same bound (u3's split points are computed in plain FP32 and may differ slightly, which
    moves it either way)."""
    # the re-triangulated torus pair (reduced): B's triangles do not follow A's, so the three
    # vertices of a sub-triangle usually have different nearest triangles (not the exact case)
    p = mg.workload(2, 0.02)
    bvh = hd.hd_build_B(p.VB, p.FB)
    rng = np.random.default_rng(11)
    V = np.asarray(p.VA, float)
    n = 400
    f = rng.integers(0, len(p.FA), n)
    W = rng.dirichlet([1, 1, 1], size=(n, 3))
    s = rng.choice([3.0, 2.0, 1.0, 0.3], size=n)[:, None, None]  # above 1: past the face (any T is valid)
    c = rng.dirichlet([1, 1, 1], size=n)[:, None, :]
    T = np.einsum("nkj,njd->nkd", c + s * (W - c), V[p.FA[f]])
    d, I, q = orc.nearest(T.reshape(-1, 3), p.VB, p.FB)
    d, I, q = d.reshape(n, 3), I.reshape(n, 3), q.reshape(n, 3, 3)
    assert np.sum((I[:, 0] != I[:, 1]) | (I[:, 1] != I[:, 2])) >= n // 4
    l0 = float(np.quantile(d, 0.8))
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    opt = hd.hd_options_default(precision=hd.HD_MIXED, bound_order=order)
    U, code = hd.hd_upper_bounds(bvh, t(T.reshape(n, 9)), t(d), t(I.astype(np.int32)), t(q.reshape(n, 9)), l0, opt)
    U, code = U.cpu().numpy(), code.cpu().numpy()
    assert np.all(np.isfinite(U)) and np.all((code >= 0) & (code <= 5))
    G = _bary_grid(12)
    S = np.einsum("gk,nkd->ngd", G, T)
    ds, _, _ = orc.nearest(S.reshape(-1, 3), p.VB, p.FB)
    smax = ds.reshape(n, len(G)).max(1)
    assert np.all(U >= smax - 1e-12 * np.maximum(1.0, smax)), np.min(U - smax)
    if len(order) == 1:
        k = order[0]
        M = np.abs(T - T[:, :1]).max((1, 2)) + np.abs(q - T).max((1, 2)) + d.max(1)
        sel = np.nonzero(code != 0)[0]
        assert len(sel) >= n // 4
        ref = np.array([orc.bounds_all(T[i], d[i], I[i], q[i], p.VB, p.FB)[k] for i in sel])
        rel = (U[sel] - ref) / M[sel]
        if k != 3:
            # certified: never below the exact value of the same bound
            assert np.all(U[sel] >= ref - 1e-12 * np.maximum(1.0, ref)), (k, np.min(U[sel] - ref))
            # tight: almost always within a few hundred float roundings (an edge nearly parallel
            # to u4's bisector plane may fall back to the edge's farther endpoint)
            assert np.quantile(rel, 0.99) <= 2000 * 2.0**-24, (k, np.quantile(rel, 0.99))
        else:
            # u3 of kept items (a discarded item stops at min_i h(T, S_i) once that is below l,
            # where the oracle goes on to min(u3~, ...)); its case-1 split points are computed in
            # plain FP32, so near the fallback to midpoints the two may take different points
            kept = code[sel] == 5
            assert kept.sum() >= 20
            assert np.quantile(np.abs(rel[kept]), 0.95) <= 1e-3, np.quantile(np.abs(rel[kept]), 0.95)


# ---------------------------------------------------------------- the FP64 certification phase


def _tight_parity(orc, p, r, tol, mode, eps):
    """r is within eps, meets the oracle's bracket at the same tolerance and at 1/100 of it."""
    assert r["status"] == 0, r
    assert r["upper"] - r["lower"] <= eps * (1 + 1e-12), (r["upper"] - r["lower"], eps)
    for t in (tol, tol / 100):
        ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, t, mode)
        assert ro["status"] == orc.OK
        assert max(r["lower"], ro["lower"]) <= min(r["upper"], ro["upper"]) + ORACLE_REL * ro["upper"], (t, r, ro)


def test_closed_forms_promote_to_fp64_at_tight_tolerance(hd):
    """At tol 1e-6 the closed-form pairs end with gaps U - l below the FP32 error width of
    their vertex distances (about 2^-18 of U), which FP32 refinement cannot resolve: those
    sub-triangles are finished in the FP64 phase (Section 5.3's rounding limit), and every
    bracket still holds the hand-derived h."""
    total = 0
    for case in _load_golden():
        VA, FA = np.array(case["VA"], float), np.array(case["FA"], np.int32)
        VB, FB = np.array(case["VB"], float), np.array(case["FB"], np.int32)
        r = hd.hd_hausdorff(hd.hd_build_B(VB, FB), VA, FA, case["tol"], hd.hd_options_default(precision=hd.HD_MIXED))
        assert r["status"] == hd.HD_OK, (case["name"], r)
        assert r["lower"] <= case["h"] <= r["upper"] and r["upper"] - r["lower"] <= case["tol"], case["name"]
        total += r["stats"]["promoted"]
        print(case["name"], "promoted", r["stats"]["promoted"])
    assert total > 0


@pytest.mark.parametrize("k,scale,tol", [(2, 0.02, 1e-8), (5, 0.005, 1e-8)])
def test_promotion_on_reduced_workloads(hd, orc, k, scale, tol):
    """Reduced workloads at tol 1e-8 dA: the last items' gaps are below FP32 resolution, so
    the run promotes them and finishes them in FP64; the bracket meets the oracle's at the
    same tolerance and at 1/100 of it."""
    p = mg.workload(k, scale)
    bvh = hd.hd_build_B(p.VB, p.FB)
    r = hd.hd_hausdorff(bvh, p.VA, p.FA, tol, hd.hd_options_default(tol_mode=p.tol_mode, precision=hd.HD_MIXED))
    print(p.name, "promoted", r["stats"]["promoted"], "splits", r["stats"]["splits"])
    assert r["stats"]["promoted"] > 0
    _tight_parity(orc, p, r, tol, p.tol_mode, tol * _dA(p.VA, p.FA))


@pytest.mark.parametrize("tol", [1e-4, 1e-5, 1e-6, 1e-7, 1e-8])
@pytest.mark.parametrize("k,scale", [(2, 0.02), (5, 0.005)])
def test_tolerance_ladder_mixed(hd, orc, k, scale, tol):
    """Runtime-versus-eps ladder (Section 5) in MIXED: at every tolerance from 1e-4 to 1e-8
    of dA the bracket is within eps and meets the oracle's at that tolerance and at 1/100 of
    it (the tight end is where the FP64 phase takes over)."""
    p = mg.workload(k, scale)
    bvh = hd.hd_build_B(p.VB, p.FB)
    r = hd.hd_hausdorff(bvh, p.VA, p.FA, tol, hd.hd_options_default(tol_mode=p.tol_mode, precision=hd.HD_MIXED))
    _tight_parity(orc, p, r, tol, p.tol_mode, tol * _dA(p.VA, p.FA))


def test_sliver_B_escalates_to_fp64(hd, orc):
    """B made of slivers up to aspect 1e6 (plus zero-area and repeated-vertex triangles), A a
    mesh of small triangles hugging their long edges: the FP32 point-triangle certificate is
    loose there, so tests are redone in FP64 (fp64_escalations > 0), and the bracket still
    meets the oracle's."""
    rng = np.random.default_rng(606)
    n = 300
    a = rng.normal(size=(n, 3))
    d = rng.normal(size=(n, 3))
    side = np.cross(d, rng.normal(size=(n, 3)))
    side /= np.linalg.norm(side, axis=1, keepdims=True)
    L = np.linalg.norm(d, axis=1, keepdims=True)
    aspect = 10.0 ** rng.uniform(3, 6, size=(n, 1))
    T = np.stack([a, a + d, a + 0.37 * d + side * L / aspect], 1)
    T[::17, 2] = T[::17, 0]
    T[::23, 2] = 0.5 * (T[::23, 0] + T[::23, 1])
    VB = T.reshape(-1, 3)
    FB = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    # A: one small triangle near the middle of each sliver's long edge, slightly off it
    c = a + 0.5 * d + rng.normal(size=(n, 3)) * 1e-3
    u = rng.normal(size=(n, 3)) * 1e-3
    w = rng.normal(size=(n, 3)) * 1e-3
    VA = np.stack([c, c + u, c + w], 1).reshape(-1, 3)
    FA = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    tol = 1e-6
    r = hd.hd_hausdorff(hd.hd_build_B(VB, FB), VA, FA, tol, hd.hd_options_default(precision=hd.HD_MIXED))
    print("sliver B: escalations", r["stats"]["fp64_escalations"], "promoted", r["stats"]["promoted"])
    assert r["stats"]["fp64_escalations"] > 0
    ro = orc.hausdorff(VA, FA, VB, FB, tol, 0)
    assert r["status"] == hd.HD_OK and r["upper"] - r["lower"] <= tol * (1 + 1e-12)
    assert max(r["lower"], ro["lower"]) <= min(r["upper"], ro["upper"]) + ORACLE_REL * ro["upper"]


@pytest.mark.parametrize("clamp", [True, False])
def test_bracket_all_bound_orders_mixed(hd, orc, clamp):
    """Every one of the 64 cascades (ordered subsets of u1..u4, Section 5's bound-order
    benchmark) in MIXED on workload 1: each bracket meets the oracle's at eps and, when the
    run finished, at eps / 100.  The paper's order runs the straight-line kernels, every
    other order the general ones; with the parent clamp on and off."""
    import itertools

    p = mg.workload(1)
    ref = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, 0)
    tight = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol / 100, 0)
    bvh = hd.hd_build_B(p.VB, p.FB)
    flags = 0 if clamp else hd.HD_FLAG_NO_PARENT_CLAMP
    n = 0
    for kk in range(1, 5):
        for order in itertools.permutations((1, 2, 3, 4), kk):
            o = hd.hd_options_default(precision=hd.HD_MIXED, bound_order=order, max_face_factor=2000, flags=flags)
            r = hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol, o)
            assert r["status"] in (hd.HD_OK, hd.HD_ERR_CAPACITY), (order, r)
            for ro in (ref, tight):
                assert max(r["lower"], ro["lower"]) <= min(r["upper"], ro["upper"]) + 1e-12, (order, r, ro)
            if r["status"] == hd.HD_OK:
                assert r["upper"] - r["lower"] <= p.tol * (1 + 1e-12), order
            n += 1
    assert n == 64
