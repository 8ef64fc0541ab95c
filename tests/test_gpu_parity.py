"""CUDA path against the FP64 oracle, through the C ABI.

Per-query parity (HD_FP64): the distance of each point to B matches the oracle's brute
force to 1e-6 relative (the tolerance the workloads are specified with); nearest indices
may differ only where two triangles tie, so the distance to the returned triangle is
checked instead of the index.  Bracket parity: the GPU bracket [l, u] and the oracle's
both contain h, so they must intersect, and both gaps are within eps.
"""
import json
import math
import os

import numpy as np
import pytest

import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")
REL = 1e-6
SHARED_MAX_PER_SPLIT = 2.6  # midpoints per split on workload 3 with shared midpoints (2.03 measured at full size)


@pytest.fixture(scope="module")
def hd():
    from paper_2406_10357_gb300 import build

    build.build()
    import paper_2406_10357_gb300 as hd

    return hd


def _dA(V, F):
    R = np.asarray(V, float)[np.unique(np.asarray(F).ravel())]
    return float(np.linalg.norm(R.max(0) - R.min(0)))


def _pts_parity(hd, orc, bvh, VB, FB, P, precision):
    Pt = torch.from_numpy(np.ascontiguousarray(P, dtype=np.float64)).cuda()
    d, idx, foot, dlo = hd.hd_nearest(bvh, Pt, precision)
    torch.cuda.synchronize()
    d, idx, foot, dlo = d.cpu().numpy(), idx.cpu().numpy(), foot.cpu().numpy(), dlo.cpu().numpy()
    do, io, qo = orc.nearest(P, VB, FB)
    scale = max(1e-12 * _dA(VB, FB), 1e-300)
    err = np.abs(d - do) / np.maximum(do, scale)
    assert np.all(idx >= 0) and np.all(idx < len(FB))
    # the returned foot lies on the returned triangle: its oracle distance to that triangle is ~0
    for i in np.random.default_rng(0).choice(len(P), size=min(50, len(P)), replace=False):
        f = FB[idx[i]]
        dd, _ = orc.point_triangle(foot[i], *np.asarray(VB, float)[f])
        assert dd <= 1e-9 * max(1.0, d[i])
        assert abs(np.linalg.norm(P[i] - foot[i]) - d[i]) <= 1e-9 * max(1.0, d[i])
    return err, d, dlo, do


@pytest.mark.parametrize("k,scale,npts", [(1, 1.0, 400), (2, 0.05, 2000), (3, 0.02, 2000), (5, 0.01, 2000)])
def test_nearest_fp64_matches_bruteforce(hd, orc, k, scale, npts):
    p = mg.workload(k, scale)
    bvh = hd.hd_build_B(p.VB, p.FB)
    rng = np.random.default_rng(k)
    V = np.asarray(p.VA, float)
    P = np.concatenate([V[rng.choice(len(V), size=min(npts, len(V)), replace=False)],
                        V.mean(0) + rng.normal(size=(200, 3)) * V.std(0) * 1.5])
    err, *_ = _pts_parity(hd, orc, bvh, p.VB, p.FB, P, hd.HD_FP64)
    assert err.max() <= REL, err.max()


@pytest.mark.parametrize("scale", [0.02, 0.2])
def test_nearest_fp64_deep_interior_points(hd, orc, scale):
    """Points deep inside workload 3's superquadric: their queries are finished by whole warps
    (k_query_long); distances match brute force to 1e-6 relative, like the lane traversal's."""
    p = mg.workload(3, scale)
    bvh = hd.hd_build_B(p.VB, p.FB)
    rng = np.random.default_rng(32)
    u = rng.normal(size=(1500, 3))
    P = u / np.linalg.norm(u, axis=1, keepdims=True) * rng.uniform(0, 0.7, size=(1500, 1))
    err, *_ = _pts_parity(hd, orc, bvh, p.VB, p.FB, P, hd.HD_FP64)
    assert err.max() <= REL, err.max()


@pytest.mark.parametrize("leaf", [1, 4, 16])
def test_nearest_every_leaf_size_and_tiny_B(hd, orc, leaf):
    rng = np.random.default_rng(leaf)
    for nB in (1, 2, 3, 5, 17, 100):
        VB = rng.normal(size=(3 * nB, 3))
        FB = np.arange(3 * nB, dtype=np.int32).reshape(nB, 3)
        bvh = hd.hd_build_B(VB, FB, hd.hd_options_default(leaf_size=leaf))
        P = rng.normal(size=(300, 3)) * 2
        err, *_ = _pts_parity(hd, orc, bvh, VB, FB, P, hd.HD_FP64)
        assert err.max() <= REL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nearest_large_B_multi_block_sort(hd, orc, precision):
    """A B of 400,000 triangles (the large soup's superquadric at 1/5): its Morton sort runs
    the multi-block path (per-digit totals and a scan per digit) instead of the fused one;
    nearest distances of 3,500 points, most of them off the surface (their queries are
    reordered along a Morton curve before the cooperative pass), match brute force."""
    p = mg.workload(5, 0.2)
    assert len(p.FB) > 64 * 4096
    bvh = hd.hd_build_B(p.VB, p.FB)
    rng = np.random.default_rng(55)
    V = np.asarray(p.VA, float)
    P = np.concatenate([V[rng.choice(len(V), size=1000, replace=False)],
                        V.mean(0) + rng.normal(size=(2500, 3)) * V.std(0)])
    if precision == "fp64":
        err, *_ = _pts_parity(hd, orc, bvh, p.VB, p.FB, P, hd.HD_FP64)
        assert err.max() <= REL, err.max()
    else:
        Pt = torch.from_numpy(np.ascontiguousarray(P)).cuda()
        hi, idx, foot, lo = (x.cpu().numpy() for x in hd.hd_nearest(bvh, Pt, hd.HD_MIXED))
        do, _, _ = orc.nearest(P, p.VB, p.FB)
        slack = 1e-12 * np.maximum(1.0, do)
        assert np.all(lo <= do + slack) and np.all(hi >= do - slack)
        assert np.max((hi - lo) / np.maximum(do, 1e-3)) < 1e-4


def test_nearest_full_size_workload2_sampled(hd, orc):
    """The benchmark's workload at full size: 2000 sampled vertices of A against brute force."""
    p = mg.workload(2)
    bvh = hd.hd_build_B(p.VB, p.FB)
    rng = np.random.default_rng(2)
    P = np.asarray(p.VA, float)[rng.choice(len(p.VA), size=2000, replace=False)]
    err, *_ = _pts_parity(hd, orc, bvh, p.VB, p.FB, P, hd.HD_FP64)
    assert err.max() <= REL


def test_upper_bounds_match_oracle(hd, orc):
    """UpperBound(T, l) on the GPU against the oracle for identical vertex data."""
    p = mg.workload(1)
    bvh = hd.hd_build_B(p.VB, p.FB)
    rng = np.random.default_rng(5)
    V = np.asarray(p.VA, float)
    n = 600
    # sub-triangles of A's faces at random barycentric positions and sizes
    f = rng.integers(0, len(p.FA), n)
    W = rng.dirichlet([1, 1, 1], size=(n, 3))
    s = rng.choice([1.0, 0.3, 0.05, 0.01], size=n)[:, None, None]
    c = rng.dirichlet([1, 1, 1], size=n)[:, None, :]
    W = c + s * (W - c)
    T = np.einsum("nkj,njd->nkd", W, V[p.FA[f]])
    d, I, q = orc.nearest(T.reshape(-1, 3), p.VB, p.FB)
    d, I, q = d.reshape(n, 3), I.reshape(n, 3), q.reshape(n, 3, 3)
    l0 = float(np.quantile(d, 0.8))
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    U, code = hd.hd_upper_bounds(bvh, t(T.reshape(n, 9)), t(d), t(I.astype(np.int32)), t(q.reshape(n, 9)), l0)
    U, code = U.cpu().numpy(), code.cpu().numpy()
    names = {"exact": 0, "u1": 1, "u2": 2, "u3": 3, "u4": 4, "kept": 5}
    for i in range(n):
        Uo, co = orc.upper_bound(T[i], d[i], I[i], q[i], p.VB, p.FB, l0)
        assert abs(U[i] - Uo) <= 1e-9 * max(1.0, Uo), (i, U[i], Uo)
        if abs(Uo - l0) > 1e-9:
            assert code[i] == names[co], (i, code[i], co)


def _soup(V, F):
    """Every triangle with its own three vertices (positions copied exactly)."""
    V = np.asarray(V)
    return np.ascontiguousarray(V[np.asarray(F)].reshape(-1, 3)), np.arange(3 * len(F), dtype=np.int32).reshape(-1, 3)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_weld_soup_bounds_equal_indexed_mesh(hd, orc, dtype):
    """HD_FLAG_WELD_B: a soup of B's triangles, welded, gives exactly the UpperBounds of the
    indexed mesh (u3's shared-edge case finds the same neighbours), which match the oracle's."""
    p = mg.workload(1)
    VB = np.asarray(p.VB, dtype)
    VS, FS = _soup(VB, p.FB)
    idx = hd.hd_build_B(VB, p.FB)
    welded = hd.hd_build_B(VS, FS, hd.hd_options_default(flags=hd.HD_FLAG_WELD_B))
    rng = np.random.default_rng(15)
    V = np.asarray(p.VA, float)
    n = 800
    f = rng.integers(0, len(p.FA), n)
    W = rng.dirichlet([1, 1, 1], size=(n, 3))
    c = rng.dirichlet([1, 1, 1], size=n)[:, None, :]
    W = c + rng.choice([1.0, 0.3, 0.05], size=n)[:, None, None] * (W - c)
    T = np.einsum("nkj,njd->nkd", W, V[p.FA[f]])
    VBd = np.asarray(VB, float)
    d, I, q = orc.nearest(T.reshape(-1, 3), VBd, p.FB)
    d, I, q = d.reshape(n, 3), I.reshape(n, 3), q.reshape(n, 3, 3)
    l0 = float(np.quantile(d, 0.8))
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    args = (t(T.reshape(n, 9)), t(d), t(I.astype(np.int32)), t(q.reshape(n, 9)), l0)
    o3 = hd.hd_options_default(bound_order=(3,))  # u3 alone, so that every item reaches it
    U1, c1 = (x.cpu().numpy() for x in hd.hd_upper_bounds(idx, *args, opt=o3))
    U2, c2 = (x.cpu().numpy() for x in hd.hd_upper_bounds(welded, *args, opt=o3))
    assert np.array_equal(U1, U2) and np.array_equal(c1, c2)
    # without the weld the soup has no shared edges: some u3 values change
    U3, _ = (x.cpu().numpy() for x in hd.hd_upper_bounds(hd.hd_build_B(VS, FS), *args, opt=o3))
    assert np.any(U3 != U1)
    for i in rng.choice(n, size=150, replace=False):
        Uo, _ = orc.upper_bound(T[i], d[i], I[i], q[i], VBd, p.FB, l0, order=(3,))
        assert abs(U2[i] - Uo) <= 1e-9 * max(1.0, Uo), (i, U2[i], Uo)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_weld_soup_run_equals_indexed_run(hd, orc, precision):
    """The whole run on a welded soup of B is the run on the indexed mesh: same BVH (same
    triangles, same Morton order), same neighbours for u3, so the same bracket and counts.
    Without the weld the soup's bracket is still valid."""
    p = mg.workload(1)
    prec = hd.HD_FP64 if precision == "fp64" else hd.HD_MIXED
    o = hd.hd_options_default(tol_mode=p.tol_mode, precision=prec)
    VS, FS = _soup(p.VB, p.FB)
    r1 = hd.hd_hausdorff(hd.hd_build_B(p.VB, p.FB), p.VA, p.FA, p.tol, o)
    r2 = hd.hd_hausdorff(hd.hd_build_B(VS, FS, hd.hd_options_default(flags=hd.HD_FLAG_WELD_B)), p.VA, p.FA, p.tol, o)
    assert (r1["lower"], r1["upper"], r1["status"]) == (r2["lower"], r2["upper"], r2["status"])
    for k in ("rounds", "splits", "queries", "pointtri_evals", "retired"):
        assert r1["stats"][k] == r2["stats"][k], k
    r3 = hd.hd_hausdorff(hd.hd_build_B(VS, FS), p.VA, p.FA, p.tol, o)
    ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, p.tol_mode)
    assert r3["status"] == hd.HD_OK and r3["upper"] - r3["lower"] <= p.tol * (1 + 1e-12)
    assert max(r3["lower"], ro["lower"]) <= min(r3["upper"], ro["upper"]) + 1e-12


def _load_golden():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _load_golden(), ids=lambda c: c["name"])
def test_closed_form_pairs_gpu(hd, case):
    VA, FA = np.array(case["VA"], float), np.array(case["FA"], np.int32)
    VB, FB = np.array(case["VB"], float), np.array(case["FB"], np.int32)
    bvh = hd.hd_build_B(VB, FB)
    r = hd.hd_hausdorff(bvh, VA, FA, case["tol"])
    assert r["status"] == hd.HD_OK, r
    assert r["lower"] <= case["h"] + 1e-12 and case["h"] <= r["upper"] + 1e-12
    assert r["upper"] - r["lower"] <= case["tol"]


def _bracket_parity(hd, orc, p, precision=None, tight=True, opt=None):
    bvh = hd.hd_build_B(p.VB, p.FB)
    o = opt or hd.hd_options_default(tol_mode=p.tol_mode)
    if precision is not None:
        o.precision = precision
    r = hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol, o)
    ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, p.tol_mode)
    eps = p.tol * (_dA(p.VA, p.FA) if p.tol_mode else 1.0)
    assert r["status"] == hd.HD_OK, r
    assert ro["status"] == orc.OK
    assert r["upper"] - r["lower"] <= eps * (1 + 1e-12)
    assert max(r["lower"], ro["lower"]) <= min(r["upper"], ro["upper"]) + 1e-12 * eps
    if tight:
        rt = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol / 100, p.tol_mode)
        assert r["lower"] <= rt["upper"] + 1e-12 and rt["lower"] <= r["upper"] + 1e-12
    return r, ro


def test_bracket_workload1_fp64(hd, orc):
    r, ro = _bracket_parity(hd, orc, mg.workload(1))
    assert r["stats"]["splits"] > 0


@pytest.mark.parametrize("k,scale", [(2, 0.02), (2, 0.1), (3, 0.01), (5, 0.005)])
def test_bracket_reduced_workloads_fp64(hd, orc, k, scale):
    _bracket_parity(hd, orc, mg.workload(k, scale), tight=(k != 3))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("k,scale", [(1, 1.0), (2, 0.02), (5, 0.005)])
def test_two_sided_matches_oracle(hd, orc, precision, k, scale):
    """H(A, B) = max(h(A, B), h(B, A)) with the second run's l warm-started from the first's
    lower bound: the bracket is within eps and meets the one the oracle gets from two
    independent one-sided runs."""
    p = mg.workload(k, scale)
    prec = hd.HD_FP64 if precision == "fp64" else hd.HD_MIXED
    bvhB, bvhA = hd.hd_build_B(p.VB, p.FB), hd.hd_build_B(p.VA, p.FA)
    H, ab, ba = hd.hd_hausdorff_sym(bvhB, p.VA, p.FA, bvhA, p.VB, p.FB, p.tol,
                                    hd.hd_options_default(tol_mode=p.tol_mode, precision=prec))
    eps = p.tol * (_dA(p.VA, p.FA) if p.tol_mode else 1.0)
    o_ab = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, eps, 0)
    o_ba = orc.hausdorff(p.VB, p.FB, p.VA, p.FA, eps, 0)
    Ho = (max(o_ab["lower"], o_ba["lower"]), max(o_ab["upper"], o_ba["upper"]))
    assert H["status"] == hd.HD_OK, H
    assert H["upper"] - H["lower"] <= eps * (1 + 1e-12)
    assert max(H["lower"], Ho[0]) <= min(H["upper"], Ho[1]) + 1e-12 * eps
    assert abs(ab["stats"]["eps_abs"] - eps) <= 1e-9 * eps and abs(ba["stats"]["eps_abs"] - eps) <= 1e-9 * eps
    assert ba["lower"] >= ab["lower"]  # warm start: l never starts below h(A, B)'s lower bound
    assert H["lower"] == max(ab["lower"], ba["lower"]) and H["upper"] == max(ab["upper"], ba["upper"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_pairs_match_oracle(hd, orc, precision):
    """Workload 4's generator at reduced sizes: every pair of the concurrent batched call is
    within eps and meets the oracle's bracket, and agrees with the same pair run alone."""
    pairs = mg.batch_workload(n_pairs=12, lo=300, hi=3000)
    prec = hd.HD_FP64 if precision == "fp64" else hd.HD_MIXED
    o = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=prec)
    bvhs = [hd.hd_build_B(p.VB, p.FB) for p in pairs]
    rs = hd.hd_hausdorff_batched(bvhs, [(p.VA, p.FA) for p in pairs], pairs[0].tol, o)
    assert len(rs) == len(pairs)
    for p, b, r in zip(pairs, bvhs, rs):
        assert p.tol == pairs[0].tol and p.tol_mode == hd.HD_TOL_REL
        eps = p.tol * _dA(p.VA, p.FA)
        ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, p.tol_mode)
        assert r["status"] == hd.HD_OK, (p.name, r)
        assert r["upper"] - r["lower"] <= eps * (1 + 1e-12), p.name
        # up to the rounding of FP64 distances (the oracle may round h's vertex distance
        # differently in the last bit)
        slack = 1e-12 * max(eps, ro["upper"])
        assert max(r["lower"], ro["lower"]) <= min(r["upper"], ro["upper"]) + slack, p.name
        r1 = hd.hd_hausdorff(b, p.VA, p.FA, p.tol, o)
        assert max(r["lower"], r1["lower"]) <= min(r["upper"], r1["upper"]) + slack, p.name


def test_batched_invalid_pair_is_reported(hd):
    p = mg.workload(1)
    bvh = hd.hd_build_B(p.VB, p.FB)
    bad = np.array(p.FA, copy=True)
    bad[0, 0] = len(p.VA) + 5
    with pytest.raises(hd.HdError):
        hd.hd_hausdorff_batched([bvh, bvh], [(p.VA, p.FA), (p.VA, bad)], 1e-4,
                                hd.hd_options_default(tol_mode=hd.HD_TOL_ABS))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_face_split_pair_gpu(hd, orc, precision):
    """One pair with A's faces split in three parts, as three ranks would run it (here one
    after another on one GPU): the shared seed, hd_hausdorff_from per part and the max of the
    brackets give a bracket within eps that meets the oracle's for the whole pair."""
    from paper_2406_10357_gb300 import multi

    p = mg.workload(2, 0.02)
    prec = hd.HD_FP64 if precision == "fp64" else hd.HD_MIXED
    bvh = hd.hd_build_B(p.VB, p.FB)
    engine, seed = multi.gpu_engine(bvh, hd.hd_options_default(precision=prec))
    eps = p.tol * multi.referenced_diagonal(p.VA, p.FA)
    FA = np.asarray(p.FA)
    parts = [FA[slice(*multi.shard_faces(len(FA), r, 3))] for r in range(3)]
    l0 = max(seed(p.VA, part) for part in parts)
    brs = [engine(p.VA, part, eps, l0) for part in parts]
    lo, up = max(b[0] for b in brs), max(b[1] for b in brs)
    assert all(b[2] == hd.HD_OK for b in brs) and all(b[0] >= l0 for b in brs)
    assert up - lo <= eps * (1 + 1e-12)
    ref = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, p.tol_mode)
    assert max(lo, ref["lower"]) <= min(up, ref["upper"]) + 1e-12 * eps


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_async_build_matches_sync(hd, orc, precision):
    """HD_FLAG_ASYNC_BUILD returns before the build ends; the run that follows on the stream
    gives a bracket within eps that meets the synchronous build's and the oracle's."""
    p = mg.workload(2, 0.02)
    prec = hd.HD_FP64 if precision == "fp64" else hd.HD_MIXED
    oa = hd.hd_options_default(tol_mode=p.tol_mode, precision=prec, flags=hd.HD_FLAG_ASYNC_BUILD)
    os_ = hd.hd_options_default(tol_mode=p.tol_mode, precision=prec)
    ra = hd.hd_hausdorff(hd.hd_build_B(p.VB, p.FB, oa), p.VA, p.FA, p.tol, oa)
    rs = hd.hd_hausdorff(hd.hd_build_B(p.VB, p.FB, os_), p.VA, p.FA, p.tol, os_)
    ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, p.tol_mode)
    eps = p.tol * _dA(p.VA, p.FA)
    for r in (ra, rs):
        assert r["status"] == hd.HD_OK and r["upper"] - r["lower"] <= eps * (1 + 1e-12)
        assert max(r["lower"], ro["lower"]) <= min(r["upper"], ro["upper"]) + 1e-12 * eps
    # float64 B: eta comes from the device in both modes
    V64 = np.asarray(p.VB, np.float64) + 1e-9
    for o in (oa, os_):
        r = hd.hd_hausdorff(hd.hd_build_B(V64, p.FB, o), p.VA, p.FA, p.tol, o)
        assert r["status"] == hd.HD_OK


@pytest.mark.parametrize("what", ["index", "nan"])
def test_async_build_invalid_B_reported_by_the_run(hd, what):
    """An invalid B built asynchronously is reported by the first bracket call that uses it
    (the synchronous build reports it itself)."""
    p = mg.workload(1)
    VB, FB = np.array(p.VB, dtype=np.float64), np.array(p.FB, copy=True)
    if what == "index":
        FB[3, 1] = len(VB) + 7
    else:
        VB[FB[5, 0], 2] = np.nan
    oa = hd.hd_options_default(tol_mode=hd.HD_TOL_ABS, flags=hd.HD_FLAG_ASYNC_BUILD)
    bvh = hd.hd_build_B(VB, FB, oa)  # queued, not checked yet
    with pytest.raises(hd.HdError):
        hd.hd_hausdorff(bvh, p.VA, p.FA, 1e-4, oa)
    with pytest.raises(hd.HdError):
        hd.hd_build_B(VB, FB)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parent_clamp_on_and_off(hd, orc, precision):
    """Clamping a child's U to its parent's is sound (the child lies inside the parent): with
    and without it the bracket is within eps and meets the oracle's."""
    p = mg.workload(1)
    prec = hd.HD_FP64 if precision == "fp64" else hd.HD_MIXED
    on = _bracket_parity(hd, orc, p, opt=hd.hd_options_default(tol_mode=p.tol_mode, precision=prec))[0]
    off = _bracket_parity(hd, orc, p, opt=hd.hd_options_default(tol_mode=p.tol_mode, precision=prec,
                                                                  flags=hd.HD_FLAG_NO_PARENT_CLAMP))[0]
    assert on["stats"]["splits"] > 0 and off["stats"]["splits"] > 0
    assert max(on["lower"], off["lower"]) <= min(on["upper"], off["upper"]) + 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("k,scale,chunk", [(1, 1.0, 0), (2, 0.02, 0), (3, 0.01, 0), (3, 0.01, 256)])
def test_shared_midpoints(hd, orc, precision, k, scale, chunk):
    """HD_FLAG_SHARE_MIDPOINTS: an edge split by two sub-triangles of one round gets one
    midpoint.  The bracket stays within eps and meets the oracle's; the run makes no more
    midpoints than 3 per split, and fewer where neighbours split together
    (workload 3 splits each face of A a few times); a small chunk (many rounds, the table
    cleared and reused between them) too."""
    p = mg.workload(k, scale)
    prec = hd.HD_FP64 if precision == "fp64" else hd.HD_MIXED
    mk = lambda f: hd.hd_options_default(tol_mode=p.tol_mode, precision=prec, frontier_chunk=chunk, flags=f)
    on = _bracket_parity(hd, orc, p, opt=mk(hd.HD_FLAG_SHARE_MIDPOINTS), tight=(k != 3))[0]
    off = _bracket_parity(hd, orc, p, opt=mk(0), tight=(k != 3))[0]
    assert max(on["lower"], off["lower"]) <= min(on["upper"], off["upper"]) + 1e-12
    s_on, s_off = on["stats"], off["stats"]
    assert s_off["pool_vertices"] - len(p.VA) == 3 * s_off["splits"]
    made = s_on["pool_vertices"] - len(p.VA)
    assert 0 < made <= 3 * s_on["splits"]
    if k == 3:
        print("shared midpoints: splits", s_on["splits"], "made", made, "queries", s_on["queries"], s_off["queries"])
        assert made < SHARED_MAX_PER_SPLIT * s_on["splits"], (made, s_on["splits"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scale", [0.01, 0.05])
def test_cooperative_queries(hd, orc, precision, scale):
    """Workload 3's sub-triangle vertices deep inside the sliver sphere have much of B within
    their distance: their lane traversals pass the node budget and a warp finishes each.  The
    bracket with those queries stays within eps and meets the oracle's."""
    p = mg.workload(3, scale)
    prec = hd.HD_FP64 if precision == "fp64" else hd.HD_MIXED
    r = _bracket_parity(hd, orc, p, opt=hd.hd_options_default(tol_mode=p.tol_mode, precision=prec), tight=False)[0]
    s = r["stats"]
    print("cooperative queries:", s["long_queries"], "of", s["queries"])
    assert 0 < s["long_queries"] < s["queries"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_block_size_limits(hd, orc, precision):
    """Block sizes the round kernels launch with give the oracle's bracket; one above what
    their register use allows is refused with HD_ERR_INVALID instead of a failed launch."""
    p = mg.workload(1)
    prec = hd.HD_FP64 if precision == "fp64" else hd.HD_MIXED
    bvh = hd.hd_build_B(p.VB, p.FB)
    for bs in (32, 96, 256):
        _bracket_parity(hd, orc, p, opt=hd.hd_options_default(tol_mode=p.tol_mode, precision=prec, block_size=bs))
    with pytest.raises(hd.HdError) as e:
        hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol, hd.hd_options_default(tol_mode=p.tol_mode, precision=prec,
                                                                     block_size=1024))
    assert e.value.status == hd.HD_ERR_INVALID


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("k,scale,chunk", [(1, 1.0, 0), (1, 1.0, 16), (2, 0.02, 0), (3, 0.01, 0), (4, None, 0)])
def test_small_round_kernel_same_result(hd, orc, precision, k, scale, chunk):
    """Rounds over small frontiers run in one single-block kernel (k_tail_rounds) unless
    HD_FLAG_NO_SMALL_ROUNDS: both paths give the same bracket and counts, and the bracket meets
    the oracle's.  A chunk of 16 splits per round makes the frontier cross the small-round
    limit back and forth."""
    p = mg.batch_workload(n_pairs=1)[0] if k == 4 else mg.workload(k, scale)
    prec = hd.HD_FP64 if precision == "fp64" else hd.HD_MIXED
    mk = lambda f: hd.hd_options_default(tol_mode=p.tol_mode, precision=prec, frontier_chunk=chunk, flags=f)
    bvh = hd.hd_build_B(p.VB, p.FB)
    a = hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol, mk(0))
    b = hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol, mk(hd.HD_FLAG_NO_SMALL_ROUNDS))
    if chunk == 0:  # every item above l + eps splits each round: the same sets on both paths
        assert (a["lower"], a["upper"], a["status"]) == (b["lower"], b["upper"], b["status"])
        for key in ("rounds", "splits", "queries", "retired", "peak_frontier"):
            assert a["stats"][key] == b["stats"][key], key
    else:  # which 16 items split first depends on the order in the frontier
        eps = a["stats"]["eps_abs"]
        for r in (a, b):
            assert r["status"] == hd.HD_OK and r["upper"] - r["lower"] <= eps * (1 + 1e-12)
        assert max(a["lower"], b["lower"]) <= min(a["upper"], b["upper"]) + 1e-12
    assert a["stats"]["kernel_launches"] <= b["stats"]["kernel_launches"]
    if k == 1:  # its last rounds are small: one launch for them instead of six per round
        assert a["stats"]["kernel_launches"] < b["stats"]["kernel_launches"]
    if k != 4:
        ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, p.tol_mode)
        assert max(a["lower"], ro["lower"]) <= min(a["upper"], ro["upper"]) + 1e-12


def test_bracket_all_bound_orders_fp64(hd, orc):
    import itertools

    p = mg.workload(1)
    ref = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, 1e-6, 0)
    bvh = hd.hd_build_B(p.VB, p.FB)
    for kk in range(1, 5):
        for order in itertools.permutations((1, 2, 3, 4), kk):
            o = hd.hd_options_default(bound_order=order, max_face_factor=2000)
            r = hd.hd_hausdorff(bvh, p.VA, p.FA, 1e-4, o)
            assert r["status"] in (hd.HD_OK, hd.HD_ERR_CAPACITY), (order, r)
            assert max(r["lower"], ref["lower"]) <= min(r["upper"], ref["upper"]) + 1e-12, order


def test_full_size_workload2_fp64_properties(hd, orc):
    """The benchmark's workload at full size: the bracket is within eps and holds the
    oracle's distances of 3000 sampled vertices (each d(v, B) <= h <= u, and l is the
    maximum over all vertices, so l >= each sample)."""
    p = mg.workload(2)
    bvh = hd.hd_build_B(p.VB, p.FB)
    r = hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol, hd.hd_options_default(tol_mode=p.tol_mode))
    eps = p.tol * _dA(p.VA, p.FA)
    assert r["status"] == hd.HD_OK and r["upper"] - r["lower"] <= eps
    rng = np.random.default_rng(9)
    P = np.asarray(p.VA, float)[rng.choice(len(p.VA), size=3000, replace=False)]
    do, _, _ = orc.nearest(P, p.VB, p.FB)
    assert do.max() <= r["lower"] * (1 + REL) and do.max() <= r["upper"]


def test_invalid_inputs_gpu(hd):
    V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]])
    F = np.array([[0, 1, 2]], np.int32)
    bvh = hd.hd_build_B(V, F)
    with pytest.raises(hd.HdError):
        hd.hd_hausdorff(bvh, V, np.array([[0, 1, 3]], np.int32), 1e-3)
    Vn = V.copy()
    Vn[2, 2] = np.nan
    with pytest.raises(hd.HdError):
        hd.hd_hausdorff(bvh, Vn, F, 1e-3)
    with pytest.raises(hd.HdError):
        hd.hd_build_B(Vn, F)
    with pytest.raises(hd.HdError):
        hd.hd_hausdorff(bvh, V, F, 0.0)


def test_capacity_returns_valid_bracket(hd, orc):
    p = mg.workload(1)
    bvh = hd.hd_build_B(p.VB, p.FB)
    ref = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, 1e-7, 0)
    r = hd.hd_hausdorff(bvh, p.VA, p.FA, 1e-7, hd.hd_options_default(max_face_factor=1.5))
    assert r["status"] == hd.HD_ERR_CAPACITY
    assert r["lower"] <= ref["upper"] + 1e-12 and ref["lower"] <= r["upper"] + 1e-12


def test_identical_meshes_gpu(hd):
    V, F = mg.icosphere(2)
    bvh = hd.hd_build_B(V, F)
    r = hd.hd_hausdorff(bvh, V, F, 1e-3)
    assert r["status"] == hd.HD_OK and 0 <= r["lower"] <= 1e-12 and r["upper"] <= 1e-3


def test_device_inputs_and_streams(hd):
    """Device tensors on a side stream give the same bracket as host arrays."""
    p = mg.workload(1)
    bvh = hd.hd_build_B(p.VB, p.FB)
    r1 = hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        VA = torch.from_numpy(p.VA).cuda()
        FA = torch.from_numpy(p.FA).cuda()
        r2 = hd.hd_hausdorff(bvh, VA, FA, p.tol)
    assert r1["lower"] == r2["lower"] and abs(r1["upper"] - r2["upper"]) <= p.tol
