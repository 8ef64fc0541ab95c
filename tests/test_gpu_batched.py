"""The batched run (hd_hausdorff_batched's default): all pairs in one frontier-parallel branch
and bound, every launch taking its work from a device-side queue of all pairs' items, each pair
with its own l, u, tolerance, status and stop on its own gap (Sections 3.1 and 4 per pair).

Every pair's bracket must be within eps and meet the oracle's and its own single run's, in
FP64 and MIXED; per-pair limits (the face cap m, the round limit) stop only the pairs that
reach them; MIXED pairs whose last items fall below FP32 resolution are finished in the
batched FP64 phase; host and device inputs mix; the host-threaded path (HD_FLAG_BATCH_STREAMS)
gives brackets that meet the batched ones.
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


@pytest.fixture(scope="module")
def hd():
    from paper_2406_10357_gb300 import build

    build.build()
    import paper_2406_10357_gb300 as hd

    return hd


def _dA(V, F):
    R = np.asarray(V, float)[np.unique(np.asarray(F).ravel())]
    return float(np.linalg.norm(R.max(0) - R.min(0)))


def _meet(a, b, eps):
    """Both brackets contain h: they intersect, up to the rounding of FP64 distances (the FP64
    path and the oracle round the same distance differently in the last bits)."""
    return max(a["lower"], b["lower"]) <= min(a["upper"], b["upper"]) + 1e-12 * max(eps, abs(b["upper"]), 1e-300)


def _uneven_pairs():
    """Reduced pairs of the batched workload plus the extremes: a one-triangle A against a
    sphere, and the reduced torus benchmark pair."""
    pairs = mg.batch_workload(n_pairs=16, lo=300, hi=3000)
    V, F = mg.icosphere(3)
    pairs.append(mg.Pair("one-triangle-A", np.array([[0.0, 0, 1.3], [0.2, 0, 1.25], [0, 0.2, 1.25]]),
                         np.array([[0, 1, 2]], np.int32), V, F, 1e-4, mg.TOL_REL))
    pairs.append(mg.workload(2, 0.02))
    return pairs


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batched_matches_oracle_single_runs_and_streams(hd, orc, precision):
    pairs = _uneven_pairs()
    prec = hd.HD_MIXED if precision == "mixed" else hd.HD_FP64
    o = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=prec)
    bvhs = [hd.hd_build_B(p.VB, p.FB) for p in pairs]
    As = [(p.VA, p.FA) for p in pairs]
    tol = 1e-4
    rs = hd.hd_hausdorff_batched(bvhs, As, tol, o)
    ostreams = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=prec, flags=hd.HD_FLAG_BATCH_STREAMS)
    rs_streams = hd.hd_hausdorff_batched(bvhs, As, tol, ostreams)
    launches = {r["stats"]["kernel_launches"] for r in rs}
    assert len(launches) == 1  # every result holds the batch's totals
    for p, b, r, r2 in zip(pairs, bvhs, rs, rs_streams):
        eps = tol * _dA(p.VA, p.FA)
        assert r["status"] == hd.HD_OK, (p.name, r)
        assert r["upper"] - r["lower"] <= eps * (1 + 1e-12), p.name
        assert abs(r["stats"]["eps_abs"] - eps) <= 1e-9 * eps
        ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, tol, hd.HD_TOL_REL, max_face_factor=200)
        assert ro["status"] in (orc.OK, orc.CAPACITY)
        assert _meet(r, ro, eps), (p.name, r, ro)
        r1 = hd.hd_hausdorff(b, p.VA, p.FA, tol, o)
        assert _meet(r, r1, eps) and _meet(r, r2, eps), p.name
        # the batch bounds the same items as the single run: the same vertex queries of A
        assert r["stats"]["queries"] >= len(np.unique(p.FA))


def test_batched_device_and_host_inputs(hd):
    """Pairs given as host arrays and as CUDA tensors in one call: the same brackets as all-host."""
    pairs = mg.batch_workload(n_pairs=6, lo=300, hi=2000)
    o = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=hd.HD_MIXED)
    bvhs = [hd.hd_build_B(p.VB, p.FB) for p in pairs]
    host = hd.hd_hausdorff_batched(bvhs, [(p.VA, p.FA) for p in pairs], 1e-4, o)
    mixed_in = [(torch.from_numpy(p.VA).cuda(), torch.from_numpy(p.FA).cuda()) if i % 2 else (p.VA, p.FA)
                for i, p in enumerate(pairs)]
    both = hd.hd_hausdorff_batched(bvhs, mixed_in, 1e-4, o)
    for p, a, b in zip(pairs, host, both):
        eps = 1e-4 * _dA(p.VA, p.FA)
        assert a["status"] == b["status"] == hd.HD_OK and a["lower"] == b["lower"]
        assert abs(a["upper"] - b["upper"]) <= eps


def test_batched_face_cap_stops_only_its_pairs(hd, orc):
    """The face cap m n_A (Section 4) is per pair: with m = 1.5 the pairs that need more splits
    stop with CAPACITY and a valid bracket (it meets the oracle's), the others finish."""
    pairs = mg.batch_workload(n_pairs=8, lo=300, hi=2000) + [mg.workload(1)]
    o = hd.hd_options_default(tol_mode=hd.HD_TOL_ABS, precision=hd.HD_FP64, max_face_factor=1.5)
    bvhs = [hd.hd_build_B(p.VB, p.FB) for p in pairs]
    tol = 1e-7
    rs = hd.hd_hausdorff_batched(bvhs, [(p.VA, p.FA) for p in pairs], tol, o)
    st = [r["status"] for r in rs]
    assert hd.HD_ERR_CAPACITY in st
    for p, r in zip(pairs, rs):
        assert r["status"] in (hd.HD_OK, hd.HD_ERR_CAPACITY)
        assert r["stats"]["splits"] <= (1.5 * len(p.FA) - len(p.FA)) / 4 + 1
        ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, tol, 0, max_face_factor=50)
        assert _meet(r, ro, tol), (p.name, r, ro)
        if r["status"] == hd.HD_OK:
            assert r["upper"] - r["lower"] <= tol * (1 + 1e-12)


def test_batched_round_limit_per_pair(hd, orc):
    """max_rounds stops the pairs that need more rounds with TIMEOUT and a valid bracket."""
    pairs = [mg.workload(1), mg.workload(2, 0.02)]
    o = hd.hd_options_default(tol_mode=hd.HD_TOL_ABS, precision=hd.HD_MIXED, max_rounds=1)
    bvhs = [hd.hd_build_B(p.VB, p.FB) for p in pairs]
    rs = hd.hd_hausdorff_batched(bvhs, [(p.VA, p.FA) for p in pairs], 1e-7, o)
    assert any(r["status"] == hd.HD_ERR_TIMEOUT for r in rs)
    for p, r in zip(pairs, rs):
        assert r["stats"]["rounds"] <= 1
        ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, 1e-7, 0)
        assert _meet(r, ro, 1e-7), (p.name, r, ro)


def test_batched_closed_forms_promote_and_hold_h(hd):
    """The closed-form pairs in one batched MIXED call at tol 1e-6: their last items fall below
    FP32 resolution and are finished in the batched FP64 phase; every bracket holds the
    hand-derived h and is within tol."""
    cases = json.load(open(GOLDEN))["cases"]
    bvhs = [hd.hd_build_B(np.array(c["VB"], float), np.array(c["FB"], np.int32)) for c in cases]
    As = [(np.array(c["VA"], float), np.array(c["FA"], np.int32)) for c in cases]
    tol = cases[0]["tol"]
    assert all(c["tol"] == tol for c in cases)
    rs = hd.hd_hausdorff_batched(bvhs, As, tol, hd.hd_options_default(precision=hd.HD_MIXED))
    for c, r in zip(cases, rs):
        assert r["status"] == hd.HD_OK, (c["name"], r)
        assert r["lower"] <= c["h"] <= r["upper"] and r["upper"] - r["lower"] <= tol, (c["name"], r)
    assert sum(r["stats"]["promoted"] for r in rs) > 0


@pytest.mark.parametrize("order", [(1, 2, 3, 4), (3,), (1, 4), (2, 3, 1)])
def test_batched_bound_orders(hd, orc, order):
    """Cascades other than the paper's run the general UpperBound kernels in the batch too."""
    pairs = [mg.workload(1), mg.workload(2, 0.02)] + mg.batch_workload(n_pairs=3, lo=300, hi=1500)
    for prec in (hd.HD_MIXED, hd.HD_FP64):
        o = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=prec, bound_order=order, max_face_factor=2000)
        bvhs = [hd.hd_build_B(p.VB, p.FB) for p in pairs]
        rs = hd.hd_hausdorff_batched(bvhs, [(p.VA, p.FA) for p in pairs], 1e-4, o)
        for p, r in zip(pairs, rs):
            eps = 1e-4 * _dA(p.VA, p.FA)
            assert r["status"] in (hd.HD_OK, hd.HD_ERR_CAPACITY), (order, p.name, r)
            ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, 1e-4, hd.HD_TOL_REL, max_face_factor=200)
            assert _meet(r, ro, eps), (order, p.name, r, ro)


def test_batched_buffers_exhausted_pairs_finish_on_their_own(hd, orc):
    """With a budget (12 MB) that each pair's single run fits but the batch as a whole does not
    (all pairs' frontiers and midpoints share it), the pairs still running when it runs out are
    finished as single runs: every pair ends OK, within eps, meeting the oracle's bracket, and
    some pairs were indeed finished that way (their statistics are their own run's, not the
    batch's totals)."""
    pairs = mg.batch_workload(n_pairs=8, lo=300, hi=2000)
    o = hd.hd_options_default(tol_mode=hd.HD_TOL_REL, precision=hd.HD_MIXED, max_frontier_bytes=12 << 20)
    bvhs = [hd.hd_build_B(p.VB, p.FB) for p in pairs]
    single = [hd.hd_hausdorff(b, p.VA, p.FA, 1e-4, o) for p, b in zip(pairs, bvhs)]
    keep = [i for i, r in enumerate(single) if r["status"] == hd.HD_OK]
    assert len(keep) >= 6
    pairs, bvhs = [pairs[i] for i in keep], [bvhs[i] for i in keep]
    rs = hd.hd_hausdorff_batched(bvhs, [(p.VA, p.FA) for p in pairs], 1e-4, o)
    batch_total = max(r["stats"]["kernel_launches"] for r in rs)
    assert any(r["stats"]["kernel_launches"] != batch_total for r in rs)  # some pairs were finished singly
    for p, r in zip(pairs, rs):
        eps = 1e-4 * _dA(p.VA, p.FA)
        assert r["status"] == hd.HD_OK, (p.name, r)
        assert r["upper"] - r["lower"] <= eps * (1 + 1e-12)
        ro = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, 1e-4, hd.HD_TOL_REL, max_face_factor=200)
        assert _meet(r, ro, eps), (p.name, r, ro)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batched_one_pair_equals_single_run(hd, orc, precision):
    """A batch of one pair: the same bracket, status and counts as the single run (the same
    items are split in the same rounds), and an empty batch returns at once."""
    p = mg.workload(2, 0.02)
    prec = hd.HD_MIXED if precision == "mixed" else hd.HD_FP64
    o = hd.hd_options_default(tol_mode=p.tol_mode, precision=prec, flags=hd.HD_FLAG_NO_SMALL_ROUNDS)
    bvh = hd.hd_build_B(p.VB, p.FB)
    (r,) = hd.hd_hausdorff_batched([bvh], [(p.VA, p.FA)], p.tol, o)
    r1 = hd.hd_hausdorff(bvh, p.VA, p.FA, p.tol, o)
    assert (r["lower"], r["upper"], r["status"]) == (r1["lower"], r1["upper"], r1["status"])
    for k in ("rounds", "splits", "queries", "retired", "promoted"):
        assert r["stats"][k] == r1["stats"][k], k
    assert hd.hd_hausdorff_batched([], [], p.tol, o) == []
