"""Cut queries against exact ones, through the C ABI.

A vertex query may stop once the triangle of B it has found lies within l - e of the vertex
(l the running lower bound, e the longest edge of A): bound u1 (Eq. u1) then discards every
sub-triangle at that vertex whatever its exact distance.  The discarded sub-triangles, the
splits, the rounds and the bracket must therefore be those of exact queries
(HD_FLAG_EXACT_QUERIES, the paper's Section 4): this file checks that equality on the
workloads, in both precisions, and that the cut is off where u1 is not in the cascade.  The
brackets themselves are checked against the oracle by the parity tests, which run with the
default (cutting) options.
"""
import numpy as np
import pytest

import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def hd():
    from paper_2406_10357_gb300 import build

    build.build()
    import paper_2406_10357_gb300 as hd

    return hd


def _dev(p):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (p.VA, p.FA, p.VB, p.FB)]


def _run(hd, d, p, precision, flags=0, **kw):
    o = hd.hd_options_default(tol_mode=p.tol_mode, precision=precision, flags=flags, **kw)
    bvh = hd.hd_build_B(d[2], d[3], o)
    r = hd.hd_hausdorff(bvh, d[0], d[1], p.tol, o)
    del bvh
    return r


def _same_run(a, b):
    """The fields that exact queries fix: the bracket, the status and the refinement."""
    sa, sb = a["stats"], b["stats"]
    assert a["status"] == b["status"]
    assert a["lower"] == b["lower"] and a["upper"] == b["upper"], (a["lower"], b["lower"], a["upper"], b["upper"])
    for k in ("splits", "rounds", "queries", "retired", "promoted", "peak_frontier", "pool_vertices"):
        assert sa[k] == sb[k], (k, sa[k], sb[k])
    # a face may be discarded by the exact case instead of u1 when a cut vertex kept the
    # triangle its neighbours are nearest to: the total is the same
    assert sum(sa["discards"].values()) == sum(sb["discards"].values())


CASES = [(1, 0.25), (2, 0.25), (2, 1.0), (3, 0.05), (5, 1 / 64), (5, 1 / 4)]


@pytest.mark.parametrize("k,scale", CASES)
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_cut_equals_exact(hd, k, scale, precision):
    p = mg.workload(k, scale)
    d = _dev(p)
    prec = hd.HD_MIXED if precision == "mixed" else hd.HD_FP64
    exact = _run(hd, d, p, prec, hd.HD_FLAG_EXACT_QUERIES)
    cut = _run(hd, d, p, prec)
    assert exact["stats"]["queries_cut"] == 0
    _same_run(exact, cut)
    # the cut queries do less traversal work, never more
    assert cut["stats"]["node_visits"] <= exact["stats"]["node_visits"]


def test_cut_happens_on_the_soup(hd):
    """The random triangles of the large soup lie up to 0.1 off B: most of their vertices are
    well below h, so most of their queries stop early."""
    p = mg.workload(5, 1 / 16)
    d = _dev(p)
    r = _run(hd, d, p, hd.HD_MIXED)
    assert r["status_str"] == "HD_OK"
    n_random = 3 * max(4, int(100_000 / 16))
    assert r["stats"]["queries_cut"] > n_random // 2, r["stats"]["queries_cut"]


@pytest.mark.parametrize("order", [(2, 3, 4), (3,), (4, 3, 2)])
def test_no_cut_without_u1(hd, order):
    """Without u1 in the cascade nothing guarantees that a cut vertex's faces are discarded,
    so every query runs to its nearest triangle."""
    p = mg.workload(5, 1 / 64)
    d = _dev(p)
    r = _run(hd, d, p, hd.HD_MIXED, bound_order=order)
    assert r["stats"]["queries_cut"] == 0
    with_u1 = _run(hd, d, p, hd.HD_MIXED, bound_order=order + (1,))
    assert with_u1["stats"]["queries_cut"] > 0
    assert r["status"] == with_u1["status"] == hd.HD_OK


def test_cut_sharded_and_warm_start(hd):
    """hd_hausdorff_from with a warm-start l: the cut uses it from the first query."""
    p = mg.workload(5, 1 / 64)
    d = _dev(p)
    full = _run(hd, d, p, hd.HD_MIXED, hd.HD_FLAG_EXACT_QUERIES)
    o = hd.hd_options_default(tol_mode=p.tol_mode, precision=hd.HD_MIXED)
    bvh = hd.hd_build_B(d[2], d[3], o)
    warm = hd.hd_hausdorff_from(bvh, d[0], d[1], p.tol, 0.5 * full["lower"], o)
    assert warm["status"] == hd.HD_OK
    assert warm["lower"] <= full["upper"] and full["lower"] <= warm["upper"]
    assert warm["stats"]["queries_cut"] > 0
