"""hd_nearest_noalloc: the nearest-triangle queries for callers that cannot let the library
allocate device memory (caller-owned allocators, fixed memory budgets, latency-critical loops).

It must give the same results as hd_nearest through the C ABI, on consecutive calls that
reuse its fixed scratch array, and reject sizes beyond HD_NOALLOC_MAX_POINTS.  This file is
named so that pytest collects it last; it builds the library itself, so it also runs alone
in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

REL = 1e-6  # the per-query tolerance of the other parity tests


@pytest.fixture(scope="module")
def hd():
    from paper_2406_10357_gb300 import build

    build.build()
    import paper_2406_10357_gb300 as hd

    return hd


def _outputs(n):
    return (torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"),
            torch.empty((n, 3), dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda"))


def _noalloc_c_abi(hd, bvh, P, precision):
    """Call the entry point directly through the C ABI with raw device pointers."""
    n = P.shape[0]
    d, i, f, lo = _outputs(n)
    ptype = hd.HD_F64 if P.dtype == torch.float64 else hd.HD_F32
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = hd.lib().hd_nearest_noalloc(bvh.handle, C.c_void_p(P.data_ptr()), ptype, n, precision, stream,
                                     C.c_void_p(d.data_ptr()), C.c_void_p(i.data_ptr()), C.c_void_p(f.data_ptr()),
                                     C.c_void_p(lo.data_ptr()))
    assert rc == hd.HD_OK, hd.hd_status_str(rc)
    torch.cuda.synchronize()
    return d.cpu().numpy(), i.cpu().numpy(), f.cpu().numpy(), lo.cpu().numpy()


def _reference(hd, bvh, P, precision):
    d, i, f, lo = hd.hd_nearest(bvh, P, precision)
    torch.cuda.synchronize()
    return d.cpu().numpy(), i.cpu().numpy(), f.cpu().numpy(), lo.cpu().numpy()


def _same(a, b):
    d1, i1, f1, lo1 = a
    d2, i2, f2, lo2 = b
    assert np.all(np.abs(d1 - d2) <= REL * np.maximum(d2, 1e-12))
    assert np.all(np.abs(lo1 - lo2) <= REL * np.maximum(d2, 1e-12))
    assert np.all(np.abs(f1 - f2) <= REL * np.maximum(d2[:, None], 1e-9) + 1e-12)
    # indices agree except where two triangles are equally near (then the distance checks above hold)
    assert np.mean(i1 == i2) > 0.99


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_hd_nearest_on_two_calls(hd, precision):
    prec = hd.HD_FP64 if precision == "fp64" else hd.HD_MIXED
    p = mg.workload(2, 0.1)
    bvh = hd.hd_build_B(p.VB, p.FB)
    rng = np.random.default_rng(77)
    V = p.VA.astype(np.float64)
    # first call: many points (both float32 and float64 inputs over the two calls)
    P1 = torch.from_numpy(V[rng.choice(len(V), size=9000, replace=False)].astype(np.float32)).cuda()
    _same(_noalloc_c_abi(hd, bvh, P1, prec), _reference(hd, bvh, P1, prec))
    # second call right after, fewer points, reusing the same scratch array
    P2 = torch.from_numpy(V.mean(0) + rng.normal(size=(1234, 3)) * V.std(0) * 1.5).cuda()
    _same(_noalloc_c_abi(hd, bvh, P2, prec), _reference(hd, bvh, P2, prec))


def test_noalloc_rejects_too_many_points(hd):
    p = mg.workload(1)
    bvh = hd.hd_build_B(p.VB, p.FB)
    n = hd.HD_NOALLOC_MAX_POINTS + 1
    P = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    d, i, f, lo = _outputs(n)
    rc = hd.lib().hd_nearest_noalloc(bvh.handle, C.c_void_p(P.data_ptr()), hd.HD_F64, n, hd.HD_FP64, None,
                                     C.c_void_p(d.data_ptr()), C.c_void_p(i.data_ptr()), C.c_void_p(f.data_ptr()),
                                     C.c_void_p(lo.data_ptr()))
    assert rc == hd.HD_ERR_INVALID
