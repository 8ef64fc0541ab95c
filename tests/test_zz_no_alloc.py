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


def _against_oracle(orc, res, P, VB, FB, precision):
    """The oracle's brute-force distance: equal to 1e-6 relative in FP64, inside the certified
    interval [dist_lo, dist] in MIXED (with the oracle's own ~1e-16 rounding allowed)."""
    d, _, _, lo = res
    do, _, _ = orc.nearest(np.asarray(P, np.float64), np.asarray(VB, np.float64), FB)
    if precision == "fp64":
        assert np.all(np.abs(d - do) <= REL * np.maximum(do, 1e-12))
    else:
        slack = 1e-12 * np.maximum(1.0, do)
        assert np.all(lo <= do + slack) and np.all(d >= do - slack)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_hd_nearest_on_two_calls(hd, orc, precision):
    prec = hd.HD_FP64 if precision == "fp64" else hd.HD_MIXED
    p = mg.workload(2, 0.1)
    bvh = hd.hd_build_B(p.VB, p.FB)
    rng = np.random.default_rng(77)
    V = p.VA.astype(np.float64)
    # first call: many points (both float32 and float64 inputs over the two calls)
    P1 = torch.from_numpy(V[rng.choice(len(V), size=9000, replace=False)].astype(np.float32)).cuda()
    r1 = _noalloc_c_abi(hd, bvh, P1, prec)
    _same(r1, _reference(hd, bvh, P1, prec))
    _against_oracle(orc, r1, P1.cpu().numpy(), p.VB, p.FB, precision)
    # second call right after, fewer points, reusing the same scratch array
    P2 = torch.from_numpy(V.mean(0) + rng.normal(size=(1234, 3)) * V.std(0) * 1.5).cuda()
    r2 = _noalloc_c_abi(hd, bvh, P2, prec)
    _same(r2, _reference(hd, bvh, P2, prec))
    _against_oracle(orc, r2, P2.cpu().numpy(), p.VB, p.FB, precision)


def _cudart():
    for name in ("libcudart.so", "libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return C.CDLL(name)
        except OSError:
            continue
    return None


def test_noalloc_allocates_no_device_memory(hd):
    """The property the entry point exists for: a call takes no memory from the device's
    stream-ordered pool (which the library's other entry points allocate from) and none from
    torch's allocator, not even for a moment (the pools' high-water marks are reset first).
    The output tensors are the caller's, passed through the binding's ``out``."""
    rt = _cudart()
    if rt is None:
        pytest.skip("libcudart not found for the pool query")
    USED_CUR, USED_HIGH, RES_CUR, RES_HIGH = 7, 8, 5, 6  # cudaMemPoolAttr values (cuda_runtime_api.h)
    pool = C.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(C.byref(pool), torch.cuda.current_device()) == 0

    def attr(a):
        v = C.c_uint64()
        assert rt.cudaMemPoolGetAttribute(pool, a, C.byref(v)) == 0
        return v.value

    p = mg.workload(1)
    bvh = hd.hd_build_B(p.VB, p.FB)
    P = torch.from_numpy(np.random.default_rng(5).normal(size=(5000, 3))).cuda()
    n = P.shape[0]
    for prec in (hd.HD_FP64, hd.HD_MIXED):
        out = _outputs(n)
        hd.hd_nearest_noalloc(bvh, P, prec, out=out)  # the first call on the device looks up the scratch
        torch.cuda.synchronize()
        zero = C.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, USED_HIGH, C.byref(zero)) == 0
        assert rt.cudaMemPoolSetAttribute(pool, RES_HIGH, C.byref(zero)) == 0
        used, res = attr(USED_CUR), attr(RES_CUR)
        t_alloc = torch.cuda.memory_allocated()
        for _ in range(2):
            hd.hd_nearest_noalloc(bvh, P, prec, out=out)
        torch.cuda.synchronize()
        assert attr(USED_HIGH) <= used and attr(USED_CUR) == used
        assert attr(RES_HIGH) <= res and attr(RES_CUR) == res
        assert torch.cuda.memory_allocated() == t_alloc


def test_noalloc_binding_with_and_without_out(hd, orc):
    """Through the Python binding: with the caller's ``out`` tensors and without, the same
    results as hd_nearest; ``out`` tensors of the wrong type, size or device are refused
    before anything is launched."""
    p = mg.workload(1)
    bvh = hd.hd_build_B(p.VB, p.FB)
    P = torch.from_numpy(np.random.default_rng(8).normal(size=(3000, 3)).astype(np.float32)).cuda()
    ref = _reference(hd, bvh, P, hd.HD_FP64)
    a = [x.cpu().numpy() for x in hd.hd_nearest_noalloc(bvh, P, hd.HD_FP64)]
    out = _outputs(P.shape[0])
    b = [x.cpu().numpy() for x in hd.hd_nearest_noalloc(bvh, P, hd.HD_FP64, out=out)]
    _same(a, ref)
    _same(b, ref)
    _against_oracle(orc, b, P.cpu().numpy(), p.VB, p.FB, "fp64")
    d, i, f, lo = _outputs(P.shape[0])
    for bad in ((d[:-1], i, f, lo), (d.float(), i, f, lo), (d, i.long(), f, lo), (d, i, f.cpu(), lo)):
        with pytest.raises(ValueError):
            hd.hd_nearest_noalloc(bvh, P, hd.HD_FP64, out=bad)


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
