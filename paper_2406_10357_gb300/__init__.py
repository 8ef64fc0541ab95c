"""Python binding of the GB300 Hausdorff branch-and-bound library (``include/hd.h``).

Argument marshalling only: every step of the computation runs in ``libhd.so``'s CUDA
kernels.  Arrays may be NumPy (host) or PyTorch tensors (host or CUDA); CUDA tensors are
passed as device pointers on torch's current stream.  There is no CPU fallback: if the
library is not built, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhd.so")

HD_OK, HD_ERR_INVALID, HD_ERR_CAPACITY, HD_ERR_NUMERIC, HD_ERR_TIMEOUT, HD_ERR_CUDA = range(6)
HD_F32, HD_F64 = 0, 1
HD_TOL_ABS, HD_TOL_REL = 0, 1
HD_FP64, HD_MIXED = 0, 1
HD_FLAG_NO_PARENT_CLAMP = 1
HD_FLAG_ASYNC_BUILD = 2
HD_FLAG_SHARE_MIDPOINTS = 4
HD_FLAG_WELD_B = 8
HD_FLAG_NO_SMALL_ROUNDS = 16
HD_FLAG_BATCH_STREAMS = 32
HD_FLAG_EXACT_QUERIES = 64
BOUND_NAMES = ("exact", "u1", "u2", "u3", "u4", "late")


class HdMesh(C.Structure):
    _fields_ = [("V", C.c_void_p), ("nV", C.c_int64), ("F", C.c_void_p), ("nF", C.c_int64), ("vtype", C.c_int32),
                ("on_device", C.c_int32)]


class HdOptions(C.Structure):
    _fields_ = [("tol_mode", C.c_int32), ("precision", C.c_int32), ("max_face_factor", C.c_double),
                ("frontier_chunk", C.c_int64), ("leaf_size", C.c_int32), ("block_size", C.c_int32),
                ("bound_order", C.c_uint8 * 4), ("n_bounds", C.c_int32), ("max_rounds", C.c_int64),
                ("max_frontier_bytes", C.c_int64), ("flags", C.c_int32), ("reserved", C.c_int32)]


class HdStats(C.Structure):
    _fields_ = [("rounds", C.c_int64), ("splits", C.c_int64), ("queries", C.c_int64), ("pointtri_evals", C.c_int64),
                ("leaf_tests", C.c_int64), ("box_tests", C.c_int64), ("discards", C.c_int64 * 6), ("retired", C.c_int64),
                ("fp64_escalations", C.c_int64), ("peak_frontier", C.c_int64), ("pool_vertices", C.c_int64),
                ("eps_abs", C.c_double), ("dA", C.c_double), ("long_queries", C.c_int64),
                ("kernel_launches", C.c_int64), ("d2h_bytes", C.c_int64), ("promoted", C.c_int64),
                ("node_visits", C.c_int64), ("long_node_visits", C.c_int64), ("long_leaf_tests", C.c_int64),
                ("queries_cut", C.c_int64)]


class HdResult(C.Structure):
    _fields_ = [("lower", C.c_double), ("upper", C.c_double), ("status", C.c_int32), ("stats", HdStats)]


class HdTrace(C.Structure):
    _fields_ = [("launches", C.c_int64 * 8), ("ms", C.c_double * 8)]


HD_K_BUILD, HD_K_QUERY, HD_K_BOUND, HD_K_SELECT, HD_K_PREP, HD_K_SMALL, HD_K_LONG = range(7)
KERNEL_KINDS = ("build", "query", "bound", "select", "prep", "small_rounds", "query_long")


_lib = None


def lib():
    """The loaded ``libhd.so``.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_2406_10357_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        L.hd_options_default.argtypes = [C.POINTER(HdOptions)]
        L.hd_options_default.restype = None
        L.hd_build_B.argtypes = [C.POINTER(HdMesh), C.POINTER(HdOptions), vp, C.POINTER(vp)]
        L.hd_free_B.argtypes = [vp]
        L.hd_free_B.restype = None
        L.hd_bvh_num_faces.argtypes = [vp]
        L.hd_bvh_num_faces.restype = i64
        L.hd_hausdorff.argtypes = [vp, C.POINTER(HdMesh), d, C.POINTER(HdOptions), vp, C.POINTER(HdResult)]
        L.hd_hausdorff_batched.argtypes = [C.POINTER(vp), C.POINTER(HdMesh), i64, d, C.POINTER(HdOptions), vp,
                                           C.POINTER(HdResult)]
        L.hd_hausdorff_from.argtypes = [vp, C.POINTER(HdMesh), d, d, C.POINTER(HdOptions), vp, C.POINTER(HdResult)]
        L.hd_hausdorff_sym.argtypes = [vp, C.POINTER(HdMesh), vp, C.POINTER(HdMesh), d, C.POINTER(HdOptions), vp,
                                       C.POINTER(HdResult), C.POINTER(HdResult), C.POINTER(HdResult)]
        L.hd_nearest.argtypes = [vp, vp, i32, i64, i32, vp, vp, vp, vp, vp]
        L.hd_upper_bounds.argtypes = [vp, vp, vp, vp, vp, i64, d, C.POINTER(HdOptions), vp, vp, vp]
        L.hd_nearest_noalloc.argtypes = [vp, vp, i32, i64, i32, vp, vp, vp, vp, vp]
        L.hd_nearest_noalloc.restype = C.c_int
        L.hd_trace_enable.argtypes = [C.c_int]
        L.hd_trace_enable.restype = None
        L.hd_trace_read.argtypes = [C.POINTER(HdTrace), C.c_int]
        L.hd_trace_read.restype = C.c_int
        L.hd_status_str.argtypes = [C.c_int]
        L.hd_status_str.restype = C.c_char_p
        L.hd_last_error.restype = C.c_char_p
        for f in ("hd_build_B", "hd_hausdorff", "hd_hausdorff_batched", "hd_hausdorff_from", "hd_hausdorff_sym",
                  "hd_nearest", "hd_upper_bounds"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


class HdError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = f"{what}: {hd_status_str(status)}"
        if status == HD_ERR_CUDA:
            msg += f" ({lib().hd_last_error().decode()})"
        super().__init__(msg)
        self.status = status


def _check(rc: int, what: str):
    if rc != HD_OK:
        raise HdError(rc, what)


def hd_status_str(status: int) -> str:
    return lib().hd_status_str(status).decode()


def hd_options_default(**kw) -> HdOptions:
    """Defaults of ``hd_options_default``; keyword arguments override fields
    (``bound_order`` may be a sequence of 1..4, which also sets ``n_bounds``)."""
    o = HdOptions()
    lib().hd_options_default(C.byref(o))
    for k, v in kw.items():
        if k == "bound_order":
            v = list(v)
            for i in range(4):
                o.bound_order[i] = v[i] if i < len(v) else 0
            o.n_bounds = len(v)
        else:
            setattr(o, k, v)
    return o


def _is_torch(x) -> bool:
    return hasattr(x, "data_ptr") and hasattr(x, "is_cuda")


def _stream(on_device: bool, stream):
    if stream is not None:
        return C.c_void_p(stream)
    if on_device:
        import torch

        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(0)


def _mesh(V, F):
    """HdMesh view of (V, F) plus the objects that must stay alive during the call."""
    if _is_torch(V):
        import torch

        V = V.contiguous()
        if V.dtype not in (torch.float32, torch.float64):
            V = V.double()
        F = F.to(device=V.device, dtype=torch.int32).contiguous()
        m = HdMesh(V.data_ptr(), V.shape[0], F.data_ptr(), F.shape[0], HD_F64 if V.dtype == torch.float64 else HD_F32,
                   1 if V.is_cuda else 0)
        return m, (V, F), bool(V.is_cuda)
    V = np.ascontiguousarray(V)
    if V.dtype not in (np.float32, np.float64):
        V = V.astype(np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    m = HdMesh(V.ctypes.data, V.shape[0], F.ctypes.data, F.shape[0], HD_F64 if V.dtype == np.float64 else HD_F32, 0)
    return m, (V, F), False


class Bvh:
    """Owner of an ``hd_bvh*`` (freed with ``hd_free_B`` when collected)."""

    def __init__(self, handle: int, nF: int):
        self.handle = C.c_void_p(handle)
        self.nF = nF

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.hd_free_B(self.handle)
            self.handle = C.c_void_p(0)


def hd_build_B(V, F, opt: HdOptions | None = None, stream=None) -> Bvh:
    """Build the BVH of B (host or device arrays)."""
    m, keep, dev = _mesh(V, F)
    out = C.c_void_p(0)
    _check(lib().hd_build_B(C.byref(m), C.byref(opt) if opt else None, _stream(dev, stream), C.byref(out)),
           "hd_build_B")
    return Bvh(out.value, int(m.nF))


def hd_free_B(bvh: Bvh):
    if bvh.handle.value:
        lib().hd_free_B(bvh.handle)
        bvh.handle = C.c_void_p(0)


def hd_trace_enable(on: bool = True):
    """Record CUDA events around the library's kernels (per kind: launches, total ms)."""
    lib().hd_trace_enable(1 if on else 0)


def hd_trace_read(reset: bool = False) -> dict:
    t = HdTrace()
    _check(lib().hd_trace_read(C.byref(t), 1 if reset else 0), "hd_trace_read")
    return {KERNEL_KINDS[k]: dict(launches=t.launches[k], ms=t.ms[k]) for k in range(len(KERNEL_KINDS))}


def _result(r: HdResult) -> dict:
    s = r.stats
    return dict(lower=r.lower, upper=r.upper, status=r.status, status_str=hd_status_str(r.status),
                stats=dict(rounds=s.rounds, splits=s.splits, queries=s.queries, pointtri_evals=s.pointtri_evals,
                           leaf_tests=s.leaf_tests,
                           box_tests=s.box_tests, discards={BOUND_NAMES[k]: s.discards[k] for k in range(6)},
                           retired=s.retired, fp64_escalations=s.fp64_escalations, peak_frontier=s.peak_frontier,
                           pool_vertices=s.pool_vertices, eps_abs=s.eps_abs, dA=s.dA,
                           long_queries=s.long_queries, kernel_launches=s.kernel_launches,
                           d2h_bytes=s.d2h_bytes, promoted=s.promoted, node_visits=s.node_visits,
                           long_node_visits=s.long_node_visits, long_leaf_tests=s.long_leaf_tests,
                           queries_cut=s.queries_cut))


def hd_hausdorff(bvh: Bvh, VA, FA, tol: float, opt: HdOptions | None = None, stream=None) -> dict:
    """h(A, B) bracket: dict(lower, upper, status, stats).  Raises on INVALID/CUDA errors;
    CAPACITY/TIMEOUT/NUMERIC come back in ``status``."""
    m, keep, dev = _mesh(VA, FA)
    r = HdResult()
    rc = lib().hd_hausdorff(bvh.handle, C.byref(m), float(tol), C.byref(opt) if opt else None, _stream(dev, stream),
                            C.byref(r))
    if rc in (HD_ERR_INVALID, HD_ERR_CUDA):
        raise HdError(rc, "hd_hausdorff")
    return _result(r)


def hd_hausdorff_from(bvh: Bvh, VA, FA, tol: float, l0: float, opt: HdOptions | None = None, stream=None) -> dict:
    """hd_hausdorff with l starting at l0 (a known lower bound); brackets max(l0, h(A, B))."""
    m, keep, dev = _mesh(VA, FA)
    r = HdResult()
    rc = lib().hd_hausdorff_from(bvh.handle, C.byref(m), float(tol), float(l0), C.byref(opt) if opt else None,
                                 _stream(dev, stream), C.byref(r))
    if rc in (HD_ERR_INVALID, HD_ERR_CUDA):
        raise HdError(rc, "hd_hausdorff_from")
    return _result(r)


def hd_hausdorff_sym(bvhB: Bvh, VA, FA, bvhA: Bvh, VB, FB, tol: float, opt: HdOptions | None = None,
                     stream=None) -> tuple[dict, dict, dict]:
    """Two-sided H(A, B): (H bracket, h(A, B) run, h(B, A) run warm-started from it)."""
    mA, keepA, devA = _mesh(VA, FA)
    mB, keepB, devB = _mesh(VB, FB)
    r, rab, rba = HdResult(), HdResult(), HdResult()
    rc = lib().hd_hausdorff_sym(bvhB.handle, C.byref(mA), bvhA.handle, C.byref(mB), float(tol),
                                C.byref(opt) if opt else None, _stream(devA or devB, stream), C.byref(r),
                                C.byref(rab), C.byref(rba))
    if rc in (HD_ERR_INVALID, HD_ERR_CUDA):
        raise HdError(rc, "hd_hausdorff_sym")
    return _result(r), _result(rab), _result(rba)


def hd_hausdorff_batched(bvhs, As, tol: float, opt: HdOptions | None = None, stream=None) -> list[dict]:
    """Independent pairs h(As[i], Bs[i]); As is a list of (V, F)."""
    n = len(bvhs)
    handles = (C.c_void_p * n)(*[b.handle.value for b in bvhs])
    meshes = (HdMesh * n)()
    keep, dev = [], False
    for i, (V, F) in enumerate(As):
        m, k, d = _mesh(V, F)
        meshes[i] = m
        keep.append(k)
        dev = dev or d
    outs = (HdResult * n)()
    _check(lib().hd_hausdorff_batched(handles, meshes, n, float(tol), C.byref(opt) if opt else None,
                                      _stream(dev, stream), outs), "hd_hausdorff_batched")
    return [_result(outs[i]) for i in range(n)]


def _points(P):
    """P as a contiguous (n, 3) float32 or float64 CUDA tensor (other real dtypes become float64)."""
    import torch

    if not (_is_torch(P) and P.is_cuda):
        raise ValueError("P must be a CUDA tensor")
    if P.ndim != 2 or P.shape[1] != 3:
        raise ValueError(f"P must have shape (n, 3), not {tuple(P.shape)}")
    if P.dtype not in (torch.float32, torch.float64):
        P = P.double()
    return P.contiguous()


def hd_nearest(bvh: Bvh, P, precision: int = HD_FP64, stream=None):
    """Nearest triangle of B for each row of P (a CUDA tensor, float32 or float64).
    Returns CUDA tensors (dist, idx, foot, dist_lo); in HD_MIXED dist is a certified upper
    bound and dist_lo a certified lower bound of d(p, B)."""
    import torch

    P = _points(P)
    n = P.shape[0]
    dev = P.device
    dist = torch.empty(n, dtype=torch.float64, device=dev)
    dlo = torch.empty(n, dtype=torch.float64, device=dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    foot = torch.empty((n, 3), dtype=torch.float64, device=dev)
    _check(lib().hd_nearest(bvh.handle, P.data_ptr(), HD_F64 if P.dtype == torch.float64 else HD_F32, n, precision,
                            _stream(True, stream), dist.data_ptr(), idx.data_ptr(), foot.data_ptr(), dlo.data_ptr()),
           "hd_nearest")
    return dist, idx, foot, dlo


HD_NOALLOC_MAX_POINTS = 65536  # as include/hd.h defines it (a CPU test compares the two)


def _check_out(out, n, device):
    """The caller's output tensors (dist, idx, foot, dist_lo) must match what the kernels write:
    float64 / int32 / float64 / float64, n / n / 3 n / n elements, contiguous, on P's device."""
    import torch

    if len(out) != 4:
        raise ValueError("out must be (dist, idx, foot, dist_lo)")
    want = ((torch.float64, n), (torch.int32, n), (torch.float64, 3 * n), (torch.float64, n))
    for name, t, (dt, k) in zip(("dist", "idx", "foot", "dist_lo"), out, want):
        if not _is_torch(t) or t.dtype != dt or t.numel() != k or not t.is_contiguous() or t.device != device:
            raise ValueError(f"out {name}: need a contiguous {dt} tensor of {k} elements on {device}")


def hd_nearest_noalloc(bvh: Bvh, P, precision: int = HD_FP64, out=None, stream=None):
    """hd_nearest without any device allocation inside the library (at most
    HD_NOALLOC_MAX_POINTS points).  The output tensors may be passed in ``out`` =
    (dist, idx, foot, dist_lo) so that the call allocates nothing at all; they are checked
    (type, size, device, layout) before anything is launched."""
    import torch

    P = _points(P)
    n = P.shape[0]
    if n > HD_NOALLOC_MAX_POINTS:
        raise ValueError(f"hd_nearest_noalloc takes at most {HD_NOALLOC_MAX_POINTS} points, not {n}")
    dev = P.device
    if out is None:
        out = (torch.empty(n, dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.int32, device=dev),
               torch.empty((n, 3), dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.float64, device=dev))
    else:
        _check_out(out, n, dev)
    dist, idx, foot, dlo = out
    _check(lib().hd_nearest_noalloc(bvh.handle, P.data_ptr(), HD_F64 if P.dtype == torch.float64 else HD_F32, n,
                                    precision, _stream(True, stream), dist.data_ptr(), idx.data_ptr(),
                                    foot.data_ptr(), dlo.data_ptr()), "hd_nearest_noalloc")
    return dist, idx, foot, dlo


def hd_upper_bounds(bvh: Bvh, T, Td, TI, Tq, l: float, opt: HdOptions | None = None, stream=None):
    """UpperBound(T, l) for n triangles (CUDA tensors): returns (U, code).  FP64 by default;
    with ``opt.precision = HD_MIXED`` the certified FP32 arithmetic of the rounds."""
    import torch

    T, Td, Tq = (x.to(torch.float64).contiguous() for x in (T, Td, Tq))
    TI = TI.to(torch.int32).contiguous()
    n = T.shape[0]
    U = torch.empty(n, dtype=torch.float64, device=T.device)
    code = torch.empty(n, dtype=torch.int32, device=T.device)
    _check(lib().hd_upper_bounds(bvh.handle, T.data_ptr(), Td.data_ptr(), TI.data_ptr(), Tq.data_ptr(), n, float(l),
                                 C.byref(opt) if opt else None, _stream(True, stream), U.data_ptr(),
                                 code.data_ptr()), "hd_upper_bounds")
    return U, code
