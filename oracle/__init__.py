"""Python access to the FP64 CPU oracle (``hd_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg are the only users.  The library under ``paper_2406_10357_gb300`` never
imports this package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hd_oracle.cpp")
_LIB = os.path.join(_HERE, "libhd_oracle.so")
_lib = None

OK, INVALID, CAPACITY, NUMERIC = 0, 1, 2, 3
BOUND_NAMES = ("exact", "u1", "u2", "u3", "u4", "kept")


class Stats(C.Structure):
    _fields_ = [("splits", C.c_int64), ("pointtri_evals", C.c_int64), ("discards", C.c_int64 * 6),
                ("max_queue", C.c_int64), ("iterations", C.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source (g++, OpenMP)."""
    stale = not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(__file__))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        # IEEE double with every operation rounded as written (no fused multiply-add
        # contraction, which g++ applies by default on some targets): the same results on x86
        # and Arm hosts
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", _SRC,
                               "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i64, i32, u8 = C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_uint8)
        _lib.or_point_triangle.argtypes = [d, d, d, d, d, d]
        _lib.or_nearest.argtypes = [d, i64, d, i64, i32, i64, d, i32, d]
        _lib.or_bounds_all.argtypes = [d, d, i32, d, d, i64, i32, i64, d]
        _lib.or_upper_bound.argtypes = [d, d, i32, d, d, i64, i32, i64, C.c_double, u8, C.c_int, C.POINTER(C.c_int)]
        _lib.or_upper_bound.restype = C.c_double
        _lib.or_hausdorff.argtypes = [d, i64, i32, i64, d, i64, i32, i64, C.c_double, C.c_int, C.c_double, u8,
                                      C.c_int, d, d, C.POINTER(Stats), d, i64, C.POINTER(C.c_int64)]
        _lib.or_hausdorff.restype = C.c_int
        _lib.or_sampling_bracket.argtypes = [d, i64, i32, i64, d, i64, i32, i64, C.c_int, d, d]
        _lib.or_num_threads.restype = C.c_int
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def num_threads() -> int:
    return lib().or_num_threads()


def point_triangle(p, a, b, c):
    """Distance from p to triangle (a, b, c) and the closest point."""
    bufs = [_d(x) for x in (p, a, b, c)]
    d = np.zeros(1)
    q = np.zeros(3)
    lib().or_point_triangle(*[x[1] for x in bufs], _d(d)[1], _d(q)[1])
    return float(d[0]), q


def nearest(P, VB, FB):
    """Brute-force d(p, B), nearest triangle index and closest point for each row of P."""
    P, pP = _d(np.reshape(P, (-1, 3)))
    VB, pV = _d(VB)
    FB, pF = _i(FB)
    n = len(P)
    d, idx, q = np.zeros(n), np.zeros(n, np.int32), np.zeros((n, 3))
    lib().or_nearest(pP, n, pV, len(VB), pF, len(FB), _d(d)[1], _i(idx)[1], _d(q)[1])
    return d, idx, q


def bounds_all(tv, td, tI, tq, VB, FB):
    """{exact (NaN unless one nearest triangle), u1, u2, u3, u4, g} of one triangle."""
    out = np.zeros(6)
    args = [_d(tv), _d(td), _i(tI), _d(tq)]
    VB, pV = _d(VB)
    FB, pF = _i(FB)
    lib().or_bounds_all(*[x[1] for x in args], pV, len(VB), pF, len(FB), _d(out)[1])
    return out


def upper_bound(tv, td, tI, tq, VB, FB, l, order=(1, 2, 3, 4)):
    """UpperBound(T, l): (U, deciding bound name)."""
    args = [_d(tv), _d(td), _i(tI), _d(tq)]
    VB, pV = _d(VB)
    FB, pF = _i(FB)
    o = np.ascontiguousarray(np.array(list(order) + [0] * (4 - len(order)), dtype=np.uint8))
    code = C.c_int(0)
    U = lib().or_upper_bound(*[x[1] for x in args], pV, len(VB), pF, len(FB), float(l),
                             o.ctypes.data_as(C.POINTER(C.c_uint8)), len(order), C.byref(code))
    return U, BOUND_NAMES[code.value]


def hausdorff(VA, FA, VB, FB, tol, tol_mode=0, max_face_factor=1e7, order=(1, 2, 3, 4), trace=False,
              max_trace=1 << 20):
    """Run the branch and bound.  Returns dict(lower, upper, status, stats, trace)."""
    VA, pVA = _d(VA)
    FA, pFA = _i(FA)
    VB, pVB = _d(VB)
    FB, pFB = _i(FB)
    o = np.ascontiguousarray(np.array(list(order) + [0] * (4 - len(order)), dtype=np.uint8))
    lo, up = np.zeros(1), np.zeros(1)
    st = Stats()
    tr = np.zeros((max_trace if trace else 1, 2))
    nt = C.c_int64(0)
    status = lib().or_hausdorff(pVA, len(VA), pFA, len(FA), pVB, len(VB), pFB, len(FB), float(tol), int(tol_mode),
                                float(max_face_factor), o.ctypes.data_as(C.POINTER(C.c_uint8)), len(order),
                                _d(lo)[1], _d(up)[1], C.byref(st), _d(tr)[1] if trace else None,
                                max_trace if trace else 0, C.byref(nt))
    stats = dict(splits=st.splits, pointtri_evals=st.pointtri_evals, iterations=st.iterations,
                 max_queue=st.max_queue, discards={BOUND_NAMES[k]: st.discards[k] for k in range(6)})
    return dict(lower=float(lo[0]), upper=float(up[0]), status=status, stats=stats,
                trace=tr[: nt.value].copy() if trace else None)


def sampling_bracket(VA, FA, VB, FB, k):
    """[max sampled d, max over faces (max sampled d + longest edge / k)], a bracket of h."""
    VA, pVA = _d(VA)
    FA, pFA = _i(FA)
    VB, pVB = _d(VB)
    FB, pFB = _i(FB)
    lo, hi = np.zeros(1), np.zeros(1)
    lib().or_sampling_bracket(pVA, len(VA), pFA, len(FA), pVB, len(VB), pFB, len(FB), int(k), _d(lo)[1],
                              _d(hi)[1])
    return float(lo[0]), float(hi[0])
