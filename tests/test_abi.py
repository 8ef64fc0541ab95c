"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/hd.h declares.  No GPU work is launched here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hd():
    from paper_2406_10357_gb300 import build

    build.build()
    import paper_2406_10357_gb300 as hd

    hd.lib()
    return hd


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hd_[A-Za-z_0-9]+)\s*\(", text)))


def _has_gpu():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def test_every_declared_symbol_is_exported(hd):
    names = declared_symbols()
    assert {"hd_build_B", "hd_hausdorff", "hd_hausdorff_batched", "hd_free_B", "hd_status_str"} <= set(names)
    L = C.CDLL(hd.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_struct_layouts_match_header(hd):
    # sizes of the ABI structs as laid out by a C compiler for this header
    assert C.sizeof(hd.HdMesh) == 40
    assert C.sizeof(hd.HdOptions) == 64
    assert C.sizeof(hd.HdStats) == 8 * 26
    assert C.sizeof(hd.HdResult) == 24 + 8 * 26
    assert C.sizeof(hd.HdTrace) == 128


def test_options_default_and_status_strings(hd):
    o = hd.hd_options_default()
    assert o.tol_mode == hd.HD_TOL_ABS and o.precision == hd.HD_FP64
    assert o.max_face_factor == 1e7 and list(o.bound_order) == [1, 2, 3, 4] and o.n_bounds == 4
    assert o.leaf_size == 1 and o.block_size == 64
    assert hd.hd_status_str(hd.HD_ERR_CAPACITY) == "HD_ERR_CAPACITY"
    assert hd.hd_status_str(99) == "HD_UNKNOWN"


def test_invalid_arguments_rejected_before_any_launch(hd):
    L = hd.lib()
    r = hd.HdResult()
    assert L.hd_hausdorff(None, None, 1e-3, None, None, C.byref(r)) == hd.HD_ERR_INVALID
    out = C.c_void_p(0)
    assert L.hd_build_B(None, None, None, C.byref(out)) == hd.HD_ERR_INVALID
    m = hd.HdMesh(0, 0, 0, 0, 0, 0)
    assert L.hd_build_B(C.byref(m), None, None, C.byref(out)) == hd.HD_ERR_INVALID
    bad = hd.hd_options_default(leaf_size=40)
    assert L.hd_build_B(C.byref(m), C.byref(bad), None, C.byref(out)) == hd.HD_ERR_INVALID
    # a valid host mesh: unknown flag bits or a nonzero reserved field are rejected before
    # any CUDA call (a good option set gets past validation)
    V = np.zeros((3, 3), np.float64)
    V[1, 0] = V[2, 1] = 1.0
    Fi = np.array([[0, 1, 2]], np.int32)
    mv = hd.HdMesh(V.ctypes.data, 3, Fi.ctypes.data, 1, hd.HD_F64, 0)
    for b in (hd.hd_options_default(flags=128), hd.hd_options_default(reserved=1)):
        assert L.hd_build_B(C.byref(mv), C.byref(b), None, C.byref(out)) == hd.HD_ERR_INVALID
    if not _has_gpu():
        good = hd.hd_options_default(flags=hd.HD_FLAG_NO_PARENT_CLAMP)
        assert L.hd_build_B(C.byref(mv), C.byref(good), None, C.byref(out)) == hd.HD_ERR_CUDA


def test_noalloc_limit_matches_header(hd):
    text = open(os.path.join(ROOT, "include", "hd.h")).read()
    m = re.search(r"#define\s+HD_NOALLOC_MAX_POINTS\s+(\d+)", text)
    assert m and int(m.group(1)) == hd.HD_NOALLOC_MAX_POINTS
    assert "hd_nearest_noalloc" in declared_symbols()


def test_noalloc_invalid_arguments_rejected_before_any_launch(hd):
    """Every check below returns before the handle is read or any CUDA call is made (the
    non-null handle is a dummy host buffer that is never dereferenced)."""
    L = hd.lib()
    dummy = (C.c_char * 64)()
    B = C.cast(dummy, C.c_void_p)
    buf = (C.c_double * 8)()
    p = C.cast(buf, C.c_void_p)
    args = lambda b, ptype, n, prec: (b, p, ptype, n, prec, None, p, p, p, p)
    assert L.hd_nearest_noalloc(*args(None, hd.HD_F64, 1, hd.HD_FP64)) == hd.HD_ERR_INVALID
    assert L.hd_nearest_noalloc(*args(B, hd.HD_F64, -1, hd.HD_FP64)) == hd.HD_ERR_INVALID
    assert L.hd_nearest_noalloc(*args(B, hd.HD_F64, hd.HD_NOALLOC_MAX_POINTS + 1, hd.HD_FP64)) == hd.HD_ERR_INVALID
    assert L.hd_nearest_noalloc(*args(B, 7, 1, hd.HD_FP64)) == hd.HD_ERR_INVALID
    assert L.hd_nearest_noalloc(*args(B, hd.HD_F32, 1, 9)) == hd.HD_ERR_INVALID
    assert L.hd_nearest_noalloc(B, None, hd.HD_F64, 1, hd.HD_FP64, None, p, p, p, p) == hd.HD_ERR_INVALID


def test_noalloc_binding_checks_before_any_launch(hd):
    """The Python binding refuses points that are not an (n, 3) CUDA tensor and output tensors
    of the wrong type, size, layout or device, before it calls the library."""
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        hd.hd_nearest_noalloc(None, torch.zeros((4, 3), dtype=torch.float64))
    with pytest.raises(ValueError):
        hd.hd_nearest(None, np.zeros((4, 3)))
    dev = torch.device("cpu")
    good = (torch.zeros(5, dtype=torch.float64), torch.zeros(5, dtype=torch.int32), torch.zeros((5, 3), dtype=torch.float64),
            torch.zeros(5, dtype=torch.float64))
    hd._check_out(good, 5, dev)
    bad = [
        (good[0][:4], *good[1:]),                                   # too small
        (good[0].float(), *good[1:]),                               # wrong type
        (good[0], good[1].long(), *good[2:]),                       # wrong index type
        (good[0], good[1], torch.zeros((3, 5), dtype=torch.float64).t(), good[3]),  # not contiguous
        good[:3],                                                   # missing dist_lo
    ]
    for out in bad:
        with pytest.raises(ValueError):
            hd._check_out(out, 5, dev)
    with pytest.raises(ValueError):
        hd._check_out(good, 5, torch.device("meta"))
