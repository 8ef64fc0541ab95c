"""Pick launch and build parameters by timing them on a sample of the user's own pairs.

The parameters are the threads per block of the round kernels, the BVH leaf size and the
frontier chunk (most sub-triangles split per round); optionally also the cascade order of the
upper bounds (the paper's order u1, u2, u3, u4 stays the default: a different order changes
which bounds run, not the validity of the bracket).  Every candidate runs the same batched
call, hd_hausdorff_batched, on the sample; the one with the least median time wins.

    opt, table = autotune(sample, tol, precision=hd.HD_MIXED)
"""
from __future__ import annotations

import itertools
import time

BLOCK_SIZES = (32, 64, 128)
LEAF_SIZES = (1, 2, 4)
CHUNKS = (0, 16384)  # 0: the library's automatic chunk
ORDERS = ((1, 2, 3, 4), (1, 3), (3,), (2, 3), (1, 3, 4))


def candidates(tune_order: bool = False):
    """The option sets tried: every combination of the grids above (orders only if asked)."""
    orders = ORDERS if tune_order else (ORDERS[0],)
    return [dict(block_size=b, leaf_size=l, frontier_chunk=c, bound_order=o)
            for b, l, c, o in itertools.product(BLOCK_SIZES, LEAF_SIZES, CHUNKS, orders)]


def autotune(sample, tol: float, precision: int, tol_mode: int | None = None, tune_order: bool = False,
             reps: int = 3):
    """sample: list of (VA, FA, VB, FB) device tensors.  Returns (best HdOptions, table), the
    table listing every candidate with its median time over `reps` calls."""
    import torch

    import paper_2406_10357_gb300 as hd

    mode = hd.HD_TOL_REL if tol_mode is None else tol_mode
    table = []
    by_leaf = {}
    for cand in candidates(tune_order):
        leaf = cand["leaf_size"]
        if leaf not in by_leaf:  # the BVHs depend on the leaf size only
            ob = hd.hd_options_default(leaf_size=leaf)
            by_leaf[leaf] = [hd.hd_build_B(VB, FB, ob) for (_, _, VB, FB) in sample]
        o = hd.hd_options_default(tol_mode=mode, precision=precision, **cand)
        As = [(VA, FA) for (VA, FA, _, _) in sample]
        hd.hd_hausdorff_batched(by_leaf[leaf], As, tol, o)  # warm-up
        ts = []
        ok = True
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rs = hd.hd_hausdorff_batched(by_leaf[leaf], As, tol, o)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            ok = ok and all(r["status"] == hd.HD_OK for r in rs)
        ts.sort()
        table.append(dict(cand, bound_order=list(cand["bound_order"]), seconds=ts[len(ts) // 2], all_ok=ok))
    good = [r for r in table if r["all_ok"]] or table
    best = min(good, key=lambda r: r["seconds"])
    opt = hd.hd_options_default(tol_mode=mode, precision=precision, block_size=best["block_size"],
                                leaf_size=best["leaf_size"], frontier_chunk=best["frontier_chunk"],
                                bound_order=best["bound_order"])
    return opt, table
