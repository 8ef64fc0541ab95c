"""Several GPUs (one process per GPU), two ways.

Independent pairs: the unit of work is one (A, B) pair; pairs never exchange data, so ranks
need no collective on the data path.  The only collectives are bookkeeping: the slowest
rank's time for throughput, and the gather of each pair's bracket (two doubles) on rank 0.

One pair split over ranks: A's faces are partitioned and B (with its BVH) is replicated.
h(A, B) is the maximum of h(A_r, B) over the parts, so each rank brackets its part alone;
the ranks exchange only a lower bound before (the largest vertex distance of any part, a
lower bound of h(A, B) that lets every rank discard sub-triangles bounded below it) and
(l, u, status) after.  Every rank's gap is within eps, hence so is the maximum's.

Works with any torch.distributed backend (nccl between GPUs, gloo on CPU for tests).
"""
from __future__ import annotations

import numpy as np


def world():
    """(rank, world size) of the default process group, or (0, 1) without one."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def shard(n_units: int, rank: int, size: int) -> list[int]:
    """Round-robin share of units [0, n_units) for `rank` of `size` ranks: every unit goes to
    exactly one rank, and rank loads differ by at most one unit."""
    if size < 1 or not 0 <= rank < size:
        raise ValueError("bad rank/size")
    return list(range(rank, n_units, size))


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a scalar over all ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist

    rank, size = world()
    if size == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_brackets(local_idx: list[int], local_brackets, n_units: int, device=None):
    """Rank 0 receives an (n_units, 3) array [lower, upper, status] assembled from every
    rank's shard; other ranks receive None."""
    import torch
    import torch.distributed as dist

    rank, size = world()
    mine = np.full((n_units, 3), np.nan)
    for i, b in zip(local_idx, local_brackets):
        mine[i] = b
    if size == 1:
        return mine
    t = torch.from_numpy(mine).to(device=device)
    parts = [torch.empty_like(t) for _ in range(size)] if rank == 0 else None
    dist.gather(t, parts, dst=0)
    if rank != 0:
        return None
    out = np.full((n_units, 3), np.nan)
    for p in parts:
        p = p.cpu().numpy()
        have = ~np.isnan(p[:, 0])
        out[have] = p[have]
    return out


def hausdorff_sharded(pairs, tol: float, opt=None, device=None):
    """h(A_i, B_i) for a list of pairs (objects with VA, FA, VB, FB), each rank computing its
    round-robin shard on its own GPU; returns the gathered [lower, upper, status] rows on
    rank 0 (None elsewhere)."""
    import paper_2406_10357_gb300 as hd

    rank, size = world()
    idx = shard(len(pairs), rank, size)
    res = []
    for i in idx:
        p = pairs[i]
        bvh = hd.hd_build_B(p.VB, p.FB)
        r = hd.hd_hausdorff(bvh, p.VA, p.FA, tol, opt)
        res.append((r["lower"], r["upper"], float(r["status"])))
    return gather_brackets(idx, res, len(pairs), device=device)


def shard_faces(n_faces: int, rank: int, size: int) -> tuple[int, int]:
    """Contiguous block [lo, hi) of A's faces for `rank` of `size` (meshes list neighbouring
    faces together, so blocks keep each rank's traversals coherent); blocks cover every face
    once and differ in size by at most one."""
    if size < 1 or not 0 <= rank < size:
        raise ValueError("bad rank/size")
    q, r = divmod(n_faces, size)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def referenced_diagonal(VA, FA) -> float:
    """Bounding-box diagonal of A's referenced vertices (the dA of a relative tolerance)."""
    R = np.asarray(VA, dtype=np.float64)[np.unique(np.asarray(FA).ravel())]
    return float(np.linalg.norm(R.max(0) - R.min(0)))


def hausdorff_face_sharded(VA, FA, tol: float, tol_mode: int, engine, lower_seed=None, device=None):
    """Bracket [lower, upper] of h(A, B) with A's faces split over the ranks.

    engine(VA, F_part, eps_abs, l0) -> (lower, upper, status) brackets max(l0, h(A_part, B))
    on this rank (hd_hausdorff_from on the GPU); lower_seed(VA, F_part) -> a certified lower
    bound of h(A_part, B), e.g. the largest vertex distance (None: 0).  The tolerance is made
    absolute from the whole of A, so that every rank works to the same eps.  Returns
    (lower, upper, status, eps_abs) on every rank; status is the largest of the ranks'."""
    rank, size = world()
    FA = np.asarray(FA)
    eps = tol * referenced_diagonal(VA, FA) if tol_mode else tol
    lo, hi = shard_faces(len(FA), rank, size)
    part = FA[lo:hi]
    l0 = max_over_ranks(float(lower_seed(VA, part)) if (lower_seed and len(part)) else 0.0, device=device)
    if len(part):
        l_r, u_r, st = engine(VA, part, eps, l0)
    else:
        l_r, u_r, st = l0, l0, 0
    lower = max_over_ranks(max(l_r, l0), device=device)
    upper = max_over_ranks(max(u_r, l0), device=device)
    status = max_over_ranks(float(st), device=device)
    return lower, upper, int(status), eps


def gpu_engine(bvh, opt=None):
    """engine and lower_seed for hausdorff_face_sharded on this rank's GPU."""
    import paper_2406_10357_gb300 as hd

    def engine(VA, F, eps, l0):
        o = opt if opt is not None else hd.hd_options_default()
        o.tol_mode = hd.HD_TOL_ABS
        r = hd.hd_hausdorff_from(bvh, VA, F, eps, l0, o)
        return r["lower"], r["upper"], r["status"]

    def lower_seed(VA, F):
        import torch

        o = opt if opt is not None else hd.hd_options_default()
        P = torch.from_numpy(np.ascontiguousarray(np.asarray(VA, np.float64)[np.unique(F.ravel())])).cuda()
        d, _, _, dlo = hd.hd_nearest(bvh, P, o.precision)
        # less a 1e-12 relative margin: points given as doubles are split into float pairs
        # by rounding (about 2^-48 relative), which the certified bound does not cover
        return float(dlo.max().item()) * (1.0 - 1e-12)

    return engine, lower_seed
