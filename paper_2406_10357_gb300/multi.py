"""Several GPUs: independent pairs sharded over ranks (one process per GPU).

The unit of work is one (A, B) pair; pairs never exchange data, so ranks need no collective
on the data path.  The only collectives are bookkeeping: the slowest rank's time for
throughput, and the gather of each pair's bracket (two doubles) on rank 0.  Works with any
torch.distributed backend (nccl between GPUs, gloo on CPU for tests).
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
