"""Host logic of the multi-GPU path with world size 2 on CPU (gloo): sharding covers every
pair exactly once, the slowest rank's time is taken, and brackets gather on rank 0."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2406_10357_gb300 import multi  # noqa: E402


def test_shard_partitions_units():
    for n in (0, 1, 5, 1024):
        for size in (1, 2, 3, 8):
            got = sorted(i for r in range(size) for i in multi.shard(n, r, size))
            assert got == list(range(n))
            loads = [len(multi.shard(n, r, size)) for r in range(size)]
            assert max(loads) - min(loads) <= 1
    with pytest.raises(ValueError):
        multi.shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, size, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=size)
    try:
        assert multi.world() == (rank, size)
        # slowest rank's time
        t = multi.max_over_ranks(10.0 + 5.0 * rank)
        # fake per-pair brackets for this rank's shard (no GPU needed)
        n = 7
        idx = multi.shard(n, rank, size)
        br = [(float(i), float(i) + 0.5, 0.0) for i in idx]
        out = multi.gather_brackets(idx, br, n)
        if rank == 0:
            np.save(out_path, np.concatenate([[t, 0, 0]], 0).reshape(1, 3).tolist() + out.tolist())
        else:
            assert out is None
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo(tmp_path):
    out = str(tmp_path / "res.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    res = np.load(out)
    assert res[0, 0] == 15.0  # max over ranks
    gathered = res[1:]
    assert gathered.shape == (7, 3)
    assert np.allclose(gathered[:, 0], np.arange(7)) and np.allclose(gathered[:, 1], np.arange(7) + 0.5)


def test_shard_faces_covers_every_face():
    for n in (0, 1, 7, 1000):
        for size in (1, 2, 3, 5):
            blocks = [multi.shard_faces(n, r, size) for r in range(size)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(blocks[i][1] == blocks[i + 1][0] for i in range(size - 1))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1


def _face_worker(rank, size, port, out_path):
    import meshgen as mg
    import oracle as orc

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=size)
    try:
        p = mg.workload(2, 0.02)
        seen = {}

        def engine(VA, F, eps, l0):
            # the oracle brackets h(A_part, B); the contract is a bracket of max(l0, h)
            r = orc.hausdorff(VA, F, p.VB, p.FB, eps, 0)
            seen["eps"] = eps
            seen["l0"] = l0
            return max(l0, r["lower"]), max(l0, r["upper"]), r["status"]

        def lower_seed(VA, F):
            d, _, _ = orc.nearest(np.asarray(VA, float)[np.unique(F.ravel())], p.VB, p.FB)
            return float(d.max())

        lo, up, st, eps = multi.hausdorff_face_sharded(p.VA, p.FA, p.tol, p.tol_mode, engine, lower_seed)
        if rank == 0:
            np.save(out_path, np.array([lo, up, st, eps, seen["eps"], seen["l0"]]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_one_pair_face_sharded_two_ranks(tmp_path):
    """A's faces split over two gloo ranks, each bracketing its part with the oracle: the
    combined bracket is within eps (eps from the whole of A) and meets the oracle's bracket
    of the whole pair."""
    import meshgen as mg
    import oracle as orc

    out = str(tmp_path / "face.npy")
    mp.spawn(_face_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    lo, up, st, eps, eps_seen, l0 = np.load(out)
    p = mg.workload(2, 0.02)
    eps_full = p.tol * multi.referenced_diagonal(p.VA, p.FA)
    assert st == 0 and abs(eps - eps_full) <= 1e-15 * eps_full and eps_seen == eps
    assert up - lo <= eps * (1 + 1e-12)
    ref = orc.hausdorff(p.VA, p.FA, p.VB, p.FB, p.tol, p.tol_mode)
    assert max(lo, ref["lower"]) <= min(up, ref["upper"]) + 1e-12
    # the shared seed is the largest vertex distance of all of A, a lower bound of h
    d, _, _ = orc.nearest(np.asarray(p.VA, float), p.VB, p.FB)
    assert abs(l0 - d.max()) <= 1e-12 and l0 <= ref["upper"]
