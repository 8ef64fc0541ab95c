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
