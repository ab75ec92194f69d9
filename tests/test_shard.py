"""Host logic of the data-parallel path on world_size-2 gloo process groups
(CPU): pose ranges cover every pose once, instance assignment balances work,
results gather on rank 0 in rank order, times reduce to the maximum."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

from paper_2607_04310_b300 import shard


def test_shard_range_covers_once():
    for n in (0, 1, 7, 1003, 4096):
        for world in (1, 2, 3, 8):
            seen = np.zeros(n, dtype=int)
            sizes = []
            for r in range(world):
                a, b = shard.shard_range(n, r, world)
                seen[a:b] += 1
                sizes.append(b - a)
            assert np.all(seen == 1)
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


def test_shard_instances_balances_work():
    g = np.random.default_rng(0)
    work = np.exp(g.uniform(np.log(16), np.log(65536), size=1024)) * g.integers(10, 101, 1024)
    owner = shard.shard_instances(work, 8)
    load = np.bincount(owner, weights=work, minlength=8)
    assert load.max() <= load.mean() + work.max()  # LPT bound
    assert load.max() / load.mean() < 1.05


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, b = shard.shard_range(n, rank, world)
        # stand-in for the rank's results: a function of the global pose index
        local = np.stack([np.arange(a, b, dtype=np.float64) ** 0.5,
                          np.full(b - a, rank, dtype=np.float64)], axis=1)
        full = shard.gather_to_rank0(local)
        t = shard.max_over_ranks(1.0 + rank)
        if rank == 0:
            np.save(out_path, full)
            with open(out_path + ".t", "w") as f:
                f.write(repr(t))
        else:
            assert full is None
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_gather_and_max_over_gloo_ranks(tmp_path, world):
    import torch.multiprocessing as mp
    n = 1001
    out = str(tmp_path / "full.npy")
    mp.spawn(_worker, args=(world, _free_port(), n, out), nprocs=world, join=True)
    full = np.load(out)
    assert full.shape == (n, 2)
    assert np.array_equal(full[:, 0], np.arange(n, dtype=np.float64) ** 0.5)
    # rank order: rank 0's range first
    a1, _ = shard.shard_range(n, 1, world)
    assert np.all(full[:a1, 1] == 0) and np.all(full[a1:, 1] == 1)
    with open(out + ".t") as f:
        assert float(f.read()) == float(world)
