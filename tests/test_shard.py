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


# ---------------------------------------------------------------------------
# edge sharding: every rank a consecutive range of obstacles, one all-reduce
# of the 64-bit keys, the owner of each pose's winning obstacle
# ---------------------------------------------------------------------------
def test_split_rows_covers_obstacles_once():
    from paper_2607_04310_b300 import scenegen as sg
    w = sg.octagon_lidar(1, n_inst=2, horizon=5, n_rects=300, n_lines=10, segs_per_line=20)
    for parts in (1, 2, 3, 8):
        sp = shard.split_rows(w.offsets, parts)
        assert sp[0][0] == 0 and sp[-1][1] == len(w.offsets) - 1
        for (o0, o1, r0, r1), nxt in zip(sp, sp[1:] + [None]):
            assert o0 <= o1 and r0 == w.offsets[o0] and r1 == w.offsets[o1]
            if nxt is not None:
                assert nxt[0] == o1
        rows = [r1 - r0 for _, _, r0, r1 in sp]
        assert sum(rows) == w.E and max(rows) - min(rows) <= 2 * 4 + w.E // 50
        e, o = shard.part_csr(w.edges, w.offsets, sp[-1])
        assert e.shape[0] == o[-1] and o[0] == 0


def _ordered_bits32(x):
    b = np.asarray(x, dtype=np.float32).copy()
    b += np.float32(0.0)  # -0 folded onto +0
    u = b.view(np.uint32).astype(np.uint64)
    return np.where(u & 0x80000000, (~u) & 0xFFFFFFFF, u | 0x80000000)


def _keys(sd, first_rows):
    """Per-pose minimum over the given obstacles of (ordered float32 value <<
    32 | rank), the min-key of Eq. psdf_value with its lowest-rank tie-break."""
    k = (_ordered_bits32(sd) << np.uint64(32)) | np.asarray(first_rows, dtype=np.uint64)[None, :]
    return k.min(axis=1) if k.shape[1] else np.full(sd.shape[0], ~np.uint64(0))


def _edge_worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2607_04310_b300 import scenegen as sg
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = sg.plain_rect_small(0)
        g = np.random.default_rng(5)
        poses = np.concatenate([w.poses, np.concatenate(
            [g.uniform(0, 20, size=(60, 2)), g.uniform(-3, 3, size=(60, 1))], axis=1)])
        parts = shard.split_rows(w.offsets, world)
        o0, o1, r0, r1 = parts[rank]
        # this rank's obstacles only: their signed distances by the oracle
        sd = oracle.obstacle_sd(w.footprint, w.edges, w.offsets, poses)[:, o0:o1]
        local = _keys(sd, np.asarray(w.offsets[o0:o1]))
        t = torch.as_tensor(local.view(np.int64).copy())
        shard.allreduce_min_keys(t)
        if rank == 0:
            np.save(out_path, t.numpy())
    finally:
        dist.destroy_process_group()


def test_edge_sharded_key_minimum_over_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    from paper_2607_04310_b300 import scenegen as sg
    out = str(tmp_path / "keys.npy")
    world = 2
    mp.spawn(_edge_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    merged = np.load(out).view(np.uint64)
    # the whole scene on one rank
    w = sg.plain_rect_small(0)
    g = np.random.default_rng(5)
    poses = np.concatenate([w.poses, np.concatenate(
        [g.uniform(0, 20, size=(60, 2)), g.uniform(-3, 3, size=(60, 1))], axis=1)])
    sd = oracle.obstacle_sd(w.footprint, w.edges, w.offsets, poses)
    whole = _keys(sd, np.asarray(w.offsets[:-1]))
    assert np.array_equal(merged, whole)
    # the value and the obstacle the key names are the oracle's minimum
    ref = oracle.psdf_eval(w.footprint, w.edges, w.offsets, poses)
    assert np.array_equal((merged >> np.uint64(32)), _ordered_bits32(ref["phi"]))
    rank = (merged & np.uint64(0xFFFFFFFF)).astype(np.int64)
    obst = np.searchsorted(np.asarray(w.offsets), rank, side="right") - 1
    assert np.array_equal(sd[np.arange(len(poses)), obst].astype(np.float32),
                          ref["phi"].astype(np.float32))
    # the owner of each pose is the part whose rows hold the winning obstacle
    parts = shard.split_rows(w.offsets, world)
    own = shard.owner(merged.view(np.int64), parts)
    for i, (o0, o1, _r0, _r1) in enumerate(parts):
        sel = own == i
        assert np.all((obst[sel] >= o0) & (obst[sel] < o1))
    assert np.all(own >= 0)


def test_key_order_conversion_round_trips():
    g = np.random.default_rng(1)
    k = g.integers(0, 2 ** 63, size=1000, dtype=np.uint64) * np.uint64(2) + \
        g.integers(0, 2, size=1000, dtype=np.uint64)
    k[:3] = [0, ~np.uint64(0), np.uint64(1) << np.uint64(63)]
    o = shard.keys_to_ordered(k.view(np.int64))
    assert np.array_equal(shard.keys_from_ordered(o).view(np.uint64), k)
    assert np.array_equal(np.argsort(o, kind="stable"), np.argsort(k, kind="stable"))
