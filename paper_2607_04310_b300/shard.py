"""Data-parallel sharding across ranks (one process per GPU).

The PSDF path shards without any exchange on the data path: the scene (or a
plan's instances' scenes) is replicated on every rank, the poses -- or whole
instances of a batched plan -- are partitioned, every rank evaluates its own
part on its own GPU, and results meet only on the host (a gather to rank 0).
Timing across ranks takes the maximum.  These helpers hold that host logic;
they run on any torch.distributed backend (gloo on CPU in the tests, NCCL for
CUDA tensors).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np


def shard_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [start, stop) of n items for `rank`; sizes differ by at most
    one, earlier ranks take the larger shares."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside world %d" % (rank, world))
    if n < 0:
        raise ValueError("n < 0")
    q, r = divmod(n, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def shard_instances(work: Sequence[float], world: int) -> List[int]:
    """Rank of every instance: largest work first onto the least loaded rank
    (longest-processing-time rule); ties go to the lower rank."""
    if world < 1:
        raise ValueError("world < 1")
    load = [0.0] * world
    owner = [0] * len(work)
    for i in sorted(range(len(work)), key=lambda k: (-float(work[k]), k)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += float(work[i])
    return owner


def gather_to_rank0(local: np.ndarray, group=None) -> Optional[np.ndarray]:
    """Concatenation of every rank's array in rank order on rank 0 (None on
    the others).  Host-side: arrays travel as objects, not on the data path."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    parts = [None] * world if rank == 0 else None
    dist.gather_object(np.ascontiguousarray(local), parts, dst=0, group=group)
    if rank != 0:
        return None
    return np.concatenate(parts, axis=0)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Maximum of a per-rank scalar (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
