"""Sharding across ranks (one process per GPU).

Two ways.  By poses: the scene (or a plan's instances' scenes) is replicated
on every rank, the poses -- or whole instances of a batched plan -- are
partitioned, every rank evaluates its own part on its own GPU, and results
meet only on the host (a gather to rank 0); no exchange on the data path.
By edges, for edge sets too large for one GPU: each rank holds a
consecutive range of the obstacles (split_rows) as a scene part, computes its
per-pose 64-bit keys (psdf_eval_keys), one all-reduce takes their minimum
(allreduce_min_keys), and the rank that holds each pose's winning obstacle
runs its epilogue (psdf_finish_keys with owner()).  Timing across ranks takes
the maximum.  These helpers hold the host logic; they run on any
torch.distributed backend (gloo on CPU in the tests, NCCL for CUDA tensors).
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


# --------------------------------------------------------------------------
# edge sharding: scene parts, key minimum, owner of each pose
# --------------------------------------------------------------------------
def split_rows(offsets, parts: int) -> List[Tuple[int, int, int, int]]:
    """Consecutive obstacle ranges of a CSR edge set for `parts` ranks, of
    about equal row (edge) counts: (first obstacle, end obstacle, first row,
    end row) per part; empty parts when there are fewer obstacles than
    parts."""
    off = np.asarray(offsets, dtype=np.int64)
    M = len(off) - 1
    if parts < 1:
        raise ValueError("parts < 1")
    E = int(off[-1]) if M > 0 else 0
    bounds = [0]
    for r in range(1, parts):
        target = E * r / parts
        i = int(np.searchsorted(off, target, side="left"))
        bounds.append(min(max(i, bounds[-1]), M))
    bounds.append(M)
    return [(bounds[r], bounds[r + 1], int(off[bounds[r]]) if M > 0 else 0,
             int(off[bounds[r + 1]]) if M > 0 else 0) for r in range(parts)]


def part_csr(edges, offsets, part) -> Tuple[np.ndarray, np.ndarray]:
    """The edge rows and rebased offsets of one part from split_rows."""
    o0, o1, r0, r1 = part
    off = np.asarray(offsets, dtype=np.int64)
    return (np.ascontiguousarray(np.asarray(edges, dtype=np.float32)[r0:r1]),
            (off[o0:o1 + 1] - r0).astype(np.int32))


_SIGN = np.int64(-0x8000000000000000)


def keys_to_ordered(keys_i64):
    """Unsigned 64-bit keys held in int64 (numpy or torch) -> int64 values
    that order as the unsigned keys do (top bit flipped)."""
    return keys_i64 ^ _SIGN if isinstance(keys_i64, np.ndarray) else keys_i64 ^ int(_SIGN)


def keys_from_ordered(ordered_i64):
    return keys_to_ordered(ordered_i64)


def allreduce_min_keys(keys_i64, group=None):
    """In place: every rank's keys (an int64 tensor holding the unsigned key
    bits) become their minimum over the ranks -- the whole scene's keys."""
    import torch.distributed as dist
    keys_i64.copy_(keys_to_ordered(keys_i64))
    dist.all_reduce(keys_i64, op=dist.ReduceOp.MIN, group=group)
    keys_i64.copy_(keys_from_ordered(keys_i64))
    return keys_i64


def owner(keys_i64: np.ndarray, parts) -> np.ndarray:
    """The part holding each pose's winning obstacle (its key's rank within
    the part's rows), -1 for a key that names no obstacle."""
    k = np.asarray(keys_i64).astype(np.int64)
    rank = k & 0xFFFFFFFF
    none = k == -1
    out = np.full(k.shape, -1, dtype=np.int64)
    for i, (_o0, _o1, r0, r1) in enumerate(parts):
        out[(~none) & (rank >= r0) & (rank < r1)] = i
    return out
