"""Work model of the PSDF kernels: algorithmic FP32 flops and bytes.

Counts follow the arithmetic the paper's stages require per (pose, edge)
pair (Sec. IV-A.3), as the scan kernel performs it: adds, subtracts and
multiplies count 1, fused multiply-adds 2; min/max, compares and selects
are not counted as flops.  Pose-invariant precompute (per-edge reciprocals,
footprint constants) is excluded.

Per edge of a closed polygon with an m-vertex footprint:
  stage 1 transform of the next vertex (2 sub, 2 mul, 2 fma)      8
  edge vector (2 sub)                                              2
  per robot vertex l (x m):
    w = v_l - A (2), projection dot (mul+fma 3), scale (1),
    residual (2 fma 4), |r|^2 (mul+fma 3)                         13
    robot projection on the edge normal (mul+fma)                  3
    obstacle vertex -> robot edge: t' (mul+fma+mul 4),
    residual (2 fma 4), |r'|^2 (3)                                11
    obstacle vertex on robot axis n_l (mul+fma)                    3
  overlap on the edge's own axis (2 fma)                           4
  => 14 + 30 m per edge, plus 2 m per obstacle (robot-axis overlaps).
A one-edge obstacle (segment): 22 + 50 m (both endpoints transformed, the
far-endpoint select, and the B endpoint's robot-edge and robot-axis terms).
"""
from __future__ import annotations

import numpy as np

FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (sm_100 family)


def flops_per_pose(m: int, offsets) -> float:
    counts = np.diff(np.asarray(offsets, dtype=np.int64))
    seg = counts == 1
    poly = ~seg
    f = float(np.sum(counts[poly] * (14 + 30 * m) + 2 * m)) + float(np.sum(seg)) * (22 + 50 * m)
    return f


def flops_evaluated(m: int, n_edges: int, n_obstacles: int) -> float:
    """Flops of the obstacles a cull evaluated exactly (closed polygons):
    14 + 30 m per edge plus 2 m per obstacle."""
    return float(n_edges) * (14 + 30 * m) + float(n_obstacles) * 2 * m


def flops_propose(bound_evaluations: int, circle_evaluations: int) -> float:
    """FP32 flops of the cull's proposal kernel: the squared distance to a
    tile's AABB (4 sub, 2 max, mul, fma: 7 counted) per tile bound it
    computed (both passes, as counted by the kernel) and one circle upper
    bound (2 sub, mul, fma, sqrt, 3 add, fma = 10) per obstacle circle of
    the proposed tiles.  The network's tensor-core flops are not FP32."""
    return 7.0 * bound_evaluations + 10.0 * circle_evaluations


def pair_flops_fixed(m: int) -> float:
    """The fixed per-(pose, edge) flop count of the hot path's stages,
    independent of any kernel: transform 14, vertex -> edge 16 m, edge
    vertex -> robot edge 14 m, robot-axis projections 5 m, obstacle-axis
    interval 5 m + 12; F(m) = 40 m + 26 (186 at m = 4, 346 at m = 8).  It
    counts work the kernels share across an edge's two ends or skip (the
    far-end clamps), so it exceeds the instruction-level count above."""
    return 40.0 * m + 26.0


def flops_fixed(m: int, pairs: float) -> float:
    """Flops of `pairs` evaluated (pose, edge) pairs by the fixed count."""
    return pair_flops_fixed(m) * float(pairs)


MLP_FLOPS_PER_ROW = (16 * 64 + 64 * 1) * 2  # one network score: 2,176 flops


def flops_network(rows: float) -> float:
    """Tensor-core flops of the tile-proposal network for `rows` scored
    (pose, tile) rows (16 -> 64 -> 1, FP16 operands)."""
    return MLP_FLOPS_PER_ROW * float(rows)


def fp32_peak_tflops(sms: int, sm_mhz: float) -> float:
    """Dense FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return sms * FP32_LANES_PER_SM * 2.0 * sm_mhz * 1e6 / 1e12


def scan_bytes(n_edges: int, n_obstacles: int, P: int, pose_blocks: int) -> float:
    """Algorithmic DRAM bytes of one full scan: poses in (12 B), keys out
    (8 B per pose), the edge records (32 B per edge + 16 B per obstacle)
    once; the CTAs' re-reads of the edge set hit L2."""
    return 12.0 * P + 8.0 * P + 32.0 * n_edges + 16.0 * n_obstacles
