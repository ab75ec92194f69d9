"""Seeded synthetic inputs for the PSDF hot path.

This module only *builds inputs*: robot footprints, obstacle edge sets and
pose batches, shaped like the workloads of the paper (random obstacle sets
and query poses, Sec. VI-B; LiDAR line-fitted obstacles, Sec. VI-D;
MPC horizons of poses, Sec. V-B).  It contains none of the signed-distance
arithmetic, so both the CUDA path and the CPU oracle can draw from it.

Conventions
-----------
* footprint: float32 [m, 2], counter-clockwise, robot-local frame (Sec. IV-A.1).
* edges:     float32 [E, 4] rows (Ax, Ay, Bx, By) in the world frame.
* offsets:   int32 [M + 1]; obstacle i owns edges offsets[i] .. offsets[i+1]-1.
  An obstacle is either a closed convex CCW polygon (>= 3 edges, B_j equal to
  the next edge's A bit for bit) or a single segment (1 edge).
* poses:     float32 [P, 3] rows (x, y, theta).

Every generator takes a seed (or a numpy Generator) so results are
reproducible bit for bit (numpy PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

F32 = np.float32


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------
# footprints (convex, CCW, local frame)
# --------------------------------------------------------------------------
def footprint_rect(width: float = 0.6, height: float = 0.4) -> np.ndarray:
    """Axis-aligned rectangle centred at the pose origin (Fig. 2 robots)."""
    a, b = width / 2.0, height / 2.0
    return np.array([[-a, -b], [a, -b], [a, b], [-a, b]], dtype=F32)


def footprint_regular(k: int, radius: float, phase: float = 0.0) -> np.ndarray:
    """Regular k-gon of circumradius `radius`.

    For even k the second half of the vertex list is the exact negation of
    the first half, so opposite edges are exactly antiparallel in float32.
    """
    ang = phase + 2.0 * math.pi * np.arange(k) / k
    v = np.stack([radius * np.cos(ang), radius * np.sin(ang)], axis=1).astype(F32)
    if k % 2 == 0:
        v[k // 2:] = -v[: k // 2]
    return v


def footprint_random_convex(g: np.random.Generator, k: int, rmin: float = 0.3,
                            rmax: float = 0.6, min_gap: float = 0.15) -> np.ndarray:
    """k points at sorted random angles on a circle (convex by construction).

    Angles are redrawn until consecutive gaps exceed `min_gap` radians, which
    keeps every edge well above the degenerate-length threshold.
    """
    if k < 3:
        raise ValueError("a convex footprint needs at least 3 vertices")
    r = g.uniform(rmin, rmax)
    while True:
        ang = np.sort(g.uniform(-math.pi, math.pi, size=k))
        gaps = np.diff(np.concatenate([ang, ang[:1] + 2 * math.pi]))
        if gaps.min() > min_gap and gaps.max() < math.pi - 1e-3:
            break
    return np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1).astype(F32)


# --------------------------------------------------------------------------
# obstacle edge sets
# --------------------------------------------------------------------------
def _csr_from_polygons(polys: Sequence[np.ndarray]) -> Tuple[np.ndarray, np.ndarray]:
    """Closed polygons (float32 [n_i, 2] CCW vertex lists) -> CSR edges."""
    counts = np.array([len(p) for p in polys], dtype=np.int64)
    offs = np.zeros(len(polys) + 1, dtype=np.int32)
    offs[1:] = np.cumsum(counts)
    edges = np.empty((int(offs[-1]), 4), dtype=F32)
    for i, p in enumerate(polys):
        s = offs[i]
        n = len(p)
        edges[s:s + n, 0:2] = p
        edges[s:s + n, 2:4] = np.roll(p, -1, axis=0)
    return edges, offs


def regular_polygons(centres: Sequence[Tuple[float, float]], ks: Sequence[int],
                     radii: Sequence[float]) -> Tuple[np.ndarray, np.ndarray]:
    """Regular k-gons (CCW) at the given centres, as CSR edges; closure is
    exact (B of an edge is the next edge's A bit for bit)."""
    polys = [(footprint_regular(k, r).astype(np.float64) + np.asarray(c)).astype(F32)
             for c, k, r in zip(centres, ks, radii)]
    return _csr_from_polygons(polys)


def rects(g: np.random.Generator, n: int, side_lo: float, side_hi: float,
          field_lo: float, field_hi: float,
          field_hi_y: Optional[float] = None) -> Tuple[np.ndarray, np.ndarray]:
    """n random-yaw rectangles: sides U[side_lo, side_hi], centres uniform in
    the field, yaw U[-pi, pi].  Four CCW edges each; closure is exact."""
    fy = field_hi if field_hi_y is None else field_hi_y
    cx = g.uniform(field_lo, field_hi, size=n)
    cy = g.uniform(field_lo, fy, size=n)
    w = g.uniform(side_lo, side_hi, size=n)
    h = g.uniform(side_lo, side_hi, size=n)
    yaw = g.uniform(-math.pi, math.pi, size=n)
    loc = np.array([[-0.5, -0.5], [0.5, -0.5], [0.5, 0.5], [-0.5, 0.5]])
    c, s = np.cos(yaw), np.sin(yaw)
    lx = loc[None, :, 0] * w[:, None]
    ly = loc[None, :, 1] * h[:, None]
    X = cx[:, None] + c[:, None] * lx - s[:, None] * ly
    Y = cy[:, None] + s[:, None] * lx + c[:, None] * ly
    verts = np.stack([X, Y], axis=2).astype(F32)          # [n, 4, 2]
    edges = np.empty((n, 4, 4), dtype=F32)
    edges[:, :, 0:2] = verts
    edges[:, :, 2:4] = np.roll(verts, -1, axis=1)
    offs = (4 * np.arange(n + 1)).astype(np.int32)
    return edges.reshape(4 * n, 4), offs


def convex_polygons(g: np.random.Generator, n: int, kmin: int, kmax: int,
                    rad_lo: float, rad_hi: float, field_lo: float,
                    field_hi: float) -> Tuple[np.ndarray, np.ndarray]:
    """n random convex polygons (k in [kmin, kmax] points on a circle at
    sorted random angles), generally without parallel edges."""
    polys = []
    for _ in range(n):
        k = int(g.integers(kmin, kmax + 1))
        fp = footprint_random_convex(g, k, rad_lo, rad_hi,
                                     min_gap=min(0.3, math.pi / k))
        c = g.uniform(field_lo, field_hi, size=2)
        polys.append((fp.astype(np.float64) + c).astype(F32))
    return _csr_from_polygons(polys)


def polyline_segments(g: np.random.Generator, n_lines: int, segs_per_line: int,
                      len_lo: float, len_hi: float, field_lo: float,
                      field_hi: float, dtheta: float = math.pi / 6
                      ) -> Tuple[np.ndarray, np.ndarray]:
    """LiDAR-like line segments: random walks whose heading turns by
    U[-dtheta, dtheta] per step.  Every segment is its own one-edge obstacle;
    consecutive segments share an endpoint bit for bit."""
    segs = []
    for _ in range(n_lines):
        p = g.uniform(field_lo, field_hi, size=2)
        hd = g.uniform(-math.pi, math.pi)
        pts = [p.copy()]
        for _k in range(segs_per_line):
            hd += g.uniform(-dtheta, dtheta)
            L = g.uniform(len_lo, len_hi)
            p = p + L * np.array([math.cos(hd), math.sin(hd)])
            pts.append(p.copy())
        pts = np.asarray(pts).astype(F32)
        e = np.concatenate([pts[:-1], pts[1:]], axis=1)
        segs.append(e)
    edges = np.concatenate(segs, axis=0).astype(F32)
    offs = np.arange(edges.shape[0] + 1, dtype=np.int32)
    return edges, offs


def concat(*parts: Tuple[np.ndarray, np.ndarray]) -> Tuple[np.ndarray, np.ndarray]:
    """Concatenate CSR edge sets (obstacle order is preserved)."""
    edges = np.concatenate([p[0] for p in parts], axis=0).astype(F32)
    offs = [np.zeros(1, dtype=np.int64)]
    base = 0
    for e, o in parts:
        offs.append(o[1:].astype(np.int64) + base)
        base += e.shape[0]
    return edges, np.concatenate(offs).astype(np.int32)


def to_padded(edges: np.ndarray, offs: np.ndarray, mbar: Optional[int] = None
              ) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """CSR -> the paper's padded tensors A, B [Mbar, mbar, 2] and mask S
    [Mbar, mbar] (Sec. IV-A.2).  Valid entries come first in each row."""
    M = len(offs) - 1
    counts = np.diff(offs)
    mb = int(counts.max()) if mbar is None else int(mbar)
    A = np.zeros((M, mb, 2), dtype=F32)
    B = np.zeros((M, mb, 2), dtype=F32)
    S = np.zeros((M, mb), dtype=np.uint8)
    for i in range(M):
        n = counts[i]
        A[i, :n] = edges[offs[i]:offs[i + 1], 0:2]
        B[i, :n] = edges[offs[i]:offs[i + 1], 2:4]
        S[i, :n] = 1
    return A, B, S


# --------------------------------------------------------------------------
# poses
# --------------------------------------------------------------------------
def poses_uniform(g: np.random.Generator, n: int, lo: float, hi: float,
                  hi_y: Optional[float] = None) -> np.ndarray:
    hy = hi if hi_y is None else hi_y
    x = g.uniform(lo, hi, size=n)
    y = g.uniform(lo, hy, size=n)
    th = g.uniform(-math.pi, math.pi, size=n)
    return np.stack([x, y, th], axis=1).astype(F32)


def poses_paths(g: np.random.Generator, n_inst: int, horizon: int, lo: float,
                hi: float, step: float = 0.1, dtheta: float = 0.1) -> np.ndarray:
    """MPC-rollout-like horizons: each instance starts uniformly in the field
    with a random heading and advances `step` metres per stage while the
    heading random-walks by U[-dtheta, dtheta]."""
    out = np.empty((n_inst, horizon, 3), dtype=np.float64)
    for i in range(n_inst):
        p = g.uniform(lo, hi, size=2)
        th = g.uniform(-math.pi, math.pi)
        for k in range(horizon):
            out[i, k] = (p[0], p[1], th)
            p = p + step * np.array([math.cos(th), math.sin(th)])
            th += g.uniform(-dtheta, dtheta)
    th = out[:, :, 2]
    out[:, :, 2] = (th + math.pi) % (2 * math.pi) - math.pi
    return out.reshape(n_inst * horizon, 3).astype(F32)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    footprint: np.ndarray
    edges: np.ndarray
    offsets: np.ndarray
    poses: np.ndarray
    info: Dict = field(default_factory=dict)

    @property
    def P(self) -> int:
        return int(self.poses.shape[0])

    @property
    def E(self) -> int:
        return int(self.edges.shape[0])

    @property
    def M(self) -> int:
        return int(len(self.offsets) - 1)


def plain_rect_small(seed: int = 0) -> Workload:
    """Rectangle footprint 0.6 x 0.4, N = 20 poses uniform in [0, 20]^2,
    50 random-yaw rectangles (sides U[0.2, 2]) in a 20 x 20 m field."""
    g = rng(seed)
    fp = footprint_rect(0.6, 0.4)
    edges, offs = rects(g, 50, 0.2, 2.0, 0.0, 20.0)
    poses = poses_uniform(g, 20, 0.0, 20.0)
    return Workload("rect-footprint 20 poses x 200 edges", fp, edges, offs, poses,
                    {"seed": seed})


def octagon_lidar(seed: int = 1, n_inst: int = 64, horizon: int = 50,
                  n_rects: int = 4000, n_lines: int = 200,
                  segs_per_line: int = 20) -> Workload:
    """Octagon footprint (circumradius 0.5), 64 rollouts x 50 stages,
    4,000 random-yaw rectangles + 4,000 polyline segments in 40 x 40 m."""
    g = rng(seed)
    fp = footprint_regular(8, 0.5)
    r = rects(g, n_rects, 0.2, 2.0, 0.0, 40.0)
    s = polyline_segments(g, n_lines, segs_per_line, 0.1, 1.0, 0.0, 40.0)
    edges, offs = concat(r, s)
    poses = poses_paths(g, n_inst, horizon, 0.0, 40.0, step=0.1, dtheta=0.1)
    return Workload("octagon-footprint 3200 poses x 20000 edges (rects + lidar segments)",
                    fp, edges, offs, poses, {"seed": seed, "n_inst": n_inst,
                                             "horizon": horizon})


def dense_clutter(seed: int = 4, n_rects: int = 25000, n_poses: int = 4096,
                  field_side: float = 200.0) -> Workload:
    """Rectangle footprint 0.6 x 0.4, 25,000 rectangles (sides U[0.2, 1.0])
    = 100,000 edges in a 200 x 200 m field, 4,096 uniform pose queries."""
    g = rng(seed)
    fp = footprint_rect(0.6, 0.4)
    edges, offs = rects(g, n_rects, 0.2, 1.0, 0.0, field_side)
    poses = poses_uniform(g, n_poses, 0.0, field_side)
    return Workload("dense clutter %d poses x %d edges" % (n_poses, 4 * n_rects),
                    fp, edges, offs, poses, {"seed": seed, "field": field_side})


def backward_rects(seed: int = 3, n_inst: int = 256, horizon: int = 40,
                   n_rects: int = 2500) -> Workload:
    """Rectangle footprint, 256 x 40 poses, 2,500 random-yaw rectangles
    (10,000 edges) in a 40 x 40 m field."""
    g = rng(seed)
    fp = footprint_rect(0.6, 0.4)
    edges, offs = rects(g, n_rects, 0.2, 2.0, 0.0, 40.0)
    poses = poses_paths(g, n_inst, horizon, 0.0, 40.0, step=0.1, dtheta=0.1)
    return Workload("backward 10240 poses x 10000 edges", fp, edges, offs, poses,
                    {"seed": seed})


@dataclass
class Instance:
    footprint: np.ndarray
    edges: np.ndarray
    offsets: np.ndarray
    poses: np.ndarray


def uneven_instances(seed: int = 2, n_inst: int = 1024, hmin: int = 10, hmax: int = 100,
                     emin: int = 16, emax: int = 65536, kmin: int = 4, kmax: int = 12
                     ) -> List[Instance]:
    """Uneven MPC instances: horizon U{hmin..hmax}, edge count log-uniform in
    [emin, emax] (random-yaw rectangles, 4 edges each, field side sqrt(E)*1.5 m),
    footprints with k in U{kmin..kmax} vertices on a circle."""
    g = rng(seed)
    out = []
    for _ in range(n_inst):
        N = int(g.integers(hmin, hmax + 1))
        E = int(4 * max(1, round(math.exp(g.uniform(math.log(emin), math.log(emax))) / 4)))
        side = math.sqrt(E) * 1.5
        k = int(g.integers(kmin, kmax + 1))
        fp = footprint_random_convex(g, k, 0.3, 0.6, min_gap=min(0.3, math.pi / k))
        edges, offs = rects(g, E // 4, 0.2, 2.0, 0.0, side)
        poses = poses_paths(g, 1, N, 0.0, side, step=0.1, dtheta=0.1)
        out.append(Instance(fp, edges, offs, poses))
    return out


def training_scene(index: int, n_rects: int = 1024, n_poses: int = 64,
                   density: float = 0.625) -> Workload:
    """One scene for the tile-proposal network's training set: rectangles at
    the dense-clutter density (sides U[0.2, 1.0]), uniform poses.  Seeds
    1000 + index."""
    g = rng(1000 + index)
    side = math.sqrt(n_rects / density)
    fp = footprint_rect(0.6, 0.4)
    edges, offs = rects(g, n_rects, 0.2, 1.0, 0.0, side)
    poses = poses_uniform(g, n_poses, 0.0, side)
    return Workload("training scene %d" % index, fp, edges, offs, poses,
                    {"seed": 1000 + index, "field": side})


def moving_obstacle_stages(seed: int = 5, n_mpc: int = 64, horizon: int = 15,
                           n_rects: int = 200, field: float = 30.0, dt: float = 0.1,
                           speed: float = 1.0) -> List[Instance]:
    """Time-varying per-stage edge sets: n_mpc MPC problems, each a horizon
    of `horizon` stages; stage s sees its own edge set (random-yaw rectangles
    translated by velocity * s * dt, velocities uniform in direction with
    |v| <= speed) and the nominal pose of that stage.  One instance per
    (problem, stage), one pose each.  Translations are added in FP64 and
    rounded once, so polygon closure stays exact."""
    g = rng(seed)
    fp = footprint_rect(0.6, 0.4)
    out = []
    for _ in range(n_mpc):
        edges, offs = rects(g, n_rects, 0.2, 2.0, 0.0, field)
        n = n_rects
        ang = g.uniform(-math.pi, math.pi, size=n)
        vel = g.uniform(0.0, speed, size=n)[:, None] * np.stack([np.cos(ang), np.sin(ang)], 1)
        path = poses_paths(g, 1, horizon, 0.0, field, step=0.1, dtheta=0.1)
        base = edges.astype(np.float64).reshape(n, 4, 4)
        for s_ in range(horizon):
            d = vel * (s_ * dt)                               # [n, 2]
            e = base.copy()
            e[:, :, 0:2] += d[:, None, :]
            e[:, :, 2:4] += d[:, None, :]
            out.append(Instance(fp, e.reshape(4 * n, 4).astype(F32), offs, path[s_:s_ + 1]))
    return out
