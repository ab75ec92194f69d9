"""Independent brute-force signed distance via the Minkowski difference.

For convex sets P and Q, sd(P, Q) (Sec. III-B: dist - pen, the minimum
translation that makes them touch or separates them) equals the signed
distance from the origin to D = P (-) Q = hull{a - b}: positive when the
origin lies outside D (the distance to D), negative when it lies inside
(minus the distance to the boundary of D).  This route shares nothing with
the oracle's edge/SAT pipeline; it is used only on tiny scenes.
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np


def _cross(o, a, b) -> float:
    return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])


def convex_hull(points: np.ndarray) -> np.ndarray:
    """Andrew's monotone chain; CCW, collinear points dropped."""
    pts = sorted(set((float(x), float(y)) for x, y in points))
    if len(pts) <= 2:
        return np.array(pts)
    lower: List = []
    for p in pts:
        while len(lower) >= 2 and _cross(lower[-2], lower[-1], p) <= 0:
            lower.pop()
        lower.append(p)
    upper: List = []
    for p in reversed(pts):
        while len(upper) >= 2 and _cross(upper[-2], upper[-1], p) <= 0:
            upper.pop()
        upper.append(p)
    return np.array(lower[:-1] + upper[:-1])


def _point_segment(p, a, b) -> float:
    ab = b - a
    t = float(np.dot(p - a, ab) / np.dot(ab, ab))
    t = min(1.0, max(0.0, t))
    q = a + t * ab
    return float(math.hypot(p[0] - q[0], p[1] - q[1]))


def signed_distance_origin(hull: np.ndarray) -> float:
    """Signed distance from the origin to a CCW convex polygon."""
    o = np.zeros(2)
    n = len(hull)
    d = min(_point_segment(o, hull[k], hull[(k + 1) % n]) for k in range(n))
    inside = all(_cross(hull[k], hull[(k + 1) % n], o) > 0 for k in range(n))
    return -d if inside else d


def world_footprint(footprint: np.ndarray, pose: Sequence[float]) -> np.ndarray:
    c, s = math.cos(pose[2]), math.sin(pose[2])
    fp = np.asarray(footprint, dtype=np.float64)
    return np.stack([c * fp[:, 0] - s * fp[:, 1] + pose[0],
                     s * fp[:, 0] + c * fp[:, 1] + pose[1]], axis=1)


def obstacle_vertices(edges: np.ndarray, offsets: np.ndarray, i: int) -> np.ndarray:
    e = np.asarray(edges, dtype=np.float64)[offsets[i]:offsets[i + 1]]
    if len(e) == 1:
        return np.array([e[0, 0:2], e[0, 2:4]])
    return e[:, 0:2]


def sd_pair(robot_world: np.ndarray, obstacle: np.ndarray) -> float:
    diff = (robot_world[:, None, :] - obstacle[None, :, :]).reshape(-1, 2)
    return signed_distance_origin(convex_hull(diff))


def phi(footprint, edges, offsets, pose) -> float:
    rw = world_footprint(footprint, pose)
    M = len(offsets) - 1
    if M == 0:
        return math.inf
    return min(sd_pair(rw, obstacle_vertices(edges, offsets, i)) for i in range(M))


def overlaps(footprint, edges, offsets, pose) -> bool:
    """True iff the origin lies strictly inside some Minkowski difference,
    i.e. the robot's interior meets an obstacle."""
    rw = world_footprint(footprint, pose)
    for i in range(len(offsets) - 1):
        if sd_pair(rw, obstacle_vertices(edges, offsets, i)) < 0:
            return True
    return False
