"""Pins for the FP64 oracle: closed forms, hand-worked examples, an
independent Minkowski-difference brute force, invariants, and central finite
differences.  CPU only (no GPU marker)."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
import brute_minkowski as bm
from paper_2607_04310_b300 import scenegen as sg

HERE = os.path.dirname(os.path.abspath(__file__))


def _box(x0, x1, y0, y1):
    return np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], dtype=np.float64)


def _csr(polys):
    """Polygons (>= 3 points) or segments (2 points) -> CSR float64 edges."""
    rows, offs = [], [0]
    for p in polys:
        p = np.asarray(p, dtype=np.float64)
        if len(p) == 2:
            rows.append(np.concatenate([p[0], p[1]])[None])
        else:
            rows.append(np.concatenate([p, np.roll(p, -1, axis=0)], axis=1))
        offs.append(offs[-1] + len(rows[-1]))
    return np.concatenate(rows, axis=0), np.array(offs, dtype=np.int32)


# ---------------------------------------------------------------------------
# hand-worked examples (tests/golden/worked_examples.txt)
# ---------------------------------------------------------------------------
def _num(tok):
    return float(eval(tok, {"__builtins__": {}}, {"pi": math.pi, "sqrt": math.sqrt}))


def _load_golden():
    cases = []
    with open(os.path.join(HERE, "golden", "worked_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            fields = [x.strip() for x in line.split("|")]
            name = fields[0]
            fp = np.array([_num(t) for t in fields[1].split()]).reshape(-1, 2)
            pose = [_num(t) for t in fields[2].split()]
            val = _num(fields[3])
            obs = [np.array([_num(t) for t in f.split()]).reshape(-1, 2) for f in fields[4:]]
            cases.append((name, fp, pose, val, obs))
    return cases


GOLDEN = _load_golden()


@pytest.mark.parametrize("case", GOLDEN, ids=[c[0] for c in GOLDEN])
def test_worked_examples(case):
    name, fp, pose, val, obs = case
    edges, offs = _csr(obs)
    r = oracle.psdf_eval(fp, edges, offs, [pose])
    assert abs(r["phi"][0] - val) < 1e-12, (name, r["phi"][0], val)


def test_golden_count():
    assert len(GOLDEN) >= 15


# ---------------------------------------------------------------------------
# closed forms: point-to-segment and axis-aligned boxes
# ---------------------------------------------------------------------------
def test_point_segment_closed_forms():
    a = 0.25  # exactly representable square footprint, half size a
    fp = np.array([[-a, -a], [a, -a], [a, a], [-a, a]])
    g = np.random.default_rng(7)
    for _ in range(200):
        b = a + g.uniform(0.01, 3.0)
        L = g.uniform(0.1, 2.0)
        # segment on the x axis starting at (b, 0): the start point projects
        # inside the right robot face -> gap b - a, active pair: obstacle
        # vertex A of edge 0 to robot edge 1 (interior)
        e, o = _csr([[[b, 0.0], [b + L, 0.0]]])
        r = oracle.psdf_eval(fp, e, o, [[0, 0, 0]])
        assert abs(r["phi"][0] - (b - a)) < 1e-12
        assert oracle.pair_fields(r["pair"][0]) == (0, 1, 1)
        # segment from (b, b) along (1, 2): closest to robot vertex 2 at its start
        e, o = _csr([[[b, b], [b + L, b + 2 * L]]])
        r = oracle.psdf_eval(fp, e, o, [[0, 0, 0]])
        assert abs(r["phi"][0] - math.sqrt(2.0) * (b - a)) < 1e-12
        assert oracle.pair_fields(r["pair"][0]) == (0, 0, 2)
        # segment seen from its far end: reversed direction, B endpoint nearest
        e, o = _csr([[[b + L, b + 2 * L], [b, b]]])
        r = oracle.psdf_eval(fp, e, o, [[0, 0, 0]])
        assert abs(r["phi"][0] - math.sqrt(2.0) * (b - a)) < 1e-12
        # point projecting inside a long segment: y = h line, x in [-L-1, L+1]
        h = a + g.uniform(0.01, 2.0)
        x0 = g.uniform(-0.2, 0.2)
        e, o = _csr([[[x0 + L + 1, h], [x0 - L - 1, h]]])
        r = oracle.psdf_eval(fp, e, o, [[0, 0, 0]])
        assert abs(r["phi"][0] - (h - a)) < 1e-12


def _box_sd(w1, h1, cx, cy, w2, h2):
    gx = abs(cx) - (w1 + w2) / 2
    gy = abs(cy) - (h1 + h2) / 2
    if gx > 0 or gy > 0:
        return math.hypot(max(gx, 0.0), max(gy, 0.0))
    return -min(-gx, -gy)


@pytest.mark.parametrize("quarter", [0, 1, 2, 3])
def test_box_box_closed_form(quarter):
    g = np.random.default_rng(11 + quarter)
    for _ in range(300):
        w1, h1 = g.uniform(0.2, 2.0, size=2)
        w2, h2 = g.uniform(0.2, 2.0, size=2)
        cx, cy = g.uniform(-3.0, 3.0, size=2)
        fp = _box(-w1 / 2, w1 / 2, -h1 / 2, h1 / 2)
        e, o = _csr([_box(-w2 / 2, w2 / 2, -h2 / 2, h2 / 2)])
        th = quarter * math.pi / 2
        r = oracle.psdf_eval(fp, e, o, [[cx, cy, th]])
        W1, H1 = (w1, h1) if quarter % 2 == 0 else (h1, w1)
        assert abs(r["phi"][0] - _box_sd(W1, H1, cx, cy, w2, h2)) < 1e-12


def test_separated_penetrating_and_contained():
    fp = _box(-0.3, 0.3, -0.2, 0.2)
    e, o = _csr([_box(-5, 5, -5, 5)])
    # robot fully inside a large box: push out through the nearest face
    r = oracle.psdf_eval(fp, e, o, [[4.0, 0.0, 0.0]])
    assert abs(r["phi"][0] - (-(5 - 4 + 0.3))) < 1e-12
    # large robot containing a small obstacle
    big = _box(-5, 5, -5, 5)
    e2, o2 = _csr([_box(0.9, 1.1, -0.1, 0.1)])
    r = oracle.psdf_eval(big, e2, o2, [[0.0, 0.0, 0.0]])
    assert abs(r["phi"][0] - (-(5 - 0.9))) < 1e-12


def test_empty_scene_is_infinite():
    fp = sg.footprint_rect()
    r = oracle.psdf_eval(fp, np.zeros((0, 4)), np.zeros(1, dtype=np.int32), [[0, 0, 0]])
    assert math.isinf(r["phi"][0]) and r["phi"][0] > 0
    assert r["pair"][0] == oracle.PID_NONE
    assert np.all(r["grad"][0] == 0)


# ---------------------------------------------------------------------------
# brute force (Minkowski difference) on tiny scenes
# ---------------------------------------------------------------------------
def _tiny_scene(g, k):
    polys = []
    nobs = int(g.integers(1, 4))
    for _ in range(nobs):
        kind = g.integers(0, 3)
        c = g.uniform(-2.0, 2.0, size=2)
        if kind == 0:
            e, o = sg.rects(g, 1, 0.2, 1.5, -2.0, 2.0)
            polys.append(e[:, 0:2].astype(np.float64))
        elif kind == 1:
            kk = int(g.integers(3, 7))
            p = sg.footprint_random_convex(g, kk, 0.2, 0.8, min_gap=0.3).astype(np.float64) + c
            polys.append(p)
        else:
            ang = g.uniform(-math.pi, math.pi)
            L = g.uniform(0.1, 1.5)
            polys.append(np.array([c, c + L * np.array([math.cos(ang), math.sin(ang)])]))
    if k == 0:
        fp = sg.footprint_rect(g.uniform(0.3, 1.0), g.uniform(0.2, 0.8)).astype(np.float64)
    else:
        fp = sg.footprint_random_convex(g, k, 0.3, 0.7, min_gap=0.3).astype(np.float64)
    return fp, polys


def test_brute_force_minkowski():
    g = np.random.default_rng(1234)
    n_pen = n_sep = 0
    for trial in range(250):
        fp, polys = _tiny_scene(g, int(g.integers(3, 9)) if trial % 3 else 0)
        e, o = _csr(polys)
        poses = np.concatenate([g.uniform(-2.5, 2.5, size=(6, 2)),
                                g.uniform(-math.pi, math.pi, size=(6, 1))], axis=1)
        r = oracle.psdf_eval(fp, e, o, poses)
        for q in range(len(poses)):
            want = bm.phi(fp, e, o, poses[q])
            assert abs(r["phi"][q] - want) < 1e-10, (trial, q, r["phi"][q], want)
            if want < 0:
                n_pen += 1
            else:
                n_sep += 1
    # both regimes are exercised
    assert n_pen > 100 and n_sep > 300


def test_sign_matches_overlap_predicate():
    g = np.random.default_rng(99)
    for trial in range(150):
        fp, polys = _tiny_scene(g, 0)
        e, o = _csr(polys)
        poses = np.concatenate([g.uniform(-2.5, 2.5, size=(5, 2)),
                                g.uniform(-math.pi, math.pi, size=(5, 1))], axis=1)
        r = oracle.psdf_eval(fp, e, o, poses)
        for q in range(len(poses)):
            if abs(r["phi"][q]) < 1e-9:
                continue
            assert (r["phi"][q] < 0) == bm.overlaps(fp, e, o, poses[q])


def test_obstacle_sd_min_is_phi():
    w = sg.plain_rect_small(0)
    sd = oracle.obstacle_sd(w.footprint, w.edges, w.offsets, w.poses)
    r = oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses)
    assert np.array_equal(sd.min(axis=1), r["phi"])
    # the reported pair's edge lies in the minimising obstacle
    obs = np.searchsorted(w.offsets, (r["pair"] >> 8).astype(np.int64), side="right") - 1
    assert np.all(sd[np.arange(w.P), obs] == r["phi"])


def test_padded_equals_csr_order():
    """The padded (A, B, S) encoding of Sec. IV-A.2 holds the same edges."""
    w = sg.octagon_lidar(1, n_inst=2, horizon=5, n_rects=20, n_lines=3, segs_per_line=4)
    A, B, S = sg.to_padded(w.edges, w.offsets)
    M, mb = S.shape
    rows = [np.concatenate([A[i, j], B[i, j]]) for i in range(M) for j in range(mb) if S[i, j]]
    assert np.array_equal(np.array(rows, dtype=np.float32), w.edges)


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
def _se2(edges, poses, ang, tx, ty):
    c, s = math.cos(ang), math.sin(ang)
    e = np.asarray(edges, dtype=np.float64).copy()
    for col in (0, 2):
        x, y = e[:, col].copy(), e[:, col + 1].copy()
        e[:, col] = c * x - s * y + tx
        e[:, col + 1] = s * x + c * y + ty
    p = np.asarray(poses, dtype=np.float64).copy()
    x, y = p[:, 0].copy(), p[:, 1].copy()
    p[:, 0] = c * x - s * y + tx
    p[:, 1] = s * x + c * y + ty
    p[:, 2] = p[:, 2] + ang
    return e, p


def test_rigid_motion_invariance():
    w = sg.octagon_lidar(1, n_inst=4, horizon=10, n_rects=200, n_lines=10, segs_per_line=20)
    base = oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses)
    g = np.random.default_rng(5)
    for _ in range(3):
        ang, tx, ty = g.uniform(-math.pi, math.pi), g.uniform(-50, 50), g.uniform(-50, 50)
        e, p = _se2(w.edges, w.poses, ang, tx, ty)
        r = oracle.psdf_eval(w.footprint, e, w.offsets, p)
        assert np.max(np.abs(r["phi"] - base["phi"])) < 1e-11
        ok = base["margin"] > 1e-6
        same = (r["pair"] == base["pair"]) | (r["pair"] == base["twin"])
        assert np.all(same[ok])


def test_one_lipschitz_in_translation():
    w = sg.plain_rect_small(0)
    g = np.random.default_rng(6)
    base = oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses)["phi"]
    for _ in range(20):
        d = g.normal(size=(w.P, 2)) * g.uniform(1e-4, 1.0)
        p = w.poses.astype(np.float64).copy()
        p[:, 0:2] += d
        phi = oracle.psdf_eval(w.footprint, w.edges, w.offsets, p)["phi"]
        assert np.all(np.abs(phi - base) <= np.linalg.norm(d, axis=1) + 1e-12)


@pytest.mark.parametrize("eta", [50.0, 200.0, 1000.0])
def test_soft_min_bounds(eta):
    w = sg.plain_rect_small(0)
    g = np.random.default_rng(8)
    poses = w.poses.astype(np.float64).copy()
    # move half of the poses onto obstacle corners to get penetrations
    idx = g.integers(0, w.E, size=w.P // 2)
    poses[: w.P // 2, 0:2] = w.edges[idx, 0:2] + g.normal(size=(w.P // 2, 2)) * 0.1
    hard = oracle.psdf_eval(w.footprint, w.edges, w.offsets, poses)["phi"]
    soft = oracle.psdf_eval(w.footprint, w.edges, w.offsets, poses, eta=eta)["phi"]
    K = 4 + 4  # robot axes + obstacle axes of a rectangle
    assert np.all(soft >= hard - 1e-12)
    assert np.all(soft - hard <= math.log(K) / eta + 1e-12)
    assert np.sum(hard < 0) >= 3
    # separated poses are unaffected by the smoothing
    assert np.array_equal(soft[hard > 0], hard[hard > 0])


def test_soft_min_tends_to_hard():
    w = sg.plain_rect_small(0)
    p = w.poses.astype(np.float64).copy()
    p[:, 0:2] = w.edges[: w.P, 0:2]
    hard = oracle.psdf_eval(w.footprint, w.edges, w.offsets, p)["phi"]
    soft = oracle.psdf_eval(w.footprint, w.edges, w.offsets, p, eta=1e7)["phi"]
    assert np.max(np.abs(soft - hard)) < 1e-6


# ---------------------------------------------------------------------------
# gradients: central finite differences of the FP64 value (h = 1e-6)
# ---------------------------------------------------------------------------
def _fd_pose(fp, e, o, poses, h=1e-6, **kw):
    out = np.empty((len(poses), 3))
    for k in range(3):
        pp = np.asarray(poses, dtype=np.float64).copy()
        pm = pp.copy()
        pp[:, k] += h
        pm[:, k] -= h
        out[:, k] = (oracle.psdf_eval(fp, e, o, pp, **kw)["phi"]
                     - oracle.psdf_eval(fp, e, o, pm, **kw)["phi"]) / (2 * h)
    return out


@pytest.mark.parametrize("scene", ["rects", "octagon_mixed", "convex"])
def test_fd_pose_gradient(scene):
    g = np.random.default_rng(21)
    if scene == "rects":
        w = sg.plain_rect_small(0)
        fp, e, o = w.footprint, w.edges, w.offsets
    elif scene == "octagon_mixed":
        w = sg.octagon_lidar(1, n_inst=4, horizon=10, n_rects=150, n_lines=10, segs_per_line=15)
        fp, e, o = w.footprint, w.edges, w.offsets
    else:
        e, o = sg.convex_polygons(g, 40, 3, 7, 0.3, 1.2, 0.0, 15.0)
        fp = sg.footprint_random_convex(g, 6, 0.3, 0.6, min_gap=0.4)
    # half near obstacles (penetration and contact-scale distances), half uniform
    n = 120
    idx = g.integers(0, len(e), size=n)
    poses = np.concatenate([e[idx, 0:2] + g.normal(size=(n, 2)) * 0.4,
                            g.uniform(-math.pi, math.pi, size=(n, 1))], axis=1)
    r = oracle.psdf_eval(fp, e, o, poses)
    keep = r["margin"] > 1e-3
    assert keep.sum() > 40
    fd = _fd_pose(fp, e, o, poses[keep])
    err = np.abs(fd - r["grad"][keep])
    assert np.max(err) < 1e-6, np.max(err)
    assert np.sum(r["phi"][keep] < 0) > 5


def _fd_vertices(fp, e, o, i, pose, h=1e-6, **kw):
    """Central differences with respect to obstacle i's vertices.  A closed
    polygon's vertex k is stored as A of edge k and B of edge k-1; both
    copies move together.  Returns [rows, 4] laid out like the backward's
    output (vertex gradient in the A slot, zero B slots for polygons)."""
    e0, n = int(o[i]), int(o[i + 1] - o[i])
    out = np.zeros((n, 4))
    slots = [(k, 0) for k in range(n)] + ([(0, 2)] if n == 1 else [])
    for k, col in slots:
        for c in range(2):
            ep = np.asarray(e, dtype=np.float64).copy()
            em = ep.copy()
            copies = [(e0 + k, col + c)]
            if n > 1:
                copies.append((e0 + (k - 1) % n, 2 + c))
            for r_, c_ in copies:
                ep[r_, c_] += h
                em[r_, c_] -= h
            out[k, col + c] = (oracle.psdf_eval(fp, ep, o, [pose], **kw)["phi"][0]
                               - oracle.psdf_eval(fp, em, o, [pose], **kw)["phi"][0]) / (2 * h)
    return out


@pytest.mark.parametrize("scene", ["convex", "segments"])
def test_fd_edge_gradient(scene):
    """d phi / d (obstacle vertices) against central differences on each
    vertex coordinate of the active obstacle (Sec. IV-D active-branch
    subgradient)."""
    g = np.random.default_rng(31)
    if scene == "convex":
        e, o = sg.convex_polygons(g, 30, 3, 7, 0.3, 1.2, 0.0, 12.0)
    else:
        e, o = sg.polyline_segments(g, 6, 8, 0.2, 1.0, 0.0, 12.0)
    fp = sg.footprint_random_convex(g, 5, 0.3, 0.6, min_gap=0.4)
    n = 80
    idx = g.integers(0, len(e), size=n)
    poses = np.concatenate([e[idx, 0:2] + g.normal(size=(n, 2)) * 0.4,
                            g.uniform(-math.pi, math.pi, size=(n, 1))], axis=1)
    r = oracle.psdf_eval(fp, e, o, poses)
    good = np.nonzero((r["egap"] > 1e-3) & (r["twin"] == oracle.PID_NONE))[0]
    assert len(good) > 20
    kinds = set()
    for q in good[:40]:
        edge = int(r["pair"][q]) >> 8
        kinds.add((int(r["pair"][q]) >> 4) & 0xF)
        i = int(np.searchsorted(o, edge, side="right") - 1)
        onehot = np.zeros(len(poses))
        onehot[q] = 1.0
        _, ge = oracle.psdf_backward(fp, e, o, poses, onehot)
        fd = _fd_vertices(fp, e, o, i, poses[q])
        got = ge[o[i]:o[i + 1]]
        assert np.max(np.abs(fd - got)) < 1e-6, (q, np.max(np.abs(fd - got)))
        # nothing outside the active obstacle
        rest = np.delete(ge, np.arange(o[i], o[i + 1]), axis=0)
        assert np.all(rest == 0)
    assert len(kinds) >= 3, kinds


def test_edge_gradient_rigid_invariants():
    """Moving every stored endpoint by d equals moving the pose by -d;
    rotating them about the origin with the pose leaves phi unchanged."""
    w = sg.octagon_lidar(1, n_inst=4, horizon=10, n_rects=150, n_lines=10, segs_per_line=15)
    gphi = np.random.default_rng(3).normal(size=w.P)
    gp, ge = oracle.psdf_backward(w.footprint, w.edges, w.offsets, w.poses, gphi)
    # translation
    tx = ge[:, 0].sum() + ge[:, 2].sum()
    ty = ge[:, 1].sum() + ge[:, 3].sum()
    assert abs(tx + gp[:, 0].sum()) < 1e-9
    assert abs(ty + gp[:, 1].sum()) < 1e-9
    # rotation: sum over stored points X of dphi/dX . (J X) + dphi/dp . (J p) + dphi/dtheta = 0
    e = w.edges.astype(np.float64)
    p = w.poses.astype(np.float64)
    rot = 0.0
    for col in (0, 2):
        rot += np.sum(ge[:, col] * (-e[:, col + 1]) + ge[:, col + 1] * e[:, col])
    rot += np.sum(gp[:, 0] * (-p[:, 1]) + gp[:, 1] * p[:, 0]) + gp[:, 2].sum()
    assert abs(rot) < 1e-8


@pytest.mark.parametrize("eta", [50.0, 500.0])
def test_fd_soft_gradient(eta):
    g = np.random.default_rng(41)
    e, o = sg.convex_polygons(g, 25, 3, 6, 0.4, 1.2, 0.0, 10.0)
    fp = sg.footprint_random_convex(g, 6, 0.3, 0.6, min_gap=0.4)
    n = 120
    idx = g.integers(0, len(e), size=n)
    poses = np.concatenate([e[idx, 0:2] + g.normal(size=(n, 2)) * 0.2,
                            g.uniform(-math.pi, math.pi, size=(n, 1))], axis=1)
    r = oracle.psdf_eval(fp, e, o, poses, eta=eta)
    hard = oracle.psdf_eval(fp, e, o, poses)
    keep = (hard["margin"] > 1e-3) & (r["phi"] < -1e-3)
    assert keep.sum() > 10
    fd = _fd_pose(fp, e, o, poses[keep], eta=eta)
    assert np.max(np.abs(fd - r["grad"][keep])) < 1e-5
