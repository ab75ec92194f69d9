"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check
that the pins catch every one: a dropped term, a wrong sign, a swapped
operand, a wrong index, a wrong clamp, a wrong gradient weight."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import brute_minkowski as bm
import test_oracle_pins as pins
from paper_2607_04310_b300 import scenegen as sg

MUTATIONS = {
    "transform_sign": ("out[1] = -s * dx + c * dy;", "out[1] = s * dx + c * dy;"),
    "drop_obstacle_vertex_pool": ("      if (t <= 0.0 || t >= 1.0) continue;\n      double r[2] = {w[0] - t * e[0], w[1] - t * e[1]};",
                                  "      if (1) continue;\n      double r[2] = {w[0] - t * e[0], w[1] - t * e[1]};"),
    "no_upper_clamp": ("double t = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);\n      if (!seg && t == 1.0) continue;",
                       "double t = u < 0.0 ? 0.0 : u;\n      if (!seg && t == 1.0) continue;"),
    "overlap_side_swapped": ("    double da = bi - aP, db = bP - ai;\n    double dn = da < db ? da : db;\n    axd[l] = dn;",
                             "    double da = bi - ai, db = bP - aP;\n    double dn = da < db ? da : db;\n    axd[l] = dn;"),
    "separated_test_sign": ("if (axd[a] < -P->eps_sat) { separated = 1; break; }",
                            "if (axd[a] > -P->eps_sat) { separated = 1; break; }"),
    "sqrt_dropped": ("    sd = sqrt(dmin2);", "    sd = dmin2;"),
    "obstacle_axis_not_normal": ("double nj[2] = {-u[1] / un, u[0] / un};",
                                 "double nj[2] = {u[1] / un, u[0] / un};"),
    "theta_grad_sign": ("out->g[0] = wr[0]; out->g[1] = wr[1]; out->g[2] = dot2(rh, jv);",
                        "out->g[0] = wr[0]; out->g[1] = wr[1]; out->g[2] = -dot2(rh, jv);"),
    "edge_grad_weights_swapped": ("gedge[4 * j + 0] -= (1.0 - a->t) * wr[0];",
                                  "gedge[4 * j + 0] -= a->t * wr[0];"),
    "robot_edge_index": ("const double *a = fp + 2 * l, *b = fp + 2 * ((l + 1) % m);",
                         "const double *a = fp + 2 * l, *b = fp + 2 * ((l + 2) % m);"),
    "obstacle_min_over_obstacles_dropped": ("    if (best < 0 || ob.sd < bsd) { best = i; bsd = ob.sd; }",
                                            "    if (best < 0) { best = i; bsd = ob.sd; }"),
    "robot_axis_grad_sign": ("gp[0] = sg * Rn[0]; gp[1] = sg * Rn[1];",
                             "gp[0] = -sg * Rn[0]; gp[1] = sg * Rn[1];"),
    "axis_grad_du_term": ("double ddu[2] = {gden * JtD[0] + gpr * uh[0] * JuD, gden * JtD[1] + gpr * uh[1] * JuD};",
                          "double ddu[2] = {gden * JtD[0], gden * JtD[1]};"),
}


def _battery() -> list:
    """Run a compact copy of the pins; return the names of those that fail."""
    failed = []

    def check(name, fn):
        try:
            ok = fn()
        except Exception:  # a crash in the mutated oracle counts as caught
            ok = False
        if not ok:
            failed.append(name)

    def golden():
        for name, fp, pose, val, obs in pins.GOLDEN:
            e, o = pins._csr(obs)
            if abs(oracle.psdf_eval(fp, e, o, [pose])["phi"][0] - val) > 1e-12:
                return False
        return True

    def brute():
        g = np.random.default_rng(1234)
        for trial in range(60):
            fp, polys = pins._tiny_scene(g, int(g.integers(3, 9)) if trial % 3 else 0)
            e, o = pins._csr(polys)
            poses = np.concatenate([g.uniform(-2.5, 2.5, size=(6, 2)),
                                    g.uniform(-math.pi, math.pi, size=(6, 1))], axis=1)
            r = oracle.psdf_eval(fp, e, o, poses)
            for q in range(len(poses)):
                if abs(r["phi"][q] - bm.phi(fp, e, o, poses[q])) > 1e-10:
                    return False
        return True

    def fd_pose():
        g = np.random.default_rng(21)
        e, o = sg.convex_polygons(g, 40, 3, 7, 0.3, 1.2, 0.0, 15.0)
        fp = sg.footprint_random_convex(g, 6, 0.3, 0.6, min_gap=0.4)
        idx = g.integers(0, len(e), size=80)
        poses = np.concatenate([e[idx, 0:2] + g.normal(size=(80, 2)) * 0.4,
                                g.uniform(-math.pi, math.pi, size=(80, 1))], axis=1)
        r = oracle.psdf_eval(fp, e, o, poses)
        keep = r["margin"] > 1e-3
        if keep.sum() < 20:
            return False
        fd = pins._fd_pose(fp, e, o, poses[keep])
        return bool(np.max(np.abs(fd - r["grad"][keep])) < 1e-6)

    def fd_edges():
        g = np.random.default_rng(31)
        e, o = sg.convex_polygons(g, 30, 3, 7, 0.3, 1.2, 0.0, 12.0)
        fp = sg.footprint_random_convex(g, 5, 0.3, 0.6, min_gap=0.4)
        idx = g.integers(0, len(e), size=60)
        poses = np.concatenate([e[idx, 0:2] + g.normal(size=(60, 2)) * 0.4,
                                g.uniform(-math.pi, math.pi, size=(60, 1))], axis=1)
        r = oracle.psdf_eval(fp, e, o, poses)
        good = np.nonzero((r["egap"] > 1e-3) & (r["twin"] == oracle.PID_NONE))[0]
        if len(good) < 10:
            return False
        for q in good[:20]:
            i = int(np.searchsorted(o, int(r["pair"][q]) >> 8, side="right") - 1)
            onehot = np.zeros(len(poses))
            onehot[q] = 1.0
            _, ge = oracle.psdf_backward(fp, e, o, poses, onehot)
            fd = pins._fd_vertices(fp, e, o, i, poses[q])
            if np.max(np.abs(fd - ge[o[i]:o[i + 1]])) > 1e-6:
                return False
        return True

    check("golden", golden)
    check("brute", brute)
    check("fd_pose", fd_pose)
    check("fd_edges", fd_edges)
    return failed


def test_unmutated_battery_passes():
    oracle.use_library(None)
    assert _battery() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, tmp_path):
    find, repl = MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(find) == 1, "mutation anchor not found: %s" % name
    path = oracle.compile_variant(src.replace(find, repl), str(tmp_path / ("m_%s.so" % name)))
    oracle.use_library(path)
    try:
        failed = _battery()
    finally:
        oracle.use_library(None)
    assert failed, "planted mistake %s passed every pin" % name
