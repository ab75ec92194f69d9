"""torch.autograd.Function over the C ABI: gradients reach poses and edges
and agree with the FP64 oracle's backward."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2607_04310_b300 import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def test_autograd_function_matches_oracle():
    from paper_2607_04310_b300.autograd import PSDF
    g = sg.rng(21)
    fp = sg.footprint_random_convex(g, 6, 0.3, 0.6, min_gap=0.4)
    e1, o1 = sg.convex_polygons(g, 50, 3, 7, 0.3, 1.0, 0.0, 12.0)
    e2, o2 = sg.polyline_segments(g, 6, 10, 0.2, 1.0, 0.0, 12.0)
    edges, offs = sg.concat((e1, o1), (e2, o2))
    n = 800
    idx = g.integers(0, len(edges), size=n)
    poses = np.concatenate([edges[idx, 0:2] + g.normal(size=(n, 2)) * 0.5,
                            g.uniform(-math.pi, math.pi, size=(n, 1))], axis=1).astype(np.float32)
    ref = oracle.psdf_eval(fp, edges, offs, poses)
    keep = (ref["egap"] >= 1e-3) & (ref["twin"] == oracle.PID_NONE) & \
           ((ref["phi"] < 0) | (ref["phi"] >= 1e-2))
    poses = poses[keep]
    model = PSDF(edges, offs, fp)
    p = torch.tensor(poses, device="cuda", requires_grad=True)
    e = torch.tensor(edges, device="cuda", requires_grad=True)
    w = torch.tensor(g.normal(size=len(poses)), dtype=torch.float32, device="cuda")
    phi = model(p, e)
    (phi * w).sum().backward()
    rp, re_ = oracle.psdf_backward(fp, edges, offs, poses, w.double().cpu().numpy())
    assert p.grad is not None and e.grad is not None
    assert np.max(np.abs(p.grad.cpu().numpy() - rp)) <= 1e-4
    err = np.abs(e.grad.cpu().numpy() - re_) / np.maximum(1.0, np.abs(re_))
    assert err.max() <= 2e-4
    assert np.max(np.abs(phi.detach().cpu().numpy() - ref["phi"][keep])) <= 1e-5


def test_autograd_pose_only():
    from paper_2607_04310_b300.autograd import PSDF
    w = sg.plain_rect_small(0)
    model = PSDF(w.edges, w.offsets, w.footprint)
    p = torch.tensor(w.poses, device="cuda", requires_grad=True)
    phi = model(p)
    phi.sum().backward()
    ref = oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses)
    ok = (ref["margin"] >= 1e-3) & ((ref["phi"] < 0) | (ref["phi"] >= 1e-2))
    assert np.max(np.abs(p.grad.cpu().numpy()[ok] - ref["grad"][ok])) <= 1e-4


def test_autograd_soft_minimum_matches_oracle():
    """eta > 0: the wrapper's forward and recomputing backward against the
    oracle's soft mode (the hard mode above goes through the saved rows)."""
    from paper_2607_04310_b300 import psdf
    from paper_2607_04310_b300.autograd import psdf_phi
    g = sg.rng(19)
    fp = sg.footprint_random_convex(g, 7, 0.3, 0.6, min_gap=0.3)
    edges, offs = sg.convex_polygons(g, 60, 3, 8, 0.3, 1.0, 0.0, 15.0)
    n = 600
    idx = g.integers(0, len(edges), size=n)
    poses = np.concatenate([edges[idx, 0:2] + g.normal(size=(n, 2)) * 0.3,
                            g.uniform(-math.pi, math.pi, size=(n, 1))], axis=1).astype(np.float32)
    eta = 200.0
    ref = oracle.psdf_eval(fp, edges, offs, poses, eta=eta)
    keep = (ref["egap"] >= 1e-3) & (ref["twin"] == oracle.PID_NONE) & \
           ((ref["phi"] < 0) | (ref["phi"] >= 1e-2))
    poses = poses[keep]
    prm = psdf.make_params(eta=eta)
    scene = psdf.Scene.from_csr(edges, offs, params=prm)
    p = torch.tensor(poses, device="cuda", requires_grad=True)
    wt = torch.tensor(g.normal(size=len(poses)), dtype=torch.float32, device="cuda")
    phi = psdf_phi(p, None, scene, fp, prm)
    (phi * wt).sum().backward()
    rp, _ = oracle.psdf_backward(fp, edges, offs, poses, wt.double().cpu().numpy(), eta=eta)
    assert np.sum(ref["phi"][keep] < 0) >= 20
    assert np.max(np.abs(phi.detach().cpu().numpy() - ref["phi"][keep])) <= 1e-5
    assert np.max(np.abs(p.grad.cpu().numpy() - rp)) <= 1e-4 * max(1.0, np.abs(rp).max())
