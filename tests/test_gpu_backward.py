"""Hand-written backward kernel (d phi / d pose, d phi / d edge endpoints)
against the FP64 oracle's analytic backward and its central differences."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import parity
from paper_2607_04310_b300 import psdf
from paper_2607_04310_b300 import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _gpu_backward(w, scene, poses_np, gphi_np):
    dev = torch.device("cuda")
    poses = torch.as_tensor(poses_np.astype(np.float32), device=dev)
    phi, dphi, act = psdf.eval_grad(scene, w.footprint, poses)
    gphi = torch.as_tensor(gphi_np.astype(np.float32), device=dev)
    gpose = torch.empty((len(poses_np), 3), device=dev)
    gedges = torch.zeros((w.E, 4), device=dev)
    psdf.psdf_backward(w.footprint, scene, poses, scene.params, act, gphi, gpose, gedges)
    torch.cuda.synchronize()
    return (phi.cpu().numpy(), psdf.pair_ids(act), dphi.cpu().numpy(), gpose.cpu().numpy(),
            gedges.cpu().numpy())


def _check_backward(w, poses, n_check=400, seed=0):
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    ref = oracle.psdf_eval(w.footprint, w.edges, w.offsets, poses)
    g = np.random.default_rng(seed)
    good = np.nonzero((ref["egap"] >= 1e-3) & (ref["twin"] == oracle.PID_NONE)
                      & ((ref["phi"] < 0) | (ref["phi"] >= 1e-2)))[0]
    assert len(good) >= min(n_check, 50)
    good = g.choice(good, size=min(n_check, len(good)), replace=False)
    gphi = np.zeros(len(poses))
    gphi[good] = g.normal(size=len(good))
    gphi = gphi.astype(np.float32).astype(np.float64)
    phi, pair, dphi, gpose, gedges = _gpu_backward(w, scene, poses, gphi)
    assert np.array_equal(pair[good], ref["pair"][good])
    rp, re_ = oracle.psdf_backward(w.footprint, w.edges, w.offsets, poses, gphi)
    # pose gradients: every pose (zero seed -> zero gradient)
    assert np.max(np.abs(gpose - rp)) <= 1e-4 * max(1.0, np.abs(rp).max())
    # edge gradients, accumulated over the checked poses
    scale = np.maximum(1.0, np.abs(re_))
    err = np.abs(gedges - re_) / scale
    assert err.max() <= 2e-4, (float(err.max()), np.unravel_index(err.argmax(), err.shape))
    # the reported layout: closed-polygon B slots stay zero
    poly_rows = np.repeat(np.diff(w.offsets) > 1, np.diff(w.offsets))
    assert np.all(gedges[poly_rows, 2:4] == 0)
    return len(good)


def test_backward_rects_small():
    w = sg.backward_rects(3, n_inst=32, horizon=40, n_rects=600)
    g = np.random.default_rng(2)
    n = 1500
    idx = g.integers(0, w.E, size=n)
    poses = np.concatenate([w.edges[idx, 0:2] + g.normal(size=(n, 2)) * 0.5,
                            g.uniform(-math.pi, math.pi, size=(n, 1))], axis=1).astype(np.float32)
    assert _check_backward(w, poses) >= 100


def test_backward_convex_and_segments():
    g = sg.rng(9)
    fp = sg.footprint_random_convex(g, 7, 0.3, 0.6, min_gap=0.3)
    e1, o1 = sg.convex_polygons(g, 60, 3, 8, 0.3, 1.0, 0.0, 15.0)
    e2, o2 = sg.polyline_segments(g, 8, 10, 0.2, 1.0, 0.0, 15.0)
    edges, offs = sg.concat((e1, o1), (e2, o2))
    n = 1500
    idx = g.integers(0, len(edges), size=n)
    poses = np.concatenate([edges[idx, 0:2] + g.normal(size=(n, 2)) * 0.5,
                            g.uniform(-math.pi, math.pi, size=(n, 1))], axis=1).astype(np.float32)
    w = sg.Workload("convex+segments", fp, edges, offs, poses)
    assert _check_backward(w, poses) >= 100


def test_backward_full_size_sampled():
    """256 x 40 poses x 10,000 edges on the GPU; the upstream gradient is
    nonzero on up to 400 poses >= 1e-3 m from argmin ties."""
    w = sg.backward_rects(3)
    g = np.random.default_rng(4)
    cand = np.sort(g.choice(w.P, size=3000, replace=False))
    ref = oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses[cand])
    keep = cand[(ref["egap"] >= 1e-3) & (ref["twin"] == oracle.PID_NONE)
                & ((ref["phi"] < 0) | (ref["phi"] >= 1e-2))][:400]
    assert len(keep) >= 150
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    gphi = np.zeros(w.P)
    gphi[keep] = g.normal(size=len(keep))
    gphi = gphi.astype(np.float32).astype(np.float64)
    phi, pair, dphi, gpose, gedges = _gpu_backward(w, scene, w.poses, gphi)
    rp, re_ = oracle.psdf_backward(w.footprint, w.edges, w.offsets, w.poses[keep], gphi[keep])
    assert np.max(np.abs(gpose[keep] - rp)) <= 1e-4
    assert np.all(gpose[np.setdiff1d(np.arange(w.P), keep)] == 0)
    err = np.abs(gedges - re_) / np.maximum(1.0, np.abs(re_))
    assert err.max() <= 2e-4


def test_backward_matches_fd_of_oracle():
    """GPU edge-endpoint gradients against central differences (h = 1e-6)
    of the FP64 oracle value, vertex by vertex."""
    g = sg.rng(12)
    fp = sg.footprint_random_convex(g, 5, 0.3, 0.6, min_gap=0.4)
    edges, offs = sg.convex_polygons(g, 30, 3, 7, 0.3, 1.2, 0.0, 12.0)
    n = 300
    idx = g.integers(0, len(edges), size=n)
    poses = np.concatenate([edges[idx, 0:2] + g.normal(size=(n, 2)) * 0.4,
                            g.uniform(-math.pi, math.pi, size=(n, 1))], axis=1).astype(np.float32)
    w = sg.Workload("fd", fp, edges, offs, poses)
    scene = psdf.Scene.from_csr(edges, offs)
    ref = oracle.psdf_eval(fp, edges, offs, poses)
    good = np.nonzero((ref["egap"] >= 1e-3) & (ref["twin"] == oracle.PID_NONE)
                      & ((ref["phi"] < 0) | (ref["phi"] >= 1e-2)))[0][:30]
    h = 1e-6
    e64 = edges.astype(np.float64)
    for q in good:
        gphi = np.zeros(n)
        gphi[q] = 1.0
        _, _, _, _, ge = _gpu_backward(w, scene, poses, gphi)
        i = int(np.searchsorted(offs, int(ref["pair"][q]) >> 8, side="right") - 1)
        e0, k = int(offs[i]), int(offs[i + 1] - offs[i])
        for v in range(k):
            for c in range(2):
                ep, em = e64.copy(), e64.copy()
                rows = [(e0 + v, c)] + ([(e0 + (v - 1) % k, 2 + c)] if k > 1 else [])
                for r_, c_ in rows:
                    ep[r_, c_] += h
                    em[r_, c_] -= h
                fd = (oracle.psdf_eval(fp, ep, offs, poses[q:q + 1])["phi"][0]
                      - oracle.psdf_eval(fp, em, offs, poses[q:q + 1])["phi"][0]) / (2 * h)
                assert abs(ge[e0 + v, c] - fd) <= 1e-4 * max(1.0, abs(fd)), (q, v, c, ge[e0 + v, c], fd)


def test_backward_pose_gradient_equals_forward_at_every_batch_size():
    """The backward's pose gradient with a unit upstream gradient is the
    forward's d phi / d pose bit for bit, for batch sizes that give the
    backward launch every spread of lanes per pose (a warp per pose for
    small batches, down to a thread per pose above about 600 K poses) and a
    ragged tail."""
    w = sg.backward_rects(3, n_inst=8, horizon=8, n_rects=400)
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    g = np.random.default_rng(31)
    dev = torch.device("cuda")
    for P in (1, 37, 4096, 25_001, 75_003, 700_001):
        poses = torch.as_tensor(np.concatenate(
            [g.uniform(0.0, 40.0, size=(P, 2)), g.uniform(-math.pi, math.pi, size=(P, 1))],
            axis=1).astype(np.float32), device=dev)
        phi, dphi, act = psdf.eval_grad(scene, w.footprint, poses)
        gpose = torch.empty((P, 3), device=dev)
        psdf.psdf_backward(w.footprint, scene, poses, scene.params, act,
                           torch.ones(P, device=dev), gpose, None)
        torch.cuda.synchronize()
        assert torch.equal(gpose.view(torch.int32), dphi.view(torch.int32)), P
