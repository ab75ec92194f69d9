"""Soft-min penetration (Eq. penetration_depth, eta > 0) on the GPU: values,
active pairs, pose gradients and backward against the FP64 oracle's soft
mode; the soft <= hard bounds; separated poses unchanged."""
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


def _penetrating(w, seed, frac=0.5, spread=0.1):
    """Half of the poses moved onto obstacle vertices (penetrations)."""
    g = np.random.default_rng(seed)
    poses = w.poses.astype(np.float64).copy()
    n = int(len(poses) * frac)
    idx = g.integers(0, w.E, size=n)
    poses[:n, 0:2] = w.edges[idx, 0:2] + g.normal(size=(n, 2)) * spread
    return poses.astype(np.float32)


@pytest.mark.parametrize("eta", [50.0, 200.0, 1000.0])
def test_soft_rects_against_oracle(eta):
    w = sg.plain_rect_small(0)
    poses = np.concatenate([_penetrating(w, 1), _penetrating(w, 2, spread=0.3)])
    prm = psdf.make_params(eta=eta)
    gpu, _ = parity.gpu_eval(w, poses=poses, params=prm)
    ref = parity.oracle_eval(w, poses=poses, eta=eta)
    st = parity.compare(gpu, ref)
    assert np.sum(ref["phi"] < 0) >= 5
    assert st["grad_checked"] >= 10


@pytest.mark.parametrize("eta", [50.0, 1000.0])
def test_soft_octagon_segments_against_oracle(eta):
    w = sg.octagon_lidar(1)
    g = np.random.default_rng(5)
    sel = g.choice(w.P, size=600, replace=False)
    w2 = sg.Workload(w.name, w.footprint, w.edges, w.offsets, w.poses[sel], w.info)
    poses = _penetrating(w2, 6, frac=0.7, spread=0.3)
    prm = psdf.make_params(eta=eta)
    gpu, _ = parity.gpu_eval(w2, poses=poses, params=prm)
    ref = parity.oracle_eval(w2, poses=poses, eta=eta)
    parity.compare(gpu, ref)


def test_soft_bounds_and_separated_unchanged():
    w = sg.plain_rect_small(0)
    poses = _penetrating(w, 3)
    hard, _ = parity.gpu_eval(w, poses=poses)
    for eta in (50.0, 200.0, 1000.0):
        soft, _ = parity.gpu_eval(w, poses=poses, params=psdf.make_params(eta=eta))
        K = 8  # robot + obstacle axes of a rectangle against a rectangle
        assert np.all(soft["phi"] >= hard["phi"] - 1e-6)
        assert np.all(soft["phi"] - hard["phi"] <= math.log(K) / eta + 1e-6)
        sep = hard["phi"] > 0
        assert np.array_equal(soft["phi"][sep].view(np.uint32), hard["phi"][sep].view(np.uint32))


@pytest.mark.parametrize("eta", [50.0, 500.0])
def test_soft_backward_against_oracle(eta):
    """Random convex polygons and segments: unlike rectangles they have no
    exactly tied far vertices, so the soft sum's edge attribution (every axis
    with delta > 0 contributes) is unique and comparable row by row."""
    g = sg.rng(19)
    fp = sg.footprint_random_convex(g, 7, 0.3, 0.6, min_gap=0.3)
    e1, o1 = sg.convex_polygons(g, 60, 3, 8, 0.3, 1.0, 0.0, 15.0)
    e2, o2 = sg.polyline_segments(g, 8, 10, 0.2, 1.0, 0.0, 15.0)
    edges, offs = sg.concat((e1, o1), (e2, o2))
    n = 1500
    idx = g.integers(0, len(edges), size=n)
    poses = np.concatenate([edges[idx, 0:2] + g.normal(size=(n, 2)) * 0.3,
                            g.uniform(-math.pi, math.pi, size=(n, 1))], axis=1).astype(np.float32)
    prm = psdf.make_params(eta=eta)
    scene = psdf.Scene.from_csr(edges, offs, params=prm)
    dev = torch.device("cuda")
    ps = torch.as_tensor(poses, device=dev)
    phi, dphi, act = psdf.eval_grad(scene, fp, ps, params=prm)
    ref = oracle.psdf_eval(fp, edges, offs, poses, eta=eta)
    good = np.nonzero((ref["egap"] >= 1e-3) & (ref["twin"] == oracle.PID_NONE)
                      & ((ref["phi"] < 0) | (ref["phi"] >= 1e-2)))[0]
    assert np.sum(ref["phi"][good] < 0) >= 50
    gphi = np.zeros(n)
    gphi[good] = g.normal(size=len(good))
    gphi = gphi.astype(np.float32).astype(np.float64)
    gpose = torch.empty((n, 3), device=dev)
    gedges = torch.zeros((len(edges), 4), device=dev)
    psdf.psdf_backward(fp, scene, ps, prm, act,
                       torch.as_tensor(gphi.astype(np.float32), device=dev), gpose, gedges)
    torch.cuda.synchronize()
    rp, re_ = oracle.psdf_backward(fp, edges, offs, poses, gphi, eta=eta)
    gp = gpose.cpu().numpy()
    assert np.max(np.abs(gp - rp)) <= 1e-4 * max(1.0, np.abs(rp).max())
    ge = gedges.cpu().numpy()
    err = np.abs(ge - re_) / np.maximum(1.0, np.abs(re_))
    assert err.max() <= 2e-4, (float(err.max()), np.unravel_index(err.argmax(), err.shape))


def test_soft_rejected_where_unsupported():
    w = sg.plain_rect_small(0)
    prm = psdf.make_params(eta=100.0)
    sc = psdf.Scene.from_csr(w.edges, w.offsets, params=prm)
    ps = torch.as_tensor(w.poses, device="cuda")
    n_tiles = sc.info().n_tiles
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.psdf_tile_values(w.footprint, sc, ps, prm,
                              torch.empty((w.P, n_tiles), device="cuda"))
    assert ei.value.code == psdf.PSDF_ERR_ARG
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.Plan([(w.footprint, w.edges, w.offsets, w.P)],
                  params=psdf.make_params(eta=float("inf")))
    assert ei.value.code == psdf.PSDF_ERR_ARG
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.eval_grad(sc, w.footprint, ps, params=psdf.make_params(eta=float("nan")))
    assert ei.value.code == psdf.PSDF_ERR_ARG


def _bits(t):
    return t.detach().cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("eta", [1.0, 50.0, 1000.0])
def test_soft_cull_equals_full_scan(eta):
    """The exact tile cull with the soft minimum (its upper bound raised by
    log(K) / eta, the most a penetrating obstacle's soft value can exceed
    zero): every output bit equal to the full scan's soft evaluation, with
    half of the poses penetrating, for two tilings and two proposal sizes."""
    w = sg.dense_clutter(4, n_rects=4000, n_poses=1024, field_side=80.0)
    poses = torch.as_tensor(_penetrating(w, 7, frac=0.5, spread=0.2), device="cuda")
    prm = psdf.make_params(eta=eta)
    hard_phi = None
    for te in (0, 32):
        scene = psdf.Scene.from_csr(w.edges, w.offsets, tile_edges=te)
        phi0, dphi0, act0 = psdf.eval_grad(scene, w.footprint, poses, params=prm)
        if hard_phi is None:
            hard_phi = psdf.eval_grad(scene, w.footprint, poses)[0]
        for k in (1, 3):
            phi1, dphi1, act1, _ws = psdf.eval_culled(scene, w.footprint, poses, k=k, params=prm)
            torch.cuda.synchronize()
            assert np.array_equal(_bits(phi0), _bits(phi1)), (te, k)
            assert np.array_equal(_bits(act0), _bits(act1)), (te, k)
            assert np.array_equal(_bits(dphi0), _bits(dphi1)), (te, k)
    # the soft minimum changes the penetrating poses' values
    pen = (hard_phi < 0).cpu().numpy()
    assert pen.sum() >= 100
    assert np.any(_bits(phi0)[pen] != _bits(hard_phi)[pen])
