"""Largest supported sizes and the rejections just past them: obstacles of
256 edges (one per tile), a 16-vertex footprint, through the full scan, the
cull and a batched plan; 257-edge obstacles and 17-vertex footprints are
refused before any launch."""
from __future__ import annotations

import numpy as np
import pytest

import parity
from paper_2607_04310_b300 import psdf
from paper_2607_04310_b300 import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _scene():
    g = np.random.default_rng(21)
    big, bo = sg.regular_polygons([(5.0, 5.0), (9.0, 4.0)], [256, 255], [1.5, 1.0])
    small, so = sg.rects(g, 40, 0.2, 1.0, 0.0, 12.0)
    edges, offs = sg.concat((big, bo), (small, so))
    fp = sg.footprint_regular(16, 0.45)
    n = 600
    centre = np.array([[5.0, 5.0]] * (n // 2) + [[9.0, 4.0]] * (n - n // 2))
    ang = g.uniform(-np.pi, np.pi, size=n)
    rad = g.uniform(0.0, 2.6, size=n)
    poses = np.concatenate([centre + np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1),
                            g.uniform(-np.pi, np.pi, size=(n, 1))], axis=1).astype(np.float32)
    return sg.Workload("limits", fp, edges, offs, poses)


def test_max_obstacle_and_footprint_against_oracle():
    w = _scene()
    gpu, sc = parity.gpu_eval(w, tile_edges=256)
    assert sc.info().max_obstacle_edges == 256
    ref = parity.oracle_eval(w)
    parity.compare(gpu, ref)
    assert np.sum(ref["phi"] < 0) >= 50 and np.sum(ref["phi"] > 0) >= 50


def test_max_sizes_cull_and_plan_bitwise():
    w = _scene()
    sc = psdf.Scene.from_csr(w.edges, w.offsets)
    ps = torch.as_tensor(w.poses, device="cuda")
    phi0, dphi0, act0 = psdf.eval_grad(sc, w.footprint, ps)
    phi1, dphi1, act1, _ = psdf.eval_culled(sc, w.footprint, ps, k=1)
    plan = psdf.Plan([(w.footprint, w.edges, w.offsets, w.P)])
    phi2, dphi2, act2 = psdf.eval_batched(plan, ps)
    torch.cuda.synchronize()
    for a, b, c in ((phi0, phi1, phi2), (dphi0, dphi1, dphi2), (act0, act1, act2)):
        x = a.cpu().numpy().view(np.uint32)
        assert np.array_equal(x, b.cpu().numpy().view(np.uint32))
        assert np.array_equal(x, c.cpu().numpy().view(np.uint32))


def test_oversize_inputs_rejected():
    e257, o257 = sg.regular_polygons([(0.0, 0.0)], [257], [2.0])
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.Scene.from_csr(e257, o257)
    assert ei.value.code == psdf.PSDF_ERR_CAPACITY
    w = _scene()
    sc = psdf.Scene.from_csr(w.edges, w.offsets)
    fp17 = sg.footprint_regular(17, 0.45)
    ps = torch.as_tensor(w.poses[:4], device="cuda")
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.eval_grad(sc, fp17, ps)
    assert ei.value.code == psdf.PSDF_ERR_FOOTPRINT
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.Plan([(fp17, w.edges, w.offsets, 4)])
    assert ei.value.code == psdf.PSDF_ERR_FOOTPRINT
    # an obstacle larger than the tile
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.Scene.from_csr(w.edges, w.offsets, tile_edges=128)
    assert ei.value.code == psdf.PSDF_ERR_ARG
