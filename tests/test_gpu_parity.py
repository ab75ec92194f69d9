"""GPU (CUDA, sm_103a) vs the FP64 oracle, element by element, through the
C ABI.  Values within 1e-5 m; active pair bit-exact (or its antiparallel
twin) where the FP64 runner-up is >= 1e-5 m away; pose gradients within 1e-4
relative away from ties."""
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


def test_plain_rect_small_full():
    """rect footprint, 20 poses x 200 edges (50 rectangles), seed 0."""
    w = sg.plain_rect_small(0)
    gpu, _ = parity.gpu_eval(w)
    ref = parity.oracle_eval(w)
    st = parity.compare(gpu, ref)
    assert st["pair_checked"] >= 15


def test_plain_rect_dense_poses():
    """many poses on the same scene, with penetrations (poses near corners)."""
    w = sg.plain_rect_small(0)
    g = np.random.default_rng(5)
    n = 3000
    idx = g.integers(0, w.E, size=n)
    poses = np.concatenate([w.edges[idx, 0:2] + g.normal(size=(n, 2)) * 0.5,
                            g.uniform(-math.pi, math.pi, size=(n, 1))], axis=1).astype(np.float32)
    gpu, _ = parity.gpu_eval(w, poses=poses)
    ref = parity.oracle_eval(w, poses=poses)
    st = parity.compare(gpu, ref)
    assert np.sum(ref["phi"] < 0) > 300
    assert st["grad_checked"] > 1500
    # a centrally symmetric footprint ties every "robot max - obstacle min"
    # overlap (kind 4) exactly with kind 3 on the antiparallel axis; the
    # lowest pair id is kind 3, so kind 4 cannot be reported here
    kinds = set((gpu["pair"] >> 4) & 0xF)
    assert {0, 1, 3, 7, 8} <= kinds and 4 not in kinds, kinds


def test_octagon_lidar_sampled():
    """octagon footprint, 3,200 poses x 20,000 edges (rects + polyline segments);
    every pose on the GPU in one launch, 256 sampled poses checked."""
    w = sg.octagon_lidar(1)
    gpu, sc = parity.gpu_eval(w)
    assert sc.info().n_edges == 20000
    g = np.random.default_rng(0)
    idx = np.sort(g.choice(w.P, size=256, replace=False))
    ref = parity.oracle_eval(w, poses=w.poses[idx])
    parity.compare(gpu, ref, idx=idx)


def test_octagon_lidar_near_segments():
    """poses pushed onto the polyline segments: shared endpoints, segment B
    kinds, penetration of one-edge obstacles."""
    w = sg.octagon_lidar(1, n_inst=2, horizon=5, n_rects=300, n_lines=30, segs_per_line=20)
    seg0 = 4 * 300
    g = np.random.default_rng(1)
    n = 2000
    idx = g.integers(seg0, w.E, size=n)
    poses = np.concatenate([w.edges[idx, 0:2] + g.normal(size=(n, 2)) * 0.4,
                            g.uniform(-math.pi, math.pi, size=(n, 1))], axis=1).astype(np.float32)
    gpu, _ = parity.gpu_eval(w, poses=poses)
    ref = parity.oracle_eval(w, poses=poses)
    parity.compare(gpu, ref)
    kinds = set((gpu["pair"] >> 4) & 0xF)
    assert {0, 2, 5, 6} & kinds, kinds


@pytest.mark.parametrize("m", list(range(3, 17)))
def test_every_footprint_size(m):
    g = sg.rng(100 + m)
    fp = sg.footprint_random_convex(g, m, 0.3, 0.6, min_gap=min(0.3, math.pi / m))
    e1, o1 = sg.convex_polygons(g, 40, 3, 8, 0.2, 1.0, 0.0, 12.0)
    e2, o2 = sg.polyline_segments(g, 5, 10, 0.2, 1.0, 0.0, 12.0)
    edges, offs = sg.concat((e1, o1), (e2, o2))
    n = 600
    idx = g.integers(0, len(edges), size=n)
    poses = np.concatenate([edges[idx, 0:2] + g.normal(size=(n, 2)) * 0.5,
                            g.uniform(-math.pi, math.pi, size=(n, 1))], axis=1).astype(np.float32)
    w = sg.Workload("m%d" % m, fp, edges, offs, poses)
    gpu, _ = parity.gpu_eval(w)
    ref = parity.oracle_eval(w)
    parity.compare(gpu, ref)
    kinds = set((gpu["pair"] >> 4) & 0xF)
    assert {0, 1} <= kinds and ({3, 4} & kinds) and ({7, 8} & kinds), kinds
    if m % 2:
        # an odd hull has no antiparallel twin, so the "robot max - obstacle
        # min" robot-axis side (kind 4) is reported, unlike kind 3 ties
        assert 4 in kinds, kinds


def test_tiling_and_ragged_sizes_bitwise():
    """tile size and pose count do not change a single bit of the result."""
    w = sg.octagon_lidar(1, n_inst=3, horizon=43, n_rects=500, n_lines=20, segs_per_line=10)
    base, _ = parity.gpu_eval(w, tile_edges=256)
    for te in (4, 7, 64, 100):
        other, _ = parity.gpu_eval(w, tile_edges=te)
        assert np.array_equal(base["phi"].view(np.uint32), other["phi"].view(np.uint32))
        assert np.array_equal(base["pair"], other["pair"])
        assert np.array_equal(base["grad"].view(np.uint32), other["grad"].view(np.uint32))
    for P in (1, 127, 128, 129, 5):
        sub, _ = parity.gpu_eval(w, poses=w.poses[:P])
        assert np.array_equal(sub["phi"].view(np.uint32), base["phi"][:P].view(np.uint32))
    again, _ = parity.gpu_eval(w, tile_edges=256)
    assert np.array_equal(base["phi"].view(np.uint32), again["phi"].view(np.uint32))


def test_padded_layout_matches_csr():
    w = sg.octagon_lidar(1, n_inst=2, horizon=20, n_rects=100, n_lines=10, segs_per_line=5)
    A, B, S = sg.to_padded(w.edges, w.offsets, mbar=6)
    csr, _ = parity.gpu_eval(w)
    sc = psdf.Scene.from_padded(A, B, S)
    pad, _ = parity.gpu_eval(w, scene=sc)
    assert np.array_equal(csr["phi"].view(np.uint32), pad["phi"].view(np.uint32))
    # padded ids report i * mbar + j
    counts = np.diff(w.offsets)
    row_of_edge = np.concatenate([i * 6 + np.arange(c) for i, c in enumerate(counts)])
    e_csr = csr["pair"] >> 8
    assert np.array_equal(row_of_edge[e_csr], pad["pair"] >> 8)
    assert np.array_equal(csr["pair"] & 0xFF, pad["pair"] & 0xFF)


def test_empty_scene_and_empty_batch():
    fp = sg.footprint_rect()
    sc = psdf.Scene.from_csr(np.zeros((0, 4), np.float32), np.zeros(1, np.int32))
    ps = torch.tensor([[1.0, 2.0, 0.3]], device="cuda")
    phi, dphi, act = psdf.eval_grad(sc, fp, ps)
    torch.cuda.synchronize()
    assert math.isinf(phi.item()) and phi.item() > 0
    assert psdf.pair_ids(act)[0] == psdf.PAIR_NONE
    assert torch.all(dphi == 0)
    w = sg.plain_rect_small(0)
    sc2 = psdf.Scene.from_csr(w.edges, w.offsets)
    empty = torch.zeros((0, 3), device="cuda")
    phi, dphi, act = psdf.eval_grad(sc2, fp, empty)
    assert phi.numel() == 0


def test_argument_errors():
    w = sg.plain_rect_small(0)
    sc = psdf.Scene.from_csr(w.edges, w.offsets)
    ps = torch.as_tensor(w.poses, device="cuda")
    phi = torch.empty(w.P, device="cuda")
    act = torch.empty(w.P, dtype=torch.int32, device="cuda")
    ws = psdf.workspace(w.P)
    prm = psdf.make_params()
    with pytest.raises(psdf.PsdfError) as ei:  # clockwise footprint
        psdf.psdf_eval(w.footprint[::-1].copy(), sc, ps, prm, phi, act, ws)
    assert ei.value.code == psdf.PSDF_ERR_FOOTPRINT
    with pytest.raises(psdf.PsdfError) as ei:  # eps differs from the scene's
        psdf.psdf_eval(w.footprint, sc, ps, psdf.make_params(eps_seg=1e-9), phi, act, ws)
    assert ei.value.code == psdf.PSDF_ERR_ARG
    with pytest.raises(psdf.PsdfError) as ei:  # workspace too small
        psdf.psdf_eval(w.footprint, sc, ps, prm, phi, act, ws[:64])
    assert ei.value.code in (psdf.PSDF_ERR_CAPACITY, psdf.PSDF_ERR_ARG)
    with pytest.raises(psdf.PsdfError) as ei:  # host poses
        psdf.psdf_eval(w.footprint, sc, torch.as_tensor(w.poses), prm, phi, act, ws)
    assert ei.value.code == psdf.PSDF_ERR_ARG
    # a valid call after the rejected ones writes the status word
    psdf.psdf_eval(w.footprint, sc, ps, prm, phi, act, ws)
    assert psdf.psdf_workspace_status(ws) == psdf.PSDF_OK


def test_eps_variants():
    """eps_seg / eps_axis / eps_sat > 0 follow the oracle."""
    w = sg.plain_rect_small(0)
    prm = psdf.make_params(eps_seg=1e-6, eps_axis=1e-6, eps_sat=1e-4)
    gpu, _ = parity.gpu_eval(w, params=prm)
    ref = parity.oracle_eval(w, eps_seg=1e-6, eps_axis=1e-6, eps_sat=1e-4)
    parity.compare(gpu, ref)


def test_gradient_against_fd_of_oracle():
    """GPU pose gradient vs central differences (h = 1e-6) of the FP64 oracle
    value, at poses >= 1e-3 m from any argmin tie."""
    w = sg.backward_rects(3, n_inst=8, horizon=40, n_rects=400)
    gpu, _ = parity.gpu_eval(w)
    ref = parity.oracle_eval(w)
    sel = np.nonzero((ref["margin"] >= 1e-3) & ((ref["phi"] < 0) | (ref["phi"] >= 1e-2)))[0]
    assert len(sel) > 100
    h = 1e-6
    fd = np.empty((len(sel), 3))
    for k in range(3):
        pp = w.poses[sel].astype(np.float64)
        pm = pp.copy()
        pp[:, k] += h
        pm[:, k] -= h
        fd[:, k] = (parity.oracle_eval(w, poses=pp)["phi"] - parity.oracle_eval(w, poses=pm)["phi"]) / (2 * h)
    rel = np.linalg.norm(gpu["grad"][sel] - fd, axis=1) / np.maximum(np.linalg.norm(fd, axis=1), 1.0)
    assert rel.max() <= parity.GRAD_RTOL, rel.max()
