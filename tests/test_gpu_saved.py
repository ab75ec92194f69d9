"""Backward from records saved by the forward (psdf_eval_grad_save,
psdf_eval_culled_save -> psdf_backward_saved): the same gradients as the
recomputing backward (which the backward tests pin to the FP64 oracle), the
cull's records equal to the full scan's bit for bit, and the argument and
bounds checks."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2607_04310_b300 import psdf
from paper_2607_04310_b300 import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

DEV = "cuda"


def _bits(t):
    return t.detach().cpu().numpy().view(np.uint32)


def _forward_save(w, scene, poses):
    P = poses.shape[0]
    phi = torch.empty(P, device=DEV)
    dphi = torch.empty((P, 3), device=DEV)
    act = torch.empty(P, dtype=torch.int32, device=DEV)
    saved = torch.full((P, psdf.SAVED_FLOATS), float("nan"), device=DEV)
    psdf.psdf_eval_grad_save(w.footprint, scene, poses, scene.params, phi, dphi, act, saved,
                             psdf.workspace(P, poses.device))
    return phi, dphi, act, saved


def _backward_both(w, scene, poses, act, saved, gphi):
    P = poses.shape[0]
    gp0 = torch.empty((P, 3), device=DEV)
    ge0 = torch.zeros((w.E, 4), device=DEV)
    psdf.psdf_backward(w.footprint, scene, poses, scene.params, act, gphi, gp0, ge0)
    gp1 = torch.empty((P, 3), device=DEV)
    ge1 = torch.zeros((w.E, 4), device=DEV)
    psdf.psdf_backward_saved(scene, saved, gphi, gp1, ge1)
    torch.cuda.synchronize()
    return gp0, ge0, gp1, ge1


def _check_records(w, saved, dphi, act):
    s = saved.cpu().numpy()
    nrow = s[:, 3].view(np.int32)
    assert set(np.unique(nrow)) <= {-1, 0, 1, 2, 3}
    has = nrow >= 0
    # the pose gradient is the forward's dphi, bit for bit
    d = dphi.detach().cpu().numpy()
    assert np.array_equal(s[has, 0:3].view(np.uint32), d[has].view(np.uint32))
    assert np.all(d[~has] == 0) and np.all(s[~has, 0:3] == 0)
    # rows: caller edge row * 4 + column (0 or 2) of a valid row, unused ones -1
    idx = s[:, [4, 7, 10]].view(np.int32)
    used = np.arange(3)[None, :] < nrow[:, None]
    assert np.all(idx[~used] == -1)
    iu = idx[used]
    assert np.all((iu >= 0) & (iu < 4 * w.E) & (iu % 2 == 0))
    # a pose with a gradient has an active pair; its rows name that pair's obstacle
    pid = psdf.pair_ids(act)
    assert np.all(pid[has] != psdf.PAIR_NONE)
    return int(has.sum())


@pytest.mark.parametrize("name", ["rects", "octagon_lidar"])
def test_saved_backward_equals_recomputing_backward(name):
    if name == "rects":
        w = sg.backward_rects(3, n_inst=32, horizon=40, n_rects=600)
    else:
        w = sg.octagon_lidar(1)
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    poses = torch.as_tensor(w.poses, device=DEV)
    phi, dphi, act, saved = _forward_save(w, scene, poses)
    # the same forward outputs as psdf_eval_grad
    phi0, dphi0, act0 = psdf.eval_grad(scene, w.footprint, poses)
    assert np.array_equal(_bits(phi), _bits(phi0))
    assert np.array_equal(_bits(dphi), _bits(dphi0))
    assert np.array_equal(_bits(act), _bits(act0))
    assert _check_records(w, saved, dphi, act) > 100
    g = np.random.default_rng(7)
    gphi = torch.as_tensor(g.normal(size=w.P).astype(np.float32), device=DEV)
    gp0, ge0, gp1, ge1 = _backward_both(w, scene, poses, act, saved, gphi)
    assert np.array_equal(_bits(gp0), _bits(gp1))
    e0, e1 = ge0.cpu().numpy(), ge1.cpu().numpy()
    # float atomics: the same addends in another order
    assert np.allclose(e0, e1, rtol=1e-5, atol=1e-6 * max(1.0, np.abs(e0).max()))
    assert np.array_equal(e0 != 0, e1 != 0)
    if name == "octagon_lidar":  # one-edge obstacles put gradients in their B slots
        seg_rows = np.repeat(np.diff(w.offsets) == 1, np.diff(w.offsets))
        assert np.any(e1[seg_rows, 2:4] != 0)


@pytest.mark.parametrize("k", [1, 3])
def test_culled_records_equal_full_scan(k):
    w = sg.dense_clutter(4, n_rects=4000, n_poses=1024, field_side=80.0)
    scene = psdf.Scene.from_csr(w.edges, w.offsets, tile_edges=32)
    poses = torch.as_tensor(w.poses, device=DEV)
    _, dphi0, act0, saved0 = _forward_save(w, scene, poses)
    P = w.P
    phi = torch.empty(P, device=DEV)
    dphi = torch.empty((P, 3), device=DEV)
    act = torch.empty(P, dtype=torch.int32, device=DEV)
    saved = torch.full((P, psdf.SAVED_FLOATS), float("nan"), device=DEV)
    ws = torch.empty(psdf.psdf_cull_workspace_bytes(P, scene), dtype=torch.uint8, device=DEV)
    psdf.psdf_eval_culled_save(w.footprint, scene, None, psdf.CullOpts(psdf.PROPOSE_BOUND, k),
                               poses, scene.params, phi, dphi, act, saved, ws)
    torch.cuda.synchronize()
    assert np.array_equal(_bits(saved), _bits(saved0))
    assert np.array_equal(_bits(act), _bits(act0))
    gphi = torch.ones(P, device=DEV)
    gp0, ge0, gp1, ge1 = _backward_both(w, scene, poses, act, saved, gphi)
    assert np.array_equal(_bits(gp0), _bits(gp1))
    assert np.allclose(ge0.cpu().numpy(), ge1.cpu().numpy(), rtol=1e-5, atol=1e-6)


def test_saved_empty_scene_and_zero_poses():
    w = sg.plain_rect_small(0)
    empty = psdf.Scene.from_csr(np.zeros((0, 4), np.float32), np.zeros(1, np.int32))
    poses = torch.as_tensor(w.poses[:5], device=DEV)
    _, dphi, _, saved = _forward_save(w, empty, poses)
    s = saved.cpu().numpy()
    assert np.all(s[:, 3].view(np.int32) == -1)
    gp = torch.full((5, 3), 7.0, device=DEV)
    psdf.psdf_backward_saved(empty, saved, torch.ones(5, device=DEV), gp, None)
    torch.cuda.synchronize()
    assert torch.all(gp == 0)
    # P = 0 is a no-op
    psdf.psdf_backward_saved(empty, saved[:0], torch.ones(0, device=DEV), gp[:0], None)


def test_saved_rejects_soft_and_misaligned():
    w = sg.plain_rect_small(0)
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    poses = torch.as_tensor(w.poses, device=DEV)
    P = w.P
    phi = torch.empty(P, device=DEV)
    dphi = torch.empty((P, 3), device=DEV)
    act = torch.empty(P, dtype=torch.int32, device=DEV)
    saved = torch.empty((P + 1, psdf.SAVED_FLOATS), device=DEV)
    ws = psdf.workspace(P, poses.device)
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.psdf_eval_grad_save(w.footprint, scene, poses, psdf.make_params(eta=100.0), phi,
                                 dphi, act, saved, ws)
    assert ei.value.code == psdf.PSDF_ERR_ARG
    cws = torch.empty(psdf.psdf_cull_workspace_bytes(P, scene), dtype=torch.uint8, device=DEV)
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.psdf_eval_culled_save(w.footprint, scene, None, psdf.CullOpts(psdf.PROPOSE_BOUND, 1),
                                   poses, psdf.make_params(eta=100.0), phi, dphi, act, saved, cws)
    assert ei.value.code == psdf.PSDF_ERR_ARG
    off = saved.view(-1)[1:1 + P * psdf.SAVED_FLOATS].view(P, psdf.SAVED_FLOATS)  # 4-byte offset
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.psdf_eval_grad_save(w.footprint, scene, poses, scene.params, phi, dphi, act, off, ws)
    assert ei.value.code == psdf.PSDF_ERR_ARG
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.psdf_backward_saved(scene, off, torch.ones(P, device=DEV), None, None)
    assert ei.value.code == psdf.PSDF_ERR_ARG


def test_saved_rows_outside_the_scene_are_skipped():
    """Records that name rows beyond the scene (not written by a forward on
    this scene) touch nothing outside grad_edges."""
    w = sg.plain_rect_small(0)
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    rec = np.zeros((3, psdf.SAVED_FLOATS), np.float32)
    iv = rec.view(np.int32)
    iv[:, 3] = 3
    iv[:, [4, 7, 10]] = -1
    iv[0, 4] = 4 * w.E          # first row past the end
    iv[1, 4] = 4 * w.E - 1      # its second column past the end
    iv[2, 4] = -8               # negative
    iv[2, 7] = 0                # one valid row (edge 0, A)
    rec[:, [5, 6, 8, 9, 11, 12]] = 1.0
    saved = torch.as_tensor(rec, device=DEV)
    ge = torch.zeros((w.E + 1, 4), device=DEV)  # one guard row past the scene's rows
    psdf.psdf_backward_saved(scene, saved, torch.ones(3, device=DEV), None, ge[:w.E])
    torch.cuda.synchronize()
    g = ge.cpu().numpy()
    assert np.all(g[w.E] == 0)
    assert g[0, 0] == 1.0 and g[0, 1] == 1.0
    assert np.count_nonzero(g) == 2


def test_zero_copy_host_buffers_equal_device_buffers():
    """Poses read and outputs written by the kernels in pinned, device-mapped
    host memory give the device-buffer results bit for bit; pageable host
    poses stay rejected."""
    w = sg.dense_clutter(4, n_rects=4000, n_poses=1024, field_side=80.0)
    scene = psdf.Scene.from_csr(w.edges, w.offsets, tile_edges=32)
    P = w.P
    poses = torch.as_tensor(w.poses, device=DEV)
    _, dphi0, act0, saved0 = _forward_save(w, scene, poses)
    phi0 = psdf.eval_grad(scene, w.footprint, poses)[0]
    h_poses = torch.as_tensor(w.poses).pin_memory()
    h_phi = torch.empty(P).pin_memory()
    h_dphi = torch.empty((P, 3)).pin_memory()
    h_act = torch.empty(P, dtype=torch.int32).pin_memory()
    saved = torch.empty((P, psdf.SAVED_FLOATS), device=DEV)
    ws = torch.empty(psdf.psdf_cull_workspace_bytes(P, scene), dtype=torch.uint8, device=DEV)
    psdf.psdf_eval_culled_save(w.footprint, scene, None, psdf.CullOpts(psdf.PROPOSE_BOUND, 2),
                               h_poses, scene.params, h_phi, h_dphi, h_act, saved, ws)
    torch.cuda.synchronize()
    assert np.array_equal(h_phi.numpy().view(np.uint32), _bits(phi0))
    assert np.array_equal(h_dphi.numpy().view(np.uint32), _bits(dphi0))
    assert np.array_equal(h_act.numpy(), act0.cpu().numpy())
    assert np.array_equal(_bits(saved), _bits(saved0))
    with pytest.raises(psdf.PsdfError) as ei:  # pageable host poses
        psdf.psdf_eval_culled_save(w.footprint, scene, None, psdf.CullOpts(psdf.PROPOSE_BOUND, 2),
                                   torch.as_tensor(w.poses), scene.params, h_phi, h_dphi, h_act,
                                   saved, ws)
    assert ei.value.code == psdf.PSDF_ERR_ARG


@pytest.mark.parametrize("mode", [psdf.PROPOSE_CIRCLES, psdf.PROPOSE_BOUND])
@pytest.mark.parametrize("P", [1, 7, 1021])
def test_cull_outputs_in_blocks_ragged_host_and_absent(mode, P):
    """The cull stores each CTA's phi, active pairs and pose gradients as
    contiguous blocks: with a pose count that fills no whole CTA, outputs in
    pinned host memory, and some outputs absent, every written value equals
    the full scan's bit for bit and nothing past the last pose is touched."""
    w = sg.dense_clutter(4, n_rects=4000, n_poses=1024, field_side=80.0)
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    poses = torch.as_tensor(w.poses[:P].copy(), device=DEV)
    phi0, dphi0, act0, saved0 = _forward_save(w, scene, poses)
    opts = psdf.CullOpts(mode, 1)
    ws = torch.empty(psdf.psdf_cull_workspace_bytes(P, scene), dtype=torch.uint8, device=DEV)
    # host outputs with a sentinel tail after the last pose
    h_phi = torch.full((P + 9,), 7.0).pin_memory()
    h_dphi = torch.full((P + 9, 3), 7.0).pin_memory()
    h_act = torch.full((P + 9,), 12345, dtype=torch.int32).pin_memory()
    saved = torch.full((P, psdf.SAVED_FLOATS), float("nan"), device=DEV)
    psdf.psdf_eval_culled_save(w.footprint, scene, None, opts, poses, scene.params, h_phi[:P],
                               h_dphi[:P], h_act[:P], saved, ws)
    torch.cuda.synchronize()
    assert np.array_equal(h_phi[:P].numpy().view(np.uint32), _bits(phi0))
    assert np.array_equal(h_dphi[:P].numpy().view(np.uint32), _bits(dphi0))
    assert np.array_equal(h_act[:P].numpy(), act0.cpu().numpy())
    assert np.array_equal(_bits(saved), _bits(saved0))
    assert np.all(h_phi[P:].numpy() == 7.0) and np.all(h_dphi[P:].numpy() == 7.0)
    assert np.all(h_act[P:].numpy() == 12345)
    # phi alone (no gradient, no active pair) into device memory
    phi1 = torch.full((P + 9,), 7.0, device=DEV)
    psdf.psdf_eval_culled(w.footprint, scene, None, opts, poses, scene.params, phi1[:P], None,
                          None, ws)
    torch.cuda.synchronize()
    assert np.array_equal(_bits(phi1[:P]), _bits(phi0))
    assert np.all(phi1[P:].cpu().numpy() == 7.0)


def test_zero_copy_full_scan_and_backward():
    """The full scan with pinned, device-mapped host poses and outputs, then
    the saved-row backward: the device-buffer results bit for bit."""
    w = sg.octagon_lidar(1)
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    P = w.P
    poses = torch.as_tensor(w.poses, device=DEV)
    phi0, dphi0, act0, saved0 = _forward_save(w, scene, poses)
    h_poses = torch.as_tensor(w.poses).pin_memory()
    h_phi = torch.empty(P).pin_memory()
    h_dphi = torch.empty((P, 3)).pin_memory()
    h_act = torch.empty(P, dtype=torch.int32).pin_memory()
    saved = torch.empty((P, psdf.SAVED_FLOATS), device=DEV)
    psdf.psdf_eval_grad_save(w.footprint, scene, h_poses, scene.params, h_phi, h_dphi, h_act,
                             saved, psdf.workspace(P, poses.device))
    gp = torch.empty((P, 3), device=DEV)
    psdf.psdf_backward_saved(scene, saved, torch.ones(P, device=DEV), gp, None)
    torch.cuda.synchronize()
    assert np.array_equal(h_phi.numpy().view(np.uint32), _bits(phi0))
    assert np.array_equal(h_dphi.numpy().view(np.uint32), _bits(dphi0))
    assert np.array_equal(h_act.numpy(), act0.cpu().numpy())
    assert np.array_equal(_bits(saved), _bits(saved0))
    assert np.array_equal(_bits(gp), _bits(dphi0))
