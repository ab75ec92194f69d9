"""The no-allocation entry point (psdf_eval_grad_noalloc), called through the
C ABI, must reproduce psdf_eval_grad (the workspace entry point) bit for bit
(it runs the same kernels on the same inputs), on two calls in a row, and
must leave the device's free memory unchanged.  It exists for callers that
may not allocate device memory while running (hard-period control loops,
plug-ins in a host framework that owns the memory pool).  This file is
collected last."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2607_04310_b300 import psdf
from paper_2607_04310_b300 import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _noalloc(w, scene, poses):
    P = poses.shape[0]
    phi = torch.full((P,), float("nan"), device="cuda")
    dphi = torch.full((P, 3), float("nan"), device="cuda")
    act = torch.zeros(P, dtype=torch.int32, device="cuda")
    fp = np.ascontiguousarray(w.footprint, dtype=np.float32)
    rc = psdf.load().psdf_eval_grad_noalloc(
        fp.ctypes.data, fp.shape[0], scene.handle, poses.data_ptr(), P,
        ctypes.byref(scene.params), phi.data_ptr(), dphi.data_ptr(), act.data_ptr(),
        torch.cuda.current_stream().cuda_stream)
    assert rc == psdf.PSDF_OK, psdf.last_error()
    torch.cuda.synchronize()
    return phi.cpu().numpy(), dphi.cpu().numpy(), psdf.pair_ids(act)


def _close(a, b):
    """Bit-for-bit equality (the parity tolerances, 1e-5 m and 1e-4, hold a
    fortiori)."""
    phi_a, g_a, p_a = a
    phi_b, g_b, p_b = b
    assert np.array_equal(phi_a.view(np.uint32), phi_b.view(np.uint32))
    assert np.array_equal(g_a.view(np.uint32), g_b.view(np.uint32))
    assert np.array_equal(p_a, p_b)


def test_noalloc_matches_workspace_entry_point_twice():
    w = sg.octagon_lidar(1, n_inst=16, horizon=50, n_rects=800, n_lines=40, segs_per_line=20)
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    poses = torch.as_tensor(w.poses, device="cuda")
    phi, dphi, act = psdf.eval_grad(scene, w.footprint, poses)
    torch.cuda.synchronize()
    ref = (phi.cpu().numpy(), dphi.cpu().numpy(), psdf.pair_ids(act))
    first = _noalloc(w, scene, poses)
    second = _noalloc(w, scene, poses)
    _close(first, ref)
    _close(second, ref)
    # a smaller batch after a larger one: the shared scratch is re-initialized
    part = _noalloc(w, scene, poses[:37])
    _close(part, tuple(x[:37] for x in ref))


def test_noalloc_leaves_free_memory_unchanged():
    """After a first call (which may load the library's kernels), further
    calls change the device's free memory by nothing."""
    w = sg.octagon_lidar(1, n_inst=8, horizon=50, n_rects=400, n_lines=20, segs_per_line=20)
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    poses = torch.as_tensor(w.poses, device="cuda")
    _noalloc(w, scene, poses)
    torch.cuda.synchronize()
    free0, _total = torch.cuda.mem_get_info()
    P = poses.shape[0]
    phi = torch.empty(P, device="cuda")
    dphi = torch.empty((P, 3), device="cuda")
    act = torch.empty(P, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free1, _total = torch.cuda.mem_get_info()
    for _ in range(5):
        rc = psdf.psdf_eval_grad_noalloc(w.footprint, scene, poses, scene.params, phi, dphi, act)
        assert rc == psdf.PSDF_OK, psdf.last_error()
    torch.cuda.synchronize()
    free2, _total = torch.cuda.mem_get_info()
    assert free2 == free1, (free0, free1, free2)


def test_noalloc_rejects_oversize_batch():
    w = sg.plain_rect_small(0)
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    P = psdf.NOALLOC_MAX_POSES + 1
    poses = torch.zeros((P, 3), device="cuda")
    out = torch.empty(P, device="cuda")
    g = torch.empty((P, 3), device="cuda")
    act = torch.empty(P, dtype=torch.int32, device="cuda")
    rc = psdf.psdf_eval_grad_noalloc(w.footprint, scene, poses, scene.params, out, g, act)
    assert rc == psdf.PSDF_ERR_CAPACITY
    assert "at most" in psdf.last_error()
