"""Failure detection without a fault: the bounded device-side waits (the
tile copies of the full scan and of a batched plan) are made to give up at
once (poll limit 0).  The failure must be reported on the host
(PSDF_ERR_TIMEOUT), the affected outputs must be NaN / PSDF_PAIR_NONE, the
copies already issued still land before the kernel exits (nothing is left in
flight), and the next call with the default limit must be clean and exact."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2607_04310_b300 import psdf
from paper_2607_04310_b300 import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


class _WaitLimit:
    def __init__(self, polls):
        self.polls = polls

    def __enter__(self):
        self.prev = psdf.psdf_debug_set_wait_limit(self.polls)
        assert self.prev == psdf.DEFAULT_WAIT_LIMIT
        return self

    def __exit__(self, *a):
        psdf.psdf_debug_set_wait_limit(self.prev)


def _outputs(P, dev):
    return (torch.zeros(P, device=dev), torch.zeros((P, 3), device=dev),
            torch.zeros(P, dtype=torch.int32, device=dev))


def test_full_scan_wait_timeout_is_reported_and_the_next_call_is_clean():
    w = sg.plain_rect_small(0)
    dev = torch.device("cuda")
    scene = psdf.Scene.from_csr(w.edges, w.offsets, tile_edges=16)  # several tiles
    poses = torch.as_tensor(w.poses, device=dev)
    ws = psdf.workspace(w.P, dev)
    phi, dphi, act = _outputs(w.P, dev)
    with _WaitLimit(0):
        psdf.psdf_eval_grad(w.footprint, scene, poses, scene.params, phi, dphi, act, ws)
        rc = psdf.psdf_workspace_status(ws)
    assert rc == psdf.PSDF_ERR_TIMEOUT
    assert "ran out" in psdf.last_error()
    assert torch.isnan(phi).all() and torch.isnan(dphi).all()
    assert act.eq(-1).all()  # PSDF_PAIR_NONE read as int32
    # default limit again: clean status, oracle values
    psdf.psdf_eval_grad(w.footprint, scene, poses, scene.params, phi, dphi, act, ws)
    assert psdf.psdf_workspace_status(ws) == psdf.PSDF_OK
    ref = oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses)
    assert np.abs(phi.cpu().numpy() - ref["phi"]).max() <= 1e-5


def test_value_only_and_stage_params_report_the_timeout():
    w = sg.plain_rect_small(0)
    dev = torch.device("cuda")
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    poses = torch.as_tensor(w.poses, device=dev)
    ws = psdf.workspace(w.P, dev)
    phi, _dphi, act = _outputs(w.P, dev)
    stage = torch.zeros((w.P, 4), device=dev)
    with _WaitLimit(0):
        psdf.psdf_eval(w.footprint, scene, poses, scene.params, phi, act, ws)
        assert psdf.psdf_workspace_status(ws) == psdf.PSDF_ERR_TIMEOUT
        psdf.psdf_stage_params(w.footprint, scene, poses, scene.params, 0.01, stage, act, ws)
        assert psdf.psdf_workspace_status(ws) == psdf.PSDF_ERR_TIMEOUT
    assert torch.isnan(phi).all() and torch.isnan(stage).all()
    psdf.psdf_eval(w.footprint, scene, poses, scene.params, phi, act, ws)
    assert psdf.psdf_workspace_status(ws) == psdf.PSDF_OK
    assert torch.isfinite(phi).all()


def test_plan_wait_timeout_is_reported_and_the_next_call_is_clean():
    w = sg.plain_rect_small(0)
    dev = torch.device("cuda")
    h = w.P // 2
    plan = psdf.Plan([(w.footprint, w.edges, w.offsets, h),
                      (w.footprint, w.edges, w.offsets, w.P - h)], tile_edges=16)
    poses = torch.as_tensor(w.poses, device=dev)
    phi, dphi, act = _outputs(w.P, dev)
    with _WaitLimit(0):
        psdf.psdf_eval_batched(plan, poses, phi, dphi, act)
        rc = psdf.psdf_plan_status(plan)
    assert rc == psdf.PSDF_ERR_TIMEOUT
    assert torch.isnan(phi).all() and torch.isnan(dphi).all()
    assert act.eq(-1).all()
    psdf.psdf_eval_batched(plan, poses, phi, dphi, act)
    assert psdf.psdf_plan_status(plan) == psdf.PSDF_OK
    scene = psdf.Scene.from_csr(w.edges, w.offsets, tile_edges=16)
    phi1, dphi1, act1 = psdf.eval_grad(scene, w.footprint, poses)
    torch.cuda.synchronize()
    assert torch.equal(phi.view(torch.int32), phi1.view(torch.int32))
    assert torch.equal(act, act1)
