"""SQP-RTI stage parameters (Alg. 1: h = phi - d_min, J_g = -grad phi) from
the fused epilogue: bitwise equal to psdf_eval_grad's outputs converted on
the host, and, for time-varying per-stage edge sets through a batched plan
(one instance per stage), against the FP64 oracle stage by stage."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2607_04310_b300 import psdf
from paper_2607_04310_b300 import scenegen as sg

from parity import CONTACT, GRAD_RTOL, GRAD_TAU, TIE_TAU, VALUE_TOL

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

D_MIN = 0.01  # m, the clearance of the paper's MPC settings


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


def test_stage_params_equal_eval_grad():
    w = sg.octagon_lidar(1)
    sc = psdf.Scene.from_csr(w.edges, w.offsets)
    ps = torch.as_tensor(w.poses, device="cuda")
    phi, dphi, act = psdf.eval_grad(sc, w.footprint, ps)
    stage = torch.empty((w.P, 4), device="cuda")
    act2 = torch.empty(w.P, dtype=torch.int32, device="cuda")
    psdf.psdf_stage_params(w.footprint, sc, ps, sc.params, D_MIN, stage, act2,
                           psdf.workspace(w.P))
    torch.cuda.synchronize()
    st = stage.cpu().numpy()
    h = (phi.cpu().numpy() - np.float32(D_MIN)).astype(np.float32)
    assert np.array_equal(_bits(st[:, 0]), _bits(h))
    assert np.array_equal(_bits(st[:, 1:]), _bits(-dphi.cpu().numpy()))
    assert torch.equal(act, act2)


def test_stage_params_time_varying_edge_sets():
    """64 MPC problems x 15 stages, each stage its own (moving) obstacles."""
    insts = sg.moving_obstacle_stages(5, n_mpc=64, horizon=15)
    plan = psdf.Plan([(w.footprint, w.edges, w.offsets, 1) for w in insts])
    poses = torch.as_tensor(np.concatenate([w.poses for w in insts]), device="cuda")
    P = plan.n_poses
    stage = torch.empty((P, 4), device="cuda")
    act = torch.empty(P, dtype=torch.int32, device="cuda")
    psdf.psdf_stage_params_batched(plan, poses, D_MIN, stage, act)
    torch.cuda.synchronize()
    st = stage.cpu().numpy()
    pair = psdf.pair_ids(act)
    n_grad = 0
    for i, w in enumerate(insts):
        ref = oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses)
        h_ref = ref["phi"][0] - D_MIN
        assert abs(st[i, 0] - h_ref) <= VALUE_TOL, (i, st[i, 0], h_ref)
        if ref["margin"][0] >= TIE_TAU:
            assert pair[i] in (ref["pair"][0], ref["twin"][0])
        if ref["margin"][0] >= GRAD_TAU and (ref["phi"][0] < 0 or ref["phi"][0] >= CONTACT):
            J_ref = -ref["grad"][0]
            err = np.linalg.norm(st[i, 1:] - J_ref) / max(1.0, np.linalg.norm(J_ref))
            assert err <= GRAD_RTOL, (i, st[i, 1:], J_ref)
            n_grad += 1
    assert n_grad >= 0.8 * len(insts)
    # sign convention: h(x + dx) = h(x) - J_g dx to first order (J_g = -grad phi)
    g = np.random.default_rng(0)
    dx = (g.normal(size=(P, 3)) * 1e-4).astype(np.float32)
    stage2 = torch.empty((P, 4), device="cuda")
    psdf.psdf_stage_params_batched(plan, poses + torch.as_tensor(dx, device="cuda"), D_MIN,
                                   stage2)
    torch.cuda.synchronize()
    st2 = stage2.cpu().numpy().astype(np.float64)
    lin = st[:, 0] - np.sum(st[:, 1:] * dx, axis=1)
    ok = (st[:, 0] > 0.05) & (st2[:, 0] > 0.05)
    assert ok.sum() >= 100
    err = np.abs(st2[ok, 0] - lin[ok])
    # second order in |dx| ~ 1e-4 except where the active pair changes within the step
    assert np.quantile(err, 0.95) <= 2e-6, np.quantile(err, 0.95)
    assert err.max() <= 1e-3


def test_stage_params_rejects_bad_arguments():
    w = sg.plain_rect_small(0)
    sc = psdf.Scene.from_csr(w.edges, w.offsets)
    ps = torch.as_tensor(w.poses, device="cuda")
    stage = torch.empty((w.P, 4), device="cuda")
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.psdf_stage_params(w.footprint, sc, ps, sc.params, float("inf"), stage, None,
                               psdf.workspace(w.P))
    assert ei.value.code == psdf.PSDF_ERR_ARG
