"""Batched plan: many uneven instances (footprint, own edge set, run of poses)
in one persistent launch.  Checked bit for bit against the single-scene path
per instance, against the FP64 oracle, across every autotuner candidate, and
under CUDA-graph replay."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2607_04310_b300 import psdf
from paper_2607_04310_b300 import scenegen as sg

from parity import compare

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _bits(t):
    return t.detach().cpu().numpy().view(np.uint32)


def _mixed_instances(seed, n_inst=36):
    """Footprints of 3..16 vertices, rectangles + one-edge segments, empty
    edge sets, zero / one / many poses (more than one pose block)."""
    g = np.random.default_rng(seed)
    out = []
    horizons = [0, 1, 7, 50, 127, 128, 129, 300]
    for i in range(n_inst):
        k = int(g.integers(3, 17))
        fp = sg.footprint_random_convex(g, k, 0.3, 0.6, min_gap=min(0.3, math.pi / k))
        side = float(g.uniform(5.0, 30.0))
        parts = []
        nr = int(g.integers(0, 400)) if i % 9 else 0
        if nr:
            parts.append(sg.rects(g, nr, 0.2, 2.0, 0.0, side))
        if i % 3 == 0 and i % 9:
            parts.append(sg.polyline_segments(g, 3, 10, 0.1, 1.0, 0.0, side))
        if parts:
            edges, offs = sg.concat(*parts)
        else:
            edges, offs = np.zeros((0, 4), np.float32), np.zeros(1, np.int64)
        N = horizons[i % len(horizons)]
        poses = sg.poses_uniform(g, N, 0.0, side)
        out.append(sg.Instance(fp, edges, offs, poses))
    return out


def _plan(insts, **kw):
    return psdf.Plan([(w.footprint, w.edges, w.offsets, w.poses.shape[0]) for w in insts], **kw)


def _poses(insts):
    ps = [w.poses for w in insts if w.poses.shape[0]]
    arr = np.concatenate(ps) if ps else np.zeros((0, 3), np.float32)
    return torch.as_tensor(arr, device="cuda").contiguous()


def _single_scene(insts):
    """phi, dphi, active of every instance through psdf_eval_grad."""
    phis, dphis, acts = [], [], []
    for w in insts:
        if w.poses.shape[0] == 0:
            continue
        sc = psdf.Scene.from_csr(w.edges, w.offsets)
        ps = torch.as_tensor(w.poses, device="cuda").contiguous()
        phi, dphi, act = psdf.eval_grad(sc, w.footprint, ps)
        phis.append(phi)
        dphis.append(dphi)
        acts.append(act)
    torch.cuda.synchronize()
    return torch.cat(phis), torch.cat(dphis), torch.cat(acts)


def test_plan_equals_single_scene_bit_for_bit():
    insts = _mixed_instances(11)
    plan = _plan(insts)
    info = plan.info()
    assert info.n_inst == len(insts)
    assert info.n_poses == sum(w.poses.shape[0] for w in insts)
    poses = _poses(insts)
    phi, dphi, act = psdf.eval_batched(plan, poses)
    torch.cuda.synchronize()
    assert psdf.psdf_plan_status(plan) == psdf.PSDF_OK
    rphi, rdphi, ract = _single_scene(insts)
    assert np.array_equal(_bits(phi), _bits(rphi))
    assert np.array_equal(_bits(dphi), _bits(rdphi))
    assert np.array_equal(_bits(act), _bits(ract))
    # instances without obstacles: phi = +inf, no pair, zero gradient
    p0 = 0
    for w in insts:
        n = w.poses.shape[0]
        if n and w.edges.shape[0] == 0:
            assert torch.all(torch.isinf(phi[p0:p0 + n]))
            assert torch.all(act[p0:p0 + n] == -1)
            assert torch.all(dphi[p0:p0 + n] == 0)
        p0 += n


def test_plan_against_oracle():
    insts = _mixed_instances(12)
    plan = _plan(insts)
    poses = _poses(insts)
    phi, dphi, act = psdf.eval_batched(plan, poses)
    torch.cuda.synchronize()
    phi_n, dphi_n, pair_n = phi.cpu().numpy(), dphi.cpu().numpy(), psdf.pair_ids(act)
    p0 = 0
    for w in insts:
        n = w.poses.shape[0]
        if n and w.edges.shape[0]:
            ref = oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses)
            got = {"phi": phi_n[p0:p0 + n], "pair": pair_n[p0:p0 + n], "grad": dphi_n[p0:p0 + n]}
            compare(got, ref)
        p0 += n


@pytest.mark.parametrize("threads", [128, 256])
@pytest.mark.parametrize("tpi", [1, 3, 64])
def test_every_config_gives_the_same_bits(threads, tpi):
    insts = _mixed_instances(13, n_inst=20)
    plan = _plan(insts)
    poses = _poses(insts)
    ref = psdf.eval_batched(plan, poses)
    psdf.psdf_plan_set_config(plan, threads, tpi)
    info = plan.info()
    assert (info.config.threads, info.config.tiles_per_item) == (threads, tpi)
    got = psdf.eval_batched(plan, poses)
    torch.cuda.synchronize()
    for a, b in zip(ref, got):
        assert np.array_equal(_bits(a), _bits(b))


def test_autotune_picks_a_candidate_and_caches_it():
    insts = _mixed_instances(14, n_inst=24)
    plan = _plan(insts)
    poses = _poses(insts)
    ref = psdf.eval_batched(plan, poses)
    cfg, hit = psdf.psdf_plan_autotune(plan, poses, reps=2)
    assert not hit
    assert cfg.threads in (128, 256) and 1 <= cfg.tiles_per_item <= 32
    got = psdf.eval_batched(plan, poses)
    torch.cuda.synchronize()
    for a, b in zip(ref, got):
        assert np.array_equal(_bits(a), _bits(b))
    # a second plan of the same shape reuses the choice
    plan2 = _plan(insts)
    cfg2, hit2 = psdf.psdf_plan_autotune(plan2, poses, reps=2)
    assert hit2 and (cfg2.threads, cfg2.tiles_per_item) == (cfg.threads, cfg.tiles_per_item)


def test_graph_replay_with_new_poses():
    insts = _mixed_instances(15, n_inst=16)
    plan = _plan(insts)
    poses = _poses(insts)
    P = plan.n_poses
    phi = torch.empty(P, device="cuda")
    dphi = torch.empty((P, 3), device="cuda")
    act = torch.empty(P, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        psdf.psdf_eval_batched(plan, poses, phi, dphi, act)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        psdf.psdf_eval_batched(plan, poses, phi, dphi, act)
    for shift in (0.0, 0.37, -1.25):
        new = poses.clone()
        new[:, 0] += shift
        new[:, 2] += 0.5 * shift
        poses.copy_(new)
        g.replay()
        torch.cuda.synchronize()
        ref = psdf.eval_batched(plan, new)
        torch.cuda.synchronize()
        for a, b in zip((phi, dphi, act), ref):
            assert np.array_equal(_bits(a), _bits(b))


def test_backward_batched_matches_single_scene():
    insts = [w for w in _mixed_instances(16, n_inst=18) if w.poses.shape[0]]
    plan = _plan(insts)
    poses = _poses(insts)
    phi, dphi, act = psdf.eval_batched(plan, poses)
    P = plan.n_poses
    gphi = torch.linspace(0.5, 1.5, P, device="cuda")
    gpose = torch.empty((P, 3), device="cuda")
    gedges = torch.zeros((plan.edges.shape[0], 4), device="cuda")
    psdf.psdf_backward_batched(plan, poses, act, gphi, gpose, gedges)
    torch.cuda.synchronize()
    p0, r0 = 0, 0
    for w in insts:
        n, E = w.poses.shape[0], w.edges.shape[0]
        sc = psdf.Scene.from_csr(w.edges, w.offsets)
        ps = poses[p0:p0 + n].contiguous()
        ga = torch.empty((n, 3), device="cuda")
        ge = torch.zeros((max(E, 1), 4), device="cuda")
        psdf.psdf_backward(w.footprint, sc, ps, sc.params, act[p0:p0 + n].contiguous(),
                           gphi[p0:p0 + n].contiguous(), ga, ge)
        torch.cuda.synchronize()
        assert np.array_equal(_bits(gpose[p0:p0 + n]), _bits(ga))
        if E:
            assert torch.allclose(gedges[r0:r0 + E], ge[:E], rtol=1e-6, atol=1e-6)
        p0 += n
        r0 += E


def test_uneven_instances_full_size_against_oracle():
    """1,024 instances, horizons 10..100, 16..65,536 edges, 4..12-vertex
    footprints (the batched-instances workload), autotuned, every pose
    checked against the oracle."""
    insts = sg.uneven_instances(2)
    plan = _plan(insts)
    poses = _poses(insts)
    cfg, _ = psdf.psdf_plan_autotune(plan, poses, reps=2)
    phi, dphi, act = psdf.eval_batched(plan, poses)
    torch.cuda.synchronize()
    assert psdf.psdf_plan_status(plan) == psdf.PSDF_OK
    phi_n, dphi_n, pair_n = phi.cpu().numpy(), dphi.cpu().numpy(), psdf.pair_ids(act)
    p0 = 0
    for w in insts:
        n = w.poses.shape[0]
        ref = oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses)
        got = {"phi": phi_n[p0:p0 + n], "pair": pair_n[p0:p0 + n], "grad": dphi_n[p0:p0 + n]}
        compare(got, ref)
        p0 += n
    assert p0 == plan.n_poses


@pytest.mark.parametrize("eta", [20.0, 500.0])
def test_soft_plan_matches_single_scene(eta):
    """The soft minimum through a plan: values, pairs and pose gradients bit
    for bit equal to one psdf_eval_grad per instance, and the backward's pose
    gradients too (edge gradients to float-atomic order), with half of every
    instance's poses moved onto obstacle vertices (penetrations)."""
    insts = [w for w in _mixed_instances(23, n_inst=18) if w.poses.shape[0] and w.edges.shape[0]]
    g = np.random.default_rng(24)
    for w in insts:
        n = w.poses.shape[0] // 2
        idx = g.integers(0, w.edges.shape[0], size=n)
        w.poses[:n, 0:2] = (w.edges[idx, 0:2] + g.normal(size=(n, 2)) * 0.2).astype(np.float32)
    prm = psdf.make_params(eta=eta)
    plan = _plan(insts, params=prm)
    poses = _poses(insts)
    phi, dphi, act = psdf.eval_batched(plan, poses)
    P = plan.n_poses
    gphi = torch.linspace(0.5, 1.5, P, device="cuda")
    gpose = torch.empty((P, 3), device="cuda")
    gedges = torch.zeros((plan.edges.shape[0], 4), device="cuda")
    psdf.psdf_backward_batched(plan, poses, act, gphi, gpose, gedges)
    torch.cuda.synchronize()
    p0, r0, n_pen = 0, 0, 0
    for w in insts:
        n, E = w.poses.shape[0], w.edges.shape[0]
        sc = psdf.Scene.from_csr(w.edges, w.offsets)
        ps = poses[p0:p0 + n].contiguous()
        rphi, rdphi, ract = psdf.eval_grad(sc, w.footprint, ps, params=prm)
        ga = torch.empty((n, 3), device="cuda")
        ge = torch.zeros((E, 4), device="cuda")
        psdf.psdf_backward(w.footprint, sc, ps, prm, ract, gphi[p0:p0 + n].contiguous(), ga, ge)
        torch.cuda.synchronize()
        assert np.array_equal(_bits(phi[p0:p0 + n]), _bits(rphi))
        assert np.array_equal(_bits(act[p0:p0 + n]), _bits(ract))
        assert np.array_equal(_bits(dphi[p0:p0 + n]), _bits(rdphi))
        assert np.array_equal(_bits(gpose[p0:p0 + n]), _bits(ga))
        assert torch.allclose(gedges[r0:r0 + E], ge, rtol=1e-5, atol=1e-6)
        n_pen += int((rphi < 0).sum())
        p0 += n
        r0 += E
    assert n_pen >= 50


def test_zz_no_index_violation_recorded():
    """Run last in this module: the debug build (libpsdf_b300_debug.so) checks every
    index the batched kernels take from their data and records the first
    violation; none may have been seen by the tests above."""
    v, enabled = psdf.psdf_plan_debug_read()
    if not enabled:
        pytest.skip("release build: the index checks are compiled out")
    assert v == 0, "site %d, index %d" % (v >> 48, v & ((1 << 48) - 1))
