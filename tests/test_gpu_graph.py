"""The evaluation entry points run under CUDA-graph capture: a captured step
replayed on new inputs (copied into the captured buffers) gives exactly the
eager results."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2607_04310_b300 import psdf
from paper_2607_04310_b300 import scenegen as sg
from paper_2607_04310_b300 import train_cull as tc

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _capture(fn):
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        fn()
    torch.cuda.synchronize()
    return g


@pytest.mark.parametrize("path", ["full", "bound", "mlp"])
def test_graph_replay_equals_eager(path):
    w = sg.dense_clutter(4, n_rects=4000, n_poses=1000, field_side=80.0)
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    W1, w2, b2, _ = tc.load_weights()
    mlp = psdf.Mlp(W1, w2, b2) if path == "mlp" else None
    P = w.P
    poses = torch.as_tensor(w.poses, device="cuda").clone()
    phi = torch.empty(P, device="cuda")
    dphi = torch.empty((P, 3), device="cuda")
    act = torch.empty(P, dtype=torch.int32, device="cuda")
    gpose = torch.empty((P, 3), device="cuda")
    gedges = torch.zeros((w.E, 4), device="cuda")
    ones = torch.ones(P, device="cuda")
    ws = psdf.workspace(P)
    cws = torch.empty(psdf.psdf_cull_workspace_bytes(P, scene), dtype=torch.uint8, device="cuda")
    opts = psdf.CullOpts(psdf.PROPOSE_MLP if path == "mlp" else psdf.PROPOSE_BOUND, 2)

    def step():
        if path == "full":
            psdf.psdf_eval_grad(w.footprint, scene, poses, scene.params, phi, dphi, act, ws)
        else:
            psdf.psdf_eval_culled(w.footprint, scene, mlp, opts, poses, scene.params, phi, dphi,
                                  act, cws)
        psdf.psdf_backward(w.footprint, scene, poses, scene.params, act, ones, gpose, gedges)

    g = _capture(step)
    for seed in (1, 2):
        new = torch.as_tensor(sg.poses_uniform(sg.rng(seed), P, 0.0, 80.0), device="cuda")
        poses.copy_(new)
        gedges.zero_()
        g.replay()
        torch.cuda.synchronize()
        got = [phi.clone(), dphi.clone(), act.clone(), gpose.clone(), gedges.clone()]
        gedges.zero_()
        step()
        torch.cuda.synchronize()
        ref = [phi, dphi, act, gpose, gedges]
        for a_, b_ in zip(got[:4], ref[:4]):
            assert torch.equal(a_.view(torch.int32) if a_.dtype == torch.float32 else a_,
                               b_.view(torch.int32) if b_.dtype == torch.float32 else b_)
        # float atomics in the edge scatter: equal up to summation order
        assert torch.allclose(got[4], ref[4], rtol=1e-5, atol=1e-5)
