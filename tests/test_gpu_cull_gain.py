"""What the trained tile-proposal network gains over the method without it
(the same exact cull with the tiles proposed by the lower bound alone)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2607_04310_b300 import psdf
from paper_2607_04310_b300 import scenegen as sg
from paper_2607_04310_b300 import train_cull as tc

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def test_trained_network_beats_bound_ordering():
    W1, w2, b2, meta = tc.load_weights()
    ev = tc.evaluate(W1, w2, b2, n_scenes=50, first=30000)
    # held-out scenes: how often the first proposed tile holds the nearest obstacle
    assert ev["top1_mlp"] > ev["top1_bound"] + 0.15, ev
    w = sg.dense_clutter(4)
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    poses = torch.as_tensor(w.poses, device="cuda")
    mlp = psdf.Mlp(W1, w2, b2)
    out = {}
    for name, net in (("mlp", mlp), ("bound", None)):
        phi, dphi, act, ws = psdf.eval_culled(scene, w.footprint, poses, mlp=net, k=1)
        st = psdf.psdf_cull_stats_read(ws)
        out[name] = (phi.clone(), act.clone(), st)
    assert torch.equal(out["mlp"][0].view(torch.int32), out["bound"][0].view(torch.int32))
    assert torch.equal(out["mlp"][1], out["bound"][1])
    sm, sb = out["mlp"][2], out["bound"][2]
    # fewer poses need tiles beyond their proposal, and less exact work overall
    assert sm.fallback_poses < sb.fallback_poses, (sm.fallback_poses, sb.fallback_poses)
    assert sm.proposed_items + sm.fallback_items < sb.proposed_items + sb.fallback_items
