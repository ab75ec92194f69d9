"""What the trained tile-proposal network gains over the method without it
(the same exact cull with the tiles proposed by the lower bound alone).

Two tilings: with Morton-packed tiles (long, overlapping AABBs) the bound's
ordering is poor and the network recovers the nearest tile far more often;
with the default sort-tile-recursive tiles (close to square) the bound is
already nearly as good, and the network matches it."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2607_04310_b300 import psdf
from paper_2607_04310_b300 import scenegen as sg
from paper_2607_04310_b300 import train_cull as tc

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _cull_stats(w, scene, net, k=1):
    poses = torch.as_tensor(w.poses, device="cuda")
    phi, dphi, act, ws = psdf.eval_culled(scene, w.footprint, poses, mlp=net, k=k)
    st = psdf.psdf_cull_stats_read(ws)
    return phi.clone(), act.clone(), st


def _compare(weights_path, flags):
    W1, w2, b2, meta = tc.load_weights(weights_path)
    ev = tc.evaluate(W1, w2, b2, n_scenes=50, first=30000, tile_flags=flags)
    w = sg.dense_clutter(4)
    scene = psdf.Scene.from_csr(w.edges, w.offsets, tile_edges=flags)
    mlp = psdf.Mlp(W1, w2, b2)
    phi_m, act_m, sm = _cull_stats(w, scene, mlp)
    phi_b, act_b, sb = _cull_stats(w, scene, None)
    # both exact: identical outputs
    assert torch.equal(phi_m.view(torch.int32), phi_b.view(torch.int32))
    assert torch.equal(act_m, act_b)
    return ev, sm, sb


def test_network_gain_on_morton_tiles():
    ev, sm, sb = _compare(tc.MORTON_WEIGHTS, tc.TILE_MORTON)
    # held-out scenes: the first proposed tile holds the nearest obstacle far more often
    assert ev["top1_mlp"] > ev["top1_bound"] + 0.15, ev
    # on the dense-clutter workload: less exact work (fewer fallback pairs)
    pairs_m = sm.proposed_items + sm.fallback_items
    pairs_b = sb.proposed_items + sb.fallback_items
    print("morton tiles: pairs mlp %d bound %d, fallback poses mlp %d bound %d"
          % (pairs_m, pairs_b, sm.fallback_poses, sb.fallback_poses))
    assert pairs_m < pairs_b, (pairs_m, pairs_b)


def test_network_on_default_tiles_matches_bound():
    ev, sm, sb = _compare(tc.DEFAULT_WEIGHTS, 0)
    assert ev["top1_mlp"] >= ev["top1_bound"] - 0.02, ev
    assert ev["top1_bound"] > 0.85, ev
    pairs_m = sm.proposed_items + sm.fallback_items
    pairs_b = sb.proposed_items + sb.fallback_items
    assert pairs_m <= 1.1 * pairs_b, (pairs_m, pairs_b)
