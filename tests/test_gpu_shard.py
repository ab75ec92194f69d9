"""A scene evaluated in parts (consecutive obstacle ranges as scenes of their
own, as an edge set sharded over GPUs or a static map plus moving
obstacles): each part's 64-bit keys (psdf_eval_keys, ranks offset to the
whole scene's rows), their minimum (psdf_merge_keys, or the all-reduce of
the sharded path), and the epilogue by the part holding each pose's winning
obstacle (psdf_finish_keys) give the whole scene's psdf_eval_grad outputs bit
for bit (Eq. psdf_value is a minimum over obstacles)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2607_04310_b300 import psdf, shard
from paper_2607_04310_b300 import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _parts_eval(w, poses, parts, prm):
    dev = poses.device
    P = poses.shape[0]
    keys = None
    ws = psdf.workspace(P, dev)
    scenes = []
    for part in parts:
        e, o = shard.part_csr(w.edges, w.offsets, part)
        sc = psdf.Scene.from_csr(e, o, params=prm)
        scenes.append(sc)
        k = torch.empty(P, dtype=torch.int64, device=dev)
        psdf.psdf_eval_keys(w.footprint, sc, poses, prm, part[2], k, ws)
        assert psdf.psdf_workspace_status(ws) == psdf.PSDF_OK
        if keys is None:
            keys = k
        else:
            psdf.psdf_merge_keys(k, keys)
    phi = torch.full((P,), float("nan"), device=dev)
    dphi = torch.full((P, 3), float("nan"), device=dev)
    act = torch.zeros(P, dtype=torch.int32, device=dev)
    for i, (part, sc) in enumerate(zip(parts, scenes)):
        psdf.psdf_finish_keys(w.footprint, sc, poses, prm, part[2], i == 0, keys, phi, dphi, act)
    torch.cuda.synchronize()
    return phi, dphi, act, keys


@pytest.mark.parametrize("n_parts,eta", [(3, 0.0), (2, 0.0), (3, 50.0)])
def test_parts_equal_whole_scene(n_parts, eta):
    w = sg.octagon_lidar(1, n_inst=16, horizon=50, n_rects=800, n_lines=40, segs_per_line=20)
    prm = psdf.make_params(eta=eta)
    whole = psdf.Scene.from_csr(w.edges, w.offsets, params=prm)
    poses = torch.as_tensor(w.poses, device="cuda")
    phi0, dphi0, act0 = psdf.eval_grad(whole, w.footprint, poses, params=prm)
    parts = shard.split_rows(w.offsets, n_parts)
    assert all(p[1] > p[0] for p in parts)
    phi, dphi, act, keys = _parts_eval(w, poses, parts, prm)
    assert torch.equal(phi.view(torch.int32), phi0.view(torch.int32))
    assert torch.equal(dphi.view(torch.int32), dphi0.view(torch.int32))
    assert torch.equal(act, act0)
    # every pose's winning obstacle was finished by the part that holds it
    own = shard.owner(keys.cpu().numpy(), parts)
    assert np.all(own >= 0) and len(np.unique(own)) == n_parts
    if eta == 0.0:  # and the whole thing agrees with the oracle
        ref = oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses)
        assert np.abs(phi.cpu().numpy() - ref["phi"]).max() <= 1e-5


def test_parts_with_an_empty_part_and_far_poses():
    """Poses far from every obstacle keep their key of the nearest part; a
    part without obstacles contributes nothing; no obstacle at all (every
    part empty) gives phi = +inf from the part that owns empty keys."""
    w = sg.plain_rect_small(0)
    prm = psdf.make_params()
    poses = torch.tensor([[500.0, -300.0, 0.1], [10.0, 10.0, 0.0], [3.0, 4.0, 1.0]],
                         device="cuda")
    whole = psdf.Scene.from_csr(w.edges, w.offsets)
    phi0, dphi0, act0 = psdf.eval_grad(whole, w.footprint, poses)
    parts = shard.split_rows(w.offsets, 2)
    phi, dphi, act, _keys = _parts_eval(w, poses, parts, prm)
    assert torch.equal(phi.view(torch.int32), phi0.view(torch.int32))
    assert torch.equal(act, act0)
    empty = psdf.Scene.from_csr(np.zeros((0, 4), np.float32), np.zeros(1, np.int32))
    ws = psdf.workspace(3)
    k = torch.empty(3, dtype=torch.int64, device="cuda")
    psdf.psdf_eval_keys(w.footprint, empty, poses, prm, 0, k, ws)
    out = torch.zeros(3, device="cuda")
    a = torch.zeros(3, dtype=torch.int32, device="cuda")
    psdf.psdf_finish_keys(w.footprint, empty, poses, prm, 0, True, k, out, None, a)
    torch.cuda.synchronize()
    assert torch.all(k == -1) and torch.all(torch.isinf(out)) and torch.all(a == -1)


def test_part_rejects_rows_beyond_the_pair_id():
    w = sg.plain_rect_small(0)
    sc = psdf.Scene.from_csr(w.edges, w.offsets)
    poses = torch.as_tensor(w.poses, device="cuda")
    k = torch.empty(w.P, dtype=torch.int64, device="cuda")
    with pytest.raises(psdf.PsdfError) as ei:
        psdf.psdf_eval_keys(w.footprint, sc, poses, sc.params, (1 << 24) - 10, k,
                            psdf.workspace(w.P))
    assert ei.value.code == psdf.PSDF_ERR_ARG
