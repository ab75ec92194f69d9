"""Shared helpers for the GPU-vs-oracle parity tests."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2607_04310_b300 import psdf

VALUE_TOL = 1e-5      # metres, |phi_gpu - phi_fp64|
GRAD_RTOL = 1e-4      # relative, on the pose gradient
TIE_TAU = 1e-5        # pair-id checks need the FP64 runner-up this far away
GRAD_TAU = 1e-3       # gradient checks need this tie margin
CONTACT = 1e-2        # separated gradients are checked at |phi| >= 1 cm


def gpu_eval(w, tile_edges=0, grad=True, poses=None, scene=None, params=None):
    import torch
    sc = scene or psdf.Scene.from_csr(w.edges, w.offsets, tile_edges=tile_edges, params=params)
    ps = torch.as_tensor(np.asarray(w.poses if poses is None else poses, dtype=np.float32),
                         device="cuda").contiguous()
    phi, dphi, act = psdf.eval_grad(sc, w.footprint, ps, params=params, grad=grad)
    torch.cuda.synchronize()
    out = {"phi": phi.cpu().numpy(), "pair": psdf.pair_ids(act),
           "grad": dphi.cpu().numpy() if dphi is not None else None}
    return out, sc


def compare(gpu, ref, idx=None, check_grad=True, tau=TIE_TAU, gtau=GRAD_TAU):
    """Element-by-element comparison; returns a stats dict, asserts the bar."""
    phi_g = gpu["phi"] if idx is None else gpu["phi"][idx]
    pair_g = gpu["pair"] if idx is None else gpu["pair"][idx]
    err = np.abs(phi_g.astype(np.float64) - ref["phi"])
    assert np.all(np.isfinite(phi_g)), "non-finite phi"
    assert err.max() <= VALUE_TOL, ("value error", float(err.max()), int(err.argmax()))
    far = ref["margin"] >= tau
    same = (pair_g == ref["pair"]) | (pair_g == ref["twin"])
    bad = np.nonzero(far & ~same)[0]
    assert len(bad) == 0, ("pair mismatch", bad[:10], pair_g[bad[:10]], ref["pair"][bad[:10]])
    stats = {"n": len(phi_g), "max_value_err": float(err.max()),
             "pair_checked": int(far.sum()), "pair_excluded": int((~far).sum())}
    if check_grad and gpu["grad"] is not None:
        g = gpu["grad"] if idx is None else gpu["grad"][idx]
        sel = (ref["margin"] >= gtau) & ((ref["phi"] < 0) | (ref["phi"] >= CONTACT))
        diff = np.linalg.norm(g[sel].astype(np.float64) - ref["grad"][sel], axis=1)
        scale = np.maximum(np.linalg.norm(ref["grad"][sel], axis=1), 1.0)
        rel = diff / scale
        assert sel.sum() == 0 or rel.max() <= GRAD_RTOL, ("grad error", float(rel.max()))
        stats["grad_checked"] = int(sel.sum())
        stats["max_grad_rel"] = float(rel.max()) if sel.any() else 0.0
    return stats


def oracle_eval(w, poses=None, **kw):
    return oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses if poses is None else poses,
                            **kw)
