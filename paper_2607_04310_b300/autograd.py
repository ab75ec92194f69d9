"""torch.autograd.Function over the C ABI (Alg. 1 PSDF_Forward / PSDF_Backward).

    phi = psdf_phi(poses, edges, scene, footprint)      # [P]
    phi.sum().backward()  ->  poses.grad [P, 3], edges.grad [E, 4]

Forward runs psdf_eval_grad_save (the hard minimum: the active pair's
gradient rows are kept per pose) and backward psdf_backward_saved, which
scales and scatters them; with the soft minimum forward runs psdf_eval_grad
and backward the recomputing psdf_backward kernel.  Both give the
active-branch subgradient of Sec. IV-D.  `edges` is the caller's [rows, 4] tensor whose values the
scene was built from; it only carries the gradient (its values are read
from the scene).  A closed polygon's vertex gradient is reported in its A
slot, its B slots receive zero.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from . import psdf


class PSDFFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, poses: torch.Tensor, edges: Optional[torch.Tensor], scene: psdf.Scene,
                footprint: np.ndarray, params: Optional[psdf.Params] = None):
        if poses.dtype != torch.float32 or not poses.is_cuda:
            raise TypeError("poses must be a float32 CUDA tensor [P, 3]")
        poses_c = poses.detach().contiguous()
        prm = params or scene.params
        ctx.scene = scene
        ctx.footprint = footprint
        ctx.params = prm
        ctx.n_rows = scene.n_rows
        if prm.eta > 0:
            phi, dphi, act = psdf.eval_grad(scene, footprint, poses_c, params=prm, grad=True)
            ctx.save_for_backward(poses_c, act, None)
        else:
            P = poses_c.shape[0]
            phi = torch.empty(P, dtype=torch.float32, device=poses.device)
            dphi = torch.empty((P, 3), dtype=torch.float32, device=poses.device)
            act = torch.empty(P, dtype=torch.int32, device=poses.device)
            saved = torch.empty((P, psdf.SAVED_FLOATS), dtype=torch.float32, device=poses.device)
            psdf.psdf_eval_grad_save(footprint, scene, poses_c, prm, phi, dphi, act, saved,
                                     psdf.workspace(P, poses.device))
            ctx.save_for_backward(poses_c, act, saved)
        ctx.mark_non_differentiable(act)
        return phi, dphi, act

    @staticmethod
    def backward(ctx, grad_phi, _grad_dphi, _grad_act):
        poses, act, saved = ctx.saved_tensors
        grad_phi = grad_phi.contiguous().float()
        need_pose = ctx.needs_input_grad[0]
        need_edges = ctx.needs_input_grad[1]
        gpose = torch.empty_like(poses) if need_pose else None
        gedges = (torch.zeros((ctx.n_rows, 4), dtype=torch.float32, device=poses.device)
                  if need_edges else None)
        if (need_pose or need_edges) and saved is not None:
            psdf.psdf_backward_saved(ctx.scene, saved, grad_phi, gpose, gedges)
        elif need_pose or need_edges:
            psdf.psdf_backward(ctx.footprint, ctx.scene, poses, ctx.params, act, grad_phi,
                               gpose, gedges)
        return gpose, gedges, None, None, None


def psdf_phi(poses: torch.Tensor, edges: Optional[torch.Tensor], scene: psdf.Scene,
             footprint: np.ndarray, params: Optional[psdf.Params] = None) -> torch.Tensor:
    """phi [P] with autograd support for poses and (optionally) edges."""
    phi, _dphi, _act = PSDFFunction.apply(poses, edges, scene, footprint, params)
    return phi


class PSDF(torch.nn.Module):
    """Module form: holds the scene and footprint; forward(poses) -> phi."""

    def __init__(self, edges, offsets, footprint, tile_edges: int = 0,
                 params: Optional[psdf.Params] = None):
        super().__init__()
        self.scene = psdf.Scene.from_csr(edges, offsets, tile_edges=tile_edges, params=params)
        self.footprint = np.ascontiguousarray(footprint, dtype=np.float32)

    def forward(self, poses: torch.Tensor, edges: Optional[torch.Tensor] = None) -> torch.Tensor:
        return psdf_phi(poses, edges, self.scene, self.footprint)
