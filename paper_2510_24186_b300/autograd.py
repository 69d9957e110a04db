"""torch.autograd.Function over trids_score_grad.

Forward scores the poses and keeps only the DOFs; backward calls the library again
with the upstream gradient, recomputing the kinematics instead of storing per-atom
intermediates (the paper's manual differentiation, Sec. 4 item 3).  Gradients flow to
the DOFs (t, q through E(q/|q|), theta), the five term weights and the per-type radii.
"""
from __future__ import annotations

import dataclasses

import torch

from . import api


class TridsScore(torch.autograd.Function):
    @staticmethod
    def forward(ctx, dof, weights, radii, pocket, batch):
        params = dataclasses.replace(pocket.params, w=[float(x) for x in weights.detach().cpu()],
                                     radius=[float(x) for x in radii.detach().cpu()])
        pocket.set_params(params)
        out = api.score_grad(pocket, batch, dof.detach().contiguous(), grad=False)
        ctx.save_for_backward(dof)
        ctx.pocket, ctx.batch, ctx.params = pocket, batch, params
        ctx.w_meta = (weights.dtype, weights.device)
        ctx.r_meta = (radii.dtype, radii.device)
        return out["energy"]

    @staticmethod
    def backward(ctx, e_bar):
        (dof,) = ctx.saved_tensors
        ctx.pocket.set_params(ctx.params)
        out = api.score_grad(ctx.pocket, ctx.batch, dof.detach().contiguous(), grad=True,
                             e_bar=e_bar.detach().contiguous().float(), param_grad=True)
        gw = out["g_w"].to(dtype=ctx.w_meta[0], device=ctx.w_meta[1])
        gr = out["g_radius"].to(dtype=ctx.r_meta[0], device=ctx.r_meta[1])
        return out["g_dof"], gw, gr, None, None


def score(dof, weights, radii, pocket, batch):
    """E_total [n_lig, P] as a differentiable function of (dof, weights, radii)."""
    return TridsScore.apply(dof, weights, radii, pocket, batch)
