"""Soft inlier score as a torch.autograd.Function over the CUDA kernels.

S(p) = sum_i w_i exp(-u_i^2 / 2) with u_i^2 = sum_j (r_ij / tol_j)^2, r_ij the
vertical residual of surface i at p (Eq. 1 in global form) and w_i the inlier
mask.  Forward and backward run in libvote (vote_softscore_fwd / _bwd); the
backward recomputes the residuals.  Gradients flow to the point and to the
surface parameters.
"""
from __future__ import annotations

import ctypes

import torch
from torch.autograd.function import once_differentiable

from . import vote


def _tol_arg(tol, nd):
    if tol is None:
        return None
    import numpy as np
    return np.ascontiguousarray(tol, dtype=np.float64).reshape(nd)


class SoftScore(torch.autograd.Function):
    """SoftScore.apply(point [d], surfaces [P, n], solver, mask_words or None, tol or None)."""

    @staticmethod
    def forward(ctx, point, surfaces, solver, mask=None, tol=None):
        if not (point.is_cuda and surfaces.is_cuda and point.dtype == torch.float64
                and surfaces.dtype == torch.float64):
            raise ValueError("point and surfaces must be CUDA float64 tensors")
        point = point.contiguous()
        surfaces = surfaces.contiguous()
        n = surfaces.shape[1]
        tl = _tol_arg(tol, solver.d - solver.k)
        score = torch.empty(1, dtype=torch.float64, device=point.device)
        vote._check(solver.lib.vote_softscore_fwd(solver.h, vote._ptr(surfaces), n, vote._ptr(mask),
                                                  vote._ptr(point), vote._ptr(tl), vote._ptr(score)))
        ctx.solver, ctx.tol, ctx.mask = solver, tl, mask
        ctx.save_for_backward(point, surfaces)
        return score[0]

    @staticmethod
    @once_differentiable
    def backward(ctx, grad):
        point, surfaces = ctx.saved_tensors
        s = ctx.solver
        n = surfaces.shape[1]
        g = grad.reshape(1).to(torch.float64).contiguous()
        gp = torch.empty_like(point) if ctx.needs_input_grad[0] else None
        gs = torch.empty_like(surfaces) if ctx.needs_input_grad[1] else None
        if gp is not None or gs is not None:
            vote._check(s.lib.vote_softscore_bwd(s.h, vote._ptr(surfaces), n, vote._ptr(ctx.mask), vote._ptr(point),
                                                 vote._ptr(ctx.tol), vote._ptr(g), vote._ptr(gp), vote._ptr(gs)))
        return gp, gs, None, None, None


def soft_score(point, surfaces, solver, mask=None, tol=None):
    return SoftScore.apply(point, surfaces, solver, mask, tol)
