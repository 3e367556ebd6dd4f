"""torch.autograd binding of the M2L translation (Sec. 4.1 steps 2-3, Eq. M2Lmat).

``M2LLevels`` runs the forward pass through ``fmm_m2l_levels`` (every level
2..max_level of a tree in one launch) and the backward pass through
``fmm_m2l_adjoint_levels`` with ``FMM_CONJ``: for a real objective J and the
complex-linear map L = A M, PyTorch's gradient convention gives
dJ/dM = A^H dJ/dL, the conjugate transpose that the library's adjoint stencil
computes (A^T(D) = -A(-D) on the symmetric lists, conjugated).  Both passes run
in the library's FP32 kernels on the caller's current stream; on an adaptive
tree they cover the V-lists, and entries of absent boxes are zero in both
directions.
"""
from __future__ import annotations

import torch

from . import fmmgb


class M2LLevels(torch.autograd.Function):
    """Ls = M2L(Ms) for levels 2..tree.max_level; Ms[i] is level 2 + i, [4^l, p] complex64 scaled."""

    @staticmethod
    def forward(ctx, tree, p, *Ms):
        Ms = [m.contiguous() for m in Ms]
        Ls = [torch.zeros_like(m) for m in Ms]
        fmmgb.fmm_m2l_levels(tree, 2, p, Ms, Ls)
        ctx.tree = tree
        ctx.p = p
        return tuple(Ls)

    @staticmethod
    def backward(ctx, *gLs):
        Ws = [g.contiguous() for g in gLs]
        Gs = [torch.zeros_like(w) for w in Ws]
        fmmgb.fmm_m2l_adjoint_levels(ctx.tree, 2, ctx.p, Ws, Gs, conj=True)
        return (None, None, *Gs)


def m2l_levels(tree, p: int, Ms):
    """Differentiable M2L of levels 2..tree.max_level (list in, tuple out)."""
    if len(Ms) != tree.max_level - 1:
        raise fmmgb.FmmError(fmmgb.FMM_EINVAL, "one ME array per level 2..max_level is required")
    for m in Ms:
        if m.dtype != torch.complex64 or not m.is_cuda:
            raise fmmgb.FmmError(fmmgb.FMM_EINVAL, "MEs must be complex64 CUDA tensors")
    return M2LLevels.apply(tree, p, *Ms)
