"""Differentiable far-field objective on a quadtree, for gradients with respect to
source positions (the P2M -> M2L -> L2L -> L2P chain of Sec. 2.1 stages 2-4).

    J = sum_j w_j Re phi_far(z_j),

phi_far(z) the local expansion of z's leaf, after M2L over the lists of every
level 2..depth and L2L down the tree, evaluated at z.  Every stage runs in the
library's kernels, forward and backward:

    forward   fmm_p2m (finest level) -> fmm_m2m (upward) -> fmm_m2l_levels -> fmm_l2l (downward)
              -> fmm_l2p
    backward  fmm_l2p_adjoint -> fmm_l2l_adjoint (upward) -> fmm_m2l_adjoint_levels (conjugate)
              -> fmm_m2m_adjoint (downward) -> fmm_p2m_adjoint, giving dJ/dx, dJ/dy per point.

Every level's MEs come from the finest level's P2M by M2M, which equals the
P2M of all points in each box (exact for truncated series); on an adaptive tree
the M2L reads existing boxes only, so a point contributes down to its leaf and
no further, which is the frozen-leaf assignment.  Units at the library boundary
are radius-scaled: M~_k = m_k / r^k, L~_n = l_n r^(n+1).
"""
from __future__ import annotations

import torch

from . import fmmgb


def leaf_boxes(tree, xy: torch.Tensor):
    """(level, box) of the deepest existing box containing each point (library
    kernel ``fmm_leaf_boxes``).  xy: [N, 2] float64 on the device; returns
    (int32, int64) device tensors."""
    xy = xy.contiguous()
    lev = torch.empty(xy.shape[0], dtype=torch.int32, device=xy.device)
    box = torch.empty(xy.shape[0], dtype=torch.int64, device=xy.device)
    fmmgb.fmm_leaf_boxes(tree, xy, lev, box)
    return lev, box


class FarFieldObjective(torch.autograd.Function):
    """J(xy) for fixed strengths, evaluation points and weights (see the module docstring)."""

    @staticmethod
    def forward(ctx, xy, tree, p, c, zxy, zlev, zbox, w):
        L = tree.max_level
        dev = xy.device
        levels = list(range(2, L + 1))
        Ms = [torch.empty((4 ** l, p), dtype=torch.complex64, device=dev) for l in levels]
        fmmgb.fmm_p2m(L, p, xy, c, Ms[-1])  # finest level, then M2M upward (exact for truncated series)
        for i in range(len(levels) - 1, 0, -1):
            fmmgb.fmm_m2m(levels[i], p, Ms[i], Ms[i - 1])
        Ls = [torch.zeros_like(M) for M in Ms]
        fmmgb.fmm_m2l_levels(tree, 2, p, Ms, Ls)
        for i in range(1, len(levels)):
            fmmgb.fmm_l2l(levels[i], p, Ls[i - 1], Ls[i], accumulate=True)
        phi = torch.empty(zxy.shape[0], dtype=torch.complex64, device=dev)
        fmmgb.fmm_l2p(p, zxy, zlev, zbox, dict(zip(levels, Ls)), L, phi)
        ctx.save_for_backward(xy, c, zxy, zlev, zbox, w)
        ctx.tree, ctx.p = tree, p
        return torch.sum(w * phi.real.to(torch.float64))

    @staticmethod
    def backward(ctx, gJ):
        xy, c, zxy, zlev, zbox, w = ctx.saved_tensors
        tree, p = ctx.tree, ctx.p
        L = tree.max_level
        levels = list(range(2, L + 1))
        dev = xy.device
        cot = (gJ * w).to(torch.complex64)  # dJ/dphi (real weights)
        Gs = [torch.zeros((4 ** l, p), dtype=torch.complex64, device=dev) for l in levels]
        fmmgb.fmm_l2p_adjoint(p, zxy, zlev, zbox, cot, dict(zip(levels, Gs)), L)
        for i in range(len(levels) - 1, 0, -1):
            fmmgb.fmm_l2l_adjoint(levels[i], p, Gs[i], Gs[i - 1], accumulate=True)
        Ws = [torch.zeros_like(G) for G in Gs]
        fmmgb.fmm_m2l_adjoint_levels(tree, 2, p, Gs, Ws, conj=True)
        for i in range(1, len(levels)):  # M_l = M2M(M_{l+1}): coarse to fine
            fmmgb.fmm_m2m_adjoint(levels[i], p, Ws[i - 1], Ws[i], accumulate=True)
        grad = torch.zeros_like(xy)
        fmmgb.fmm_p2m_adjoint(L, p, xy, c, Ws[-1], grad)
        return grad, None, None, None, None, None, None, None


def far_field_objective(tree, p: int, xy: torch.Tensor, c: torch.Tensor, leaf, z: torch.Tensor, z_leaf,
                        w: torch.Tensor) -> torch.Tensor:
    """J (a 0-d float64 tensor), differentiable in xy ([N, 2] float64, CUDA).

    c: [N] float64 strengths; z: [Z] complex128 evaluation points; z_leaf: their
    (levels, boxes) from ``leaf_boxes``; w: [Z] float64 weights.  `leaf`, the
    sources' leaves, is implied by their positions (each point is binned at
    every level and absent boxes are skipped) and is accepted for symmetry."""
    del leaf
    zxy = torch.view_as_real(z.to(torch.complex128)).contiguous()
    zlev, zbox = z_leaf
    return FarFieldObjective.apply(xy.contiguous(), tree, p, c.contiguous(), zxy, zlev.to(torch.int32).contiguous(),
                                   zbox.to(torch.int64).contiguous(), w.contiguous())


class FmmPotential:
    """The whole FMM on a uniform tree to level L (Sec. 2.1 stages 2-5), every stage a
    library kernel: P2M at level L (on the binned points), M2M up, M2L over the interaction lists of levels 2..L,
    L2L down, L2P at each target's level-L box (on the binned targets), plus the near
    field (own and adjacent boxes) by ``fmm_p2p``.

        phi(z) = sum_i c_i / (z - y_i)   (sources at exactly z skipped)

    The near field and the far field up to L2L are independent: the near field runs on
    a second stream (writing phi, with FMM_P2P_SHARE_SM so that the far-field kernels
    find room on every SM), the far field on the current one, and L2P adds into phi
    once both are done.  Buffers are allocated once; ``__call__`` enqueues the whole
    evaluation, ending on the current stream (capturable as a CUDA graph after a
    first call)."""

    def __init__(self, tree, p: int, xy: torch.Tensor, c: torch.Tensor, z: torch.Tensor, prec: int = 0):
        if tree.adaptive or tree.periodic or tree.max_level < 2:
            raise ValueError("FmmPotential takes a uniform, non-periodic tree of depth >= 2")
        self.tree, self.p, self.prec = tree, p, prec
        self.L = L = tree.max_level
        dev = xy.device
        self.xy, self.c, self.z = xy.contiguous(), c.contiguous(), z.contiguous()
        self.levels = list(range(2, L + 1))
        self.Ms = [torch.empty((4 ** l, p), dtype=torch.complex64, device=dev) for l in self.levels]
        self.Ls = [torch.empty_like(M) for M in self.Ms]
        nb = 4 ** L

        def bins(pts):
            perm = torch.empty(pts.shape[0], dtype=torch.int32, device=dev)
            start = torch.empty(nb + 1, dtype=torch.int32, device=dev)
            work = torch.empty(nb, dtype=torch.int32, device=dev)
            fmmgb.fmm_bin_points(L, pts, perm, start, work)
            return perm, start

        self.sperm, self.sstart = bins(self.xy)
        self.tperm, self.tstart = bins(self.z)
        self.phi = torch.empty(self.z.shape[0], dtype=torch.complex64, device=dev)
        self.side = torch.cuda.Stream(device=dev)

    def __call__(self) -> torch.Tensor:
        p, L = self.p, self.L
        cur = torch.cuda.current_stream(self.phi.device)
        self.side.wait_stream(cur)  # the inputs and phi are the current stream's until here
        fmmgb.fmm_p2p(L, self.xy, self.c, self.sperm, self.sstart, self.z, self.tperm, self.tstart, self.phi,
                      stream=self.side, share_sm=True)
        fmmgb.fmm_p2m_binned(L, p, self.xy, self.c, self.sperm, self.sstart, self.Ms[-1])
        for i in range(len(self.levels) - 1, 0, -1):
            fmmgb.fmm_m2m(self.levels[i], p, self.Ms[i], self.Ms[i - 1])
        fmmgb.fmm_m2l_levels(self.tree, 2, p, self.Ms, self.Ls, prec=self.prec)
        for i in range(1, len(self.levels)):
            fmmgb.fmm_l2l(self.levels[i], p, self.Ls[i - 1], self.Ls[i], accumulate=True)
        cur.wait_stream(self.side)
        fmmgb.fmm_l2p_binned(L, p, self.z, self.tperm, self.tstart, self.Ls[-1], self.phi, accumulate=True)
        return self.phi
