"""Differentiable far-field objective on a quadtree, for gradients with respect to
source positions (the P2M -> M2L -> L2L -> L2P chain of Sec. 2.1 stages 2-4).

    J = sum_j w_j Re phi_far(z_j),

phi_far(z) the local expansion of z's leaf, after M2L over the lists of every
level 2..depth and L2L down the tree, evaluated at z; each source point
contributes to the ME of the box that contains its (frozen) leaf at every level
down to that leaf.  The M2L of every level, forward and adjoint, runs in the
library's FP32 kernels (``autograd.M2LLevels``); the P2M, L2L and L2P stages are
FP64 tensor operations here, so that coordinate differences of order r_l stay
exact in the gradient.  Units at the library boundary are radius-scaled:
M~_k = m_k / r^k, L~_n = l_n r^(n+1).
"""
from __future__ import annotations

import math

import torch

from .autograd import m2l_levels


def leaf_boxes(tree, xy: torch.Tensor):
    """(level, box) of the deepest existing box containing each point, from the
    tree's existence masks.  xy: [N, 2] float64 (any device); returns int64."""
    lev = torch.zeros(xy.shape[0], dtype=torch.int64, device=xy.device)
    box = torch.zeros_like(lev)
    for l in range(tree.max_level + 1):
        n = 1 << l
        ix = torch.clamp(torch.floor(xy[:, 0] * n).to(torch.int64), 0, n - 1)
        iy = torch.clamp(torch.floor(xy[:, 1] * n).to(torch.int64), 0, n - 1)
        b = iy * n + ix
        here = torch.from_numpy(tree.exists(l)).to(xy.device)[b]
        lev = torch.where(here, torch.full_like(lev, l), lev)
        box = torch.where(here, b, box)
    return lev, box


def _ancestor(lev, box, level):
    sh = torch.clamp(lev - level, min=0)
    side = torch.bitwise_left_shift(torch.ones_like(lev), lev)
    ix = torch.bitwise_right_shift(box % side, sh)
    iy = torch.bitwise_right_shift(torch.div(box, side, rounding_mode="floor"), sh)
    return torch.where(lev >= level, iy * (1 << level) + ix, torch.full_like(box, -1))


def _centre(level, b):
    n = 1 << level
    return torch.complex(((b % n).double() + 0.5) / n, (torch.div(b, n, rounding_mode="floor").double() + 0.5) / n)


def _l2l_matrices(p: int, device):
    """Scaled L2L per child class c = (ix & 1) + 2 (iy & 1):
    L~_child[j] = sum_{n >= j} C(n, j) u^(n-j) 2^-(j+1) L~_parent[n], u = (x_child - x_parent) / r_parent."""
    T = torch.zeros((4, p, p), dtype=torch.complex128)
    for c in range(4):
        u = complex(((c & 1) - 0.5) / 2.0, ((c >> 1) - 0.5) / 2.0)
        for j in range(p):
            for n in range(j, p):
                T[c, j, n] = math.comb(n, j) * u ** (n - j) * 2.0 ** (-(j + 1))
    return T.to(device)


def far_field_objective(tree, p: int, xy: torch.Tensor, c: torch.Tensor, leaf, z: torch.Tensor, z_leaf,
                        w: torch.Tensor) -> torch.Tensor:
    """J (a 0-d float64 tensor), differentiable in xy ([N, 2] float64) and c.

    leaf, z_leaf: (levels, boxes) of the sources' and evaluation points' leaves
    (``leaf_boxes``; frozen while the points move).  z: [Z] complex128, w: [Z] float64."""
    dev = xy.device
    lev, box = leaf
    y = torch.complex(xy[:, 0], xy[:, 1])
    Ms = []
    for l in range(2, tree.max_level + 1):
        b = _ancestor(lev, box, l)
        sel = b >= 0
        bs = b[sel]
        d = (y[sel] - _centre(l, bs)) * float(1 << l)  # (y - x_b) / r
        pw = [c[sel].to(torch.complex128)]
        for _ in range(p - 1):
            pw.append(pw[-1] * d)
        contrib = torch.stack(pw, 1)  # c_i ((y_i - x_b) / r)^k
        M = torch.zeros((4 ** l, p), dtype=torch.complex128, device=dev).index_add(0, bs, contrib)
        Ms.append(M.to(torch.complex64))
    Ls = m2l_levels(tree, p, Ms)
    T = _l2l_matrices(p, dev)
    Lfull = {}
    for i, l in enumerate(range(2, tree.max_level + 1)):
        Ll = Ls[i].to(torch.complex128)
        if l > 2:
            h = 1 << (l - 1)
            Lp = Lfull[l - 1].reshape(h, h, p)  # (py, px, n)
            # child (iy, ix) = (2 py + cy, 2 px + cx) takes T_c L_parent, c = cx + 2 cy
            rows = [torch.stack([Lp @ T[cx + 2 * cy].transpose(0, 1) for cx in range(2)], dim=2) for cy in range(2)]
            Ll = Ll + torch.stack(rows, dim=1).reshape(4 ** l, p)  # (py, cy, px, cx) -> iy * 2^l + ix
        Lfull[l] = Ll
    zlev, zbox = z_leaf
    phi = torch.zeros(z.shape[0], dtype=torch.complex128, device=dev)
    for l in range(2, tree.max_level + 1):
        sel = zlev == l
        if not bool(sel.any()):
            continue
        bz = zbox[sel]
        u = (z[sel] - _centre(l, bz)) * float(1 << l)  # (z - x_t) / r
        acc = torch.zeros_like(u)
        for k in range(p - 1, -1, -1):  # Horner on sum_n L~_n u^n
            acc = acc * u + Lfull[l][bz, k]
        phi = phi.index_put((torch.nonzero(sel)[:, 0],), acc * float(1 << l))  # phi = (1/r) sum L~_n u^n
    return torch.sum(w * phi.real)
