"""FP64 CPU oracle for the M2L / FGT Hermite-to-Taylor translation path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library (``paper_1009_3457_gb300``) and imports
nothing from it.

The arithmetic lives in ``fmm_oracle.c`` (plain loops, FP64, the paper's
definitions in the paper's order).  This module only marshals numpy arrays
into that library, plus the coefficient-scaling convention used at the CUDA
library's boundary, which is a change of units and is written out here:

    scaled ME   M~[b][k] = m_{b,k} / r^k
    scaled LE   L~[b][n] = l_{b,n} * r^(n+1)          r = 2^-level (box side)

Every function cites the passage of Cruz, Layton & Barba (arXiv:1009.3457)
that it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``fmm_oracle.c`` into ``liboracle.so`` with gcc (plain C11, FP64)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_i = ctypes.c_int
_i64 = ctypes.c_int64
_d = ctypes.c_double

_SIGS = {
    "orc_binom": (_d, [_i, _i]),
    "orc_box_centre": (None, [_i, _i, _i, _D]),
    "orc_interaction_list": (_i, [_i, _i, _i, _i, _I, _I, _I, _I]),
    "orc_list_count_level": (_i64, [_i, _i]),
    "orc_p2m_box": (None, [_i64, _D, _D, _d, _d, _i, _D]),
    "orc_p2m_uniform": (None, [_i, _i, _i64, _D, _D, _D]),
    "orc_m2m_uniform": (None, [_i, _i, _D, _D]),
    "orc_m2l_pair": (None, [_i, _d, _d, _D, _D]),
    "orc_m2l_matrix": (None, [_i, _d, _d, _D]),
    "orc_m2l_uniform": (None, [_i, _i, _i, _D, _D]),
    "orc_m2l_uniform_targets": (None, [_i, _i, _i, _D, _i64, _I64, _D]),
    "orc_m2l_adjoint_uniform": (None, [_i, _i, _i, _D, _D]),
    "orc_l2p": (None, [_i, _D, _d, _d, _i64, _D, _D]),
    "orc_m2p": (None, [_i, _D, _d, _d, _i64, _D, _D]),
    "orc_direct": (None, [_i64, _D, _D, _i64, _D, _D]),
    "orc_l2l": (None, [_i, _D, _d, _d, _D]),
    "orc_level_offset": (_i64, [_i]),
    "orc_adaptive_tree": (_i, [_i64, _D, _i, _i, _U8]),
    "orc_vlist": (_i, [_i, _i, _i, _U8, _I, _I, _I, _I]),
    "orc_vlist_count_level": (_i64, [_i, _U8]),
    "orc_m2l_adaptive": (None, [_i, _i, _U8, _D, _D]),
    "orc_m2l_adjoint_adaptive": (None, [_i, _i, _U8, _D, _D]),
    "orc_m2l_adaptive_from_sources": (None, [_i, _i, _U8, _i64, _I64, _D, _D]),
    "orc_p2m_assigned": (None, [_i, _i, _i64, _D, _D, _I64, _D]),
    "orc_l2l_level": (None, [_i, _i, _U8, _D, _D]),
    "orc_hermite_functions": (None, [_i, _d, _D]),
    "orc_fgt_direct": (None, [_i64, _D, _D, _d, _i64, _D, _D]),
    "orc_fgt_p2h": (None, [_i64, _D, _D, _d, _d, _d, _i, _D]),
    "orc_fgt_hermite_eval": (None, [_i, _D, _d, _d, _d, _i64, _D, _D]),
    "orc_fgt_p2t": (None, [_i64, _D, _D, _d, _d, _d, _i, _D]),
    "orc_fgt_taylor_eval": (None, [_i, _D, _d, _d, _d, _i64, _D, _D]),
    "orc_fgt_h2t_pair": (None, [_i, _D, _d, _d, _D]),
    "orc_fgt_h2t_grid": (None, [_i, _i, _i, _d, _D, _D]),
    "orc_fgt_h2t_targets": (None, [_i, _i, _i, _d, _D, _i64, _I64, _D]),
    "orc_fgt_p2h_grid": (None, [_i, _i, _d, _i64, _D, _D, _D]),
    "orc_fgt_hermite_eval_grid": (None, [_i, _i, _i, _d, _D, _i64, _D, _D]),
    "orc_p2p_uniform": (None, [_i, _i64, _D, _D, _i64, _D, _D]),
}


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _c2r(z: np.ndarray) -> np.ndarray:
    """complex128 array -> float64 array with a trailing (re, im) axis."""
    z = np.ascontiguousarray(z, dtype=np.complex128)
    return z.view(np.float64).reshape(z.shape + (2,))


def _r2c(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.view(np.complex128).reshape(a.shape[:-1])


# ---------------------------------------------------------------------------
# quadtree and interaction lists  (Sec. 2.1; Sec. 4.1 step 1)
# ---------------------------------------------------------------------------

def binom(a: int, b: int) -> float:
    return lib().orc_binom(a, b)


def box_centre(level: int, ix: int, iy: int) -> complex:
    out = np.zeros(2)
    lib().orc_box_centre(level, ix, iy, _dp(out))
    return complex(out[0], out[1])


def interaction_list(level: int, tx: int, ty: int, periodic: bool = False):
    """List of (sx, sy, ox, oy): source box and image offset (source image minus target, box units)."""
    bufs = [np.zeros(27, dtype=np.int32) for _ in range(4)]
    ptrs = [b.ctypes.data_as(_I) for b in bufs]
    n = lib().orc_interaction_list(level, tx, ty, int(periodic), *ptrs)
    return [tuple(int(b[i]) for b in bufs) for i in range(n)]


def list_count_level(level: int, periodic: bool = False) -> int:
    return int(lib().orc_list_count_level(level, int(periodic)))


# ---------------------------------------------------------------------------
# upward sweep, M2L, far and near field (Sec. 2.1, Sec. 4.1, Eq. M2Lmat)
# ---------------------------------------------------------------------------

def p2m_box(xy, c, centre: complex, p: int) -> np.ndarray:
    xy, c = _f64(xy), _f64(c)
    m = np.zeros((p, 2))
    lib().orc_p2m_box(len(c), _dp(xy), _dp(c), centre.real, centre.imag, p, _dp(m))
    return _r2c(m)


def p2m_uniform(level: int, p: int, xy, c) -> np.ndarray:
    """Multipole coefficients of every box of a uniform level, [4^l, p] complex128."""
    xy, c = _f64(xy), _f64(c)
    n = 1 << level
    M = np.zeros((n * n, p, 2))
    lib().orc_p2m_uniform(level, p, len(c), _dp(xy), _dp(c), _dp(M))
    return _r2c(M)


def m2m_uniform(child_level: int, p: int, Mc: np.ndarray) -> np.ndarray:
    n = 1 << (child_level - 1)
    Mcr = _c2r(Mc)
    Mp = np.zeros((n * n, p, 2))
    lib().orc_m2m_uniform(child_level, p, _dp(Mcr), _dp(Mp))
    return _r2c(Mp)


def upward_uniform(max_level: int, p: int, xy, c) -> dict:
    """P2M at ``max_level`` then M2M up to level 2 -> {level: M_l}."""
    Ms = {max_level: p2m_uniform(max_level, p, xy, c)}
    for l in range(max_level, 2, -1):
        Ms[l - 1] = m2m_uniform(l, p, Ms[l])
    return Ms


def m2l_pair(p: int, d: complex, m: np.ndarray) -> np.ndarray:
    mr = _c2r(m)
    l = np.zeros((p, 2))
    lib().orc_m2l_pair(p, d.real, d.imag, _dp(mr), _dp(l))
    return _r2c(l)


def m2l_matrix(p: int, d: complex) -> np.ndarray:
    a = np.zeros((p, p, 2))
    lib().orc_m2l_matrix(p, d.real, d.imag, _dp(a))
    return _r2c(a)


def m2l_uniform(level: int, p: int, M: np.ndarray, periodic: bool = False) -> np.ndarray:
    """Physical-unit M2L + reduction over the interaction lists of a uniform level."""
    Mr = _c2r(M)
    L = np.zeros_like(Mr)
    lib().orc_m2l_uniform(level, p, int(periodic), _dp(Mr), _dp(L))
    return _r2c(L)


def m2l_uniform_targets(level: int, p: int, M: np.ndarray, targets, periodic: bool = False) -> np.ndarray:
    Mr = _c2r(M)
    t = np.ascontiguousarray(targets, dtype=np.int64)
    L = np.zeros((len(t), p, 2))
    lib().orc_m2l_uniform_targets(level, p, int(periodic), _dp(Mr), len(t), t.ctypes.data_as(_I64), _dp(L))
    return _r2c(L)


def m2l_adjoint_uniform(level: int, p: int, W: np.ndarray, periodic: bool = False) -> np.ndarray:
    """Plain transpose (no conjugation) of ``m2l_uniform``, by explicit transposed loops."""
    Wr = _c2r(W)
    G = np.zeros_like(Wr)
    lib().orc_m2l_adjoint_uniform(level, p, int(periodic), _dp(Wr), _dp(G))
    return _r2c(G)


def l2p(p: int, l: np.ndarray, centre: complex, z) -> np.ndarray:
    lr = _c2r(l)
    zr = _c2r(np.asarray(z, dtype=np.complex128))
    phi = np.zeros_like(zr)
    lib().orc_l2p(p, _dp(lr), centre.real, centre.imag, zr.shape[0], _dp(zr), _dp(phi))
    return _r2c(phi)


def m2p(p: int, m: np.ndarray, centre: complex, z) -> np.ndarray:
    mr = _c2r(m)
    zr = _c2r(np.asarray(z, dtype=np.complex128))
    phi = np.zeros_like(zr)
    lib().orc_m2p(p, _dp(mr), centre.real, centre.imag, zr.shape[0], _dp(zr), _dp(phi))
    return _r2c(phi)


def direct(xy, c, z) -> np.ndarray:
    """Eq. (n_body) with the Cauchy kernel: phi(z) = sum_i c_i / (z - y_i)."""
    xy, c = _f64(xy), _f64(c)
    zr = _c2r(np.asarray(z, dtype=np.complex128))
    phi = np.zeros_like(zr)
    lib().orc_direct(len(c), _dp(xy), _dp(c), zr.shape[0], _dp(zr), _dp(phi))
    return _r2c(phi)


def p2p_uniform(level: int, xy, c, z) -> np.ndarray:
    """Near field of a uniform tree at `level` (reading R15): at each z the direct sum over
    the sources of its box and the adjacent boxes, skipping sources at exactly z."""
    xy, c = _f64(xy), _f64(c)
    zr = _c2r(np.asarray(z, dtype=np.complex128))
    phi = np.zeros_like(zr)
    lib().orc_p2p_uniform(level, len(c), _dp(xy), _dp(c), zr.shape[0], _dp(zr), _dp(phi))
    return _r2c(phi)


def fmm_potential_uniform(level: int, p: int, xy, c, z) -> np.ndarray:
    """The whole FMM on a uniform tree to `level` (Sec. 2.1 stages 2-5): P2M at every level
    2..level, M2L over the interaction lists of each level, L2L down, L2P at each z's box of
    the finest level, plus the near field there (``p2p_uniform``)."""
    xy, c = _f64(xy), _f64(c)
    z = np.asarray(z, dtype=np.complex128)
    L = {}
    full = np.ones(sum(4 ** k for k in range(level + 1)), dtype=np.uint8)  # every box of levels 0..level exists
    for l in range(2, level + 1):
        Lr = _c2r(m2l_uniform(l, p, p2m_uniform(l, p, xy, c)))
        if l > 2:
            lib().orc_l2l_level(l, p, full.ctypes.data_as(_U8), _dp(_c2r(L[l - 1])), _dp(Lr))
        L[l] = _r2c(Lr)
    n = 1 << level
    zb = np.clip(np.floor(z.real * n), 0, n - 1).astype(np.int64) + n * np.clip(
        np.floor(z.imag * n), 0, n - 1).astype(np.int64)
    far = _l2p_at_leaves(p, L, z, np.full(len(z), level), zb) if level >= 2 else 0.0
    return far + p2p_uniform(level, xy, c, z)


def l2l(p: int, lp: np.ndarray, shift: complex) -> np.ndarray:
    lpr = _c2r(lp)
    lc = np.zeros((p, 2))
    lib().orc_l2l(p, _dp(lpr), shift.real, shift.imag, _dp(lc))
    return _r2c(lc)


# ---------------------------------------------------------------------------
# adaptive quadtree, V-lists and the far field on it (readings R12, R13)
# ---------------------------------------------------------------------------

class AdaptiveTree:
    """Box existence over levels 0..max_level of an adaptive quadtree (reading R12)."""

    def __init__(self, exists: np.ndarray, max_level: int, depth: int, q: int):
        self.exists = exists  # uint8, level-major: level l at [(4^l - 1)/3, (4^(l+1) - 1)/3)
        self.max_level = max_level
        self.depth = depth
        self.q = q

    def level(self, l: int) -> np.ndarray:
        """Existence of the 4^l boxes of level l (bool, b = iy * 2^l + ix)."""
        off = ((1 << (2 * l)) - 1) // 3
        return self.exists[off:off + (1 << (2 * l))].astype(bool)

    def _ptr(self):
        return self.exists.ctypes.data_as(_U8)


def adaptive_tree(xy, q: int, max_level: int) -> AdaptiveTree:
    """Split boxes holding more than q points down to max_level; empty children are dropped."""
    xy = _f64(xy)
    ex = np.zeros(((1 << (2 * (max_level + 1))) - 1) // 3, dtype=np.uint8)
    depth = lib().orc_adaptive_tree(xy.shape[0], _dp(xy), q, max_level, ex.ctypes.data_as(_U8))
    return AdaptiveTree(ex, max_level, int(depth), q)


def vlist(tree: AdaptiveTree, level: int, tx: int, ty: int):
    """V-list of (tx, ty): [(sx, sy, ox, oy)], offsets = source minus target in box units."""
    bufs = [np.zeros(27, dtype=np.int32) for _ in range(4)]
    ptrs = [b.ctypes.data_as(_I) for b in bufs]
    n = lib().orc_vlist(level, tx, ty, tree._ptr(), *ptrs)
    return [tuple(int(b[i]) for b in bufs) for i in range(n)]


def vlist_count_level(tree: AdaptiveTree, level: int) -> int:
    return int(lib().orc_vlist_count_level(level, tree._ptr()))


def m2l_adaptive(tree: AdaptiveTree, level: int, p: int, M: np.ndarray) -> np.ndarray:
    """Physical-unit M2L over the V-lists of one level (zero at absent boxes)."""
    Mr = _c2r(M)
    L = np.zeros_like(Mr)
    lib().orc_m2l_adaptive(level, p, tree._ptr(), _dp(Mr), _dp(L))
    return _r2c(L)


def m2l_adjoint_adaptive(tree: AdaptiveTree, level: int, p: int, W: np.ndarray) -> np.ndarray:
    """Plain transpose of ``m2l_adaptive`` by explicit transposed loops."""
    Wr = _c2r(W)
    G = np.zeros_like(Wr)
    lib().orc_m2l_adjoint_adaptive(level, p, tree._ptr(), _dp(Wr), _dp(G))
    return _r2c(G)


def leaf_boxes(tree: AdaptiveTree, xy):
    """(leaf level, leaf box index) of every point: the deepest existing box containing it (reading R5)."""
    xy = _f64(xy)
    lev = np.zeros(xy.shape[0], dtype=np.int64)
    box = np.zeros(xy.shape[0], dtype=np.int64)
    for l in range(tree.depth + 1):
        n = 1 << l
        ix = np.clip(np.floor(xy[:, 0] * n).astype(np.int64), 0, n - 1)
        iy = np.clip(np.floor(xy[:, 1] * n).astype(np.int64), 0, n - 1)
        b = iy * n + ix
        here = tree.level(l)[b]
        lev = np.where(here, l, lev)
        box = np.where(here, b, box)
    return lev, box


def ancestor_box(leaf_level, leaf_box, level: int) -> np.ndarray:
    """Box of `level` containing each leaf (-1 where the leaf is shallower than `level`)."""
    leaf_level = np.asarray(leaf_level, dtype=np.int64)
    leaf_box = np.asarray(leaf_box, dtype=np.int64)
    sh = leaf_level - level
    side = np.left_shift(1, leaf_level)
    ix = np.right_shift(leaf_box % side, np.maximum(sh, 0))
    iy = np.right_shift(leaf_box // side, np.maximum(sh, 0))
    return np.where(sh >= 0, iy * (1 << level) + ix, -1)


def p2m_assigned(level: int, p: int, xy, c, box) -> np.ndarray:
    """ME of every box of `level` from the points assigned to it (box[i] = -1: none)."""
    xy, c = _f64(xy), _f64(c)
    b = np.ascontiguousarray(box, dtype=np.int64)
    M = np.zeros(((1 << (2 * level)), p, 2))
    lib().orc_p2m_assigned(level, p, len(c), _dp(xy), _dp(c), b.ctypes.data_as(_I64), _dp(M))
    return _r2c(M)


def _l2p_at_leaves(p: int, L: dict, z, z_lev, z_box) -> np.ndarray:
    """phi(z_j) = sum_n L[leaf_j][n] (z_j - x_leaf)^n for every evaluation point."""
    z = np.asarray(z, dtype=np.complex128)
    phi = np.zeros(len(z), dtype=np.complex128)
    for l in np.unique(z_lev):
        sel = np.nonzero(z_lev == l)[0]
        if l < 2:
            continue  # no far field above level 2
        n = 1 << int(l)
        bx, by = z_box[sel] % n, z_box[sel] // n
        centre = (bx + 0.5) / n + 1j * (by + 0.5) / n
        d = z[sel] - centre
        acc = np.zeros(len(sel), dtype=np.complex128)
        for k in range(p - 1, -1, -1):  # Horner
            acc = acc * d + L[int(l)][z_box[sel], k]
        phi[sel] = acc
    return phi


def far_field_objective(tree: AdaptiveTree, p: int, xy, c, leaf, z, z_leaf, omega) -> float:
    """J = sum_j omega_j Re phi_far(z_j) (reading R13): the MEs of every level from
    the points assigned to the frozen leaves `leaf` = (levels, boxes), M2L over the
    V-lists of levels 2..depth, L2L down, L2P at each evaluation point's leaf."""
    lev, box = leaf
    L = {}
    for l in range(2, tree.depth + 1):
        M = p2m_assigned(l, p, xy, c, ancestor_box(lev, box, l))
        Lr = _c2r(m2l_adaptive(tree, l, p, M))
        if l > 2:
            lib().orc_l2l_level(l, p, tree._ptr(), _dp(_c2r(L[l - 1])), _dp(Lr))
        L[l] = _r2c(Lr)
    phi = _l2p_at_leaves(p, L, z, z_leaf[0], z_leaf[1])
    return float(np.sum(np.asarray(omega) * phi.real))


def far_field_fd_gradient(tree: AdaptiveTree, p: int, xy, c, leaf, z, z_leaf, omega, idx, h: float = 1e-4):
    """Central differences (J(y + h e) - J(y - h e)) / 2h of `far_field_objective`
    with respect to the coordinates of the points `idx` (frozen topology).  J is
    linear in the MEs, so each difference is J's pipeline applied to the
    difference of the perturbed MEs, which is non-zero only in the point's
    ancestor boxes (one per level): the M2L runs from those boxes only.
    Returns [len(idx), 2] (d/dx, d/dy)."""
    xy, c = _f64(xy), _f64(c)
    lev, box = leaf
    out = np.zeros((len(idx), 2))
    for r, i in enumerate(idx):
        for axis in range(2):
            plus, minus = xy[i].copy(), xy[i].copy()
            plus[axis] += h
            minus[axis] -= h
            L = {}
            for l in range(2, tree.depth + 1):
                Lr = np.zeros(((1 << (2 * l)), p, 2))
                b = int(ancestor_box(lev[i:i + 1], box[i:i + 1], l)[0])
                if b >= 0:
                    n = 1 << l
                    centre = complex((b % n + 0.5) / n, (b // n + 0.5) / n)
                    dM = p2m_box(plus[None, :], c[i:i + 1], centre, p) - p2m_box(minus[None, :], c[i:i + 1], centre, p)
                    src = np.array([b], dtype=np.int64)
                    lib().orc_m2l_adaptive_from_sources(l, p, tree._ptr(), 1, src.ctypes.data_as(_I64),
                                                        _dp(_c2r(dM[None, :])), _dp(Lr))
                if l > 2:
                    lib().orc_l2l_level(l, p, tree._ptr(), _dp(_c2r(L[l - 1])), _dp(Lr))
                L[l] = _r2c(Lr)
            phi = _l2p_at_leaves(p, L, z, z_leaf[0], z_leaf[1])
            out[r, axis] = float(np.sum(np.asarray(omega) * phi.real)) / (2.0 * h)
    return out


# ---------------------------------------------------------------------------
# radius scaling used at the CUDA library's boundary (a change of units)
# ---------------------------------------------------------------------------

def scale_me(M: np.ndarray, level: int) -> np.ndarray:
    """m~_k = m_k / r^k,  r = 2^-level."""
    p = M.shape[-1]
    k = np.arange(p)
    return M * np.ldexp(1.0, level * k)


def unscale_me(Ms: np.ndarray, level: int) -> np.ndarray:
    """m_k = m~_k r^k,  r = 2^-level."""
    p = Ms.shape[-1]
    k = np.arange(p)
    return Ms * np.ldexp(1.0, -level * k)


def scale_le(L: np.ndarray, level: int) -> np.ndarray:
    """l~_n = l_n * r^(n+1),  r = 2^-level."""
    p = L.shape[-1]
    n = np.arange(p)
    return L * np.ldexp(1.0, -level * (n + 1))


def unscale_le(Ls: np.ndarray, level: int) -> np.ndarray:
    p = Ls.shape[-1]
    n = np.arange(p)
    return Ls * np.ldexp(1.0, level * (n + 1))


# ---------------------------------------------------------------------------
# fast Gauss transform (Sec. 2.2, Eqs. dgt, A_alpha, B_beta, C_beta, hermite, taylor)
# ---------------------------------------------------------------------------

def hermite_functions(nmax: int, t: float) -> np.ndarray:
    h = np.zeros(max(nmax, 1))
    lib().orc_hermite_functions(nmax, float(t), _dp(h))
    return h[:nmax]


def fgt_direct(x, q, sigma: float, y) -> np.ndarray:
    x, q, y = _f64(x), _f64(q), _f64(y)
    G = np.zeros(y.shape[0])
    lib().orc_fgt_direct(len(q), _dp(x), _dp(q), sigma, y.shape[0], _dp(y), _dp(G))
    return G


def fgt_taylor_eval_grid(g: int, p: int, sigma: float, C: np.ndarray, y) -> np.ndarray:
    """Eq. (taylor) at every target from the Taylor coefficients of its own box of the
    2^g grid (box floor(y 2^g), clamped; centre the box centre)."""
    y = _f64(y)
    side = 1 << g
    ix = np.clip(np.floor(y[:, 0] * side).astype(np.int64), 0, side - 1)
    iy = np.clip(np.floor(y[:, 1] * side).astype(np.int64), 0, side - 1)
    G = np.zeros(y.shape[0])
    for b in np.unique(iy * side + ix):
        sel = np.nonzero(iy * side + ix == b)[0]
        tc = ((b % side + 0.5) / side, (b // side + 0.5) / side)
        G[sel] = fgt_taylor_eval(C[b], tc, sigma, y[sel])
    return G


def fgt_p2h(x, q, sB, sigma: float, p: int) -> np.ndarray:
    x, q = _f64(x), _f64(q)
    A = np.zeros((p, p))
    lib().orc_fgt_p2h(len(q), _dp(x), _dp(q), sB[0], sB[1], sigma, p, _dp(A))
    return A


def fgt_hermite_eval(A: np.ndarray, sB, sigma: float, y) -> np.ndarray:
    A, y = _f64(A), _f64(y)
    G = np.zeros(y.shape[0])
    lib().orc_fgt_hermite_eval(A.shape[0], _dp(A), sB[0], sB[1], sigma, y.shape[0], _dp(y), _dp(G))
    return G


def fgt_p2t(x, q, tC, sigma: float, p: int) -> np.ndarray:
    x, q = _f64(x), _f64(q)
    B = np.zeros((p, p))
    lib().orc_fgt_p2t(len(q), _dp(x), _dp(q), tC[0], tC[1], sigma, p, _dp(B))
    return B


def fgt_taylor_eval(B: np.ndarray, tC, sigma: float, y) -> np.ndarray:
    B, y = _f64(B), _f64(y)
    G = np.zeros(y.shape[0])
    lib().orc_fgt_taylor_eval(B.shape[0], _dp(B), tC[0], tC[1], sigma, y.shape[0], _dp(y), _dp(G))
    return G


def fgt_h2t_pair(A: np.ndarray, u1: float, u2: float) -> np.ndarray:
    A = _f64(A)
    C = np.zeros_like(A)
    lib().orc_fgt_h2t_pair(A.shape[0], _dp(A), float(u1), float(u2), _dp(C))
    return C


def fgt_h2t_grid(g: int, ncut: int, p: int, sigma: float, A: np.ndarray) -> np.ndarray:
    A = _f64(A)
    C = np.zeros_like(A)
    lib().orc_fgt_h2t_grid(g, ncut, p, sigma, _dp(A), _dp(C))
    return C


def fgt_h2t_targets(g: int, ncut: int, p: int, sigma: float, A: np.ndarray, targets) -> np.ndarray:
    A = _f64(A)
    t = np.ascontiguousarray(targets, dtype=np.int64)
    C = np.zeros((len(t), p, p))
    lib().orc_fgt_h2t_targets(g, ncut, p, sigma, _dp(A), len(t), t.ctypes.data_as(_I64), _dp(C))
    return C


def fgt_hermite_eval_grid(g: int, ncut: int, p: int, sigma: float, A: np.ndarray, y) -> np.ndarray:
    """Eq. (hermite) at every target, summed over the source boxes of the 2^g grid within
    Chebyshev distance ncut of the target's own box (reading R14).  A: [4^g, p, p]."""
    A, y = _f64(A), _f64(y)
    G = np.zeros(y.shape[0])
    lib().orc_fgt_hermite_eval_grid(g, ncut, p, sigma, _dp(A), y.shape[0], _dp(y), _dp(G))
    return G


def fgt_p2h_grid(g: int, p: int, sigma: float, x, q) -> np.ndarray:
    x, q = _f64(x), _f64(q)
    n = 1 << g
    A = np.zeros((n * n, p, p))
    lib().orc_fgt_p2h_grid(g, p, sigma, len(q), _dp(x), _dp(q), _dp(A))
    return A
