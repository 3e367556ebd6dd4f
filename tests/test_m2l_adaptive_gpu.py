"""GPU parity of the M2L path on adaptive trees (V-lists, reading R12) and of its
gradients (the autograd binding and the far-field objective of reading R13)
against the FP64 oracle, through the C ABI.

Bars: FP32 forward and adjoint, relative L2 of the scaled coefficients of the
existing boxes of each level <= 1e-5; absent boxes untouched; gradient of the
far-field objective with respect to 64 source positions against the oracle's
central differences (frozen topology): relative L2 <= 1e-4.  The step is
h = 1e-6: the ME terms ((y - x_b)/r)^k vary on the scale of a level-9 box
(r = 2^-9), where h = 1e-4 leaves a central-difference error of ~1e-3; at
h = 1e-6 it is ~1e-8 (h = 1e-7 agrees to 1e-7), and the oracle differences
only the perturbed point's own ME terms, so rounding does not grow as h shrinks.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5
FD_STEP = 1e-6


@pytest.fixture(scope="module")
def fmm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_3457_gb300 import build, fmmgb

    build.build()
    fmmgb.load()
    return fmmgb


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def _host(t):
    return t.cpu().numpy().astype(np.complex128)


def _rel(got, ref):
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


def _case(orc, fmm, n, q, L, seed):
    xy, c = workloads.gmm_particles(n, np.random.default_rng(seed), ncomp=8)
    tree = fmm.fmm_build_lists(xy, L, leaf_cap=q)
    otree = orc.adaptive_tree(xy, q, L)
    lev, box = orc.leaf_boxes(otree, xy)
    Ms = {l: orc.p2m_assigned(l, 16, xy, c, orc.ancestor_box(lev, box, l)) for l in range(2, L + 1)}
    return xy, c, tree, otree, Ms


@pytest.mark.parametrize("p", [8, 16])
def test_adaptive_forward_levels(fmm, orc, p):
    xy, c, tree, otree, _ = _case(orc, fmm, 30000, 40, 8, 5)
    lev, box = orc.leaf_boxes(otree, xy)
    levels = list(range(2, 9))
    Ms = {l: orc.p2m_assigned(l, p, xy, c, orc.ancestor_box(lev, box, l)) for l in levels}
    Md = [_dev(orc.scale_me(Ms[l], l)) for l in levels]
    Ld = [m.new_full(m.shape, 5.0 + 0j) for m in Md]
    fmm.fmm_m2l_levels(tree, 2, p, Md, Ld)
    fmm.fmm_sync_status()
    for l, out in zip(levels, Ld):
        ex = otree.level(l)
        got = _host(out)
        ref = orc.scale_le(orc.m2l_adaptive(otree, l, p, Ms[l]), l)
        if ex.any():
            assert _rel(got[ex], ref[ex]) <= TOL, l
        assert (got[~ex] == 5.0).all(), l  # absent boxes untouched


def test_adaptive_single_level_and_accumulate(fmm, orc):
    xy, c, tree, otree, Ms = _case(orc, fmm, 20000, 30, 7, 6)
    rng = np.random.default_rng(1)
    for l in (5, 7):
        ex = otree.level(l)
        X = rng.standard_normal((4 ** l, 16)) + 1j * rng.standard_normal((4 ** l, 16))
        Md = _dev(orc.scale_me(Ms[l], l))
        Ld = _dev(X)
        fmm.fmm_m2l(tree, l, 16, Md, Ld, accumulate=True)
        fmm.fmm_sync_status()
        got = _host(Ld) - X.astype(np.complex64).astype(np.complex128)
        ref = orc.scale_le(orc.m2l_adaptive(otree, l, 16, Ms[l]), l)
        assert _rel(got[ex], ref[ex]) <= TOL


@pytest.mark.parametrize("conj", [False, True])
def test_adaptive_adjoint(fmm, orc, conj):
    """Scaled adjoint G~ = R_M A^T R_L W~ over the V-lists (A^T from the oracle's explicit transpose)."""
    xy, c, tree, otree, _ = _case(orc, fmm, 20000, 30, 7, 7)
    rng = np.random.default_rng(9)
    p = 16
    for l in range(2, 8):
        ex = otree.level(l)
        W = rng.standard_normal((4 ** l, p)) + 1j * rng.standard_normal((4 ** l, p))
        Wd = _dev(W)
        Gd = Wd.new_zeros(Wd.shape)
        fmm.fmm_m2l_adjoint(tree, l, p, Wd, Gd, conj=conj)
        fmm.fmm_sync_status()
        Win = np.conj(W) if conj else W
        G = orc.unscale_me(orc.m2l_adjoint_adaptive(otree, l, p, orc.scale_le(Win, l)), l)
        if conj:
            G = np.conj(G)
        if ex.any() and np.linalg.norm(G[ex]) > 0:
            assert _rel(_host(Gd)[ex], G[ex]) <= TOL, l
        assert (_host(Gd)[~ex] == 0).all()


def test_autograd_m2l_backward_is_conjugate_adjoint(fmm, orc):
    """M2LLevels: d/dM of Re <W, L(M)> equals A^H W (oracle transpose, conjugated)."""
    import torch

    from paper_1009_3457_gb300 import autograd

    xy, c, tree, otree, Ms = _case(orc, fmm, 20000, 30, 6, 8)
    p = 16
    levels = list(range(2, 7))
    rng = np.random.default_rng(2)
    Md = [_dev(orc.scale_me(Ms[l], l)).requires_grad_(True) for l in levels]
    Wn = [rng.standard_normal((4 ** l, p)) + 1j * rng.standard_normal((4 ** l, p)) for l in levels]
    Ls = autograd.m2l_levels(tree, p, Md)
    J = sum((torch.conj(_dev(w)) * L).real.sum() for w, L in zip(Wn, Ls))
    J.backward()
    for l, m, w in zip(levels, Md, Wn):
        ex = otree.level(l)
        # J = Re sum conj(W) L = Re <W, A M>;  PyTorch grad = dJ/dRe M + i dJ/dIm M = A^H W
        G = np.conj(orc.unscale_me(orc.m2l_adjoint_adaptive(otree, l, p, orc.scale_le(np.conj(w), l)), l))
        assert _rel(_host(m.grad)[ex], G[ex]) <= TOL, l


def _gradient_case(orc, fmm, n, q, L, seed):
    import torch

    from paper_1009_3457_gb300 import farfield

    rng = np.random.default_rng(seed)
    xy, c = workloads.gmm_particles(n, rng)
    tree = fmm.fmm_build_lists(xy, L, leaf_cap=q)
    otree = orc.adaptive_tree(xy, q, L)
    zr = np.random.default_rng(seed + 1)
    z = zr.random(4096) + 1j * zr.random(4096)
    w = zr.uniform(-1, 1, 4096)
    xyt = torch.from_numpy(xy).cuda().requires_grad_(True)
    leaf = farfield.leaf_boxes(tree, xyt.detach())
    zl = farfield.leaf_boxes(tree, torch.from_numpy(np.stack([z.real, z.imag], 1)).cuda())
    J = farfield.far_field_objective(tree, 16, xyt, torch.from_numpy(c).cuda(), leaf, torch.from_numpy(z).cuda(), zl,
                                     torch.from_numpy(w).cuda())
    J.backward()
    fmm.fmm_sync_status()
    grad = xyt.grad.cpu().numpy()
    oleaf = orc.leaf_boxes(otree, xy)
    ozl = orc.leaf_boxes(otree, np.stack([z.real, z.imag], 1))
    idx = np.random.default_rng(seed + 2).choice(n, 64, replace=False)
    fd = orc.far_field_fd_gradient(otree, 16, xy, c, oleaf, z, ozl, w, idx, FD_STEP)
    Jo = orc.far_field_objective(otree, 16, xy, c, oleaf, z, ozl, w)
    return float(J.detach()), Jo, grad[idx], fd


def test_gradient_matches_oracle_fd_small(fmm, orc):
    J, Jo, g, fd = _gradient_case(orc, fmm, 40000, 32, 7, 12)
    assert abs(J - Jo) <= 1e-5 * abs(Jo)
    assert np.linalg.norm(g - fd) <= 1e-4 * np.linalg.norm(fd), np.linalg.norm(g - fd) / np.linalg.norm(fd)


@pytest.mark.slow
def test_gradient_matches_oracle_fd_gmm_workload(fmm, orc):
    """The differentiation workload: 2^20 Gaussian-mixture points, q = 64, levels
    to 9, p = 16, 4096 evaluation points, 64 sampled source positions."""
    cfg = workloads.CONFIGS["m2l_gmm"]
    J, Jo, g, fd = _gradient_case(orc, fmm, cfg["n"], cfg["leaf_cap"], cfg["max_level"], workloads.SEED_BASE + 4)
    assert abs(J - Jo) <= 1e-5 * abs(Jo)
    assert np.linalg.norm(g - fd) <= 1e-4 * np.linalg.norm(fd), np.linalg.norm(g - fd) / np.linalg.norm(fd)


@pytest.mark.parametrize("p,prec_name,tol", [(16, "FMM_TC_BF16X3", 1e-4), (24, "FMM_TC_BF16X3", 1e-4),
                                              (16, "FMM_TC_TF32X3", 1e-5)])
def test_tensor_core_adaptive_levels(fmm, orc, p, prec_name, tol):
    """The tensor cores on an adaptive tree, levels 2..8 in one launch: V-list translations within
    the precision's bar (BF16x3 1e-4, TF32x3 the FP32 bar 1e-5) at existing boxes; absent source
    boxes hold garbage that must not enter, absent targets keep their values; then accumulating
    into existing values."""
    prec = getattr(fmm, prec_name)
    xy, c, tree, otree, _ = _case(orc, fmm, 30000, 40, 8, 15)
    lev, box = orc.leaf_boxes(otree, xy)
    levels = list(range(2, 9))
    Ms = {l: orc.p2m_assigned(l, p, xy, c, orc.ancestor_box(lev, box, l)) for l in levels}
    Min = {}
    for l in levels:
        m = orc.scale_me(Ms[l], l)
        m[~otree.level(l)] = 1e3 + 1e3j  # absent sources: ignored on input
        Min[l] = m
    Md = [_dev(Min[l]) for l in levels]
    Ld = [m.new_full(m.shape, 5.0 + 0j) for m in Md]
    fmm.fmm_m2l_levels(tree, 2, p, Md, Ld, prec=prec)
    fmm.fmm_sync_status()
    refs = {}
    for l, out in zip(levels, Ld):
        ex = otree.level(l)
        got = _host(out)
        refs[l] = orc.scale_le(orc.m2l_adaptive(otree, l, p, Ms[l]), l)
        if ex.any():
            assert _rel(got[ex], refs[l][ex]) <= tol, l
        assert (got[~ex] == 5.0).all(), l  # absent boxes untouched
    # accumulate: L0 + M2L(M) at existing boxes
    rng = np.random.default_rng(2)
    X = {l: rng.standard_normal((4 ** l, p)) + 1j * rng.standard_normal((4 ** l, p)) for l in levels}
    Ld = [_dev(X[l]) for l in levels]
    fmm.fmm_m2l_levels(tree, 2, p, Md, Ld, prec=prec, accumulate=True)
    fmm.fmm_sync_status()
    for l, out in zip(levels, Ld):
        ex = otree.level(l)
        got = _host(out) - X[l].astype(np.complex64).astype(np.complex128)
        if ex.any():
            assert _rel(got[ex], refs[l][ex]) <= tol, l


@pytest.mark.parametrize("conj", [False, True])
def test_tensor_core_adaptive_adjoint(fmm, orc, conj):
    """The adjoint on the tensor cores over an adaptive tree's V-lists, all levels in one launch."""
    xy, c, tree, otree, _ = _case(orc, fmm, 20000, 30, 7, 17)
    rng = np.random.default_rng(19)
    p = 16
    levels = list(range(2, 8))
    W = {l: rng.standard_normal((4 ** l, p)) + 1j * rng.standard_normal((4 ** l, p)) for l in levels}
    Wd = [_dev(W[l]) for l in levels]
    Gd = [w.new_zeros(w.shape) for w in Wd]
    fmm.fmm_m2l_adjoint_levels(tree, 2, p, Wd, Gd, prec=fmm.FMM_TC_BF16X3, conj=conj)
    fmm.fmm_sync_status()
    for l, g in zip(levels, Gd):
        ex = otree.level(l)
        Win = np.conj(W[l]) if conj else W[l]
        G = orc.unscale_me(orc.m2l_adjoint_adaptive(otree, l, p, orc.scale_le(Win, l)), l)
        if conj:
            G = np.conj(G)
        if ex.any() and np.linalg.norm(G[ex]) > 0:
            assert _rel(_host(g)[ex], G[ex]) <= 1e-4, l
        assert (_host(g)[~ex] == 0).all()


@pytest.mark.parametrize("adaptive", [True, False])
def test_leaf_boxes_match_oracle_exactly(fmm, orc, adaptive):
    """fmm_leaf_boxes equals the oracle's leaf assignment bit for bit: the tree's
    own points, uniform points, and coordinates on and next to cell boundaries
    of every level (0, 1 - ulp, exact multiples of 2^-l, 1.0 and above, below 0)."""
    import torch

    from paper_1009_3457_gb300 import farfield

    rng = np.random.default_rng(91)
    xy, _ = workloads.gmm_particles(30000, rng, ncomp=8)
    L = 9
    if adaptive:
        tree = fmm.fmm_build_lists(xy, L, leaf_cap=32)
        otree = orc.adaptive_tree(xy, 32, L)
    else:
        L = 6
        tree = fmm.fmm_build_lists(None, L)
        nall = ((1 << (2 * (L + 1))) - 1) // 3
        otree = orc.AdaptiveTree(np.ones(nall, dtype=np.uint8), L, L, 0)  # every box of every level exists
    edges = np.array([0.0, np.nextafter(1.0, 0.0), 1.0, 1.5, -0.25, -0.0] +
                     [k * 2.0 ** -l for l in range(1, L + 1) for k in (1, 3, (1 << l) - 1)] +
                     [np.nextafter(k * 2.0 ** -l, 0.0) for l in range(1, L + 1) for k in (1, 3)])
    ex = np.array(np.meshgrid(edges, edges)).reshape(2, -1).T
    pts = np.concatenate([xy, rng.random((5000, 2)), ex])
    lev, box = farfield.leaf_boxes(tree, torch.from_numpy(pts).cuda())
    fmm.fmm_sync_status()
    olev, obox = orc.leaf_boxes(otree, pts)
    np.testing.assert_array_equal(lev.cpu().numpy(), olev)
    np.testing.assert_array_equal(box.cpu().numpy(), obox)
