"""GPU parity of the tensor-core M2L path (fmm_m2l with FMM_TC_BF16X3 / FMM_TC_BF16)
against the FP64 oracle, through the C ABI.

Bars:
* FMM_TC_BF16X3 (BF16 hi/lo split, three products, FP32 accumulation): relative L2
  error of the scaled local coefficients <= 1e-4 per level, and on the p = 24
  workload (4096 points, level 4) the far-field potential error vs the direct sum
  must stay within the oracle's own truncation error + 1e-4;
* FMM_TC_BF16 (plain BF16 inputs): relative L2 <= 1e-2 (8 significant bits).
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


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


def _oracle_level(orc, level, p, M, periodic=False):
    return orc.scale_le(orc.m2l_uniform(level, p, M, periodic), level)


@pytest.fixture(scope="module")
def particles():
    return workloads.uniform_particles(6000, np.random.default_rng(321))


@pytest.mark.parametrize("p", [16, 24])
def test_tc_bf16x3_levels_2_to_5(fmm, orc, particles, p):
    xy, c = particles
    Ms = orc.upward_uniform(5, p, xy, c)
    tree = fmm.fmm_build_lists(None, 5)
    for level in range(2, 6):
        Md = _dev(orc.scale_me(Ms[level], level))
        Ld = Md.new_empty(Md.shape)
        fmm.fmm_m2l(tree, level, p, Md, Ld, prec=fmm.FMM_TC_BF16X3)
        fmm.fmm_sync_status()
        err = _rel(_host(Ld), _oracle_level(orc, level, p, Ms[level]))
        assert err <= 1e-4, (level, err)


def test_tc_bf16_single_pass(fmm, orc, particles):
    xy, c = particles
    p, level = 16, 4
    Ms = orc.upward_uniform(level, p, xy, c)
    tree = fmm.fmm_build_lists(None, level)
    Md = _dev(orc.scale_me(Ms[level], level))
    Ld = Md.new_empty(Md.shape)
    fmm.fmm_m2l(tree, level, p, Md, Ld, prec=fmm.FMM_TC_BF16)
    fmm.fmm_sync_status()
    err = _rel(_host(Ld), _oracle_level(orc, level, p, Ms[level]))
    assert 1e-5 < err <= 1e-2, err


def test_tc_levels_periodic_accumulate(fmm, orc, particles):
    """All levels 2..6 in one launch, periodic lists, accumulating into existing values."""
    xy, c = particles
    p, Lmax = 16, 6
    Ms = orc.upward_uniform(Lmax, p, xy, c)
    tree = fmm.fmm_build_lists(None, Lmax, periodic=True)
    levels = list(range(2, Lmax + 1))
    rng = np.random.default_rng(5)
    X = {l: (rng.standard_normal((4 ** l, p)) + 1j * rng.standard_normal((4 ** l, p))) for l in levels}
    Md = [_dev(orc.scale_me(Ms[l], l)) for l in levels]
    Ld = [_dev(X[l]) for l in levels]
    fmm.fmm_m2l_levels(tree, 2, p, Md, Ld, prec=fmm.FMM_TC_BF16X3, accumulate=True)
    fmm.fmm_sync_status()
    for l, out in zip(levels, Ld):
        ref = _oracle_level(orc, l, p, Ms[l], periodic=True)
        got = _host(out) - X[l].astype(np.complex64).astype(np.complex128)
        assert _rel(got, ref) <= 1e-4, l


@pytest.mark.parametrize("p", [16, 24])
def test_tc_levels_free_space_accumulate(fmm, orc, particles, p):
    """Levels 2..7 in one launch (tiles cut between CTAs, every level by tensor copy),
    free-space lists, accumulating into existing values: every part of a cut tile adds."""
    xy, c = particles
    Lmax = 7
    Ms = orc.upward_uniform(Lmax, p, xy, c)
    tree = fmm.fmm_build_lists(None, Lmax)
    levels = list(range(2, Lmax + 1))
    rng = np.random.default_rng(11)
    X = {l: (rng.standard_normal((4 ** l, p)) + 1j * rng.standard_normal((4 ** l, p))) for l in levels}
    Md = [_dev(orc.scale_me(Ms[l], l)) for l in levels]
    Ld = [_dev(X[l]) for l in levels]
    fmm.fmm_m2l_levels(tree, 2, p, Md, Ld, prec=fmm.FMM_TC_BF16X3, accumulate=True)
    fmm.fmm_sync_status()
    for l, out in zip(levels, Ld):
        ref = _oracle_level(orc, l, p, Ms[l])
        got = _host(out) - X[l].astype(np.complex64).astype(np.complex128)
        assert _rel(got, ref) <= 1e-4, l


def test_tc_precision_workload_p24_potential(fmm, orc):
    """The p = 24 precision workload (4096 points, uniform tree to level 4): the far-field
    potential from the tensor-core LEs is within the oracle's own truncation error + 1e-4."""
    cfg = workloads.CONFIGS["m2l_tc"]
    p, L = cfg["p"], cfg["max_level"]
    xy, c = workloads.uniform_particles(cfg["n"], workloads.rng_for("m2l_tc"))
    Ms = orc.upward_uniform(L, p, xy, c)
    tree = fmm.fmm_build_lists(None, L)
    n = 1 << L
    side = 2.0 ** -L
    ib = np.minimum((xy * n).astype(int), n - 1)
    rng = np.random.default_rng(77)
    worst_tc, worst_orc = 0.0, 0.0
    Md = _dev(orc.scale_me(Ms[L], L))
    Ld = Md.new_empty(Md.shape)
    fmm.fmm_m2l(tree, L, p, Md, Ld, prec=fmm.FMM_TC_BF16X3)
    fmm.fmm_sync_status()
    L_tc = orc.unscale_le(_host(Ld), L)
    L_or = orc.m2l_uniform(L, p, Ms[L])
    coef_err = _rel(orc.scale_le(L_tc, L), orc.scale_le(L_or, L))
    assert coef_err <= 1e-4
    for t in rng.choice(n * n, 24, replace=False):
        tx, ty = int(t % n), int(t // n)
        ct = orc.box_centre(L, tx, ty)
        z = ct + (rng.random(16) - 0.5) * side + 1j * (rng.random(16) - 0.5) * side
        srcs = np.zeros(len(c), bool)
        for sx, sy, _, _ in orc.interaction_list(L, tx, ty):
            srcs |= (ib[:, 0] == sx) & (ib[:, 1] == sy)
        exact = orc.direct(xy[srcs], c[srcs], z)
        nrm = np.linalg.norm(exact)
        worst_orc = max(worst_orc, np.linalg.norm(orc.l2p(p, L_or[t], ct, z) - exact) / nrm)
        worst_tc = max(worst_tc, np.linalg.norm(orc.l2p(p, L_tc[t], ct, z) - exact) / nrm)
    assert worst_tc <= worst_orc + 1e-4, (worst_tc, worst_orc)


@pytest.mark.slow
def test_tc_full_size_workload(fmm, orc):
    """2^22 points, level 8, p = 16, levels 2..8 in one launch (BF16x3): levels 2..6 in full,
    level 8 on sampled targets."""
    cfg = workloads.CONFIGS["m2l_scale"]
    p, L = cfg["p"], cfg["max_level"]
    xy, c = workloads.uniform_particles(cfg["n"], workloads.rng_for("m2l_scale"))
    Ms = orc.upward_uniform(L, p, xy, c)
    tree = fmm.fmm_build_lists(None, L)
    levels = workloads.m2l_levels(L)
    Md = [_dev(orc.scale_me(Ms[l], l)) for l in levels]
    Ld = [m.new_empty(m.shape) for m in Md]
    fmm.fmm_m2l_levels(tree, 2, p, Md, Ld, prec=fmm.FMM_TC_BF16X3)
    fmm.fmm_sync_status()
    for l, out in zip(levels, Ld):
        if l <= 6:
            assert _rel(_host(out), _oracle_level(orc, l, p, Ms[l])) <= 1e-4, l
    n = 1 << L
    rng = np.random.default_rng(2)
    targets = np.unique(np.concatenate([[0, n - 1, n * (n - 1), n * n - 1], rng.integers(0, n * n, 2000)]))
    ref = orc.scale_le(orc.m2l_uniform_targets(L, p, Ms[L], targets), L)
    assert _rel(_host(Ld[-1])[targets], ref) <= 1e-4


@pytest.mark.parametrize("conj", [False, True])
@pytest.mark.parametrize("p", [16, 24])
def test_tc_bf16x3_adjoint_levels(fmm, orc, p, conj):
    """Tensor-core adjoint (the forward kernel with the image of -T or -conj T) against the
    oracle's explicit transpose, scaled units G~ = R_M A^T R_L W~, levels 2..5 in one launch."""
    rng = np.random.default_rng(40 + p + int(conj))
    levels = list(range(2, 6))
    tree = fmm.fmm_build_lists(None, 5)
    W = {l: rng.standard_normal((4 ** l, p)) + 1j * rng.standard_normal((4 ** l, p)) for l in levels}
    Wd = [_dev(W[l]) for l in levels]
    Gd = [w.new_empty(w.shape) for w in Wd]
    fmm.fmm_m2l_adjoint_levels(tree, 2, p, Wd, Gd, prec=fmm.FMM_TC_BF16X3, conj=conj)
    fmm.fmm_sync_status()
    for l, g in zip(levels, Gd):
        Win = np.conj(W[l]) if conj else W[l]
        G = orc.unscale_me(orc.m2l_adjoint_uniform(l, p, orc.scale_le(Win, l)), l)
        if conj:
            G = np.conj(G)
        assert _rel(_host(g), G) <= 1e-4, (l, _rel(_host(g), G))
