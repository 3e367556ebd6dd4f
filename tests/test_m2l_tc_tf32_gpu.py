"""GPU parity of the tensor-core M2L with TF32 operands (FMM_TC_TF32X3, p = 16)
against the FP64 oracle, through the C ABI.

FMM_TC_TF32X3 splits the operator and the MEs into TF32 hi + lo (11 significant
bits each, rounded to nearest) and issues hi*hi + hi*lo + lo*hi with FP32
accumulation: ~21 significant bits per product, so it is held to the FP32 bar,
relative L2 of the scaled local coefficients <= 1e-5 per level (FMM_TC_BF16X3
is held to 1e-4).
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def test_tf32x3_levels_2_to_5_and_tighter_than_bf16x3(fmm, orc, particles):
    """One level per call; the TF32 split is more accurate than the BF16 one at every level."""
    xy, c = particles
    p = 16
    Ms = orc.upward_uniform(5, p, xy, c)
    tree = fmm.fmm_build_lists(None, 5)
    for level in range(2, 6):
        ref = _oracle_level(orc, level, p, Ms[level])
        Md = _dev(orc.scale_me(Ms[level], level))
        errs = {}
        for name in ("FMM_TC_TF32X3", "FMM_TC_BF16X3"):
            Ld = Md.new_empty(Md.shape)
            fmm.fmm_m2l(tree, level, p, Md, Ld, prec=getattr(fmm, name))
            fmm.fmm_sync_status()
            errs[name] = _rel(_host(Ld), ref)
        assert errs["FMM_TC_TF32X3"] <= TOL, (level, errs)
        assert errs["FMM_TC_TF32X3"] < errs["FMM_TC_BF16X3"], (level, errs)


def test_tf32x3_levels_free_space_accumulate(fmm, orc, particles):
    """Levels 2..7 in one launch (tiles cut between CTAs, halos by tensor copy), accumulating
    into existing values: every part of a cut tile adds."""
    xy, c = particles
    p, Lmax = 16, 7
    Ms = orc.upward_uniform(Lmax, p, xy, c)
    tree = fmm.fmm_build_lists(None, Lmax)
    levels = list(range(2, Lmax + 1))
    rng = np.random.default_rng(12)
    X = {l: (rng.standard_normal((4 ** l, p)) + 1j * rng.standard_normal((4 ** l, p))) * 1e-3 for l in levels}
    Md = [_dev(orc.scale_me(Ms[l], l)) for l in levels]
    Ld = [_dev(X[l]) for l in levels]
    fmm.fmm_m2l_levels(tree, 2, p, Md, Ld, prec=fmm.FMM_TC_TF32X3, accumulate=True)
    fmm.fmm_sync_status()
    for l, out in zip(levels, Ld):
        ref = _oracle_level(orc, l, p, Ms[l])
        got = _host(out) - X[l].astype(np.complex64).astype(np.complex128)
        assert _rel(got, ref) <= TOL, (l, _rel(got, ref))


def test_tf32x3_periodic_levels(fmm, orc, particles):
    """Periodic lists (halos staged from global memory, wrapping), levels 2..6 in one launch."""
    xy, c = particles
    p, Lmax = 16, 6
    Ms = orc.upward_uniform(Lmax, p, xy, c)
    tree = fmm.fmm_build_lists(None, Lmax, periodic=True)
    levels = list(range(2, Lmax + 1))
    Md = [_dev(orc.scale_me(Ms[l], l)) for l in levels]
    Ld = [m.new_empty(m.shape) for m in Md]
    fmm.fmm_m2l_levels(tree, 2, p, Md, Ld, prec=fmm.FMM_TC_TF32X3)
    fmm.fmm_sync_status()
    for l, out in zip(levels, Ld):
        err = _rel(_host(out), _oracle_level(orc, l, p, Ms[l], periodic=True))
        assert err <= TOL, (l, err)


@pytest.mark.parametrize("conj", [False, True])
def test_tf32x3_adjoint_levels(fmm, orc, conj):
    """The adjoint (the forward kernel with the TF32 image of -T or -conj T) against the
    oracle's explicit transpose, scaled units, levels 2..5 in one launch."""
    p = 16
    rng = np.random.default_rng(70 + int(conj))
    levels = list(range(2, 6))
    tree = fmm.fmm_build_lists(None, 5)
    W = {l: rng.standard_normal((4 ** l, p)) + 1j * rng.standard_normal((4 ** l, p)) for l in levels}
    Wd = [_dev(W[l]) for l in levels]
    Gd = [w.new_empty(w.shape) for w in Wd]
    fmm.fmm_m2l_adjoint_levels(tree, 2, p, Wd, Gd, prec=fmm.FMM_TC_TF32X3, conj=conj)
    fmm.fmm_sync_status()
    for l, g in zip(levels, Gd):
        Win = np.conj(W[l]) if conj else W[l]
        G = orc.unscale_me(orc.m2l_adjoint_uniform(l, p, orc.scale_le(Win, l)), l)
        if conj:
            G = np.conj(G)
        assert _rel(_host(g), G) <= TOL, (l, _rel(_host(g), G))


@pytest.mark.slow
def test_tf32x3_full_size_workload(fmm, orc):
    """2^22 points, level 8, p = 16, levels 2..8 in one launch: levels 2..6 in full, level 8
    on sampled targets (corners included)."""
    cfg = workloads.CONFIGS["m2l_scale"]
    p, L = cfg["p"], cfg["max_level"]
    xy, c = workloads.uniform_particles(cfg["n"], workloads.rng_for("m2l_scale"))
    Ms = orc.upward_uniform(L, p, xy, c)
    tree = fmm.fmm_build_lists(None, L)
    levels = workloads.m2l_levels(L)
    Md = [_dev(orc.scale_me(Ms[l], l)) for l in levels]
    Ld = [m.new_empty(m.shape) for m in Md]
    fmm.fmm_m2l_levels(tree, 2, p, Md, Ld, prec=fmm.FMM_TC_TF32X3)
    fmm.fmm_sync_status()
    for l, out in zip(levels, Ld):
        if l <= 6:
            assert _rel(_host(out), _oracle_level(orc, l, p, Ms[l])) <= TOL, l
    n = 1 << L
    rng = np.random.default_rng(3)
    targets = np.unique(np.concatenate([[0, n - 1, n * (n - 1), n * n - 1], rng.integers(0, n * n, 2000)]))
    ref = orc.scale_le(orc.m2l_uniform_targets(L, p, Ms[L], targets), L)
    assert _rel(_host(Ld[-1])[targets], ref) <= TOL
