"""GPU parity of the near field (fmm_p2p, Sec. 2.1 stage 5, reading R15) and of the whole
FMM on the device (farfield.FmmPotential) against the FP64 oracle.

Bars.  The kernel keeps positions relative to the target box's centre in FP32, so a
pair's distance carries an absolute error of ~2^-24 x 1.5 box sides; a term's relative
error is that over the pair's distance, and the closest of m points in a box lies ~side/m
away.  Trees used as an FMM keep a few dozen points per finest box: there the bar is
relative L2 <= 1e-5 against the oracle's near field, every target within 1e-4 of
max |phi|.  The coarse cases below (4,000 points in one box at level 0, ~250 per box at
level 2) are checked at 2e-4 and 1e-4.  The whole FMM at p = 16 is held to 2e-5 of the
direct sum (the oracle's own FMM at p = 16 is within 3e-8 of it).
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


def _bins(fmm, level, pts):
    import torch

    perm = torch.empty(pts.shape[0], dtype=torch.int32, device="cuda")
    start = torch.empty(4 ** level + 1, dtype=torch.int32, device="cuda")
    work = torch.empty(4 ** level, dtype=torch.int32, device="cuda")
    fmm.fmm_bin_points(level, pts, perm, start, work)
    return perm, start


def _p2p(fmm, level, xy, c, z, phi0=None):
    import torch

    xyd, cd = torch.from_numpy(xy).cuda(), torch.from_numpy(c).cuda()
    zd = torch.from_numpy(np.stack([z.real, z.imag], 1).copy()).cuda()
    sp, ss = _bins(fmm, level, xyd)
    tp, ts = _bins(fmm, level, zd)
    phi = torch.zeros(len(z), dtype=torch.complex64, device="cuda") if phi0 is None else \
        torch.from_numpy(phi0.astype(np.complex64)).cuda()
    fmm.fmm_p2p(level, xyd, cd, sp, ss, zd, tp, ts, phi, accumulate=phi0 is not None)
    fmm.fmm_sync_status()
    return phi.cpu().numpy().astype(np.complex128)


def _check(got, ref, l2=1e-5, worst=1e-4):
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    w = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= l2 and w <= worst, f"relative L2 {err:.3e}, worst {w:.3e}"


@pytest.mark.parametrize("level,bar,nsrc", [(0, 2e-4, 4000), (2, 1e-4, 4000), (3, 1e-5, 4000), (5, 1e-5, 4000),
                                            (8, 1e-5, 262144), (10, 1e-5, 1048576)])
def test_p2p_matches_oracle(fmm, orc, level, bar, nsrc):
    """Levels 0 to 10, the finest (1M boxes) with ~1 source per box."""
    rng = np.random.default_rng(40 + level)
    xy, c = workloads.uniform_particles(nsrc, rng)
    z = rng.random(3000) + 1j * rng.random(3000)
    _check(_p2p(fmm, level, xy, c, z), orc.p2p_uniform(level, xy, c, z), l2=bar, worst=max(1e-4, 2 * bar))


@pytest.mark.parametrize("level,nsrc", [(3, 4000), (8, 262144)])
def test_p2p_shared_sm_grid_gives_the_same_result(fmm, orc, level, nsrc):
    """FMM_P2P_SHARE_SM only shrinks the persistent grid: on the same binning (the binning's
    order within a box is not fixed) every claim is summed the same way by whichever CTA
    takes it, so the result is bit-identical, and on the oracle's bar."""
    import torch

    rng = np.random.default_rng(60 + level)
    xy, c = workloads.uniform_particles(nsrc, rng)
    z = rng.random(3000) + 1j * rng.random(3000)
    xyd, cd = torch.from_numpy(xy).cuda(), torch.from_numpy(c).cuda()
    zd = torch.from_numpy(np.stack([z.real, z.imag], 1).copy()).cuda()
    sp, ss = _bins(fmm, level, xyd)
    tp, ts = _bins(fmm, level, zd)
    out = []
    for share in (False, True):
        phi = torch.zeros(len(z), dtype=torch.complex64, device="cuda")
        fmm.fmm_p2p(level, xyd, cd, sp, ss, zd, tp, ts, phi, share_sm=share)
        fmm.fmm_sync_status()
        out.append(phi.cpu())
    assert torch.equal(out[0], out[1])
    _check(out[1].numpy().astype(np.complex128), orc.p2p_uniform(level, xy, c, z))


def test_p2p_points_on_box_boundaries_and_outside(fmm, orc):
    """Sources on the level's box boundaries, targets one ulp either side of them, and
    points at 1.0 and just outside the unit square (clamped to the edge boxes)."""
    rng = np.random.default_rng(44)
    level, side = 3, 8
    xy, c = workloads.uniform_particles(3000, rng)
    k = np.arange(side + 1) / side
    xy[:side + 1, 0] = k
    xy[side + 1:2 * side + 2, 1] = k
    xy[-4:] = [[1.0, 0.3], [1.004, 0.6], [-0.003, 0.2], [0.7, 1.002]]
    zx = np.concatenate([np.nextafter(k, -1.0), np.nextafter(k, 2.0), rng.random(300), [1.0, 1.006, -0.002]])
    zy = rng.random(len(zx))
    _check(_p2p(fmm, level, xy, c, zx + 1j * zy), orc.p2p_uniform(level, xy, c, zx + 1j * zy))


def test_p2p_targets_on_sources_skip_themselves(fmm, orc):
    xy, c = workloads.uniform_particles(5000, np.random.default_rng(3))
    z = xy[:, 0] + 1j * xy[:, 1]
    _check(_p2p(fmm, 4, xy, c, z), orc.p2p_uniform(4, xy, c, z))


def test_p2p_clustered_sources_span_several_batches(fmm, orc):
    """Gaussian-mixture sources: boxes near the means hold thousands of points, so the
    3 x 3 neighbourhood is staged in several shared-memory batches (the coarse regime of
    the module's bars: 2e-4)."""
    xy, c = workloads.gmm_particles(30000, np.random.default_rng(8), ncomp=3)
    rng = np.random.default_rng(9)
    z = np.concatenate([rng.random(1500) + 1j * rng.random(1500), xy[:1500, 0] + 1j * xy[:1500, 1]])
    _check(_p2p(fmm, 4, xy, c, z), orc.p2p_uniform(4, xy, c, z), l2=2e-4, worst=4e-4)


def test_p2p_accumulate_and_ragged_counts(fmm, orc):
    rng = np.random.default_rng(12)
    xy, c = workloads.uniform_particles(3000, rng)
    for m in (1, 255, 257):
        z = rng.random(m) + 1j * rng.random(m)
        ref = orc.p2p_uniform(3, xy, c, z)
        base = 0.5 - 0.25j + np.zeros(m)
        _check(_p2p(fmm, 3, xy, c, z, phi0=base), ref + base)


@pytest.mark.parametrize("level,n", [(4, 8192), (5, 20000)])
def test_whole_fmm_on_device_matches_direct_sum(fmm, orc, level, n):
    """P2M, M2M, M2L, L2L, L2P and P2P, all library kernels, at the points themselves."""
    import torch
    from paper_1009_3457_gb300.farfield import FmmPotential

    xy, c = workloads.uniform_particles(n, np.random.default_rng(60 + level))
    tree = fmm.fmm_build_lists(xy, max_level=level)
    xyd = torch.from_numpy(xy).cuda()
    pot = FmmPotential(tree, 16, xyd, torch.from_numpy(c).cuda(), xyd)
    got = pot().cpu().numpy().astype(np.complex128)
    fmm.fmm_sync_status()
    pick = np.random.default_rng(1).choice(n, 400, replace=False)
    ref = orc.p2p_uniform(0, xy, c, xy[pick, 0] + 1j * xy[pick, 1])  # level 0: every other point
    assert np.linalg.norm(got[pick] - ref) / np.linalg.norm(ref) <= 2e-5
    # re-runnable: every buffer is rewritten (P2M sums with FP32 atomics, so runs agree to rounding)
    again = pot().cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(again - got) / np.linalg.norm(got) <= 1e-6


def test_whole_fmm_full_size_sampled(fmm, orc):
    """2^22 uniform points, uniform tree to level 8, p = 16 (the M2L benchmark's tree): the
    potential at 120 sampled points against the direct sum over all other points."""
    import torch
    from paper_1009_3457_gb300.farfield import FmmPotential

    n = 1 << 22
    xy, c = workloads.uniform_particles(n, np.random.default_rng(77))
    tree = fmm.fmm_build_lists(xy, max_level=8)
    xyd = torch.from_numpy(xy).cuda()
    got = FmmPotential(tree, 16, xyd, torch.from_numpy(c).cuda(), xyd)().cpu().numpy().astype(np.complex128)
    fmm.fmm_sync_status()
    pick = np.random.default_rng(2).choice(n, 120, replace=False)
    ref = orc.p2p_uniform(0, xy, c, xy[pick, 0] + 1j * xy[pick, 1])  # level 0: every other point
    assert np.linalg.norm(got[pick] - ref) / np.linalg.norm(ref) <= 2e-5


@pytest.mark.parametrize("p", [8, 16, 24])
def test_p2m_binned_matches_oracle_and_repeats_exactly(fmm, orc, p):
    """fmm_p2m_binned (one block per box, no atomics) against the oracle's P2M in
    radius-scaled units, on uniform and clustered points; two runs are bit-identical."""
    import torch

    for xy, c, level in (workloads.uniform_particles(20000, np.random.default_rng(31)) + (5,),
                         workloads.gmm_particles(20000, np.random.default_rng(32), ncomp=3) + (6,)):
        xyd, cd = torch.from_numpy(xy).cuda(), torch.from_numpy(c).cuda()
        perm, start = _bins(fmm, level, xyd)
        M = torch.empty((4 ** level, p), dtype=torch.complex64, device="cuda")
        fmm.fmm_p2m_binned(level, p, xyd, cd, perm, start, M)
        fmm.fmm_sync_status()
        got = M.cpu().numpy().astype(np.complex128)
        ref = orc.scale_me(orc.p2m_uniform(level, p, xy, c), level)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
        again = M.clone()
        fmm.fmm_p2m_binned(level, p, xyd, cd, perm, start, M)
        assert torch.equal(again, M)
