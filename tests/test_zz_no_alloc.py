"""fgt_h2t_noalloc: the allocation-free Hermite-to-Taylor entry point.

Some callers cannot allocate device memory: an application whose caching
allocator or fixed pool owns the whole device, a plugin that may not allocate
behind its host's back, or a latency-critical loop that cannot afford the
device-wide synchronisation an allocation may cause.  fgt_h2t_noalloc keeps its
intermediate in a fixed array compiled into the library instead of a buffer
from cudaMalloc.

This test calls it through the C ABI twice in a row, on two different grids,
and checks each result against the FP64 oracle (sampled target boxes, relative
L2 <= 1e-5, the FP32 bar of the other FGT tests) and against the allocating
entry point fgt_h2t; then it checks the accumulate flag (C0 + H2T(A)) and that
a grid too large for the built-in array is refused.

The file is named so that pytest collects it last; it passes both alone in a
fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL_L2 = 1e-5


@pytest.fixture(scope="module")
def fmm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_3457_gb300 import build, fmmgb

    build.build()
    fmmgb.load()
    return fmmgb


def _hermite_inputs(orc, sigma, p):
    """FP64 oracle P2H of a seeded Gaussian-mixture draw, and sampled target boxes."""
    x, q = workloads.gmm_particles(30000, np.random.default_rng(int(sigma * 1000) + p))
    g = workloads.fgt_grid_log2(sigma)
    A = orc.fgt_p2h_grid(g, p, sigma, x, q)
    n = 1 << g
    rng = np.random.default_rng(p)
    tg = np.unique(np.concatenate([[0, n - 1, n * (n - 1), n * n - 1], rng.integers(0, n * n, 36)]))
    return g, A, tg


def _rel(got, ref):
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_noalloc_matches_oracle_and_allocating_entry_point_twice(fmm, orc):
    import torch

    ncut = workloads.FGT_NCUT
    for sigma, p in [(0.05, 16), (0.1, 12)]:  # 32 x 32 boxes at p = 16 fills the built-in array exactly
        g, A, tg = _hermite_inputs(orc, sigma, p)
        ref = orc.fgt_h2t_targets(g, ncut, p, sigma, A, tg)
        Ad = torch.from_numpy(A.astype(np.float32)).cuda()
        C_ref = torch.empty_like(Ad)
        C_new = torch.full_like(Ad, float("nan"))
        fmm.fgt_h2t(g, ncut, p, sigma, Ad, C_ref)
        fmm.fgt_h2t_noalloc(g, ncut, p, sigma, Ad, C_new)
        torch.cuda.synchronize()
        got = C_new.double().cpu().numpy()
        assert np.isfinite(got).all()
        err_oracle = _rel(got[tg], ref)
        assert err_oracle <= TOL_L2, (sigma, p, err_oracle)
        err_alloc = _rel(got, C_ref.double().cpu().numpy())
        assert err_alloc <= TOL_L2, (sigma, p, err_alloc)
    fmm.fmm_sync_status()


def test_noalloc_accumulates(fmm, orc):
    import torch

    sigma, p, ncut = 0.1, 8, workloads.FGT_NCUT
    g, A, tg = _hermite_inputs(orc, sigma, p)
    ref = orc.fgt_h2t_targets(g, ncut, p, sigma, A, tg)
    C0 = (np.random.default_rng(1).standard_normal(A.shape) * 0.25 * np.abs(ref).max()).astype(np.float32)
    Ad = torch.from_numpy(A.astype(np.float32)).cuda()
    Cd = torch.from_numpy(C0).cuda()
    fmm.fgt_h2t_noalloc(g, ncut, p, sigma, Ad, Cd, accumulate=True)
    got = Cd.double().cpu().numpy()[tg] - C0.astype(np.float64)[tg]
    # the accumulated sum carries FP32 rounding of |C0| ~ max|ref|
    err = _rel(got, ref)
    assert err <= 1e-5, err
    fmm.fmm_sync_status()


def test_noalloc_rejects_grids_beyond_its_scratch(fmm):
    import torch

    A = torch.zeros((4 ** 6, 16, 16), dtype=torch.float32, device="cuda")
    C = torch.empty_like(A)
    with pytest.raises(fmm.FmmError) as e:
        fmm.fgt_h2t_noalloc(6, 10, 16, 0.02, A, C)
    assert e.value.code == fmm.FMM_EINVAL
    assert "scratch" in str(e.value)
