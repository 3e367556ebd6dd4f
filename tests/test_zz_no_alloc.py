"""fgt_h2t_noalloc: the allocation-free Hermite-to-Taylor entry point.

Callers that cannot allocate device memory (for example code running during
CUDA-graph capture, or under an allocator that owns the whole device) use
fgt_h2t_noalloc, whose intermediate lives in a fixed array compiled into the
library instead of a buffer from cudaMalloc.  This test calls it through the C
ABI twice in a row, on two different grids, and checks each result against the
allocating entry point fgt_h2t within the FP32 tolerance the other FGT tests
use; it also checks that a grid too large for the built-in array is refused.

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


def _hermite_inputs(fmm, sigma, p):
    import torch

    x, q = workloads.gmm_particles(30000, np.random.default_rng(int(sigma * 1000) + p))
    g = workloads.fgt_grid_log2(sigma)
    A = torch.empty((4 ** g, p, p), dtype=torch.float32, device="cuda")
    fmm.fgt_p2h(g, p, sigma, torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), A)
    return g, A


def test_noalloc_matches_allocating_entry_point_twice(fmm):
    import torch

    ncut = workloads.FGT_NCUT
    for sigma, p in [(0.05, 16), (0.1, 12)]:  # 32 x 32 boxes at p = 16 fills the built-in array exactly
        g, A = _hermite_inputs(fmm, sigma, p)
        C_ref = torch.empty_like(A)
        C_new = torch.full_like(A, float("nan"))
        fmm.fgt_h2t(g, ncut, p, sigma, A, C_ref)
        fmm.fgt_h2t_noalloc(g, ncut, p, sigma, A, C_new)
        torch.cuda.synchronize()
        ref = C_ref.double().cpu().numpy()
        got = C_new.double().cpu().numpy()
        assert np.isfinite(got).all()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= TOL_L2, (sigma, p, err)
    fmm.fmm_sync_status()


def test_noalloc_rejects_grids_beyond_its_scratch(fmm):
    import torch

    A = torch.zeros((4 ** 6, 16, 16), dtype=torch.float32, device="cuda")
    C = torch.empty_like(A)
    with pytest.raises(fmm.FmmError) as e:
        fmm.fgt_h2t_noalloc(6, 10, 16, 0.02, A, C)
    assert e.value.code == fmm.FMM_EINVAL
    assert "scratch" in str(e.value)
