"""GPU parity of the FGT Hermite-to-Taylor translation on the tensor cores
(fgt_h2t with FMM_TC_BF16X3 / FMM_TC_BF16, p = 16) against the FP64 oracle.

Bars (the FP32 path keeps 1e-5): FMM_TC_BF16X3 (BF16 hi/lo split, three
products, FP32 accumulation; two separable passes, each rounding its operands
to ~16 bits) relative L2 of the Taylor coefficients <= 2e-5 and every box's own
relative error <= 1e-4; FMM_TC_BF16 (8 significant bits) relative L2 <= 1e-2.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL_L2_X3, TOL_BOX_X3, TOL_L2_X1 = 2e-5, 1e-4, 1e-2


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

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _errors(got, ref):
    l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    nb = got.shape[0]
    box = np.linalg.norm((got - ref).reshape(nb, -1), axis=1) / np.maximum(
        np.linalg.norm(ref.reshape(nb, -1), axis=1), 1e-300)
    return l2, box.max()


@pytest.fixture(scope="module")
def gmm_sources():
    return workloads.gmm_particles(20000, np.random.default_rng(56))


def _sample(n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n - 1, n * n - 1, n * (n - 1), n // 2 * n + n // 2],
                                     rng.integers(0, n * n, 24)]))


@pytest.mark.parametrize("sigma", [0.05, 0.1, 0.2])
def test_fgt_h2t_tc_bf16x3(fmm, orc, gmm_sources, sigma):
    """n_cut = 10 on the 32 x 32, 16 x 16 and 8 x 8 grids (one segment of 8 boxes per
    line at 8 x 8: the window clipped on both sides); sampled boxes, corners included."""
    import torch

    x, q = gmm_sources
    p, g, ncut = 16, workloads.fgt_grid_log2(sigma), workloads.FGT_NCUT
    A = orc.fgt_p2h_grid(g, p, sigma, x, q)
    n = 1 << g
    tg = np.arange(n * n) if n <= 8 else _sample(n, g)
    ref = orc.fgt_h2t_targets(g, ncut, p, sigma, A, tg)
    Ad = _dev(A)
    Cd = torch.empty_like(Ad)
    fmm.fgt_h2t(g, ncut, p, sigma, Ad, Cd, prec=fmm.FMM_TC_BF16X3)
    fmm.fmm_sync_status()
    l2, box = _errors(Cd.cpu().numpy().astype(np.float64)[tg], ref)
    assert l2 <= TOL_L2_X3 and box <= TOL_BOX_X3, (l2, box)


@pytest.mark.parametrize("g,ncut", [(3, 0), (4, 3), (6, 2), (5, 16), (8, 10)])
def test_fgt_h2t_tc_neighbourhoods_and_grids(fmm, orc, g, ncut):
    """n_cut 0 (one offset: the second MMA issuer has none), 3, 2 on a 64 x 64 grid (several
    segments per CTA and pass), the largest n_cut, 16, and a 256 x 256 grid at n_cut 10 (8,192
    segments per pass over the co-resident CTAs)."""
    import torch
    import math

    rng = np.random.default_rng(100 * g + ncut)
    p, sigma = 16, 0.5 * 2.0 ** -g
    n = 1 << g
    fact = np.array([math.factorial(a) for a in range(p)], float)
    A = rng.standard_normal((n * n, p, p)) * (0.3 ** (np.arange(p)[:, None] + np.arange(p)[None, :])) / np.outer(fact, fact)
    tg = _sample(n, 7 * g + ncut)
    ref = orc.fgt_h2t_targets(g, ncut, p, sigma, A, tg)
    Ad = _dev(A)
    Cd = torch.empty_like(Ad)
    fmm.fgt_h2t(g, ncut, p, sigma, Ad, Cd, prec=fmm.FMM_TC_BF16X3)
    fmm.fmm_sync_status()
    l2, box = _errors(Cd.cpu().numpy().astype(np.float64)[tg], ref)
    assert l2 <= TOL_L2_X3 and box <= TOL_BOX_X3, (l2, box)


def test_fgt_h2t_tc_accumulate_work_buffer_and_single_product(fmm, orc, gmm_sources):
    """FMM_ACCUMULATE into existing values with a caller's work buffer; FMM_TC_BF16
    (one product) at its bar; two calls in a row (the grid barrier's words reset)."""
    import torch

    x, q = gmm_sources
    p, sigma = 16, 0.1
    g, ncut = workloads.fgt_grid_log2(sigma), workloads.FGT_NCUT
    A = orc.fgt_p2h_grid(g, p, sigma, x, q)
    n = 1 << g
    tg = np.arange(0, n * n, 5)
    ref = orc.fgt_h2t_targets(g, ncut, p, sigma, A, tg)
    Ad = _dev(A)
    X = np.random.default_rng(1).standard_normal(A.shape).astype(np.float32) * 0.1
    Cd = _dev(X)
    work = torch.empty_like(Ad)
    fmm.fgt_h2t(g, ncut, p, sigma, Ad, Cd, work=work, accumulate=True, prec=fmm.FMM_TC_BF16X3)
    fmm.fmm_sync_status()
    got = Cd.cpu().numpy().astype(np.float64)[tg] - X.astype(np.float64)[tg]
    l2, _ = _errors(got, ref)
    assert l2 <= TOL_L2_X3, l2
    C1 = torch.empty_like(Ad)
    for _ in range(2):
        fmm.fgt_h2t(g, ncut, p, sigma, Ad, C1, work=work, prec=fmm.FMM_TC_BF16)
    fmm.fmm_sync_status()
    l2, _ = _errors(C1.cpu().numpy().astype(np.float64)[tg], ref)
    assert l2 <= TOL_L2_X1, l2


def test_fgt_h2t_tc_graph_replay(fmm, orc, gmm_sources):
    """The cooperative launch captured in a CUDA graph and replayed."""
    import torch

    x, q = gmm_sources
    p, sigma = 16, 0.05
    g, ncut = workloads.fgt_grid_log2(sigma), workloads.FGT_NCUT
    A = orc.fgt_p2h_grid(g, p, sigma, x, q)
    n = 1 << g
    tg = _sample(n, 11)
    ref = orc.fgt_h2t_targets(g, ncut, p, sigma, A, tg)
    Ad = _dev(A)
    Cd = torch.zeros_like(Ad)
    work = torch.empty_like(Ad)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        fmm.fgt_h2t(g, ncut, p, sigma, Ad, Cd, work=work, prec=fmm.FMM_TC_BF16X3, stream=s)  # warm (image, opt-in)
    torch.cuda.synchronize()
    Cd.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        fmm.fgt_h2t(g, ncut, p, sigma, Ad, Cd, work=work, prec=fmm.FMM_TC_BF16X3, stream=s)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    fmm.fmm_sync_status()
    l2, box = _errors(Cd.cpu().numpy().astype(np.float64)[tg], ref)
    assert l2 <= TOL_L2_X3 and box <= TOL_BOX_X3, (l2, box)
