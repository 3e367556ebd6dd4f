"""GPU parity of the FGT Hermite-to-Taylor translation (fgt_h2t) against the FP64 oracle.

Bar: relative L2 error of the Taylor coefficients over all boxes and all
(b1, b2) <= 1e-5 (FP32), and every box's own relative error <= 1e-4.
"""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL_L2 = 1e-5
TOL_BOX = 1e-4


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


def _check(got, ref):
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= TOL_L2, f"relative L2 {err:.3e}"
    nb = got.shape[0]
    box = np.linalg.norm((got - ref).reshape(nb, -1), axis=1) / np.maximum(
        np.linalg.norm(ref.reshape(nb, -1), axis=1), 1e-300)
    assert box.max() <= TOL_BOX, f"worst box {box.max():.3e} at {int(box.argmax())}"
    return err


@pytest.fixture(scope="module")
def gmm_sources():
    return workloads.gmm_particles(20000, np.random.default_rng(55))


@pytest.mark.parametrize("p", [4, 8, 12, 16])
def test_fgt_h2t_small_grid_full(fmm, orc, gmm_sources, p):
    """sigma = 0.2 (g = 3, 8 x 8 boxes, fewer than one 32-box segment: ragged), n_cut = 10."""
    import torch

    x, q = gmm_sources
    sigma, g, ncut = 0.2, workloads.fgt_grid_log2(0.2), workloads.FGT_NCUT
    A = orc.fgt_p2h_grid(g, p, sigma, x, q)
    ref = orc.fgt_h2t_grid(g, ncut, p, sigma, A)
    Ad = _dev(A)
    Cd = torch.empty_like(Ad)
    fmm.fgt_h2t(g, ncut, p, sigma, Ad, Cd)
    _check(Cd.cpu().numpy().astype(np.float64), ref)


@pytest.mark.parametrize("g,ncut", [(0, 0), (1, 3), (2, 1), (6, 2)])
def test_fgt_h2t_edge_sizes(fmm, orc, g, ncut):
    import torch

    rng = np.random.default_rng(g * 10 + ncut)
    p, sigma = 8, 0.5 * 2.0 ** -g
    n = 1 << g
    fact = np.array([math.factorial(a) for a in range(p)], float)
    A = rng.standard_normal((n * n, p, p)) * (0.3 ** (np.arange(p)[:, None] + np.arange(p)[None, :])) / np.outer(fact, fact)
    if n * n <= 64:
        tg = np.arange(n * n)
    else:
        tg = np.unique(np.concatenate([[0, n - 1, n * n - 1, n * (n - 1)], rng.integers(0, n * n, 40)]))
    ref = orc.fgt_h2t_targets(g, ncut, p, sigma, A, tg)
    Ad = _dev(A)
    Cd = torch.empty_like(Ad)
    fmm.fgt_h2t(g, ncut, p, sigma, Ad, Cd)
    _check(Cd.cpu().numpy().astype(np.float64)[tg], ref)


@pytest.mark.parametrize("g,ncut,p", [(9, 10, 8), (10, 3, 4)])
def test_fgt_h2t_large_grids_sampled(fmm, orc, g, ncut, p):
    """Grids of 512 x 512 (n_cut 10, p 8) and 1024 x 1024 boxes (n_cut 3, p 4): the two pass
    kernels over thousands of segments; corners, edges and random interior boxes against the
    oracle."""
    import torch

    rng = np.random.default_rng(500 + g)
    sigma = 0.5 * 2.0 ** -g
    n = 1 << g
    fact = np.array([math.factorial(a) for a in range(p)], float)
    scale = ((0.3 ** (np.arange(p)[:, None] + np.arange(p)[None, :])) / np.outer(fact, fact)).astype(np.float32)
    A = rng.standard_normal((n * n, p, p), dtype=np.float32) * scale
    edges = [0, n - 1, n * n - 1, n * (n - 1), n // 2, n // 2 * n, n // 2 * n + n - 1, n * (n - 1) + n // 2]
    tg = np.unique(np.concatenate([edges, rng.integers(0, n * n, 40)]))
    ref = orc.fgt_h2t_targets(g, ncut, p, sigma, A, tg)
    Ad = _dev(A)
    Cd = torch.empty_like(Ad)
    fmm.fgt_h2t(g, ncut, p, sigma, Ad, Cd)
    fmm.fmm_sync_status()
    _check(Cd.cpu().numpy().astype(np.float64)[tg], ref)


def test_fgt_h2t_accumulate_and_work_buffer(fmm, orc, gmm_sources):
    import torch

    x, q = gmm_sources
    p, sigma = 12, 0.1
    g, ncut = workloads.fgt_grid_log2(sigma), workloads.FGT_NCUT
    A = orc.fgt_p2h_grid(g, p, sigma, x, q)
    n = 1 << g
    tg = np.arange(0, n * n, 7)
    ref = orc.fgt_h2t_targets(g, ncut, p, sigma, A, tg)
    Ad = _dev(A)
    X = np.random.default_rng(0).standard_normal(A.shape).astype(np.float32)
    Cd = _dev(X)
    work = torch.empty_like(Ad)
    fmm.fgt_h2t(g, ncut, p, sigma, Ad, Cd, work=work, accumulate=True)
    got = Cd.cpu().numpy().astype(np.float64)[tg] - X.astype(np.float64)[tg]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-5


@pytest.mark.slow
@pytest.mark.parametrize("sigma", [0.05, 0.1, 0.2])
@pytest.mark.parametrize("p", [8, 12, 16])
def test_fgt_h2t_full_size_workload(fmm, orc, sigma, p):
    """2^20 Gaussian-mixture sources, n_cut = 10: sampled targets (corners, edges, interior)."""
    import torch

    cfg = workloads.CONFIGS["fgt"]
    x, q = workloads.gmm_particles(cfg["n"], workloads.rng_for("fgt"))
    g, ncut = workloads.fgt_grid_log2(sigma), cfg["ncut"]
    A = orc.fgt_p2h_grid(g, p, sigma, x, q)
    Ad = _dev(A)
    Cd = torch.empty_like(Ad)
    fmm.fgt_h2t(g, ncut, p, sigma, Ad, Cd)
    n = 1 << g
    rng = np.random.default_rng(3)
    tg = np.unique(np.concatenate([[0, n - 1, n * n - 1, n * (n - 1), n // 2 * n + n // 2], rng.integers(0, n * n, 12)]))
    ref = orc.fgt_h2t_targets(g, ncut, p, sigma, A, tg)
    _check(Cd.cpu().numpy().astype(np.float64)[tg], ref)


def test_fgt_p2h_on_device(fmm, orc, gmm_sources):
    import torch

    x, q = gmm_sources
    for sigma, p in [(0.1, 8), (0.05, 16)]:
        g = workloads.fgt_grid_log2(sigma)
        ref = orc.fgt_p2h_grid(g, p, sigma, x, q)
        Ad = torch.empty((4 ** g, p, p), dtype=torch.float32, device="cuda")
        fmm.fgt_p2h(g, p, sigma, torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), Ad)
        got = Ad.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


@pytest.mark.parametrize("p", [4, 8, 12, 16])
def test_fgt_t2p_matches_oracle(fmm, orc, p):
    """fgt_t2p (Eq. taylor at each target's box) against the oracle's evaluation."""
    import torch

    rng = np.random.default_rng(70 + p)
    g = 4
    C = rng.standard_normal((4 ** g, p, p)) / (1.0 + np.add.outer(np.arange(p), np.arange(p)))[None]
    y = rng.random((3000, 2))
    # on and next to box boundaries, at the ends of [0, 1) and just outside it (the nearest box)
    k = np.arange(17) / 16
    edge = np.concatenate([k, np.nextafter(k, -1.0), np.nextafter(k, 2.0), [1 - 2.0 ** -53, 1.01, -0.01, 0.0]])
    y[:len(edge), 0] = edge
    y[len(edge):2 * len(edge), 1] = edge
    G = torch.empty(3000, dtype=torch.float32, device="cuda")
    fmm.fgt_t2p(g, p, 0.1, _dev(C), torch.from_numpy(y).cuda(), G)
    fmm.fmm_sync_status()
    ref = orc.fgt_taylor_eval_grid(g, p, 0.1, C, y)
    got = G.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-6


@pytest.mark.parametrize("p", [4, 8, 12, 16])
def test_fgt_t2p_binned_matches_oracle_and_per_target_kernel(fmm, orc, p):
    """fgt_t2p_binned (targets binned by fgt_bin_points, one block per box) against the
    oracle's evaluation and fgt_t2p, with targets on and next to box boundaries and just
    outside the unit square; accumulate."""
    import torch

    rng = np.random.default_rng(80 + p)
    g, n = 4, 3000
    C = rng.standard_normal((4 ** g, p, p)) / (1.0 + np.add.outer(np.arange(p), np.arange(p)))[None]
    y = rng.random((n, 2))
    k = np.arange(17) / 16
    edge = np.concatenate([k, np.nextafter(k, -1.0), np.nextafter(k, 2.0), [1 - 2.0 ** -53, 1.01, -0.01, 0.0]])
    y[:len(edge), 0] = edge
    y[len(edge):2 * len(edge), 1] = edge
    yd = torch.from_numpy(y).cuda()
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    start = torch.empty(4 ** g + 1, dtype=torch.int32, device="cuda")
    fmm.fgt_bin_points(g, yd, perm, start, torch.empty(4 ** g, dtype=torch.int32, device="cuda"))
    G = torch.empty(n, dtype=torch.float32, device="cuda")
    Cd = _dev(C)
    fmm.fgt_t2p_binned(g, p, 0.1, Cd, yd, perm, start, G)
    fmm.fmm_sync_status()
    ref = orc.fgt_taylor_eval_grid(g, p, 0.1, C, y)
    got = G.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-6
    G2 = torch.empty_like(G)
    fmm.fgt_t2p(g, p, 0.1, Cd, yd, G2)
    fmm.fmm_sync_status()
    assert np.linalg.norm(got - G2.cpu().numpy()) / np.linalg.norm(ref) <= 1e-6
    fmm.fgt_t2p_binned(g, p, 0.1, Cd, yd, perm, start, G, accumulate=True)
    fmm.fmm_sync_status()
    assert np.linalg.norm(G.cpu().numpy() - 2 * ref) / np.linalg.norm(2 * ref) <= 1e-6


@pytest.mark.parametrize("sigma,p", [(0.1, 8), (0.05, 12), (0.2, 16)])
def test_fgt_whole_transform_on_device(fmm, orc, sigma, p):
    """fgt_p2h -> fgt_h2t -> fgt_t2p on the device against the oracle's pipeline
    (FP32 bar 1e-5) and against the direct Gauss sum (truncation and cutoff)."""
    import torch

    rng = np.random.default_rng(int(sigma * 1000) + p)
    x, q = workloads.gmm_particles(20000, rng)
    y = rng.random((2000, 2))
    g = workloads.fgt_grid_log2(sigma)
    A = torch.empty((4 ** g, p, p), dtype=torch.float32, device="cuda")
    Cd = torch.empty_like(A)
    G = torch.empty(2000, dtype=torch.float32, device="cuda")
    fmm.fgt_p2h(g, p, sigma, torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), A)
    fmm.fgt_h2t(g, workloads.FGT_NCUT, p, sigma, A, Cd)
    fmm.fgt_t2p(g, p, sigma, Cd, torch.from_numpy(y).cuda(), G)
    fmm.fmm_sync_status()
    got = G.cpu().numpy().astype(np.float64)
    Ao = orc.fgt_p2h_grid(g, p, sigma, x, q)
    ref = orc.fgt_taylor_eval_grid(g, p, sigma, orc.fgt_h2t_grid(g, workloads.FGT_NCUT, p, sigma, Ao), y)
    direct = orc.fgt_direct(x, q, sigma, y)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    assert np.linalg.norm(got - direct) / np.linalg.norm(direct) <= 1e-5
