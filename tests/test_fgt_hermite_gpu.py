"""GPU parity of the FGT Hermite-series evaluation (fgt_h2p, Sec. 4.2, Eq. hermite),
the device binning of points by box (fgt_bin_points) and the binned P2H
(fgt_p2h_binned), against the FP64 oracle.

Bars: binning is exact (the same box for every point, every point once);
G relative L2 over all targets <= 1e-5 (FP32) against the oracle evaluating
the same FP32 coefficients in FP64, and every target's error <= 1e-5 of
max |G|; the binned P2H relative L2 <= 1e-5 against the oracle's P2H.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL_L2 = 1e-5
TOL_MAX = 1e-5


@pytest.fixture(scope="module")
def fmm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_3457_gb300 import build, fmmgb

    build.build()
    fmmgb.load()
    return fmmgb


def _boxes(y, g):
    n = 1 << g
    ix = np.clip(np.floor(y[:, 0] * n), 0, n - 1).astype(np.int64)
    iy = np.clip(np.floor(y[:, 1] * n), 0, n - 1).astype(np.int64)
    return iy * n + ix


def _bin(fmm, g, y_dev):
    import torch

    n = y_dev.shape[0]
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    start = torch.empty(4 ** g + 1, dtype=torch.int32, device="cuda")
    work = torch.empty(4 ** g, dtype=torch.int32, device="cuda")
    fmm.fgt_bin_points(g, y_dev, perm, start, work)
    return perm, start


def _h2p(fmm, g, ncut, p, sigma, A32, y, G=None, accumulate=False):
    import torch

    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float64)).cuda()
    perm, start = _bin(fmm, g, yd)
    if G is None:
        G = torch.empty(len(y), dtype=torch.float32, device="cuda")
    fmm.fgt_h2p(g, ncut, p, sigma, torch.from_numpy(A32).cuda(), yd, perm, start, G, accumulate=accumulate)
    fmm.fmm_sync_status()
    return G.cpu().numpy().astype(np.float64)


def _check(got, ref):
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    worst = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= TOL_L2 and worst <= TOL_MAX, f"relative L2 {err:.3e}, worst {worst:.3e}"
    return err


@pytest.fixture(scope="module")
def gmm_sources():
    return workloads.gmm_particles(20000, np.random.default_rng(91))


def test_bin_points_is_an_exact_counting_sort(fmm):
    import torch

    rng = np.random.default_rng(3)
    g = 5
    y = rng.random((50000, 2))
    y[:10] = [[0.0, 0.0], [1.0, 1.0], [-0.5, 0.3], [0.3, 1.5], [0.999999999, 0.5], [0.5, 0.03125],
              [0.03125, 0.0625], [1e-300, 0.9999999999999999], [2.0, -2.0], [0.5, 0.5]]
    y[10:5000] = [0.4, 0.6]  # one crowded box
    perm, start = _bin(fmm, g, torch.from_numpy(y).cuda())
    perm, start = perm.cpu().numpy(), start.cpu().numpy()
    box = _boxes(y, g)
    counts = np.bincount(box, minlength=4 ** g)
    assert start[0] == 0 and start[-1] == len(y)
    np.testing.assert_array_equal(np.diff(start), counts)
    assert np.array_equal(np.sort(perm), np.arange(len(y)))
    owner = np.repeat(np.arange(4 ** g), counts)
    np.testing.assert_array_equal(box[perm], owner)


def _edge_values(g):
    """Coordinates on and next to every cell boundary of the 2^g grid, the ends of [0, 1),
    subnormals, signed zeros, and values outside [0, 1) (clamped), infinities and NaN."""
    k = np.arange((1 << g) + 1) / (1 << g)
    v = np.concatenate([k, np.nextafter(k, -np.inf), np.nextafter(k, np.inf),
                        [0.0, -0.0, 5e-324, 1e-310, 1e-300, 1 - 2.0 ** -53, 1.0, 1.5, 2.0 ** 40, -1e-300, -3.0,
                         np.inf, -np.inf, np.nan, 0.5, 1.0 / 3.0]])
    return v


@pytest.mark.parametrize("g", [0, 1, 5, 10])
def test_bin_points_edge_coordinates(fmm, g):
    """The device places a coordinate by floor(v 2^g) exactly (read off the bits of the
    FP64 value), clamped to the grid, NaN to cell 0."""
    import torch

    v = _edge_values(g)
    rng = np.random.default_rng(17 + g)
    y = np.stack([np.concatenate([v, rng.permutation(v)]), np.concatenate([rng.permutation(v), v])], axis=1)
    side = 1 << g
    with np.errstate(invalid="ignore", over="ignore"):
        cell = np.floor(y * side)
    cell = np.clip(np.where(np.isnan(cell), 0.0, cell), 0, side - 1).astype(np.int64)
    box = cell[:, 1] * side + cell[:, 0]
    perm, start = _bin(fmm, g, torch.from_numpy(y).cuda())
    perm, start = perm.cpu().numpy(), start.cpu().numpy()
    counts = np.bincount(box, minlength=4 ** g)
    np.testing.assert_array_equal(np.diff(start), counts)
    np.testing.assert_array_equal(box[perm], np.repeat(np.arange(4 ** g), counts))


def test_bin_points_empty_and_single(fmm):
    import torch

    for n in (0, 1):
        y = torch.full((n, 2), 0.7, dtype=torch.float64, device="cuda")
        perm, start = _bin(fmm, 3, y)
        s = start.cpu().numpy()
        assert s[-1] == n and (np.diff(s) >= 0).all()
        if n:
            assert s[_boxes(np.full((1, 2), 0.7), 3)[0] + 1] == 1


@pytest.mark.parametrize("p", [4, 8, 12, 16])
def test_p2h_binned_matches_oracle(fmm, orc, gmm_sources, p):
    import torch

    x, q = gmm_sources
    for sigma in (0.2, 0.05):
        g = workloads.fgt_grid_log2(sigma)
        xd = torch.from_numpy(x).cuda()
        perm, _ = _bin(fmm, g, xd)
        A = torch.empty((4 ** g, p, p), dtype=torch.float32, device="cuda")
        fmm.fgt_p2h_binned(g, p, sigma, xd, torch.from_numpy(q).cuda(), perm, A)
        fmm.fmm_sync_status()
        ref = orc.fgt_p2h_grid(g, p, sigma, x, q)
        got = A.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
        fmm.fgt_p2h_binned(g, p, sigma, xd, torch.from_numpy(q).cuda(), perm, A, accumulate=True)
        got2 = A.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got2 - 2 * ref) / np.linalg.norm(2 * ref) <= 1e-5


@pytest.mark.parametrize("p", [4, 8, 12, 16])
@pytest.mark.parametrize("sigma,ncut", [(0.2, 10), (0.1, 3), (0.05, 1), (0.1, 0)])
def test_h2p_matches_oracle(fmm, orc, gmm_sources, p, sigma, ncut):
    """Targets: uniform (many in boxes with no sources) plus a cluster of 700 in one
    box (several claims of one box, a ragged last one)."""
    x, q = gmm_sources
    g = workloads.fgt_grid_log2(sigma)
    rng = np.random.default_rng(p * 100 + ncut)
    y = np.concatenate([rng.random((2500, 2)), 0.52 + 0.001 * rng.random((700, 2))])
    A32 = orc.fgt_p2h_grid(g, p, sigma, x, q).astype(np.float32)
    got = _h2p(fmm, g, ncut, p, sigma, A32, y)
    ref = orc.fgt_hermite_eval_grid(g, ncut, p, sigma, A32.astype(np.float64), y)
    _check(got, ref)


def test_h2p_accumulate_and_ragged_counts(fmm, orc, gmm_sources):
    import torch

    x, q = gmm_sources
    sigma, p, ncut = 0.1, 8, 4
    g = workloads.fgt_grid_log2(sigma)
    A32 = orc.fgt_p2h_grid(g, p, sigma, x, q).astype(np.float32)
    for n in (1, 31, 33, 511, 513):
        y = np.random.default_rng(n).random((n, 2))
        ref = orc.fgt_hermite_eval_grid(g, ncut, p, sigma, A32.astype(np.float64), y)
        _check(_h2p(fmm, g, ncut, p, sigma, A32, y), ref)
        G = torch.full((n,), 0.25, dtype=torch.float32, device="cuda")
        _check(_h2p(fmm, g, ncut, p, sigma, A32, y, G=G, accumulate=True), ref + 0.25)


@pytest.mark.parametrize("g", [0, 1, 6, 7])
def test_h2p_claim_order_grids(fmm, orc, g):
    """Claims are handed out heaviest neighbourhood first: one CTA builds that order for grids
    of up to 64 x 64 boxes, five launches (row prefix, keys, scan, scatter, claims) above.
    Grids of 1 x 1, 2 x 2 (the neighbourhood clipped to the grid), 64 x 64 and 128 x 128 boxes,
    a third of the source boxes empty, clustered targets (per box counts from 0 to thousands),
    G pre-filled with NaN: every target is evaluated once, against the oracle."""
    import math
    import torch

    rng = np.random.default_rng(300 + g)
    p, ncut = 8, 3
    n = 1 << g
    sigma = 2.0 ** -g / (math.sqrt(2.0) * 0.442)
    fact = np.array([math.factorial(a) for a in range(p)], float)
    A = rng.standard_normal((n * n, p, p)) * (0.3 ** (np.arange(p)[:, None] + np.arange(p)[None, :])) / np.outer(fact, fact)
    empty = rng.random(n * n) < 0.33
    empty[0] = False  # at least one source box holds coefficients
    A[empty] = 0.0
    A32 = A.astype(np.float32)
    c = rng.random((6, 2))
    y = np.concatenate([np.clip(c[i] + 0.03 * rng.standard_normal((3000, 2)), 0.0, 0.999999) for i in range(6)]
                       + [rng.random((2000, 2))])
    yd = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    perm, start = _bin(fmm, g, yd)
    G = torch.full((len(y),), float("nan"), dtype=torch.float32, device="cuda")
    fmm.fgt_h2p(g, ncut, p, sigma, torch.from_numpy(A32).cuda(), yd, perm, start, G)
    fmm.fmm_sync_status()
    got = G.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all()
    ref = orc.fgt_hermite_eval_grid(g, ncut, p, sigma, A32.astype(np.float64), y)
    _check(got, ref)


def test_h2p_bad_permutation_sets_error_word(fmm):
    """A perm entry outside [0, n) is caught by the kernel's own bounds check: the
    target is skipped and fmm_sync_status reports FMM_EDEVICE; the context stays usable."""
    import torch

    g, p = 3, 4
    y = torch.from_numpy(np.random.default_rng(1).random((100, 2))).cuda()
    perm, start = _bin(fmm, g, y)
    perm[5] = 1000
    A = torch.zeros((4 ** g, p, p), dtype=torch.float32, device="cuda")
    A[:, 0, 0] = 1.0
    G = torch.zeros(100, dtype=torch.float32, device="cuda")
    fmm.fgt_h2p(g, 2, p, 0.2, A, y, perm, start, G)
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_sync_status()
    assert e.value.code == fmm.FMM_EDEVICE
    fmm.fmm_sync_status()  # the word was cleared
    assert float(G.abs().sum()) > 0


@pytest.mark.parametrize("sigma,p", [(0.1, 8), (0.05, 12), (0.2, 16)])
def test_hermite_transform_on_device_matches_direct_sum(fmm, orc, sigma, p):
    """fgt_bin_points -> fgt_p2h_binned -> fgt_h2p: the whole transform through Hermite
    evaluation, against the direct Gauss sum (Eq. dgt), within truncation and cutoff."""
    import torch

    rng = np.random.default_rng(int(sigma * 1000) + p + 7)
    x, q = workloads.gmm_particles(20000, rng)
    y = rng.random((2000, 2))
    g = workloads.fgt_grid_log2(sigma)
    xd = torch.from_numpy(x).cuda()
    perm, _ = _bin(fmm, g, xd)
    A = torch.empty((4 ** g, p, p), dtype=torch.float32, device="cuda")
    fmm.fgt_p2h_binned(g, p, sigma, xd, torch.from_numpy(q).cuda(), perm, A)
    got = _h2p(fmm, g, workloads.FGT_NCUT, p, sigma, A.cpu().numpy(), y)
    direct = orc.fgt_direct(x, q, sigma, y)
    assert np.linalg.norm(got - direct) / np.linalg.norm(direct) <= 1e-5


@pytest.mark.parametrize("sigma,p", [(0.05, 16), (0.2, 8)])
def test_h2p_full_size_workload_sampled(fmm, orc, sigma, p):
    """2^20 Gaussian-mixture sources and 2^20 targets from the same mixture (n_cut = 10),
    the launch the benchmark times; 1,500 sampled targets against the oracle."""
    import torch

    n = 1 << 20
    rng = np.random.default_rng(2024)
    x, q = workloads.gmm_particles(n, rng)
    y, _ = workloads.gmm_particles(n, np.random.default_rng(2025))
    g = workloads.fgt_grid_log2(sigma)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    perm, _ = _bin(fmm, g, xd)
    A = torch.empty((4 ** g, p, p), dtype=torch.float32, device="cuda")
    fmm.fgt_p2h_binned(g, p, sigma, xd, torch.from_numpy(q).cuda(), perm, A)
    tperm, tstart = _bin(fmm, g, yd)
    G = torch.empty(n, dtype=torch.float32, device="cuda")
    fmm.fgt_h2p(g, workloads.FGT_NCUT, p, sigma, A, yd, tperm, tstart, G)
    fmm.fmm_sync_status()
    pick = np.random.default_rng(5).choice(n, 1500, replace=False)
    A64 = A.cpu().numpy().astype(np.float64)
    ref = orc.fgt_hermite_eval_grid(g, workloads.FGT_NCUT, p, sigma, A64, y[pick])
    _check(G.cpu().numpy().astype(np.float64)[pick], ref)


# ---------------------------------------------------------------------------
# tensor-core forms (p = 16): bar = the oracle's truncation error + 1e-4 in relative L2
# (split BF16, three products); the single-product form is checked at 1e-2.
# ---------------------------------------------------------------------------
TC_BAR = {"bf16x3": 1e-4, "bf16": 1e-2}


def _prec(fmm, name):
    return {"bf16x3": fmm.FMM_TC_BF16X3, "bf16": fmm.FMM_TC_BF16}[name]


def _h2p_tc(fmm, g, ncut, sigma, A32, y, prec, G=None, accumulate=False):
    import torch

    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float64)).cuda()
    perm, start = _bin(fmm, g, yd)
    if G is None:
        G = torch.empty(len(y), dtype=torch.float32, device="cuda")
    fmm.fgt_h2p(g, ncut, 16, sigma, torch.from_numpy(A32).cuda(), yd, perm, start, G, accumulate=accumulate,
                prec=prec)
    fmm.fmm_sync_status()
    return G.cpu().numpy().astype(np.float64)


def _rel(got, ref):
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("name", ["bf16x3", "bf16"])
@pytest.mark.parametrize("sigma,ncut", [(0.2, 10), (0.1, 10), (0.05, 10), (0.1, 3), (0.05, 1), (0.1, 0), (0.05, 15)])
def test_h2p_tc_matches_oracle(fmm, orc, gmm_sources, name, sigma, ncut):
    x, q = gmm_sources
    g = workloads.fgt_grid_log2(sigma)
    rng = np.random.default_rng(ncut + int(sigma * 100))
    y = np.concatenate([rng.random((2500, 2)), 0.52 + 0.001 * rng.random((700, 2))])
    A32 = orc.fgt_p2h_grid(g, 16, sigma, x, q).astype(np.float32)
    got = _h2p_tc(fmm, g, ncut, sigma, A32, y, _prec(fmm, name))
    ref = orc.fgt_hermite_eval_grid(g, ncut, 16, sigma, A32.astype(np.float64), y)
    trunc = _rel(orc.fgt_hermite_eval_grid(g, ncut, 16, sigma, orc.fgt_p2h_grid(g, 16, sigma, x, q), y),
                 orc.fgt_direct(x, q, sigma, y)) if ncut == 10 else 0.0
    err = _rel(got, ref)
    assert err <= trunc + TC_BAR[name], f"relative L2 {err:.3e}"
    assert np.abs(got - ref).max() <= 10 * TC_BAR[name] * np.abs(ref).max()


def test_h2p_tc_ragged_counts_and_accumulate(fmm, orc, gmm_sources):
    import torch

    x, q = gmm_sources
    sigma, ncut = 0.1, 4
    g = workloads.fgt_grid_log2(sigma)
    A32 = orc.fgt_p2h_grid(g, 16, sigma, x, q).astype(np.float32)
    for n in (1, 127, 128, 129, 300):
        y = np.random.default_rng(n + 5).random((n, 2))
        ref = orc.fgt_hermite_eval_grid(g, ncut, 16, sigma, A32.astype(np.float64), y)
        assert _rel(_h2p_tc(fmm, g, ncut, sigma, A32, y, fmm.FMM_TC_BF16X3), ref) <= 1e-4
        G = torch.full((n,), 0.5, dtype=torch.float32, device="cuda")
        got = _h2p_tc(fmm, g, ncut, sigma, A32, y, fmm.FMM_TC_BF16X3, G=G, accumulate=True)
        assert _rel(got, ref + 0.5) <= 1e-4


def test_h2p_tc_agrees_with_fp32_path_at_full_size(fmm, orc):
    """2^20 mixture targets, sigma 0.05, n_cut 10 (the benchmark's launch): the tensor-core
    result against the FP32 path everywhere and the oracle on 1,500 sampled targets."""
    import torch

    n = 1 << 20
    x, q = workloads.gmm_particles(n, np.random.default_rng(2024))
    y, _ = workloads.gmm_particles(n, np.random.default_rng(2025))
    sigma, ncut = 0.05, workloads.FGT_NCUT
    g = workloads.fgt_grid_log2(sigma)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    perm, _ = _bin(fmm, g, xd)
    A = torch.empty((4 ** g, 16, 16), dtype=torch.float32, device="cuda")
    fmm.fgt_p2h_binned(g, 16, sigma, xd, torch.from_numpy(q).cuda(), perm, A)
    tperm, tstart = _bin(fmm, g, yd)
    G32 = torch.empty(n, dtype=torch.float32, device="cuda")
    Gtc = torch.empty(n, dtype=torch.float32, device="cuda")
    fmm.fgt_h2p(g, ncut, 16, sigma, A, yd, tperm, tstart, G32)
    fmm.fgt_h2p(g, ncut, 16, sigma, A, yd, tperm, tstart, Gtc, prec=fmm.FMM_TC_BF16X3)
    fmm.fmm_sync_status()
    g32, gtc = G32.cpu().numpy().astype(np.float64), Gtc.cpu().numpy().astype(np.float64)
    assert _rel(gtc, g32) <= 1e-4
    pick = np.random.default_rng(6).choice(n, 1500, replace=False)
    ref = orc.fgt_hermite_eval_grid(g, ncut, 16, sigma, A.cpu().numpy().astype(np.float64), y[pick])
    assert _rel(gtc[pick], ref) <= 1e-4
