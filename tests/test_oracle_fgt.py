"""Pins for the FP64 fast-Gauss-transform oracle (Sec. 2.2).

* Hermite functions h_n(t) = exp(-t^2) H_n(t) against numpy's Hermite series
  (a library routine);
* Hermite expansion + evaluation (Eqs. A_alpha, hermite), Taylor expansion +
  evaluation (Eqs. B_beta, taylor) and Hermite-to-Taylor translation +
  evaluation (Eq. C_beta) against the direct Gauss sum (Eq. dgt), with the
  truncation error falling as p grows;
* the single-source case, where the H2T of A = q e_0 must equal the Taylor
  coefficients of that source exactly;
* the separable (Hankel) form that the CUDA path uses, checked in FP64.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import hermite as npherm


def test_hermite_functions_match_numpy(orc):
    for t in [-4.4, -2.0, -0.3, 0.0, 0.7, 1.9, 4.4]:
        h = orc.hermite_functions(32, t)
        for n in range(32):
            e = np.zeros(n + 1)
            e[n] = 1.0
            ref = npherm.hermval(t, e) * math.exp(-t * t)
            assert abs(h[n] - ref) <= 1e-12 * max(1.0, abs(ref)) * (1 + n)


def _cluster(rng, centre, half, n):
    x = centre + (rng.random((n, 2)) * 2 - 1) * half
    q = rng.uniform(-1, 1, n)
    return x, q


def fgt_case():
    """200 sources in one box of the sigma = 0.1 grid, and the generator for the targets."""
    sigma = 0.1
    side = 2.0 ** -4  # box side for sigma = 0.1 (g = 4): side / (sqrt(2) sigma) = 0.442
    rng = np.random.default_rng(21)
    sB = np.array([0.40625, 0.53125])
    x, q = _cluster(rng, sB, side / 2, 200)
    return sigma, side, sB, x, q, rng


@pytest.fixture(scope="module")
def fgt_setup():
    return fgt_case()


def test_hermite_expansion_converges_to_direct(orc, fgt_setup):
    sigma, side, sB, x, q, rng = fgt_setup
    y = rng.random((50, 2)) * 0.6 + 0.2
    G = orc.fgt_direct(x, q, sigma, y)
    errs = []
    for p in (4, 8, 12, 16):
        A = orc.fgt_p2h(x, q, sB, sigma, p)
        errs.append(np.abs(orc.fgt_hermite_eval(A, sB, sigma, y) - G).max() / np.abs(q).sum())
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-12


def test_taylor_expansion_converges_to_direct(orc, fgt_setup):
    sigma, side, sB, x, q, rng = fgt_setup
    tC = sB + np.array([3 * side, -2 * side])
    y = tC + (rng.random((50, 2)) * 2 - 1) * side / 2
    G = orc.fgt_direct(x, q, sigma, y)
    errs = []
    for p in (4, 8, 12, 16):
        B = orc.fgt_p2t(x, q, tC, sigma, p)
        errs.append(np.abs(orc.fgt_taylor_eval(B, tC, sigma, y) - G).max() / np.abs(q).sum())
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-9


@pytest.mark.parametrize("offset", [(1, 0), (3, -2), (-5, 4), (10, 10)])
def test_h2t_then_taylor_converges_to_direct(orc, fgt_setup, offset):
    sigma, side, sB, x, q, rng = fgt_setup
    tC = sB + side * np.array(offset, float)
    y = tC + (rng.random((40, 2)) * 2 - 1) * side / 2
    G = orc.fgt_direct(x, q, sigma, y)
    sc = math.sqrt(2.0) * sigma
    errs = []
    for p in (4, 8, 12, 16):
        A = orc.fgt_p2h(x, q, sB, sigma, p)
        C = orc.fgt_h2t_pair(A, (tC[0] - sB[0]) / sc, (tC[1] - sB[1]) / sc)
        errs.append(np.abs(orc.fgt_taylor_eval(C, tC, sigma, y) - G).max() / np.abs(q).sum())
    assert all(b < a * 1.01 + 1e-15 for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-8


def test_h2t_of_single_source_equals_its_taylor_coefficients(orc):
    sigma, p = 0.05, 10
    sc = math.sqrt(2.0) * sigma
    sB = np.array([0.3, 0.6])
    for off in [(0.02, -0.01), (-0.1, 0.07), (0.0, 0.0)]:
        tC = sB + np.array(off)
        A = np.zeros((p, p))
        A[0, 0] = 0.8
        C = orc.fgt_h2t_pair(A, (tC[0] - sB[0]) / sc, (tC[1] - sB[1]) / sc)
        B = orc.fgt_p2t(sB[None, :], np.array([0.8]), tC, sigma, p)
        np.testing.assert_allclose(C, B, rtol=1e-13, atol=1e-300)


def test_h2t_separable_hankel_form(orc):
    """C = S * (H(u1)^T A H(u2)), H(u)_ab = h_{a+b}(u), S_b1b2 = (-1)^(b1+b2)/(b1! b2!)."""
    rng = np.random.default_rng(4)
    p = 9
    A = rng.standard_normal((p, p))
    u1, u2 = -1.3, 0.4
    h1 = orc.hermite_functions(2 * p - 1, u1)
    h2 = orc.hermite_functions(2 * p - 1, u2)
    H1 = np.array([[h1[a + b] for b in range(p)] for a in range(p)])
    H2 = np.array([[h2[a + b] for b in range(p)] for a in range(p)])
    s = np.array([(-1) ** b / math.factorial(b) for b in range(p)])
    C = np.outer(s, s) * (H1.T @ A @ H2)
    np.testing.assert_allclose(orc.fgt_h2t_pair(A, u1, u2), C, rtol=1e-12, atol=1e-14 * np.abs(C).max())


def test_h2t_grid_is_sum_over_square_neighbourhood(orc):
    rng = np.random.default_rng(8)
    g, ncut, p, sigma = 3, 2, 5, 0.2
    n = 1 << g
    A = rng.standard_normal((n * n, p, p))
    C = orc.fgt_h2t_grid(g, ncut, p, sigma, A)
    sc = math.sqrt(2.0) * sigma
    side = 2.0 ** -g
    for t in [0, 13, 36, 63]:
        tx, ty = t % n, t // n
        acc = np.zeros((p, p))
        for sy in range(n):
            for sx in range(n):
                if max(abs(sx - tx), abs(sy - ty)) <= ncut:
                    acc += orc.fgt_h2t_pair(A[sy * n + sx], (tx - sx) * side / sc, (ty - sy) * side / sc)
        np.testing.assert_allclose(C[t], acc, rtol=1e-12, atol=1e-12 * np.abs(acc).max())
    Ct = orc.fgt_h2t_targets(g, ncut, p, sigma, A, [0, 13, 36, 63])
    np.testing.assert_allclose(Ct, C[[0, 13, 36, 63]], rtol=0, atol=0)


def test_full_fgt_grid_pipeline_matches_direct(orc):
    """P2H on a grid -> H2T over the cutoff neighbourhood -> Taylor evaluation equals Eq. dgt."""
    rng = np.random.default_rng(9)
    sigma = 0.2
    g = 3  # side / (sqrt 2 sigma) = 0.442
    ncut = 10
    p = 14
    x = rng.random((300, 2))
    q = rng.uniform(-1, 1, 300)
    A = orc.fgt_p2h_grid(g, p, sigma, x, q)
    C = orc.fgt_h2t_grid(g, ncut, p, sigma, A)
    n = 1 << g
    side = 2.0 ** -g
    y = rng.random((30, 2))
    G = orc.fgt_direct(x, q, sigma, y)
    approx = np.zeros(len(y))
    for j, (yx, yy) in enumerate(y):
        tx, ty = min(int(yx * n), n - 1), min(int(yy * n), n - 1)
        tC = ((tx + 0.5) * side, (ty + 0.5) * side)
        approx[j] = orc.fgt_taylor_eval(C[ty * n + tx], tC, sigma, y[j:j + 1])[0]
    assert np.abs(approx - G).max() / np.abs(q).sum() < 1e-7


def test_grid_pipeline_converges_to_direct_gauss_sum(orc):
    """P2H on the grid, H2T over the n_cut neighbourhood, Taylor evaluation at each
    target's box (Eqs. A_alpha, C_beta, taylor) against the direct sum (Eq. dgt):
    the error falls with p and is below 1e-6 from p = 8 (truncation and cutoff)."""
    import workloads

    x, q = workloads.gmm_particles(3000, np.random.default_rng(5), ncomp=4)
    y = np.random.default_rng(6).random((300, 2))
    sigma = 0.1
    g = workloads.fgt_grid_log2(sigma)
    D = orc.fgt_direct(x, q, sigma, y)
    errs = []
    for p in (4, 8, 12):
        A = orc.fgt_p2h_grid(g, p, sigma, x, q)
        C = orc.fgt_h2t_grid(g, workloads.FGT_NCUT, p, sigma, A)
        G = orc.fgt_taylor_eval_grid(g, p, sigma, C, y)
        errs.append(np.linalg.norm(G - D) / np.linalg.norm(D))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 1e-6 and errs[2] < 1e-8, errs


def test_hermite_grid_eval_converges_to_direct_gauss_sum(orc):
    """P2H on the grid, then Eq. (hermite) summed over each target's n_cut
    neighbourhood (reading R14), against the direct sum (Eq. dgt): the error
    falls with p until the cutoff (about 2e-10 here) dominates."""
    import workloads

    x, q = workloads.gmm_particles(3000, np.random.default_rng(15), ncomp=4)
    y = np.random.default_rng(16).random((300, 2))
    sigma = 0.1
    g = workloads.fgt_grid_log2(sigma)
    D = orc.fgt_direct(x, q, sigma, y)
    errs = []
    for p in (4, 8, 12, 16):
        A = orc.fgt_p2h_grid(g, p, sigma, x, q)
        G = orc.fgt_hermite_eval_grid(g, workloads.FGT_NCUT, p, sigma, A, y)
        errs.append(np.linalg.norm(G - D) / np.linalg.norm(D))
    assert errs[0] > errs[1] > errs[2] and errs[3] <= errs[2] * 1.01, errs
    assert errs[0] < 1e-3 and errs[1] < 1e-6 and errs[2] < 1e-9, errs


@pytest.mark.parametrize("ncut", [1, 2, 3, 4])
def test_hermite_grid_eval_sums_exactly_the_neighbourhood(orc, ncut):
    """With p = 16 the Hermite truncation is ~1e-13 of sum|q|, so G must equal the
    direct Gauss sum over exactly the sources whose boxes lie within Chebyshev
    distance ncut of the target's box (a box too many or too few changes G by
    ~1e-2 of sum|q| here).  The omitted part is bounded by the Gaussian tail
    sum|q| exp(-(ncut side)^2 / 2 sigma^2), since every omitted source lies at
    least ncut box sides from the target."""
    rng = np.random.default_rng(30 + ncut)
    sigma, g, p = 0.1, 4, 16
    n = 1 << g
    side = 2.0 ** -g
    x = rng.random((400, 2))
    q = rng.uniform(-1, 1, 400)
    y = rng.random((200, 2))
    A = orc.fgt_p2h_grid(g, p, sigma, x, q)
    G = orc.fgt_hermite_eval_grid(g, ncut, p, sigma, A, y)
    sbx = np.minimum((x * n).astype(int), n - 1)
    tby = np.minimum((y * n).astype(int), n - 1)
    near = np.zeros(len(y))
    for j in range(len(y)):
        keep = np.maximum(np.abs(sbx[:, 0] - tby[j, 0]), np.abs(sbx[:, 1] - tby[j, 1])) <= ncut
        d2 = ((x[keep] - y[j]) ** 2).sum(axis=1)
        near[j] = (q[keep] * np.exp(-d2 / (2 * sigma ** 2))).sum()
    assert np.abs(G - near).max() <= 1e-11 * np.abs(q).sum()
    D = orc.fgt_direct(x, q, sigma, y)
    assert np.abs(G - D).max() <= np.abs(q).sum() * math.exp(-((ncut * side) ** 2) / (2 * sigma ** 2))


def test_hermite_grid_eval_equals_taylor_route_on_same_neighbourhood(orc):
    """H2T over the n_cut neighbourhood followed by Taylor evaluation (Eqs. C_beta,
    taylor) sums the same source boxes as the Hermite evaluation (Eq. hermite,
    R14); with a small n_cut the neighbourhood decides the answer, so the two
    routes agree only if both take the same boxes.  They differ by truncation."""
    rng = np.random.default_rng(12)
    sigma, g, p, ncut = 0.2, 3, 16, 2
    x = rng.random((300, 2))
    q = rng.uniform(-1, 1, 300)
    y = rng.random((150, 2))
    A = orc.fgt_p2h_grid(g, p, sigma, x, q)
    Gh = orc.fgt_hermite_eval_grid(g, ncut, p, sigma, A, y)
    C = orc.fgt_h2t_grid(g, ncut, p, sigma, A)
    Gt = orc.fgt_taylor_eval_grid(g, p, sigma, C, y)
    D = orc.fgt_direct(x, q, sigma, y)
    assert np.linalg.norm(Gh - D) / np.linalg.norm(D) > 1e-3  # the cutoff matters here
    assert np.linalg.norm(Gh - Gt) / np.linalg.norm(Gh) < 1e-8
    # and each target box's sum is that of its own neighbourhood: brute force on two targets
    n = 1 << g
    sc = math.sqrt(2.0) * sigma
    side = 2.0 ** -g
    for j in (0, 77):
        tx, ty = min(int(y[j, 0] * n), n - 1), min(int(y[j, 1] * n), n - 1)
        acc = 0.0
        for b in range(n * n):
            sx, sy = b % n, b // n
            if max(abs(sx - tx), abs(sy - ty)) > ncut:
                continue
            t1 = (y[j, 0] - (sx + 0.5) * side) / sc
            t2 = (y[j, 1] - (sy + 0.5) * side) / sc
            h1 = orc.hermite_functions(p, t1)
            h2 = orc.hermite_functions(p, t2)
            acc += h1 @ A[b] @ h2
        assert abs(acc - Gh[j]) <= 1e-12 * max(1.0, abs(acc))
