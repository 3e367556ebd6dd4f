"""Pins for the FP64 M2L oracle against facts fixed by the paper and by mathematics.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a wrong list rule) fails at least one
of them:

* interaction lists: closed-form counts, an all-pairs brute force of the rule,
  symmetry, the 40 offset codes, and the paper's printed translation counts
  (Table m2ltesla, Sec. 4.1 worked example);
* M2L: the exact Taylor coefficients of the Cauchy kernel (closed form),
  convergence of the far-field potential to the direct sum (Eq. n_body) at a
  geometric rate, and M2M-then-M2L consistency;
* M2P: the exact potential of a centred source, one power per coefficient, a
  cluster's ME converging to the direct sum within the geometric tail bound, and
  agreement with L2P(M2L(.)) as p grows;
* adjoint: the bilinear dot-product identity.
"""
import math
import os

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(v) for v in line.split()])
    return rows


# ---------------------------------------------------------------------------
# binomials and lists
# ---------------------------------------------------------------------------

def test_binomials_match_library(orc):
    for a in range(0, 63):
        for b in range(0, a + 1):
            assert orc.binom(a, b) == float(math.comb(a, b))


def _brute_force_list(level, tx, ty):
    """All same-level boxes s with Chebyshev(parent(s), parent(t)) <= 1 and Chebyshev(s, t) >= 2."""
    n = 1 << level
    out = set()
    for sy in range(n):
        for sx in range(n):
            par = max(abs((sx >> 1) - (tx >> 1)), abs((sy >> 1) - (ty >> 1)))
            own = max(abs(sx - tx), abs(sy - ty))
            if par <= 1 and own >= 2:
                out.add((sx, sy))
    return out


@pytest.mark.parametrize("level", [2, 3, 4])
def test_list_matches_all_pairs_brute_force(orc, level):
    n = 1 << level
    for ty in range(n):
        for tx in range(n):
            lst = orc.interaction_list(level, tx, ty)
            got = {(sx, sy) for sx, sy, _, _ in lst}
            assert len(got) == len(lst)
            assert got == _brute_force_list(level, tx, ty)
            for sx, sy, ox, oy in lst:
                assert (ox, oy) == (sx - tx, sy - ty)


@pytest.mark.parametrize("level", [2, 3, 4, 5, 6, 7])
def test_list_count_closed_form(orc, level):
    n = 1 << level
    assert orc.list_count_level(level) == (6 * n - 8) ** 2 - (3 * n - 2) ** 2


def test_list_counts_of_the_workloads(orc):
    small = sum(orc.list_count_level(l) for l in workloads.m2l_levels(4))
    assert small == 156 + 1116 + 5628 == 6900
    big = sum(((6 * (1 << l) - 8) ** 2 - (3 * (1 << l) - 2) ** 2) for l in workloads.m2l_levels(8))
    assert big == 2316900


@pytest.mark.parametrize("level", [3, 4])
def test_list_symmetry_and_offsets(orc, level):
    n = 1 << level
    lists = {(tx, ty): {(sx, sy) for sx, sy, _, _ in orc.interaction_list(level, tx, ty)}
             for ty in range(n) for tx in range(n)}
    for t, srcs in lists.items():
        for s in srcs:
            assert t in lists[s]
    offsets = set()
    by_class = {}
    for ty in range(n):
        for tx in range(n):
            offs = {(ox, oy) for _, _, ox, oy in orc.interaction_list(level, tx, ty)}
            offsets |= offs
            by_class.setdefault((tx & 1, ty & 1), set()).update(offs)
    assert len(offsets) == 40
    assert all(max(abs(a), abs(b)) in (2, 3) for a, b in offsets)
    assert all(len(v) == 27 for v in by_class.values())
    # interior boxes have exactly 27
    for ty in range(2, n - 2):
        for tx in range(2, n - 2):
            assert len(orc.interaction_list(level, tx, ty)) == 27


def test_periodic_counts_match_paper_table(orc):
    rows = _load_table("m2l_table_tesla.txt")
    counts = sorted({int(r[1]) for r in rows})
    per_level = {l: orc.list_count_level(l, periodic=True) for l in range(2, 9)}
    for l in range(2, 9):
        assert per_level[l] == 27 * 4 ** l
    expected = [sum(per_level[l] for l in range(2, L + 1)) for L in range(3, 9)]
    assert counts == expected


def test_paper_example_count(orc):
    (row,) = _load_table("m2l_example_count.txt")
    assert orc.list_count_level(int(row[0]), periodic=True) == int(row[1])


def test_paper_op_count_convention():
    """28 p (p + 7) ops per translation reproduces the OPS. column from the translations/s column."""
    from paper_1009_3457_gb300.metrics import paper_ops_per_translation

    for p, ntr, secs, gops, mtr in _load_table("m2l_table_tesla.txt"):
        assert abs(mtr * 1e6 * paper_ops_per_translation(int(p)) / 1e9 - gops) / gops < 2e-3
        # the printed kernel time is rounded to 3 digits
        assert abs(ntr / secs / 1e6 - mtr) / mtr < 6e-3


# ---------------------------------------------------------------------------
# M2L against closed forms
# ---------------------------------------------------------------------------

def test_m2l_point_source_at_centre_is_exact_taylor(orc):
    """A unit-ME source c at x_s: the LE of c/(z - x_s) about x_t is (-1)^n c d^-(n+1), d = x_t - x_s."""
    p = 12
    c = 0.7 - 0.2j
    for d in [2.0 + 0.0j, -3.0 + 1.0j, 0.25 - 0.5j, -0.125 - 0.375j]:
        m = np.zeros(p, complex)
        m[0] = c
        l = orc.m2l_pair(p, d, m)
        expect = np.array([(-1) ** n * c / d ** (n + 1) for n in range(p)])
        np.testing.assert_allclose(l, expect, rtol=1e-14, atol=0)


def test_m2l_converges_to_exact_taylor_coefficients(orc):
    """Off-centre source y: as p grows the LE tends to the exact Taylor coefficients
    (-1)^n c (x_t - y)^-(n+1) of c/(z - y) about x_t."""
    rng = np.random.default_rng(7)
    for _ in range(5):
        d = complex(*rng.choice([-3, -2, 2, 3], 2)) * 0.125
        e = (rng.random() - 0.5) * 0.125 / 2 + 1j * (rng.random() - 0.5) * 0.125 / 2
        c = rng.uniform(-1, 1)
        p = 60
        m = np.array([c * e ** k for k in range(p)])  # P2M of one source
        l = orc.m2l_pair(p, d, m)
        nchk = 8
        expect = np.array([(-1) ** n * c / (d - e) ** (n + 1) for n in range(nchk)])
        np.testing.assert_allclose(l[:nchk], expect, rtol=1e-11)


def test_m2p_centred_source_is_exact(orc):
    """M2P of the ME (c, 0, ..., 0) about x_s is c/(z - x_s) exactly, at any p
    (Sec. 2.1: the ME of one source at the box centre)."""
    cs = 0.3 + 0.6j
    c = -0.8 + 0.1j
    rng = np.random.default_rng(19)
    z = cs + (rng.random(16) - 0.5) * 4 + 1j * (rng.random(16) - 0.5) * 4
    for p in (1, 5, 16):
        m = np.zeros(p, complex)
        m[0] = c
        np.testing.assert_allclose(orc.m2p(p, m, cs, z), c / (z - cs), rtol=1e-15, atol=0)


def test_m2p_single_term_powers(orc):
    """The k-th coefficient multiplies (z - x_s)^-(k+1): a unit ME in slot k alone
    gives exactly that power, so a shifted or dropped index fails."""
    cs = -0.25 + 0.5j
    z = np.array([1.5 + 0.25j, -2.0 - 1.0j, 0.75 + 3.0j])
    p = 9
    for k in range(p):
        m = np.zeros(p, complex)
        m[k] = 1.0
        np.testing.assert_allclose(orc.m2p(p, m, cs, z), (z - cs) ** -(k + 1), rtol=1e-14, atol=0)


def test_m2p_of_cluster_converges_to_direct_sum(orc):
    """The ME of a box's sources (P2M), evaluated two or more box sides away, tends
    to the direct sum (Eq. n_body) geometrically: the error of p terms is at most
    sum|c| rho^p / (|z - x_s| (1 - rho)) with rho = (side/sqrt 2) / |z - x_s|."""
    rng = np.random.default_rng(23)
    side = 0.125
    cs = 0.4375 + 0.5625j
    xy = np.column_stack([cs.real + (rng.random(200) - 0.5) * side,
                          cs.imag + (rng.random(200) - 0.5) * side])
    c = rng.uniform(-1, 1, 200)
    ang = rng.random(32) * 2 * np.pi
    rad = side * (2.0 + 2.0 * rng.random(32))
    z = cs + rad * np.exp(1j * ang)
    exact = orc.direct(xy, c, z)
    prev = np.inf
    for p in (2, 4, 8, 12, 16, 24, 32):
        got = orc.m2p(p, orc.p2m_box(xy, c, cs, p), cs, z)
        rho = (side / np.sqrt(2)) / np.abs(z - cs)
        bound = np.abs(c).sum() * rho ** p / (np.abs(z - cs) * (1 - rho))
        err = np.abs(got - exact)
        assert np.all(err <= bound * (1 + 1e-9) + 1e-13)
        e = np.linalg.norm(err)
        assert e < prev or e < 1e-13
        prev = e
    assert prev < 1e-11 * np.linalg.norm(exact)


def test_m2p_equals_l2p_of_m2l_in_the_limit(orc):
    """Evaluating the ME directly at points of a well-separated target box equals
    L2P(M2L(ME)) there as p grows (Eq. M2Lmat is the re-expansion of M2P)."""
    rng = np.random.default_rng(29)
    m = rng.normal(size=12) + 1j * rng.normal(size=12)
    m *= 0.5 ** np.arange(12)
    cs, ct = 0.0 + 0.0j, 2.0 + 1.0j
    z = ct + (rng.random(8) - 0.5) * 0.5 + 1j * (rng.random(8) - 0.5) * 0.5
    direct = orc.m2p(12, m, cs, z)
    errs = []
    for p in (12, 20, 28, 32):
        mp = np.zeros(p, complex)
        mp[:12] = m
        le = orc.m2l_pair(p, ct - cs, mp)
        errs.append(np.max(np.abs(orc.l2p(p, le, ct, z) - direct) / np.abs(direct)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[-1] < 1e-13


def test_m2m_then_m2l_equals_parent_p2m(orc):
    """P2M about the parent equals M2M of the children's P2M exactly (finite series)."""
    rng = np.random.default_rng(3)
    xy, c = workloads.uniform_particles(500, rng)
    p = 10
    M3 = orc.p2m_uniform(3, p, xy, c)
    M2 = orc.p2m_uniform(2, p, xy, c)
    M2b = orc.m2m_uniform(3, p, M3)
    scale = np.abs(M2).max(axis=0)
    np.testing.assert_allclose(M2b / scale, M2 / scale, atol=1e-12)
    L2 = orc.m2l_uniform(2, p, M2)
    L2b = orc.m2l_uniform(2, p, M2b)
    np.testing.assert_allclose(L2b, L2, rtol=1e-10, atol=1e-10 * np.abs(L2).max())


def small_tree_case():
    rng = np.random.default_rng(11)
    return workloads.uniform_particles(600, rng)


@pytest.fixture(scope="module")
def small_tree(orc):
    return small_tree_case()


def _far_field_error(orc, xy, c, level, p, tx, ty, z):
    """L2P(sum over IL of M2L(P2M)) at points z of box (tx, ty) vs the direct sum over IL sources."""
    M = orc.p2m_uniform(level, p, xy, c)
    n = 1 << level
    lst = orc.interaction_list(level, tx, ty)
    side = 2.0 ** -level
    ct = orc.box_centre(level, tx, ty)
    l = np.zeros(p, complex)
    srcs = np.zeros(len(c), bool)
    ib = np.minimum((xy * n).astype(int), n - 1)
    for sx, sy, ox, oy in lst:
        l += orc.m2l_pair(p, -(ox + 1j * oy) * side, M[sy * n + sx])
        srcs |= (ib[:, 0] == sx) & (ib[:, 1] == sy)
    approx = orc.l2p(p, l, ct, z)
    exact = orc.direct(xy[srcs], c[srcs], z)
    return np.linalg.norm(approx - exact) / np.linalg.norm(exact)


def test_far_field_potential_converges_geometrically(orc, small_tree):
    xy, c = small_tree
    level, tx, ty = 3, 3, 4
    side = 2.0 ** -level
    rng = np.random.default_rng(5)
    ct = orc.box_centre(level, tx, ty)
    z = ct + (rng.random(64) - 0.5) * side + 1j * (rng.random(64) - 0.5) * side
    errs = [_far_field_error(orc, xy, c, level, p, tx, ty, z) for p in (4, 8, 12, 16, 20, 24)]
    for a, b in zip(errs, errs[1:]):
        assert b < a
    # worst case geometry: source/target radius r/sqrt(2), separation >= 2r -> ratio ~0.55 per term
    for p, e in zip((4, 8, 12, 16, 20, 24), errs):
        assert e < 4.0 * 0.55 ** p
    assert errs[-1] < 1e-6


def test_m2l_uniform_equals_pairwise_sum(orc, small_tree):
    """The level routine is the reduction (sum) of per-pair translations over each list."""
    xy, c = small_tree
    level, p = 3, 6
    M = orc.p2m_uniform(level, p, xy, c)
    L = orc.m2l_uniform(level, p, M)
    n = 1 << level
    side = 2.0 ** -level
    for t in [0, 9, 27, 63]:
        tx, ty = t % n, t // n
        acc = np.zeros(p, complex)
        for sx, sy, ox, oy in orc.interaction_list(level, tx, ty):
            acc += orc.m2l_matrix(p, -(ox + 1j * oy) * side) @ M[sy * n + sx]
        np.testing.assert_allclose(L[t], acc, rtol=1e-12, atol=1e-12 * np.abs(acc).max())
    Lt = orc.m2l_uniform_targets(level, p, M, [0, 9, 27, 63])
    np.testing.assert_allclose(Lt, L[[0, 9, 27, 63]], rtol=0, atol=0)


def test_periodic_m2l_every_box_has_27(orc):
    rng = np.random.default_rng(2)
    level, p = 3, 4
    n = 1 << level
    M = rng.standard_normal((n * n, p)) + 1j * rng.standard_normal((n * n, p))
    L = orc.m2l_uniform(level, p, M, periodic=True)
    # periodic images: a constant ME field gives the same LE in every box of a
    # child class (the 27 offsets depend only on the class (tx & 1, ty & 1))
    Mc = np.tile(M[:1], (n * n, 1))
    Lc = orc.m2l_uniform(level, p, Mc, periodic=True)
    for t in range(n * n):
        tx, ty = t % n, t // n
        ref = Lc[(ty & 1) * n + (tx & 1)]
        np.testing.assert_allclose(Lc[t], ref, rtol=1e-12)
    assert np.all(np.isfinite(L))


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("periodic", [False, True])
def test_adjoint_dot_product(orc, periodic):
    rng = np.random.default_rng(13)
    level, p = 3, 7
    n = 1 << level
    M = rng.standard_normal((n * n, p)) + 1j * rng.standard_normal((n * n, p))
    W = rng.standard_normal((n * n, p)) + 1j * rng.standard_normal((n * n, p))
    AM = orc.m2l_uniform(level, p, M, periodic)
    AtW = orc.m2l_adjoint_uniform(level, p, W, periodic)
    lhs = np.sum(W * AM)
    rhs = np.sum(AtW * M)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_operator_transpose_identity(orc):
    """a(d)^T = -a(-d) for the Cauchy M2L matrix (the structure the adjoint relies on)."""
    for d in [2 + 1j, -3 + 0j, 0.5 - 0.75j]:
        A = orc.m2l_matrix(9, d)
        B = orc.m2l_matrix(9, -d)
        np.testing.assert_allclose(A.T, -B, rtol=1e-14)


def test_scaled_operator_depends_only_on_offset(orc):
    """With m~_k = m_k / r^k and l~_n = l_n r^(n+1), the M2L of a fixed box offset is level independent."""
    rng = np.random.default_rng(17)
    p = 10
    m_s = rng.standard_normal(p) + 1j * rng.standard_normal(p)
    outs = []
    for level in (2, 5, 8):
        r = 2.0 ** -level
        m = m_s * r ** np.arange(p)  # physical ME with this scaled value
        l = orc.m2l_pair(p, -(2 + 3j) * r, m)
        outs.append(orc.scale_le(l, level))
    np.testing.assert_allclose(outs[1], outs[0], rtol=1e-13)
    np.testing.assert_allclose(outs[2], outs[0], rtol=1e-13)
