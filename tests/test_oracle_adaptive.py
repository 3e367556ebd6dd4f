"""Pins of the FP64 oracle's adaptive-tree path (reading R12: split boxes holding
more than q points, drop empty children; V-lists; far-field objective of
reading R13) against things other than the oracle itself: an independent
recursive tree builder, brute-force list scans, the uniform special case, the
direct sum within the truncation error, and closed-form derivatives."""
import numpy as np
import pytest

import workloads


def _recursive_tree(xy, q, max_level):
    """Top-down recursion over explicit point sets: {(level, ix, iy)} of existing boxes."""
    out = set()

    def visit(level, ix, iy, pts):
        out.add((level, ix, iy))
        if level == max_level or len(pts) <= q:
            return
        n = 1 << (level + 1)
        bx = np.clip(np.floor(pts[:, 0] * n).astype(int), 0, n - 1)
        by = np.clip(np.floor(pts[:, 1] * n).astype(int), 0, n - 1)
        for cy in range(2):
            for cx in range(2):
                sel = (bx == 2 * ix + cx) & (by == 2 * iy + cy)
                if sel.any():
                    visit(level + 1, 2 * ix + cx, 2 * iy + cy, pts[sel])

    visit(0, 0, 0, np.asarray(xy))
    return out


def small_case(orc):
    """3000 mixture points, q = 20, depth <= 7, the tree built by `orc`."""
    xy, c = workloads.gmm_particles(3000, np.random.default_rng(17), ncomp=5)
    tree = orc.adaptive_tree(xy, 20, 7)
    return xy, c, tree


@pytest.fixture(scope="module")
def small(orc):
    return small_case(orc)


def test_tree_matches_recursive_builder(orc, small):
    xy, _, tree = small
    want = _recursive_tree(xy, 20, 7)
    got = set()
    for l in range(tree.max_level + 1):
        n = 1 << l
        for b in np.nonzero(tree.level(l))[0]:
            got.add((l, int(b % n), int(b // n)))
    assert got == want
    assert tree.depth == max(l for l, _, _ in want)


def test_tree_invariants(orc, small):
    xy, _, tree = small
    lev, box = orc.leaf_boxes(tree, xy)
    for l in range(1, tree.depth + 1):
        n = 1 << l
        for b in np.nonzero(tree.level(l))[0]:
            parent = (b // n // 2) * (n // 2) + (b % n) // 2
            assert tree.level(l - 1)[parent]
    # every point is in exactly one leaf; a leaf holds <= q points unless at max_level
    counts = {}
    for l, b in zip(lev, box):
        counts[(int(l), int(b))] = counts.get((int(l), int(b)), 0) + 1
    assert sum(counts.values()) == len(xy)
    for (l, b), k in counts.items():
        n = 1 << l
        kids = [(2 * (b // n) + cy) * 2 * n + 2 * (b % n) + cx for cy in range(2) for cx in range(2)]
        is_leaf = l == tree.max_level or not any(tree.level(l + 1)[k_] for k_ in kids)
        assert is_leaf
        assert k <= 20 or l == tree.max_level


def test_vlists_brute_force_and_symmetric(orc, small):
    _, _, tree = small
    for l in range(2, tree.depth + 1):
        n = 1 << l
        ex = np.nonzero(tree.level(l))[0]
        exset = set(int(b) for b in ex)
        total = 0
        for t in ex:
            tx, ty = int(t % n), int(t // n)
            want = set()
            for s in ex:  # brute force over every existing box of the level
                sx, sy = int(s % n), int(s // n)
                if max(abs(sx // 2 - tx // 2), abs(sy // 2 - ty // 2)) <= 1 and max(abs(sx - tx), abs(sy - ty)) >= 2:
                    want.add((sx, sy))
            got = orc.vlist(tree, l, tx, ty)
            assert {(a, b) for a, b, _, _ in got} == want
            assert all(ox == a - tx and oy == b - ty for a, b, ox, oy in got)
            total += len(got)
            for a, b, _, _ in got:  # symmetry: t is in V(s)
                assert (tx, ty) in {(u, v) for u, v, _, _ in orc.vlist(tree, l, a, b)}
                assert b * n + a in exset
        assert orc.vlist_count_level(tree, l) == total
        absent = np.nonzero(~tree.level(l))[0]
        if len(absent):
            assert orc.vlist(tree, l, int(absent[0] % n), int(absent[0] // n)) == []


def test_full_tree_reduces_to_uniform_lists_and_m2l(orc):
    """One point per finest box and q = 0: every box exists and V(t) = IL(t)."""
    L, p = 4, 8
    n = 1 << L
    rng = np.random.default_rng(4)
    g = (np.arange(n) + 0.5) / n
    xy = np.stack(np.meshgrid(g, g), -1).reshape(-1, 2) + rng.uniform(-0.3, 0.3, (n * n, 2)) / n
    c = rng.uniform(-1, 1, n * n)
    tree = orc.adaptive_tree(xy, 0, L)
    assert tree.depth == L and all(tree.level(l).all() for l in range(L + 1))
    for l in range(2, L + 1):
        m = 1 << l
        for t in range(m * m):
            assert orc.vlist(tree, l, t % m, t // m) == orc.interaction_list(l, t % m, t // m)
        M = orc.p2m_uniform(l, p, xy, c)
        np.testing.assert_allclose(orc.m2l_adaptive(tree, l, p, M), orc.m2l_uniform(l, p, M), rtol=0, atol=0)


def test_adjoint_dot_product(orc, small):
    _, _, tree = small
    rng = np.random.default_rng(8)
    p = 8
    for l in range(2, tree.depth + 1):
        nb = 1 << (2 * l)
        M = rng.standard_normal((nb, p)) + 1j * rng.standard_normal((nb, p))
        W = rng.standard_normal((nb, p)) + 1j * rng.standard_normal((nb, p))
        lhs = np.sum(W * orc.m2l_adaptive(tree, l, p, M))
        rhs = np.sum(orc.m2l_adjoint_adaptive(tree, l, p, W) * M)
        assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_vlist_potential_matches_direct_sum(orc, small):
    """L2P of the V-list LE of a box equals the direct sum over the points of its
    V-list boxes, within the truncation error of p = 16."""
    xy, c, tree = small
    p = 16
    l = 4
    n = 1 << l
    bx = np.clip(np.floor(xy * n).astype(int), 0, n - 1)
    bidx = bx[:, 1] * n + bx[:, 0]
    ex = tree.level(l)
    M = orc.p2m_assigned(l, p, xy, c, np.where(ex[bidx], bidx, -1))
    Lv = orc.m2l_adaptive(tree, l, p, M)
    rng = np.random.default_rng(1)
    worst = 0.0
    checked = 0
    for t in np.nonzero(ex)[0][::3]:
        vl = orc.vlist(tree, l, int(t % n), int(t // n))
        if not vl:
            continue
        src = np.isin(bidx, [b * n + a for a, b, _, _ in vl])
        ctr = orc.box_centre(l, int(t % n), int(t // n))
        z = ctr + (rng.random(8) - 0.5) / n + 1j * (rng.random(8) - 0.5) / n
        exact = orc.direct(xy[src], c[src], z)
        got = orc.l2p(p, Lv[t], ctr, z)
        worst = max(worst, np.linalg.norm(got - exact) / np.linalg.norm(exact))
        checked += 1
    assert checked >= 5
    assert worst <= 1e-5, worst


def _objective_case(orc, n=2000, seed=21, q=24, max_level=6, nz=300):
    rng = np.random.default_rng(seed)
    xy, c = workloads.gmm_particles(n, rng, ncomp=4)
    tree = orc.adaptive_tree(xy, q, max_level)
    leaf = orc.leaf_boxes(tree, xy)
    z = rng.random(nz) + 1j * rng.random(nz)
    zl = orc.leaf_boxes(tree, np.stack([z.real, z.imag], 1))
    om = rng.uniform(-1, 1, nz)
    return xy, c, tree, leaf, z, zl, om


def test_objective_is_linear_in_strengths(orc):
    xy, c, tree, leaf, z, zl, om = _objective_case(orc)
    rng = np.random.default_rng(2)
    c2 = rng.uniform(-1, 1, len(c))
    J1 = orc.far_field_objective(tree, 12, xy, c, leaf, z, zl, om)
    J2 = orc.far_field_objective(tree, 12, xy, c2, leaf, z, zl, om)
    J12 = orc.far_field_objective(tree, 12, xy, 2.0 * c - 3.0 * c2, leaf, z, zl, om)
    assert abs(J12 - (2.0 * J1 - 3.0 * J2)) <= 1e-10 * (abs(J1) + abs(J2))


def test_fd_gradient_equals_full_recomputation(orc):
    """The sparse difference propagation gives the same central difference as two
    full evaluations of the objective (frozen topology)."""
    xy, c, tree, leaf, z, zl, om = _objective_case(orc)
    p, h = 12, 1e-4
    idx = [0, 777, 1999]
    fd = orc.far_field_fd_gradient(tree, p, xy, c, leaf, z, zl, om, idx, h)
    for r, i in enumerate(idx):
        for axis in range(2):
            a, b = xy.copy(), xy.copy()
            a[i, axis] += h
            b[i, axis] -= h
            full = (orc.far_field_objective(tree, p, a, c, leaf, z, zl, om)
                    - orc.far_field_objective(tree, p, b, c, leaf, z, zl, om)) / (2 * h)
            assert abs(fd[r, axis] - full) <= 1e-6 * max(abs(full), 1e-3), (i, axis, fd[r, axis], full)


def test_fd_gradient_single_source_closed_form(orc):
    """One charged source near (0.1, 0.1) and one evaluation point near (0.9, 0.9),
    well separated at level 2: phi_far(z) = c / (z - y) up to truncation, so
    dJ/dx = w Re(c / (z - y)^2) and dJ/dy = w Re(i c / (z - y)^2)."""
    rng = np.random.default_rng(6)
    xy = rng.random((600, 2))
    c = np.zeros(600)
    xy[0] = (0.11, 0.09)
    c[0] = 0.7
    tree = orc.adaptive_tree(xy, 8, 6)
    leaf = orc.leaf_boxes(tree, xy)
    z = np.array([0.88 + 0.91j])
    zl = orc.leaf_boxes(tree, np.array([[0.88, 0.91]]))
    om = np.array([1.3])
    y = complex(*xy[0])
    fd = orc.far_field_fd_gradient(tree, 16, xy, c, leaf, z, zl, om, [0], 1e-4)[0]
    d = c[0] / (z[0] - y) ** 2
    want = np.array([om[0] * d.real, om[0] * (1j * d).real])
    assert np.linalg.norm(fd - want) <= 1e-6 * np.linalg.norm(want), (fd, want)
    J = orc.far_field_objective(tree, 16, xy, c, leaf, z, zl, om)
    assert abs(J - om[0] * (c[0] / (z[0] - y)).real) <= 1e-8


def test_fd_gradient_step_converges(orc):
    """Central differences at h and h/10 agree to O(h^2): the step used against the
    GPU gradient (1e-6) is inside the converged range even on the finest boxes."""
    xy, c, tree, leaf, z, zl, om = _objective_case(orc, n=6000, seed=3, q=8, max_level=9)
    assert tree.depth >= 8
    idx = [int(i) for i in np.nonzero(leaf[0] >= 8)[0][:4]]
    f6 = orc.far_field_fd_gradient(tree, 16, xy, c, leaf, z, zl, om, idx, 1e-6)
    f7 = orc.far_field_fd_gradient(tree, 16, xy, c, leaf, z, zl, om, idx, 1e-7)
    assert np.linalg.norm(f6 - f7) <= 1e-6 * np.linalg.norm(f6)
