"""GPU parity of the far-field stages around the M2L path (fmm_l2l, fmm_l2p and
their adjoints, fmm_p2m_adjoint) against references built from the FP64 oracle
only: the oracle's L2L and L2P routines, explicit conjugate transposes of the
maps the oracle applies to unit vectors, and central differences of the
oracle's P2M.  Scaled units at the library boundary."""
import numpy as np
import pytest

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


def _dev(a, dtype=np.complex64):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _host(t):
    return t.cpu().numpy().astype(np.complex128)


def _rel(got, ref):
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


def _oracle_l2l_scaled(orc, child_level, p, Lp):
    """Scaled L2L of a whole level from the oracle's physical-unit L2L."""
    n = 1 << child_level
    Lc = np.zeros((n * n, p), dtype=np.complex128)
    phys = orc.unscale_le(Lp, child_level - 1)
    for iy in range(n):
        for ix in range(n):
            shift = orc.box_centre(child_level, ix, iy) - orc.box_centre(child_level - 1, ix // 2, iy // 2)
            Lc[iy * n + ix] = orc.l2l(p, phys[(iy // 2) * (n // 2) + ix // 2], shift)
    return orc.scale_le(Lc, child_level)


@pytest.mark.parametrize("p", [8, 16])
def test_l2l_and_adjoint(fmm, orc, p):
    rng = np.random.default_rng(p)
    cl = 4
    nb_p, nb_c = 4 ** (cl - 1), 4 ** cl
    Lp = rng.standard_normal((nb_p, p)) + 1j * rng.standard_normal((nb_p, p))
    X = rng.standard_normal((nb_c, p)) + 1j * rng.standard_normal((nb_c, p))
    Lcd = _dev(X)
    fmm.fmm_l2l(cl, p, _dev(Lp), Lcd, accumulate=True)
    fmm.fmm_sync_status()
    ref = _oracle_l2l_scaled(orc, cl, p, Lp)
    assert _rel(_host(Lcd) - X.astype(np.complex64), ref) <= 1e-6
    # adjoint: conj transpose of the oracle's map (applied to unit parent vectors)
    W = rng.standard_normal((nb_c, p)) + 1j * rng.standard_normal((nb_c, p))
    Wp = _dev(np.zeros((nb_p, p)))
    fmm.fmm_l2l_adjoint(cl, p, _dev(W), Wp)
    fmm.fmm_sync_status()
    n = 1 << cl
    T = {}
    for c in range(4):  # T_c[j][n] from unit inputs, one child per class
        ix, iy = c & 1, c >> 1
        cols = []
        for k in range(p):
            e = np.zeros((nb_p, p), dtype=np.complex128)
            e[0, k] = 1.0
            cols.append(_oracle_l2l_scaled(orc, cl, p, e)[iy * n + ix])
        T[c] = np.stack(cols, axis=1)
    ref = np.zeros((nb_p, p), dtype=np.complex128)
    for iy in range(n):
        for ix in range(n):
            c = (ix & 1) + 2 * (iy & 1)
            ref[(iy // 2) * (n // 2) + ix // 2] += T[c].conj().T @ W[iy * n + ix]
    assert _rel(_host(Wp), ref) <= 1e-6


def _points(rng, n, level):
    import torch

    z = rng.random((n, 2))
    side = 1 << level
    ix = np.minimum((z[:, 0] * side).astype(np.int64), side - 1)
    iy = np.minimum((z[:, 1] * side).astype(np.int64), side - 1)
    box = iy * side + ix
    return z, box, torch.from_numpy(z).cuda(), torch.full((n,), level, dtype=torch.int32).cuda(), \
        torch.from_numpy(box).cuda()


@pytest.mark.parametrize("p", [8, 16])
def test_l2p_and_adjoint(fmm, orc, p):
    import torch

    rng = np.random.default_rng(10 + p)
    level, npts = 5, 300
    nb = 4 ** level
    Ls = rng.standard_normal((nb, p)) + 1j * rng.standard_normal((nb, p))
    z, box, zd, levd, boxd = _points(rng, npts, level)
    phi = torch.empty(npts, dtype=torch.complex64, device="cuda")
    fmm.fmm_l2p(p, zd, levd, boxd, {level: _dev(Ls)}, level, phi)
    fmm.fmm_sync_status()
    side = 1 << level
    phys = orc.unscale_le(Ls, level)
    ref = np.array([orc.l2p(p, phys[b], orc.box_centre(level, int(b % side), int(b // side)),
                            np.array([z[j, 0] + 1j * z[j, 1]]))[0] for j, b in enumerate(box)])
    assert _rel(_host(phi), ref) <= 1e-6
    # adjoint: G[b][n] = sum_j conj(A_jn) cot_j with A_jn = phi_j for the unit LE e_n of box b
    cot = rng.standard_normal(npts) + 1j * rng.standard_normal(npts)
    G = _dev(np.zeros((nb, p)))
    fmm.fmm_l2p_adjoint(p, zd, levd, boxd, _dev(cot), {level: G}, level)
    fmm.fmm_sync_status()
    ref = np.zeros((nb, p), dtype=np.complex128)
    for j, b in enumerate(box):
        centre = orc.box_centre(level, int(b % side), int(b // side))
        for k in range(p):
            e = np.zeros((1, p), dtype=np.complex128)
            e[0, k] = 1.0
            a = orc.l2p(p, orc.unscale_le(e, level)[0], centre, np.array([z[j, 0] + 1j * z[j, 1]]))[0]
            ref[b, k] += np.conj(a) * cot[j]
    assert _rel(_host(G), ref) <= 1e-5


@pytest.mark.parametrize("p", [8, 16])
def test_l2p_binned_matches_oracle_and_per_point_kernel(fmm, orc, p):
    """fmm_l2p_binned (one block per box over the binned points) against the oracle's
    L2P at each point's box and the per-point kernel: points in random order, on box
    boundaries, at 1.0 and just outside the unit square (clamped boxes)."""
    import torch

    rng = np.random.default_rng(40 + p)
    level, npts = 5, 3000
    side, nb = 1 << level, 4 ** level
    z = rng.random((npts, 2))
    k = np.arange(side + 1) / side
    z[:side + 1, 0] = k
    z[side + 1:2 * side + 2, 1] = np.nextafter(k, -1.0)
    z[-3:] = [[1.0, 0.5], [1.004, 0.2], [-0.002, 0.7]]
    Ls = rng.standard_normal((nb, p)) + 1j * rng.standard_normal((nb, p))
    zd = torch.from_numpy(z).cuda()
    perm = torch.empty(npts, dtype=torch.int32, device="cuda")
    start = torch.empty(nb + 1, dtype=torch.int32, device="cuda")
    fmm.fmm_bin_points(level, zd, perm, start, torch.empty(nb, dtype=torch.int32, device="cuda"))
    phi = torch.empty(npts, dtype=torch.complex64, device="cuda")
    fmm.fmm_l2p_binned(level, p, zd, perm, start, _dev(Ls), phi)
    fmm.fmm_sync_status()
    ix = np.clip(np.floor(z[:, 0] * side), 0, side - 1).astype(np.int64)
    iy = np.clip(np.floor(z[:, 1] * side), 0, side - 1).astype(np.int64)
    phys = orc.unscale_le(Ls, level)
    ref = np.array([orc.l2p(p, phys[iy[j] * side + ix[j]], orc.box_centre(level, int(ix[j]), int(iy[j])),
                            np.array([z[j, 0] + 1j * z[j, 1]]))[0] for j in range(npts)])
    got = _host(phi)
    assert _rel(got, ref) <= 1e-6
    # the per-point kernel on the same boxes
    phi2 = torch.empty_like(phi)
    lev = torch.full((npts,), level, dtype=torch.int32, device="cuda")
    fmm.fmm_l2p(p, zd, lev, torch.from_numpy(iy * side + ix).cuda(), {level: _dev(Ls)}, level, phi2)
    fmm.fmm_sync_status()
    assert _rel(got, _host(phi2)) <= 1e-6
    # accumulate
    fmm.fmm_l2p_binned(level, p, zd, perm, start, _dev(Ls), phi, accumulate=True)
    fmm.fmm_sync_status()
    assert _rel(_host(phi), 2 * ref) <= 1e-6


def test_l2p_binned_coarse_levels_and_bad_bins(fmm):
    """Levels 0 and 1 carry no LEs (phi = 0, L may be None); a box_start that does not bin
    the points sets the device error word."""
    import torch

    z = torch.rand((50, 2), dtype=torch.float64, device="cuda")
    perm = torch.arange(50, dtype=torch.int32, device="cuda")
    phi = torch.full((50,), 3.0 + 1.0j, dtype=torch.complex64, device="cuda")
    start = torch.tensor([0, 50], dtype=torch.int32, device="cuda")
    fmm.fmm_l2p_binned(0, 8, z, perm, start, None, phi)
    fmm.fmm_sync_status()
    assert float(phi.abs().max()) == 0.0
    bad = torch.tensor([0, 10, 5, 20, 50], dtype=torch.int32, device="cuda")  # a box with end < first
    L1 = torch.zeros((4, 8), dtype=torch.complex64, device="cuda")
    fmm.fmm_l2p_binned(1, 8, z, perm, bad, L1, phi)
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_sync_status()
    assert e.value.code == fmm.FMM_EDEVICE


def test_l2p_reports_bad_leaves(fmm, orc):
    import torch

    z = torch.rand((4, 2), dtype=torch.float64, device="cuda")
    lev = torch.tensor([3, 3, 9, 3], dtype=torch.int32, device="cuda")  # level 9 has no array
    box = torch.tensor([0, 63, 0, 64], dtype=torch.int64, device="cuda")  # box 64 is outside level 3
    L3 = torch.zeros((64, 8), dtype=torch.complex64, device="cuda")
    phi = torch.empty(4, dtype=torch.complex64, device="cuda")
    fmm.fmm_l2p(8, z, lev, box, {3: L3}, 3, phi)
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_sync_status()
    assert e.value.code == fmm.FMM_EDEVICE
    assert float(phi.abs().max()) == 0.0


def test_p2m_adjoint_matches_central_differences(fmm, orc):
    """grad of J = Re sum_b sum_k conj(G[b][k]) M~_b[k](y) in each point's position."""
    import torch

    rng = np.random.default_rng(3)
    p, level, n = 12, 4, 40
    xy = rng.random((n, 2))
    c = rng.uniform(-1, 1, n)
    nb = 4 ** level
    G = rng.standard_normal((nb, p)) + 1j * rng.standard_normal((nb, p))
    grad = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    fmm.fmm_p2m_adjoint(level, p, torch.from_numpy(xy).cuda(), torch.from_numpy(c).cuda(), _dev(G), grad)
    fmm.fmm_sync_status()
    side = 1 << level
    h = 1e-7

    def J(i, pos):
        ix, iy = min(int(xy[i, 0] * side), side - 1), min(int(xy[i, 1] * side), side - 1)
        b = iy * side + ix
        m = orc.scale_me(orc.p2m_box(pos[None, :], c[i:i + 1], orc.box_centre(level, ix, iy), p)[None, :], level)[0]
        return float(np.real(np.sum(np.conj(G[b]) * m)))

    ref = np.zeros((n, 2))
    for i in range(n):
        for a in range(2):
            pp, pm = xy[i].copy(), xy[i].copy()
            pp[a] += h
            pm[a] -= h
            ref[i, a] = (J(i, pp) - J(i, pm)) / (2 * h)
    got = grad.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref), np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_m2m_adjoint(fmm, orc):
    """Conjugate transpose of M2M against the oracle's M2M applied to unit child vectors."""
    rng = np.random.default_rng(21)
    p, cl = 12, 4
    nb_c, nb_p = 4 ** cl, 4 ** (cl - 1)
    W = rng.standard_normal((nb_p, p)) + 1j * rng.standard_normal((nb_p, p))
    Wc = _dev(np.zeros((nb_c, p)))
    fmm.fmm_m2m_adjoint(cl, p, _dev(W), Wc)
    fmm.fmm_sync_status()
    n = 1 << cl
    ref = np.zeros((nb_c, p), dtype=np.complex128)
    for c in range(4):  # scaled M2M matrix of child class c: parent[j] from child[k]
        ix, iy = c & 1, c >> 1
        cols = []
        for k in range(p):
            e = np.zeros((nb_c, p), dtype=np.complex128)
            e[iy * n + ix, k] = 1.0
            Mp = orc.scale_me(orc.m2m_uniform(cl, p, orc.unscale_me(e, cl)), cl - 1)
            cols.append(Mp[0])
        T = np.stack(cols, axis=1)
        for py in range(n // 2):
            for px in range(n // 2):
                ref[(2 * py + iy) * n + 2 * px + ix] = T.conj().T @ W[py * (n // 2) + px]
    assert _rel(_host(Wc), ref) <= 1e-6
