"""CPU-side checks of the C ABI library: it loads, exports every entry point the
header declares, rejects bad arguments on the host before touching the GPU,
and builds interaction lists that agree with the FP64 oracle's definition."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fmm():
    from paper_1009_3457_gb300 import build, fmmgb

    build.build()
    fmmgb.load()
    return fmmgb


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*((?:fmm|fgt)_[a-z_0-9]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


@pytest.mark.parametrize("compiler,std", [("gcc", "-std=c99"), ("g++", "-std=c++17")])
def test_header_compiles_as_plain_c_and_cpp(tmp_path, compiler, std):
    """include/fmmgb.h is a C ABI: it compiles on its own as strict C99 (pedantic, no
    warnings) and as C++, and a caller can name every status, precision and flag."""
    import shutil
    import subprocess

    if shutil.which(compiler) is None:
        pytest.skip(f"{compiler} not installed")
    src = tmp_path / "use_header.c"
    src.write_text(
        '#include "fmmgb.h"\n'
        "int main(void) {\n"
        "    fmm_host_stream_info_t hi; fmm_batch_info_t bi; fmm_level_info li;\n"
        "    (void)hi; (void)bi; (void)li;\n"
        "    return FMM_OK + FMM_EDEVICE + FMM_TC_TF32X3 + FMM_ACCUMULATE + FMM_CONJ + FMM_TREE_PERIODIC\n"
        "           + FMM_BATCH_AUTOTUNE + FMM_HOST_CONTIGUOUS + FMM_P2P_SHARE_SM + FMM_MAX_LEVEL;\n"
        "}\n")
    lang = ["-x", "c++"] if compiler == "g++" else []
    subprocess.check_call([compiler, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                           "-I", os.path.join(ROOT, "include")] + lang + [str(src)])


def test_every_declared_symbol_is_exported(fmm):
    lib = fmm.load()
    names = _declared_functions()
    assert {"fmm_build_lists", "fmm_m2l", "fmm_m2l_adjoint"} <= names
    for n in names:
        assert hasattr(lib, n), n
        assert n in fmm.SIGNATURES, f"binding lacks {n}"


def test_version(fmm):
    assert "sm_103a" in fmm.fmm_version()


def test_build_lists_rejects_bad_arguments(fmm):
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_build_lists(None, 1)
    assert e.value.code == fmm.FMM_EINVAL
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_build_lists(None, fmm.FMM_MAX_LEVEL + 1)
    assert e.value.code == fmm.FMM_EINVAL
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_build_lists(None, 5, leaf_cap=-1)
    assert e.value.code == fmm.FMM_EINVAL


def test_m2l_rejects_bad_arguments_before_launch(fmm):
    lib = fmm.load()
    tree = fmm.fmm_build_lists(None, 4)
    # NULL tree, bad level, bad p, NULL / misaligned / overlapping pointers, bad flags
    assert lib.fmm_m2l(None, 3, 8, 0, 4096, 1 << 20, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_m2l(tree.handle, 5, 8, 0, 4096, 1 << 20, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_m2l(tree.handle, -1, 8, 0, 4096, 1 << 20, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_m2l(tree.handle, 3, 7, 0, 4096, 1 << 20, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_m2l(tree.handle, 3, 8, 9, 4096, 1 << 20, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_m2l(tree.handle, 3, 8, 0, None, 1 << 20, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_m2l(tree.handle, 3, 8, 0, 4104, 1 << 20, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_m2l(tree.handle, 3, 8, 0, 4096, 4096 + 64, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_m2l(tree.handle, 3, 8, 0, 4096, 1 << 20, 8, None) == fmm.FMM_EINVAL
    assert "overlap" in fmm.fmm_last_error() or "flags" in fmm.fmm_last_error()
    assert lib.fmm_m2l_adjoint(tree.handle, 3, 8, 0, 4096, 1 << 20, 16, None) == fmm.FMM_EINVAL
    # FMM_TC_TF32X3 is provided at p = 16 only (refused before any device work); 4 is no precision
    TF = fmm.FMM_TC_TF32X3
    assert lib.fmm_m2l(tree.handle, 3, 24, TF, 1 << 20, 1 << 24, 0, None) == fmm.FMM_EUNSUPPORTED
    assert "p = 16" in fmm.fmm_last_error()
    assert lib.fmm_m2l(tree.handle, 3, 16, 4, 1 << 20, 1 << 24, 0, None) == fmm.FMM_EINVAL


def test_host_stream_rejects_bad_arguments_before_any_cuda_call(fmm):
    """fmm_host_stream_create checks its arguments before it creates a stream or allocates;
    the other entry points refuse a NULL handle."""
    import ctypes

    lib = fmm.load()
    tree = fmm.fmm_build_lists(None, 4)
    h = ctypes.c_void_p()
    create = lib.fmm_host_stream_create
    assert create(tree.handle, 2, 4, 8, 0, 2, None) == fmm.FMM_EINVAL          # NULL out
    assert create(None, 2, 4, 8, 0, 2, ctypes.byref(h)) == fmm.FMM_EINVAL       # NULL tree
    assert create(tree.handle, 2, 5, 8, 0, 2, ctypes.byref(h)) == fmm.FMM_EINVAL  # level beyond the tree
    assert create(tree.handle, 3, 2, 8, 0, 2, ctypes.byref(h)) == fmm.FMM_EINVAL  # lmin > lmax
    assert create(tree.handle, -1, 2, 8, 0, 2, ctypes.byref(h)) == fmm.FMM_EINVAL
    assert create(tree.handle, 2, 4, 7, 0, 2, ctypes.byref(h)) == fmm.FMM_EINVAL  # no such order
    assert create(tree.handle, 2, 4, 8, 9, 2, ctypes.byref(h)) == fmm.FMM_EINVAL  # no such precision
    for depth in (0, 9):
        assert create(tree.handle, 2, 4, 8, 0, depth, ctypes.byref(h)) == fmm.FMM_EINVAL
        assert "depth" in fmm.fmm_last_error()
    assert create(tree.handle, 2, 4, 8, fmm.FMM_TC_BF16X3, 2, ctypes.byref(h)) == fmm.FMM_EUNSUPPORTED
    assert create(tree.handle, 2, 4, 24, fmm.FMM_TC_TF32X3, 2, ctypes.byref(h)) == fmm.FMM_EUNSUPPORTED
    assert h.value is None
    one = (ctypes.c_void_p * 3)(4096, 8192, 16384)
    assert lib.fmm_host_stream_submit(None, one, one, 0) == fmm.FMM_EINVAL
    assert lib.fmm_host_stream_sync(None) == fmm.FMM_EINVAL
    assert lib.fmm_host_stream_info(None, ctypes.byref(fmm.fmm_host_stream_info_t())) == fmm.FMM_EINVAL
    lib.fmm_host_stream_destroy(None)


def test_p2m_m2m_reject_bad_arguments(fmm):
    lib = fmm.load()
    assert lib.fmm_p2m(-1, 8, 64, 64, 10, 64, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_p2m(3, 0, 64, 64, 10, 64, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_p2m(3, 8, None, 64, 10, 64, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_m2m(0, 8, 64, 128, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_m2m(3, 8, None, 128, 0, None) == fmm.FMM_EINVAL


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("level", [2, 3, 4, 5])
def test_library_lists_match_oracle(fmm, orc, level, periodic):
    tree = fmm.fmm_build_lists(None, 6, periodic=periodic)
    lst, code = tree.lists(level)
    n = 1 << level
    assert tree.translations(level) == orc.list_count_level(level, periodic)
    assert int((lst >= 0).sum()) == tree.translations(level)
    for t in range(n * n):
        tx, ty = t % n, t // n
        want = sorted((sy * n + sx, (oy + 3) * 7 + (ox + 3))
                      for sx, sy, ox, oy in orc.interaction_list(level, tx, ty, periodic))
        got = sorted((int(s), int(c)) for s, c in zip(lst[t], code[t]) if s >= 0)
        assert got == want, (t, got, want)
        assert all(c == -1 for s, c in zip(lst[t], code[t]) if s < 0)


def test_levels_below_two_have_no_lists(fmm):
    tree = fmm.fmm_build_lists(None, 3)
    for level in (0, 1):
        lst, code = tree.lists(level)
        assert (lst == -1).all() and (code == -1).all()
        assert tree.translations(level) == 0


def test_batch_rejects_bad_arguments_before_launch(fmm):
    """fmm_batch_create / fmm_m2l_batched validate everything on the host."""
    import ctypes

    lib = fmm.load()
    t3 = fmm.fmm_build_lists(None, 3)  # levels 2, 3 -> two pointers per problem
    vp, i32 = ctypes.c_void_p, ctypes.c_int32

    def call(trees, ps, Ms, Ls, prec=0, flags=0, nprob=None):
        n = len(trees) if nprob is None else nprob
        out = vp()
        return lib.fmm_batch_create((vp * max(len(trees), 1))(*trees), (i32 * max(len(ps), 1))(*ps), n,
                                    (vp * max(len(Ms), 1))(*Ms), (vp * max(len(Ls), 1))(*Ls), prec, flags, None,
                                    ctypes.byref(out))

    good_M, good_L = [1 << 20, 1 << 22], [1 << 24, 1 << 26]
    assert call([t3.handle], [8], good_M, good_L, nprob=0) == fmm.FMM_EINVAL
    assert call([None], [8], good_M, good_L) == fmm.FMM_EINVAL
    assert call([t3.handle], [7], good_M, good_L) == fmm.FMM_EINVAL
    assert call([t3.handle], [24], good_M, good_L) == fmm.FMM_EUNSUPPORTED
    assert call([t3.handle], [8], good_M, good_L, prec=fmm.FMM_TC_BF16X3) == fmm.FMM_EUNSUPPORTED
    assert call([t3.handle], [8], good_M, good_L, prec=fmm.FMM_TC_TF32X3) == fmm.FMM_EUNSUPPORTED
    assert call([t3.handle], [8], good_M, good_L, prec=9) == fmm.FMM_EINVAL
    assert call([t3.handle], [8], good_M, good_L, flags=16) == fmm.FMM_EINVAL
    assert call([t3.handle], [8], [1 << 20, None], good_L) == fmm.FMM_EINVAL
    assert call([t3.handle], [8], [(1 << 20) + 8, 1 << 22], good_L) == fmm.FMM_EINVAL
    # level 3 at p = 8 spans 64 * 8 * 8 = 4096 bytes: L inside M's range overlaps
    assert call([t3.handle], [8], good_M, [1 << 24, (1 << 22) + 1024]) == fmm.FMM_EINVAL
    assert "overlap" in fmm.fmm_last_error()
    out = vp()
    assert lib.fmm_batch_create(None, None, 1, None, None, 0, 0, None, ctypes.byref(out)) == fmm.FMM_EINVAL
    one = (vp * 1)(t3.handle)
    assert lib.fmm_m2l_batched(one, (i32 * 1)(8), 1, (vp * 2)(*good_M), (vp * 2)(*good_L), 0,
                               fmm.FMM_BATCH_AUTOTUNE, None) == fmm.FMM_EINVAL
    assert lib.fmm_batch_run(None, None) == fmm.FMM_EINVAL
    lib.fmm_batch_destroy(None, None)  # no-op


@pytest.fixture(scope="module")
def gmm_points():
    import workloads

    return workloads.gmm_particles(5000, np.random.default_rng(31), ncomp=6)[0]


def test_adaptive_tree_matches_oracle(fmm, orc, gmm_points):
    """Library adaptive tree (leaf_cap > 0): box existence, V-lists and their
    offset codes equal the oracle's reading R12, level by level."""
    xy = gmm_points
    q, L = 16, 8
    tree = fmm.fmm_build_lists(xy, L, leaf_cap=q)
    otree = orc.adaptive_tree(xy, q, L)
    assert tree.adaptive
    for level in range(L + 1):
        assert (tree.exists(level) == otree.level(level)).all(), level
    for level in range(2, L + 1):
        n = 1 << level
        assert tree.translations(level) == orc.vlist_count_level(otree, level)
        lst, code = tree.lists(level)
        for t in np.nonzero(otree.level(level) | (lst >= 0).any(axis=1))[0]:
            tx, ty = int(t % n), int(t // n)
            want = sorted((sy * n + sx, (oy + 3) * 7 + (ox + 3)) for sx, sy, ox, oy in orc.vlist(otree, level, tx, ty))
            got = sorted((int(s), int(c)) for s, c in zip(lst[t], code[t]) if s >= 0)
            assert got == want, (level, t)


def test_adaptive_tree_arguments(fmm, gmm_points):
    import ctypes

    lib = fmm.load()

    h = ctypes.c_void_p()
    assert lib.fmm_build_lists(None, 10, 5, 8, 0, ctypes.byref(h)) == fmm.FMM_EINVAL  # xy needed
    xy = np.ascontiguousarray(gmm_points)
    assert lib.fmm_build_lists(xy.ctypes.data, len(xy), 5, 8, fmm.FMM_TREE_PERIODIC,
                               ctypes.byref(h)) == fmm.FMM_EINVAL  # periodic + adaptive
    # a tree with no point splitting below the root: empty lists everywhere
    t = fmm.fmm_build_lists(xy[:5], 6, leaf_cap=8)
    assert all(t.translations(l) == 0 for l in range(7))
    assert t.level_info(3).nexist == 0
    # batched path takes uniform trees only
    tb = fmm.fmm_build_lists(xy, 5, leaf_cap=8)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    ptrs = (vp * 4)(*[(1 << 20) * (k + 1) for k in range(4)])
    outs = (vp * 4)(*[(1 << 28) * (k + 1) for k in range(4)])
    assert lib.fmm_batch_create((vp * 1)(tb.handle), (i32 * 1)(8), 1, ptrs, outs, 0, 0, None,
                                ctypes.byref(h)) == fmm.FMM_EUNSUPPORTED


def test_far_field_entry_points_reject_bad_arguments(fmm):
    import ctypes

    lib = fmm.load()
    vp = ctypes.c_void_p
    assert lib.fmm_l2l(0, 8, 64, 4096, 0, None) == fmm.FMM_EINVAL          # child level 0
    assert lib.fmm_l2l(3, 0, 64, 4096, 0, None) == fmm.FMM_EINVAL          # p
    assert lib.fmm_l2l(3, 8, None, 4096, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_l2l(3, 8, 68, 4096, 0, None) == fmm.FMM_EINVAL          # misaligned
    assert lib.fmm_l2l_adjoint(3, 8, 64, 4096, 2, None) == fmm.FMM_EINVAL  # flags
    tab = (vp * 4)(None, None, None, 4096)
    assert lib.fmm_l2p(8, 10, 64, 128, 256, tab, 15, 512, 0, None) == fmm.FMM_EINVAL   # max_level
    assert lib.fmm_l2p(8, 10, None, 128, 256, tab, 3, 512, 0, None) == fmm.FMM_EINVAL  # z
    assert lib.fmm_l2p(8, 10, 64, 128, 260, tab, 3, 512, 0, None) == fmm.FMM_EINVAL   # box misaligned
    assert lib.fmm_l2p_adjoint(8, 10, 64, 128, 256, None, tab, 3, None) == fmm.FMM_EINVAL
    assert lib.fmm_p2m_adjoint(3, 8, 64, 128, 10, None, 256, 0, None) == fmm.FMM_EINVAL
    assert lib.fmm_p2m_adjoint(3, 65, 64, 128, 10, 512, 256, 0, None) == fmm.FMM_EINVAL


def test_fgt_hermite_entry_points_reject_bad_arguments(fmm):
    lib = fmm.load()
    # fgt_bin_points(g, y, n, perm, box_start, work, stream)
    assert lib.fgt_bin_points(11, 64, 10, 128, 256, 512, None) == fmm.FMM_EINVAL        # grid_log2
    assert lib.fgt_bin_points(3, 64, -1, 128, 256, 512, None) == fmm.FMM_EINVAL         # n
    assert lib.fgt_bin_points(3, 64, 1 << 31, 128, 256, 512, None) == fmm.FMM_EINVAL    # n > int32
    assert lib.fgt_bin_points(3, None, 10, 128, 256, 512, None) == fmm.FMM_EINVAL       # y
    assert lib.fgt_bin_points(3, 64, 10, 128, 256, None, None) == fmm.FMM_EINVAL        # work
    assert lib.fgt_bin_points(3, 68, 10, 128, 256, 4096, None) == fmm.FMM_EINVAL        # y misaligned
    assert lib.fgt_bin_points(3, 64, 10, 128, 256, 300, None) == fmm.FMM_EINVAL         # work overlaps box_start
    # fgt_p2h_binned(g, p, sigma, x, q, n, perm, A, flags, stream)
    assert lib.fgt_p2h_binned(3, 6, 0.1, 64, 128, 10, 256, 512, 0, None) == fmm.FMM_EINVAL   # p
    assert lib.fgt_p2h_binned(3, 8, -0.1, 64, 128, 10, 256, 512, 0, None) == fmm.FMM_EINVAL  # sigma
    assert lib.fgt_p2h_binned(3, 8, 0.1, 64, 128, 10, None, 512, 0, None) == fmm.FMM_EINVAL  # perm
    assert lib.fgt_p2h_binned(3, 8, 0.1, 64, 128, 10, 256, 512, 4, None) == fmm.FMM_EINVAL   # flags
    # fgt_h2p(g, ncut, p, prec, sigma, A, y, n, perm, box_start, G, flags, stream)
    F, T3 = fmm.FMM_FP32, fmm.FMM_TC_BF16X3
    assert lib.fgt_h2p(3, 17, 8, F, 0.1, 64, 128, 10, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL  # n_cut
    assert lib.fgt_h2p(3, 2, 10, F, 0.1, 64, 128, 10, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL  # p
    assert lib.fgt_h2p(3, 2, 8, F, 0.0, 64, 128, 10, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL   # sigma
    assert lib.fgt_h2p(3, 2, 8, F, 0.1, 72, 128, 10, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL   # A misaligned
    assert lib.fgt_h2p(3, 2, 8, F, 0.1, 64, 128, 10, 256, None, 1024, 0, None) == fmm.FMM_EINVAL  # box_start
    assert lib.fgt_h2p(3, 2, 8, F, 0.1, 64, 128, 10, 256, 512, 1024, 2, None) == fmm.FMM_EINVAL   # flags
    assert "flags" in fmm.fmm_last_error()
    assert lib.fgt_h2p(3, 2, 8, 7, 0.1, 64, 128, 10, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL   # precision
    assert lib.fgt_h2p(3, 2, 8, T3, 0.1, 64, 128, 10, 256, 512, 1024, 0, None) == fmm.FMM_EUNSUPPORTED   # TC p
    assert lib.fgt_h2p(3, 16, 16, T3, 0.1, 64, 128, 10, 256, 512, 1024, 0, None) == fmm.FMM_EUNSUPPORTED  # TC n_cut
    TF = fmm.FMM_TC_TF32X3  # an M2L precision only
    assert lib.fgt_h2p(3, 2, 16, TF, 0.1, 64, 128, 10, 256, 512, 1024, 0, None) == fmm.FMM_EUNSUPPORTED
    # fgt_h2t(g, ncut, p, prec, sigma, A, C, work, flags, stream)
    A_, C_ = 1 << 20, 1 << 22
    assert lib.fgt_h2t(3, 2, 8, 7, 0.1, A_, C_, None, 0, None) == fmm.FMM_EINVAL            # precision
    assert "precision" in fmm.fmm_last_error()
    assert lib.fgt_h2t(3, 2, 8, T3, 0.1, A_, C_, None, 0, None) == fmm.FMM_EUNSUPPORTED     # TC p
    assert lib.fgt_h2t(2, 2, 16, T3, 0.1, A_, C_, None, 0, None) == fmm.FMM_EUNSUPPORTED    # TC grid under 8 x 8
    assert lib.fgt_h2t(3, 17, 16, T3, 0.1, A_, C_, None, 0, None) == fmm.FMM_EINVAL         # n_cut
    assert lib.fgt_h2t(3, 2, 16, T3, 0.1, A_, C_ + 8, None, 0, None) == fmm.FMM_EINVAL      # C misaligned
    assert lib.fgt_h2t(3, 2, 16, TF, 0.1, A_, C_, None, 0, None) == fmm.FMM_EUNSUPPORTED    # TF32x3: M2L only


def test_p2p_rejects_bad_arguments(fmm):
    lib = fmm.load()
    # fmm_p2p(level, xy, c, n, sperm, sstart, z, nz, tperm, tstart, phi, flags, stream)
    assert lib.fmm_p2p(11, 64, 128, 10, 256, 512, 1024, 10, 2048, 4096, 8192, 0, None) == fmm.FMM_EINVAL  # level
    assert lib.fmm_p2p(3, 64, 128, -1, 256, 512, 1024, 10, 2048, 4096, 8192, 0, None) == fmm.FMM_EINVAL  # n
    assert lib.fmm_p2p(3, 64, 128, 10, 256, None, 1024, 10, 2048, 4096, 8192, 0, None) == fmm.FMM_EINVAL  # src_start
    assert lib.fmm_p2p(3, 64, 128, 10, 256, 512, 1028, 10, 2048, 4096, 8192, 0, None) == fmm.FMM_EINVAL  # z misaligned
    assert lib.fmm_p2p(3, 64, 128, 10, 256, 512, 1024, 10, 2048, 4096, 8192, 8, None) == fmm.FMM_EINVAL  # flags
    assert lib.fmm_p2p(3, 64, 128, 10, 256, 512, 1024, 10, 2048, 4096, 8192, 32, None) == fmm.FMM_EINVAL
    assert lib.fmm_bin_points(11, 64, 10, 128, 256, 512, None) == fmm.FMM_EINVAL
    # fmm_l2p_binned(level, p, z, n, perm, box_start, L, phi, flags, stream)
    assert lib.fmm_l2p_binned(11, 8, 64, 10, 128, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL   # level
    assert lib.fmm_l2p_binned(3, 65, 64, 10, 128, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL   # p
    assert lib.fmm_l2p_binned(3, 8, 64, -1, 128, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL    # n
    assert lib.fmm_l2p_binned(3, 8, 64, 10, 128, 256, None, 1024, 0, None) == fmm.FMM_EINVAL   # L at level 3
    assert lib.fmm_l2p_binned(3, 8, 64, 10, 128, None, 512, 1024, 0, None) == fmm.FMM_EINVAL   # box_start
    assert lib.fmm_l2p_binned(3, 8, 68, 10, 128, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL    # z misaligned
    assert lib.fmm_l2p_binned(3, 8, 64, 10, 128, 256, 512, 1024, 2, None) == fmm.FMM_EINVAL    # flags
    assert lib.fmm_l2p_binned(3, 8, 64, 0, None, 256, None, None, 0, None) == fmm.FMM_OK       # nothing to do
    # fgt_t2p_binned(g, p, sigma, C, y, n, perm, box_start, G, flags, stream)
    assert lib.fgt_t2p_binned(11, 8, 0.1, 64, 128, 10, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL   # grid
    assert lib.fgt_t2p_binned(3, 6, 0.1, 64, 128, 10, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL    # p
    assert lib.fgt_t2p_binned(3, 8, 0.0, 64, 128, 10, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL    # sigma
    assert lib.fgt_t2p_binned(3, 8, 0.1, 64, 128, 10, None, 512, 1024, 0, None) == fmm.FMM_EINVAL   # perm
    assert lib.fgt_t2p_binned(3, 8, 0.1, 64, 132, 10, 256, 512, 1024, 0, None) == fmm.FMM_EINVAL    # y misaligned
    assert lib.fgt_t2p_binned(3, 8, 0.1, 64, 128, 10, 256, 512, 1024, 4, None) == fmm.FMM_EINVAL    # flags


def test_paper_design_rejects_bad_arguments(fmm):
    lib = fmm.load()
    assert lib.fmm_m2l_paper_design(None, 3, 8, 64, 128, 256, 0, None) == fmm.FMM_EINVAL
    tree = fmm.fmm_build_lists(None, 4)
    assert lib.fmm_m2l_paper_design(tree.handle, 1, 8, 64, 128, 256, 0, None) == fmm.FMM_EINVAL   # level
    assert lib.fmm_m2l_paper_design(tree.handle, 3, 6, 64, 128, 256, 0, None) == fmm.FMM_EINVAL   # p
    assert lib.fmm_m2l_paper_design(tree.handle, 3, 8, 64, 136, 256, 0, None) == fmm.FMM_EINVAL   # misaligned
    assert lib.fmm_m2l_paper_design(tree.handle, 3, 8, 64, 128, None, 0, None) == fmm.FMM_EINVAL  # work
    ptree = fmm.fmm_build_lists(None, 4, periodic=True)
    assert lib.fmm_m2l_paper_design(ptree.handle, 3, 8, 64, 128, 256, 0, None) == fmm.FMM_EUNSUPPORTED


def test_wait_probe_rejects_bad_arguments(fmm):
    lib = fmm.load()
    assert lib.fmm_wait_probe(-1, 1, None) == fmm.FMM_EINVAL
    assert lib.fmm_wait_probe((1 << 22) + 1, 0, None) == fmm.FMM_EINVAL
    assert "cap" in fmm.fmm_last_error()
    assert lib.fmm_wait_probe(8, 2, None) == fmm.FMM_EINVAL
