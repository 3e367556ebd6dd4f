"""GPU checks of the host-resident M2L pipeline (fmm_host_stream_*) through the C ABI:
every step's LEs, copied back to host memory, equal fmm_m2l_levels on the same MEs
in device memory (bit for bit in FP32; the tensor-core kernel adds the parts of a
tile cut between CTAs in whatever order they finish, so there to FP32 rounding),
and lie within the precision's bar of the FP64 oracle (Sec. 4.1, Eq. M2Lmat summed
over the interaction lists)."""
import ctypes

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


def _rand_levels(rng, levels, p):
    import torch

    return [torch.from_numpy((rng.standard_normal((4 ** l, p)) + 1j * rng.standard_normal((4 ** l, p)))
                             .astype(np.complex64)) for l in levels]


def _same(fmm, prec, a, b):
    import torch

    if prec == fmm.FMM_FP32:
        return torch.equal(a, b)
    return bool(torch.isfinite(a).all()) and float((a - b).abs().norm() / b.abs().norm()) <= 1e-6


def _direct(fmm, tree, lmin, p, prec, Ms):
    """fmm_m2l_levels on device copies of the same MEs."""
    import torch

    Md = [m.cuda() for m in Ms]
    Ld = [torch.empty_like(m) for m in Md]
    fmm.fmm_m2l_levels(tree, lmin, p, Md, Ld, prec=prec)
    fmm.fmm_sync_status()
    return [x.cpu() for x in Ld]


@pytest.mark.parametrize("depth,prec_name,p,tol", [
    (1, "FMM_FP32", 8, 1e-5),
    (3, "FMM_FP32", 12, 1e-5),
    (2, "FMM_TC_BF16X3", 16, 1e-4),
    (2, "FMM_TC_TF32X3", 16, 1e-5),
    (2, "FMM_FP32", 24, 1e-5),
    (4, "FMM_TC_BF16X3", 24, 1e-4),
])
def test_steps_match_direct_calls_and_oracle(fmm, orc, depth, prec_name, p, tol):
    """Seven steps, more than the buffer sets, rotating between pageable per-level tensors,
    one pinned flat tensor per direction, and separately pinned per-level tensors."""
    import torch

    prec = getattr(fmm, prec_name)
    L = 5
    levels = list(range(2, L + 1))
    tree = fmm.fmm_build_lists(None, L)
    hs = fmm.fmm_host_stream_create(tree, 2, L, p, prec, depth)
    info = hs.info()
    entries = p * sum(4 ** l for l in levels)
    assert (info["entries"], info["bytes_in"], info["bytes_out"]) == (entries, 8 * entries, 8 * entries)
    assert (info["depth"], info["lmin"], info["lmax"], info["p"], info["prec"]) == (depth, 2, L, p, prec)
    rng = np.random.default_rng(40 + depth + p)
    steps = []
    for i in range(7):
        Ms = _rand_levels(rng, levels, p)
        if i % 3 == 1:  # one pinned buffer per direction: one copy each way (FMM_HOST_CONTIGUOUS)
            flat_in = torch.cat([m.reshape(-1) for m in Ms]).pin_memory()
            flat_out = torch.full((entries,), complex(np.nan, np.nan), dtype=torch.complex64).pin_memory()
            hs.submit(flat_in, flat_out)
            Min, Lout = flat_in, _views(flat_out, levels, p)
        elif i % 3 == 2:  # every level pinned on its own (neighbouring allocations, one copy each)
            Min = [m.pin_memory() for m in Ms]
            Lout = [torch.full_like(m, complex(np.nan, np.nan)).pin_memory() for m in Ms]
            hs.submit(Min, Lout)
        else:  # pageable
            Min = Ms
            Lout = [torch.full_like(m, complex(np.nan, np.nan)) for m in Ms]
            hs.submit(Min, Lout)
        steps.append((Ms, Min, Lout))  # the host buffers stay alive until the sync
    assert hs.info()["steps"] == 7
    hs.sync()
    for Ms, _, Lout in steps:
        for a, b in zip(Lout, _direct(fmm, tree, 2, p, prec, Ms)):
            assert _same(fmm, prec, a, b)
    Ms, _, Lout = steps[3]
    for l, m, out in zip(levels, Ms, Lout):
        ref = orc.scale_le(orc.m2l_uniform(l, p, orc.unscale_me(m.numpy().astype(np.complex128), l)), l)
        got = out.numpy().astype(np.complex128)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol, l


def _views(flat, levels, p):
    out, off = [], 0
    for l in levels:
        n = 4 ** l * p
        out.append(flat[off:off + n].view(4 ** l, p))
        off += n
    return out


def test_periodic_tree_levels_from_zero(fmm):
    """Levels 0..4 of a periodic tree: levels 0 and 1 (no interaction list) come back zero."""
    import torch

    p = 8
    tree = fmm.fmm_build_lists(None, 4, periodic=True)
    levels = list(range(0, 5))
    hs = fmm.fmm_host_stream_create(tree, 0, 4, p)
    rng = np.random.default_rng(5)
    Ms = _rand_levels(rng, levels, p)
    Lout = [torch.full_like(m, 1.0) for m in Ms]
    hs.submit(Ms, Lout)
    hs.sync()
    assert not Lout[0].any() and not Lout[1].any()
    for a, b in zip(Lout, _direct(fmm, tree, 0, p, fmm.FMM_FP32, Ms)):
        assert torch.equal(a, b)


def test_adaptive_tree(fmm):
    """A Gaussian-mixture adaptive tree: existing boxes match the direct call exactly."""
    import torch

    import workloads

    xy, _ = workloads.gmm_particles(20000, np.random.default_rng(8))
    p, L = 16, 7
    tree = fmm.fmm_build_lists(xy, L, leaf_cap=64)
    levels = list(range(2, tree.max_level + 1))
    hs = fmm.fmm_host_stream_create(tree, 2, tree.max_level, p, fmm.FMM_FP32, 2)
    rng = np.random.default_rng(9)
    Ms = _rand_levels(rng, levels, p)
    Lout = [torch.zeros_like(m) for m in Ms]
    hs.submit(Ms, Lout)
    hs.sync()
    ref = _direct(fmm, tree, 2, p, fmm.FMM_FP32, Ms)
    for l, a, b in zip(levels, Lout, ref):
        ex = torch.from_numpy(tree.exists(l))
        assert torch.equal(a[ex], b[ex]), l


def test_bad_submissions_enqueue_nothing(fmm):
    """Overlapping M and L, or a NULL level pointer, are refused before any copy; the
    pipeline then still runs a good step."""
    import torch

    p, L = 8, 3
    tree = fmm.fmm_build_lists(None, L)
    levels = [2, 3]
    hs = fmm.fmm_host_stream_create(tree, 2, L, p)
    lib = fmm.load()
    Ms = _rand_levels(np.random.default_rng(2), levels, p)
    mp = (ctypes.c_void_p * 2)(*[m.data_ptr() for m in Ms])
    lp_overlap = (ctypes.c_void_p * 2)(Ms[1].data_ptr() + 64, Ms[0].data_ptr())
    assert lib.fmm_host_stream_submit(hs.handle, mp, lp_overlap, 0) == fmm.FMM_EINVAL
    assert "overlap" in fmm.fmm_last_error()
    lp_null = (ctypes.c_void_p * 2)(None, Ms[0].data_ptr() + (1 << 30))
    assert lib.fmm_host_stream_submit(hs.handle, mp, lp_null, 0) == fmm.FMM_EINVAL
    # one flat buffer each way: the L buffer starts inside the M buffer's span
    flat = torch.zeros(2 * p * (16 + 64), dtype=torch.complex64)
    m1 = (ctypes.c_void_p * 1)(flat.data_ptr())
    l1 = (ctypes.c_void_p * 1)(flat.data_ptr() + 8 * p * 80 - 8)
    assert lib.fmm_host_stream_submit(hs.handle, m1, l1, fmm.FMM_HOST_CONTIGUOUS) == fmm.FMM_EINVAL
    Lgood = [torch.empty_like(m) for m in Ms]
    lp = (ctypes.c_void_p * 2)(*[x.data_ptr() for x in Lgood])
    assert lib.fmm_host_stream_submit(hs.handle, mp, lp, 16) == fmm.FMM_EINVAL  # unknown flag
    assert hs.info()["steps"] == 0
    Lout = [torch.empty_like(m) for m in Ms]
    hs.submit(Ms, Lout)
    hs.sync()
    for a, b in zip(Lout, _direct(fmm, tree, 2, p, fmm.FMM_FP32, Ms)):
        assert torch.equal(a, b)
