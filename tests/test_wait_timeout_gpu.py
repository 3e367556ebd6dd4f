"""Failure detection on the GPU without a fault: a bounded device-side wait runs out.

The tensor-core kernels hand work between warps through shared-memory
mbarriers, and every wait there has a poll limit: a wait that reaches it sets
the timeout bit of the device error word and the kernel returns, so a lost
arrival shows up as FMM_ETIMEOUT from fmm_sync_status instead of a hung GPU.
fmm_wait_probe runs those same wait routines on a barrier that nothing
completes (a flag that nothing sets); this test checks that the waits give up,
that the timeout is reported and cleared, and that the next calls on the same
stream (the probe with an arrival, then a tensor-core M2L) are correct.
"""
import numpy as np
import pytest

import workloads

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


def test_completed_barrier_reports_ok(fmm):
    fmm.fmm_wait_probe(0, arrive=True)
    fmm.fmm_sync_status()


@pytest.mark.parametrize("polls", [1, 64, 4096])
def test_wait_that_nothing_completes_times_out_and_clears(fmm, polls):
    fmm.fmm_wait_probe(polls, arrive=False)
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_sync_status()
    assert e.value.code == fmm.FMM_ETIMEOUT
    # the error word was read and cleared: the stream and the context stay usable
    fmm.fmm_sync_status()
    fmm.fmm_wait_probe(0, arrive=True)
    fmm.fmm_sync_status()


def test_translation_after_a_timeout_is_correct(fmm, orc):
    import torch

    fmm.fmm_wait_probe(16, arrive=False)
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_sync_status()
    assert e.value.code == fmm.FMM_ETIMEOUT
    xy, c = workloads.uniform_particles(3000, np.random.default_rng(77))
    p, L = 16, 4
    Ms = orc.upward_uniform(L, p, xy, c)
    tree = fmm.fmm_build_lists(None, L)
    for prec in (fmm.FMM_TC_BF16X3, fmm.FMM_TC_TF32X3, fmm.FMM_FP32):
        for level in range(2, L + 1):
            Md = torch.from_numpy(orc.scale_me(Ms[level], level).astype(np.complex64)).cuda()
            Ld = torch.empty_like(Md)
            fmm.fmm_m2l(tree, level, p, Md, Ld, prec=prec)
            fmm.fmm_sync_status()
            ref = orc.scale_le(orc.m2l_uniform(level, p, Ms[level]), level)
            got = Ld.cpu().numpy().astype(np.complex128)
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err <= (1e-4 if prec == fmm.FMM_TC_BF16X3 else 1e-5), (prec, level, err)
