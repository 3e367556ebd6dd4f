"""CPU check of the far-field objective's tensor-op stages (P2M scaling, L2L,
L2P in paper_1009_3457_gb300.farfield) against the FP64 oracle's objective:
the M2L stage, which on a GPU runs in the library's kernels, is replaced here,
inside this test only, by the oracle's V-list M2L on the same tree."""
import numpy as np
import pytest

import workloads


@pytest.fixture(scope="module")
def fmm():
    from paper_1009_3457_gb300 import build, fmmgb

    build.build()
    fmmgb.load()
    return fmmgb


def test_far_field_glue_matches_oracle_objective(fmm, orc, monkeypatch):
    import torch

    from paper_1009_3457_gb300 import farfield

    rng = np.random.default_rng(44)
    xy, c = workloads.gmm_particles(3000, rng, ncomp=4)
    q, L, p = 24, 6, 12
    tree = fmm.fmm_build_lists(xy, L, leaf_cap=q)
    otree = orc.adaptive_tree(xy, q, L)
    z = rng.random(200) + 1j * rng.random(200)
    w = rng.uniform(-1, 1, 200)

    def oracle_m2l(tr, p_, Ms):
        out = []
        for i, M in enumerate(Ms):
            l = i + 2
            Mp = orc.unscale_me(M.numpy().astype(np.complex128), l)
            out.append(torch.from_numpy(orc.scale_le(orc.m2l_adaptive(otree, l, p_, Mp), l).astype(np.complex64)))
        return tuple(out)

    monkeypatch.setattr(farfield, "m2l_levels", oracle_m2l)
    xyt = torch.from_numpy(xy)
    leaf = farfield.leaf_boxes(tree, xyt)
    zl = farfield.leaf_boxes(tree, torch.from_numpy(np.stack([z.real, z.imag], 1)))
    J = float(farfield.far_field_objective(tree, p, xyt, torch.from_numpy(c), leaf, torch.from_numpy(z), zl,
                                           torch.from_numpy(w)))
    oleaf = orc.leaf_boxes(otree, xy)
    ozl = orc.leaf_boxes(otree, np.stack([z.real, z.imag], 1))
    assert (leaf[0].numpy() == oleaf[0]).all() and (leaf[1].numpy() == oleaf[1]).all()
    assert (zl[0].numpy() == ozl[0]).all() and (zl[1].numpy() == ozl[1]).all()
    Jo = orc.far_field_objective(otree, p, xy, c, oleaf, z, ozl, w)
    assert abs(J - Jo) <= 1e-5 * abs(Jo), (J, Jo)
