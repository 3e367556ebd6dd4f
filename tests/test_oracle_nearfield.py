"""Pins for the oracle's near field and its whole FMM (Sec. 2.1 stages 2-5; reading R15).

* At levels 0 and 1 every box is its own box or adjacent, so the near field is
  the direct sum (Eq. n_body) itself.
* Targets placed on the sources: only the coincident source is skipped.
* At a deeper level the near field is the direct sum over exactly the sources
  whose boxes touch the target's (brute force with numpy masks).
* Far field (P2M, M2L over the interaction lists, L2L, L2P) plus near field
  converges to the direct sum as p grows: a near/far partition that dropped or
  double-counted any box would leave an O(1) error.
"""
import numpy as np
import pytest

import workloads


@pytest.fixture(scope="module")
def pts():
    return workloads.uniform_particles(800, np.random.default_rng(71))


def _z(rng, m):
    return rng.random(m) + 1j * rng.random(m)


def test_near_field_at_levels_0_and_1_is_the_direct_sum(orc, pts):
    xy, c = pts
    z = _z(np.random.default_rng(1), 60)
    d = orc.direct(xy, c, z)
    for level in (0, 1):
        np.testing.assert_allclose(orc.p2p_uniform(level, xy, c, z), d, rtol=1e-12, atol=1e-12 * np.abs(d).max())


def test_near_field_skips_only_the_coincident_source(orc, pts):
    xy, c = pts
    z = xy[:40, 0] + 1j * xy[:40, 1]
    got = orc.p2p_uniform(1, xy, c, z)
    for j in range(40):
        keep = np.arange(len(c)) != j
        ref = orc.direct(xy[keep], c[keep], z[j:j + 1])[0]
        assert abs(got[j] - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("level", [2, 3, 4])
def test_near_field_is_the_sum_over_adjacent_boxes(orc, pts, level):
    xy, c = pts
    z = _z(np.random.default_rng(level), 50)
    n = 1 << level
    sb = np.minimum((xy * n).astype(int), n - 1)
    got = orc.p2p_uniform(level, xy, c, z)
    for j in range(len(z)):
        t = (min(int(z[j].real * n), n - 1), min(int(z[j].imag * n), n - 1))
        near = (np.abs(sb[:, 0] - t[0]) <= 1) & (np.abs(sb[:, 1] - t[1]) <= 1)
        ref = np.sum(c[near] / (z[j] - (xy[near, 0] + 1j * xy[near, 1])))
        assert abs(got[j] - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("level", [3, 4])
def test_whole_fmm_converges_to_the_direct_sum(orc, pts, level):
    xy, c = pts
    z = _z(np.random.default_rng(10 + level), 80)
    d = orc.direct(xy, c, z)
    errs = [np.linalg.norm(orc.fmm_potential_uniform(level, p, xy, c, z) - d) / np.linalg.norm(d)
            for p in (4, 8, 16, 24)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[2] < 1e-6 and errs[3] < 1e-9, errs
