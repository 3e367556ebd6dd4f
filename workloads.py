"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds none of the method's arithmetic (no expansions, no
translations): it only draws particle positions and strengths and states the
workload shapes.  Both the FP64 oracle (``oracle/``) and the CUDA library's
tests and benchmark take their inputs from here, so the two sides see the same
numbers without sharing any code that computes the method.

Workloads (all synthetic; the paper's own M2L benchmark is synthetic too and
uses no public dataset):

  m2l_small   4096 points U[0,1)^2, strengths U[-1,1], uniform quadtree to
              level 4, p = 8                               (levels 2..4)
  m2l_scale   2^22 points U[0,1)^2, strengths U[-1,1], uniform quadtree to
              level 8, p = 16, FP32                        (levels 2..8)
  m2l_tc      the m2l_small tree at p = 24 (tensor-core precision study)
  m2l_gmm     2^20 points from a 16-component Gaussian mixture (sigma_c in
              [0.01, 0.05], means U[0.1,0.9]^2), strengths U[-1,1], adaptive
              tree (q = 64, level <= 9), p = 16
  fgt         2^20 Gaussian-mixture sources (same generator), weights U[-1,1],
              bandwidth sigma in {0.05, 0.1, 0.2}, Hermite order p in 8..16
  m2l_batched 256 independent problems: N ~ logU[1e3, 1e5] points U[0,1)^2,
              strengths U[-1,1], uniform quadtree of depth ~ U{4..9}, p ~
              U{6, 8, 12, 16}, FP32, all translated in one launch
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20100913

WORKLOAD_IDS = {"m2l_small": 1, "m2l_scale": 2, "m2l_tc": 3, "m2l_gmm": 4, "fgt": 5, "m2l_batched": 6,
                "fgt_targets": 7}


def rng_for(workload: str, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + WORKLOAD_IDS[workload] + 1000 * salt)


def uniform_particles(n: int, rng: np.random.Generator):
    """n points U[0,1)^2 (float64, interleaved x,y) and strengths U[-1,1]."""
    xy = rng.random((n, 2))
    c = rng.uniform(-1.0, 1.0, n)
    return np.ascontiguousarray(xy), np.ascontiguousarray(c)


def gmm_particles(n: int, rng: np.random.Generator, ncomp: int = 16,
                  sigma_range=(0.01, 0.05), mean_range=(0.1, 0.9)):
    """n points from an equal-weight Gaussian mixture, kept inside [0,1)^2 by rejection."""
    means = rng.uniform(mean_range[0], mean_range[1], (ncomp, 2))
    sig = rng.uniform(sigma_range[0], sigma_range[1], ncomp)
    out = np.empty((0, 2))
    while out.shape[0] < n:
        m = n - out.shape[0]
        comp = rng.integers(0, ncomp, m)
        pts = means[comp] + sig[comp, None] * rng.standard_normal((m, 2))
        ok = np.all((pts >= 0.0) & (pts < 1.0), axis=1)
        out = np.concatenate([out, pts[ok]], axis=0)
    c = rng.uniform(-1.0, 1.0, n)
    return np.ascontiguousarray(out[:n]), np.ascontiguousarray(c)


def batched_problems(nprob: int, rng: np.random.Generator, depths=(4, 9), orders=(6, 8, 12, 16),
                     n_range=(1e3, 1e5)):
    """Shapes of a batch of independent uniform-tree problems: a list of
    dicts (n, max_level, p), n log-uniform in n_range, depth uniform in the
    closed range `depths`, p uniform over `orders`."""
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    out = []
    for _ in range(nprob):
        n = int(round(math.exp(rng.uniform(lo, hi))))
        depth = int(rng.integers(depths[0], depths[1] + 1))
        p = int(orders[int(rng.integers(0, len(orders)))])
        out.append(dict(n=n, max_level=depth, p=p))
    return out


def m2l_levels(max_level: int):
    """Levels that carry M2L translations in a uniform tree: 2..max_level."""
    return list(range(2, max_level + 1))


def fgt_grid_log2(sigma: float) -> int:
    """Boxes per side 2^g with g = ceil(log2(sqrt(2)/sigma)): side/(sqrt(2) sigma) <= 0.5."""
    return int(math.ceil(math.log2(math.sqrt(2.0) / sigma)))


FGT_NCUT = 10  # neighbourhood half-width in boxes (21 x 21 source boxes per target)

CONFIGS = {
    "m2l_small": dict(n=4096, max_level=4, p=8),
    "m2l_scale": dict(n=1 << 22, max_level=8, p=16),
    "m2l_tc": dict(n=4096, max_level=4, p=24),
    "m2l_gmm": dict(n=1 << 20, max_level=9, leaf_cap=64, p=16),
    "fgt": dict(n=1 << 20, sigmas=(0.05, 0.1, 0.2), orders=(8, 12, 16), ncut=FGT_NCUT),
    "m2l_batched": dict(nprob=256, depths=(4, 9), orders=(6, 8, 12, 16), n_range=(1e3, 1e5)),
}
