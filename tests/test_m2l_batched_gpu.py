"""GPU parity of the batched persistent M2L path (fmm_batch_* / fmm_m2l_batched)
against the FP64 oracle, through the C ABI.

Each problem of a batch is an independent uniform tree with its own depth and
p; its result must equal the oracle's M2L of every level (relative L2 of the
scaled local coefficients <= 1e-5, FP32) and, bit for bit, the per-problem
launch fmm_m2l_levels (the same FP32 work unit computes both).
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def fmm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_3457_gb300 import build, fmmgb

    build.build()
    fmmgb.load()
    return fmmgb


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def _host(t):
    return t.cpu().numpy().astype(np.complex128)


def _rel(got, ref):
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


def _small_batch(fmm, orc, seed, nprob=10, depths=(2, 5)):
    """Problems with mixed depth, p and boundary rule; oracle MEs uploaded scaled."""
    rng = np.random.default_rng(seed)
    shapes = workloads.batched_problems(nprob, rng, depths=depths, n_range=(500, 3000))
    probs = []
    for i, sh in enumerate(shapes):
        xy, c = workloads.uniform_particles(sh["n"], rng)
        periodic = bool(i % 3 == 1)
        Ms = orc.upward_uniform(sh["max_level"], sh["p"], xy, c)
        levels = workloads.m2l_levels(sh["max_level"])
        tree = fmm.fmm_build_lists(None, sh["max_level"], periodic=periodic)
        Md = [_dev(orc.scale_me(Ms[l], l)) for l in levels]
        Ld = [m.new_empty(m.shape) for m in Md]
        probs.append(dict(p=sh["p"], tree=tree, levels=levels, Ms=Ms, Md=Md, Ld=Ld, periodic=periodic))
    return probs


def _oracle(orc, pr, l):
    return orc.scale_le(orc.m2l_uniform(l, pr["p"], pr["Ms"][l], pr["periodic"]), l)


def test_batched_one_shot_matches_oracle_and_per_problem_launch(fmm, orc):
    probs = _small_batch(fmm, orc, 11)
    assert len({pr["p"] for pr in probs}) >= 3
    fmm.fmm_m2l_batched([pr["tree"] for pr in probs], [pr["p"] for pr in probs], [pr["Md"] for pr in probs],
                        [pr["Ld"] for pr in probs])
    fmm.fmm_sync_status()
    for pr in probs:
        ref_launch = [m.new_empty(m.shape) for m in pr["Md"]]
        fmm.fmm_m2l_levels(pr["tree"], 2, pr["p"], pr["Md"], ref_launch)
        fmm.fmm_sync_status()
        for l, out, same in zip(pr["levels"], pr["Ld"], ref_launch):
            assert _rel(_host(out), _oracle(orc, pr, l)) <= TOL, (pr["p"], l)
            assert bool((out == same).all()), ("batched differs from fmm_m2l_levels", pr["p"], l)


def test_batched_plan_graph_replay_and_capture_accumulate(fmm, orc):
    import torch

    probs = _small_batch(fmm, orc, 12, nprob=6)
    rng = np.random.default_rng(3)
    X = []
    for pr in probs:
        xs = []
        for l, out in zip(pr["levels"], pr["Ld"]):
            x = (rng.standard_normal(out.shape) + 1j * rng.standard_normal(out.shape)).astype(np.complex64)
            out.copy_(torch.from_numpy(x).cuda())
            xs.append(x.astype(np.complex128))
        X.append(xs)
    plan = fmm.fmm_batch_create([pr["tree"] for pr in probs], [pr["p"] for pr in probs],
                                [pr["Md"] for pr in probs], [pr["Ld"] for pr in probs], accumulate=True)
    info = plan.info()
    assert info["items"] > 0 and info["grid"] > 0
    assert info["translations"] == sum(pr["tree"].translations(l) for pr in probs for l in pr["levels"])
    plan.run()  # instantiated graph of the plan
    plan.run()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run()  # recorded by the caller's capture
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    fmm.fmm_sync_status()
    for pr, xs in zip(probs, X):
        for l, out, x in zip(pr["levels"], pr["Ld"], xs):
            got = (_host(out) - x) / 3.0  # two plan runs + one graph replay (capture itself runs nothing)
            assert _rel(got, _oracle(orc, pr, l)) <= 1e-4, (pr["p"], l)


def test_batched_autotune_writes_no_output(fmm, orc):
    import torch

    probs = _small_batch(fmm, orc, 13, nprob=5)
    for pr in probs:
        for out in pr["Ld"]:
            out.fill_(7.0 + 0j)
    plan = fmm.fmm_batch_create([pr["tree"] for pr in probs], [pr["p"] for pr in probs],
                                [pr["Md"] for pr in probs], [pr["Ld"] for pr in probs], autotune=True)
    torch.cuda.synchronize()
    for pr in probs:
        for out in pr["Ld"]:
            assert bool((out == 7.0).all())
    info = plan.info()
    assert info["tuned"] == 1 and info["tuned_ms"] > 0.0
    plan.run()
    fmm.fmm_sync_status()
    for pr in probs:
        for l, out in zip(pr["levels"], pr["Ld"]):
            assert _rel(_host(out), _oracle(orc, pr, l)) <= TOL, (pr["p"], l)


def test_batched_single_problem_is_fmm_m2l_levels(fmm, orc):
    """A batch of one problem at the headline shape p = 16, depth 6."""
    probs = _small_batch(fmm, orc, 14, nprob=1, depths=(6, 6))
    pr = probs[0]
    plan = fmm.fmm_batch_create([pr["tree"]], [pr["p"]], [pr["Md"]], [pr["Ld"]])
    plan.run()
    ref = [m.new_empty(m.shape) for m in pr["Md"]]
    fmm.fmm_m2l_levels(pr["tree"], 2, pr["p"], pr["Md"], ref)
    fmm.fmm_sync_status()
    for out, same in zip(pr["Ld"], ref):
        assert bool((out == same).all())


@pytest.mark.slow
def test_batched_full_workload(fmm, orc):
    """The 256-problem batch (depth 4..9, p in {6, 8, 12, 16}, 5.7M points, 582M
    translations) in one autotuned launch: every level <= 5 in full, deeper
    levels on sampled targets (corners + random boxes)."""
    cfg = workloads.CONFIGS["m2l_batched"]
    rng = workloads.rng_for("m2l_batched")
    shapes = workloads.batched_problems(cfg["nprob"], rng, depths=cfg["depths"], orders=cfg["orders"],
                                        n_range=cfg["n_range"])
    trees, ps, Mds, Lds, refs = [], [], [], [], []
    srng = np.random.default_rng(99)
    for sh in shapes:
        xy, c = workloads.uniform_particles(sh["n"], rng)
        L, p = sh["max_level"], sh["p"]
        Ms = orc.upward_uniform(L, p, xy, c)
        levels = workloads.m2l_levels(L)
        trees.append(fmm.fmm_build_lists(None, L))
        ps.append(p)
        Mds.append([_dev(orc.scale_me(Ms[l], l)) for l in levels])
        Lds.append([m.new_empty(m.shape) for m in Mds[-1]])
        ref = {}
        for l in levels:
            if l <= 5:
                ref[l] = (None, orc.scale_le(orc.m2l_uniform(l, p, Ms[l]), l))
            else:
                n = 1 << l
                tg = np.unique(np.concatenate([[0, n - 1, n * (n - 1), n * n - 1], srng.integers(0, n * n, 48)]))
                ref[l] = (tg, orc.scale_le(orc.m2l_uniform_targets(l, p, Ms[l], tg), l))
        refs.append(ref)
        del Ms
    plan = fmm.fmm_batch_create(trees, ps, Mds, Lds, autotune=True)
    assert plan.info()["translations"] == 582342588
    plan.run()
    fmm.fmm_sync_status()
    worst = 0.0
    for levels_out, ref, L_levels in zip(Lds, refs, Mds):
        for i, out in enumerate(levels_out):
            l = i + 2
            tg, r = ref[l]
            got = _host(out) if tg is None else _host(out)[tg]
            worst = max(worst, _rel(got, r))
    assert worst <= TOL, worst


_TUNE_CHILD = r'''
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import workloads
from paper_1009_3457_gb300 import fmmgb
fmmgb.load()
rng = np.random.default_rng(2024)
shapes = workloads.batched_problems(6, rng, depths=(3, 5), n_range=(500, 2000))
trees, ps, Ms, Ls = [], [], [], []
for sh in shapes:
    L, p = sh["max_level"], sh["p"]
    xy, c = workloads.uniform_particles(sh["n"], rng)
    M = {l: torch.empty((4 ** l, p), dtype=torch.complex64, device="cuda") for l in range(2, L + 1)}
    fmmgb.fmm_p2m(L, p, torch.from_numpy(xy).cuda(), torch.from_numpy(c).cuda(), M[L])
    for l in range(L, 2, -1):
        fmmgb.fmm_m2m(l, p, M[l], M[l - 1])
    trees.append(fmmgb.fmm_build_lists(None, L))
    ps.append(p)
    Ms.append([M[l] for l in range(2, L + 1)])
    Ls.append([torch.empty_like(M[l]) for l in range(2, L + 1)])
infos = []
for k in range(2):  # the second plan of this process reuses the first one's choice
    plan = fmmgb.fmm_batch_create(trees, ps, Ms, Ls, autotune=True)
    plan.run()
    infos.append(plan.info())
worst = 0.0
for tr, p, m, l in zip(trees, ps, Ms, Ls):
    ref = [torch.empty_like(x) for x in m]
    fmmgb.fmm_m2l_levels(tr, 2, p, m, ref)
    for a, b in zip(l, ref):
        worst = max(worst, float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)))
fmmgb.fmm_sync_status()
print(json.dumps({"infos": infos, "worst": worst}))
'''


def test_batched_autotune_choice_persists_across_processes(fmm, tmp_path):
    """FMM_BATCH_AUTOTUNE stores its choice (launch configuration and work-unit variant) in the
    cache file; a second plan in the same process and every plan of a later process reuse it
    without timing, and the tuned plans agree with fmm_m2l_levels."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.json"
    env = dict(os.environ, FMMGB_TUNE_CACHE=str(cache))
    runs = []
    for _ in range(2):
        out = subprocess.run([sys.executable, "-c", _TUNE_CHILD, root], env=env, capture_output=True, text=True,
                             timeout=600)
        assert out.returncode == 0, out.stderr[-2000:]
        runs.append(json.loads(out.stdout.strip().splitlines()[-1]))
    first, second = runs
    a, b = first["infos"]
    assert a["tuned"] == 1 and a["from_cache"] == 0 and a["tuned_ms"] > 0.0
    assert b["tuned"] == 1 and b["from_cache"] == 1
    text = cache.read_text()
    assert '"variant"' in text and "|fp32|" in text
    for info in second["infos"]:
        assert info["from_cache"] == 1
        for k in ("grid", "chunk", "persistent", "variant", "form", "loads"):
            assert info[k] == a[k], (k, info[k], a[k])
    assert a["form"] in (-1, 0, 1, 2) and a["loads"] in (2, 3)
    assert first["worst"] <= TOL and second["worst"] <= TOL
