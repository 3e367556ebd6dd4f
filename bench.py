"""Benchmark of the M2L translation path on GB300.

Workload (one "step"): the FMM downward-sweep M2L of a uniform quadtree to
level 8 built from 2^22 points U[0,1)^2 with strengths U[-1,1], p = 16, FP32,
every interaction-list translation of levels 2..8 (2,316,900 translations),
one fmm_m2l launch per level, reduction fused (Sec. 4.1).  Inputs (radius-
scaled MEs) are built on the device by fmm_p2m / fmm_m2m before timing.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is whole-job translations/s with inputs resident
in HBM; `e2e` is the same metric with a pinned-host -> device copy of the
step's MEs and a device -> host copy of its LEs inside the timed region
(the library's fmm_host_stream_submit, one C call per step with host
buffers: consecutive steps overlap on its three streams).
Under torchrun each rank runs an independent replica of the workload (the
single-tree M2L step has no cross-GPU exchange: replicas only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from paper_1009_3457_gb300 import metrics  # noqa: E402

WORKLOAD = "m2l_scale"
CFG = workloads.CONFIGS[WORKLOAD]
P = CFG["p"]
MAXL = CFG["max_level"]
LEVELS = workloads.m2l_levels(MAXL)
NTR = sum(metrics.uniform_translations(l) for l in LEVELS)
METRIC = "M2L translations/s"
UNIT = "translations/s"
CONFIG = {
    "workload": "plain M2L at scale: 2^22 points U[0,1)^2, strengths U[-1,1], uniform quadtree to level 8, "
                "p=16, FP32 complex coefficients, all interaction-list translations of levels 2-8 "
                "(one multi-level launch; one-launch-per-level timing under rows)",
    "points": CFG["n"], "max_level": MAXL, "p": P, "translations_per_step": NTR,
    "levels": f"{LEVELS[0]}-{LEVELS[-1]}",
    "l2": "flushed between timed device-resident steps (256 MiB write); in e2e every step's MEs arrive by copy",
    "timing": "device-resident step captured once as a CUDA graph (one kernel) and replayed between "
              "CUDA events; e2e makes one C call per step with host buffers (fmm_host_stream_submit), MEs "
              "in from and LEs out to pinned host memory, consecutive steps overlapped on the library's "
              "three streams",
    "parallelism": "replicas",
}
FP32_LANES_PER_SM = 128
def fgt_h2t_launches(g: int) -> int:
    """Kernel launches of one fgt_h2t call: one fused launch for grids up to 16 x 16, two passes beyond."""
    return 1 if g <= 4 else 2
# replaced at start-up by the device's own SM count and maximum SM clock (device_peaks)
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def _measured_bf16_tflops() -> float:
    """Dense BF16 GEMM throughput measured on the GB300s (burst), else the fallback figure."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


BF16_PEAK_TFLOPS = _measured_bf16_tflops()
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rate (per GPU)


def device_peaks(torch, dev):
    """SM count (device attribute), maximum SM clock (nvidia-smi clocks.max.sm) and a measured FP32
    throughput (cuBLAS SGEMM 8192^3 with TF32 off, best of 5) of the current GPU; sets the globals
    the ALU roofline uses."""
    global SM_COUNT, SM_MAX_MHZ
    SM_COUNT = torch.cuda.get_device_properties(dev).multi_processor_count
    src = "nvidia-smi clocks.max.sm"
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(dev.index or 0), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        SM_MAX_MHZ = float(out.stdout.strip().splitlines()[0])
    except Exception:
        src = "fallback 2070 MHz (nvidia-smi unavailable)"
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        n = 8192
        a = torch.randn((n, n), device=dev)
        b = torch.randn((n, n), device=dev)
        c = torch.empty((n, n), device=dev)
        torch.matmul(a, b, out=c)
        best = float("inf")
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        sgemm = 2.0 * n ** 3 / (best * 1e-3) / 1e12
        del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    return {"sm_count": SM_COUNT, "sm_max_mhz": SM_MAX_MHZ, "clock_source": src,
            "alu_peak_tflops": alu_peak_tflops(), "sgemm_fp32_tflops": sgemm}


def alu_peak_tflops() -> float:
    """FP32 FMA peak from unit counts and clock: SMs x 128 lanes x 2 flop x max SM clock."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline_run(levels=None):
    """The FP64 oracle as it stands (single thread) on the whole workload: translations/s."""
    import oracle

    levels = levels or LEVELS
    xy, c = workloads.uniform_particles(CFG["n"], workloads.rng_for(WORKLOAD))
    Ms = oracle.upward_uniform(MAXL, P, xy, c)
    t0 = time.perf_counter()
    ntr = 0
    for l in levels:
        oracle.m2l_uniform(l, P, Ms[l])
        ntr += metrics.uniform_translations(l)
    dt = time.perf_counter() - t0
    return ntr / dt, dt, ntr


# --- the oracle on all host cores: worker processes (spawned, so safe after CUDA
# work), each rebuilding the seeded MEs once and translating slices of targets
_ORC_MES = None


def _oracle_worker_init(maxl, p):
    global _ORC_MES
    import oracle

    xy, c = workloads.uniform_particles(CFG["n"], workloads.rng_for(WORKLOAD))
    _ORC_MES = oracle.upward_uniform(maxl, p, xy, c)


def _oracle_worker_task(task):
    import oracle

    level, t0, t1 = task
    oracle.m2l_uniform_targets(level, P, _ORC_MES[level], np.arange(t0, t1, dtype=np.int64))
    return t1 - t0


class OraclePool:
    """The unmodified FP64 oracle run in `cores` processes over disjoint target slices."""

    def __init__(self, cores=None):
        import multiprocessing as mp

        self.cores = cores or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init, initargs=(MAXL, P))
        self.pool.map(_oracle_worker_task, [(2, 0, 1)] * self.cores)  # workers ready

    def step(self, levels):
        tasks = []
        for l in levels:
            nb = 4 ** l
            chunk = max(1, nb // (4 * self.cores))
            tasks += [(l, t0, min(nb, t0 + chunk)) for t0 in range(0, nb, chunk)]
        self.pool.map(_oracle_worker_task, tasks, chunksize=1)

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline_all_cores(levels=None, steps=3, warmup=1):
    """Translations/s of the oracle over all host cores, timed the way the reference arm times it:
    `warmup` whole steps untimed, then `steps` whole steps; rate = translations / total time."""
    levels = levels or LEVELS
    op = OraclePool()
    try:
        for _ in range(warmup):
            op.step(levels)
        times = []
        for _ in range(steps):
            t0 = time.perf_counter()
            op.step(levels)
            times.append(time.perf_counter() - t0)
    finally:
        op.close()
    ntr = sum(metrics.uniform_translations(l) for l in levels)
    return ntr * steps / sum(times), times, ntr, op.cores


def tc_accuracy_vs_oracle(torch, fmmgb, dev):
    """Coefficient error of the FP32 and the tensor-core M2L against the FP64 oracle on the
    precision workload's tree (4096 points, uniform to level 4): relative L2 of the radius-scaled
    LEs, max over levels 2-4; at p = 24 FP32 and BF16x3, at p = 16 FP32, BF16x3 and TF32x3.  Part
    of the CPU-baseline leg (the one leg of this benchmark that runs the oracle)."""
    import oracle

    cfg = workloads.CONFIGS["m2l_tc"]
    L = cfg["max_level"]
    xy, c = workloads.uniform_particles(cfg["n"], workloads.rng_for("m2l_small"))  # the m2l_small points
    tree = fmmgb.fmm_build_lists(None, L)

    def worst(p, Ms, prec):
        w = 0.0
        for level in workloads.m2l_levels(L):
            ref = oracle.scale_le(oracle.m2l_uniform(level, p, Ms[level]), level)
            Md = torch.from_numpy(oracle.scale_me(Ms[level], level).astype(np.complex64)).to(dev)
            Ld = torch.empty_like(Md)
            fmmgb.fmm_m2l(tree, level, p, Md, Ld, prec=prec)
            got = Ld.cpu().numpy().astype(np.complex128)
            w = max(w, float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
        return w

    p = cfg["p"]
    Ms = oracle.upward_uniform(L, p, xy, c)
    out = {"tree": f"{cfg['n']} points U[0,1)^2, uniform to level {L}, p = {p}, levels 2-{L}",
           "fp32_rel_l2": worst(p, Ms, fmmgb.FMM_FP32), "bf16x3_rel_l2": worst(p, Ms, fmmgb.FMM_TC_BF16X3)}
    Ms16 = oracle.upward_uniform(L, 16, xy, c)
    out["p16"] = {"fp32_rel_l2": worst(16, Ms16, fmmgb.FMM_FP32),
                  "bf16x3_rel_l2": worst(16, Ms16, fmmgb.FMM_TC_BF16X3),
                  "tf32x3_rel_l2": worst(16, Ms16, fmmgb.FMM_TC_TF32X3)}
    fmmgb.fmm_sync_status()
    out.update({"bar_fp32": 1e-5, "bar_tc": "oracle truncation + 1e-4 (TF32x3 is tested at the FP32 bar)",
                "metric": "relative L2 of radius-scaled LEs vs FP64 oracle, max over levels"})
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle

    # one step = the whole workload (levels 2..8, 2,316,900 translations) on every host core
    op = OraclePool()
    ntr_step = NTR
    try:
        for _ in range(args.warmup):
            op.step(LEVELS)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            op.step(LEVELS)
            times.append(time.perf_counter() - t0)
    finally:
        op.close()
    tot = sum(times)
    value = ntr_step * args.steps / tot
    sample = (f"the whole step (levels 2-8, {ntr_step} translations) per step, FP64 oracle in {op.cores} "
              f"processes over disjoint target slices")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": CONFIG,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": op.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


def _fgt_hermite_setup(torch, fmmgb, dev, fxd, fqd, fyd, sigma, fp):
    """Sources binned and P2H'd, targets binned, for Hermite evaluation on the grid of sigma."""
    g = workloads.fgt_grid_log2(sigma)
    nb = 4 ** g

    def bins(pts):
        perm = torch.empty(pts.shape[0], dtype=torch.int32, device=dev)
        start = torch.empty(nb + 1, dtype=torch.int32, device=dev)
        work = torch.empty(nb, dtype=torch.int32, device=dev)
        fmmgb.fgt_bin_points(g, pts, perm, start, work)
        return perm, start, work

    sperm, sstart, swork = bins(fxd)
    A = torch.empty((nb, fp, fp), dtype=torch.float32, device=dev)
    fmmgb.fgt_p2h_binned(g, fp, sigma, fxd, fqd, sperm, A)
    tperm, tstart, twork = bins(fyd)
    G = torch.empty(fyd.shape[0], dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    counts = torch.diff(tstart).cpu().numpy()
    nonempty = (torch.diff(sstart) > 0).cpu().numpy()
    pairs = metrics.fgt_h2p_pairs(g, workloads.FGT_NCUT, counts, nonempty)
    return dict(g=g, A=A, G=G, sperm=sperm, sstart=sstart, swork=swork, tperm=tperm, tstart=tstart,
                twork=twork, pairs=pairs)


def _fgt_hermite_rows(torch, fmmgb, dev, fxd, fqd, args, stream, flush):
    """FGT Hermite evaluation (Sec. 4.2, Eq. hermite) at 2^20 Gaussian-mixture targets from the
    Hermite coefficients of 2^20 mixture sources, n_cut = 10, for every sigma and order; and the
    whole transform through it (bin sources, P2H, bin targets, evaluate) at sigma 0.05, p 16."""
    fcfg = workloads.CONFIGS["fgt"]
    ncut = fcfg["ncut"]
    fy, _ = workloads.gmm_particles(fcfg["n"], workloads.rng_for("fgt_targets"))
    fyd = torch.from_numpy(fy).to(dev)
    peak = alu_peak_tflops()
    rows = {}
    for sigma in fcfg["sigmas"]:
        for fp in fcfg["orders"]:
            st = _fgt_hermite_setup(torch, fmmgb, dev, fxd, fqd, fyd, sigma, fp)
            g = st["g"]

            def h2p():
                fmmgb.fgt_h2p(g, ncut, fp, sigma, st["A"], fyd, st["tperm"], st["tstart"], st["G"])

            ms = statistics.median(_timed(torch, _graph(torch, h2p), args.steps, stream, flush))
            flops = st["pairs"] * metrics.fgt_h2p_flops_per_pair(fp)
            rows[f"fgt_h2p_sigma{sigma}_p{fp}"] = {
                "ms": ms, "targets": int(fcfg["n"]), "targets_per_s": fcfg["n"] / (ms * 1e-3),
                "box_pairs": st["pairs"], "gflops": flops / (ms * 1e-3) / 1e9,
                "alu_frac": flops / (ms * 1e-3) / 1e12 / peak, "launches": 1, "grid": f"{1 << g}^2"}
            if fp == 16:
                for pname, prec, prods in (("bf16x3", fmmgb.FMM_TC_BF16X3, 3), ("bf16", fmmgb.FMM_TC_BF16, 1)):
                    Gt = torch.empty_like(st["G"])

                    def h2p_tc():
                        fmmgb.fgt_h2p(g, ncut, fp, sigma, st["A"], fyd, st["tperm"], st["tstart"], Gt, prec=prec)

                    ms_tc = statistics.median(_timed(torch, _graph(torch, h2p_tc), args.steps, stream, flush))
                    counts = torch.diff(st["tstart"]).cpu().numpy()
                    mma = metrics.fgt_h2p_tc_mma_flops(g, ncut, counts, products=prods)
                    rel = float(torch.linalg.vector_norm((Gt - st["G"]).double())
                                / torch.linalg.vector_norm(st["G"].double()))
                    useful = st["pairs"] * metrics.fgt_h2p_flops_per_pair(fp) * prods  # non-empty pairs only
                    rows[f"fgt_h2p_tc_{pname}_sigma{sigma}_p16"] = {
                        "ms": ms_tc, "targets_per_s": fcfg["n"] / (ms_tc * 1e-3), "launches": 3,
                        "tensor_tflops": mma / (ms_tc * 1e-3) / 1e12,
                        "tensor_frac_of_measured_bf16": mma / (ms_tc * 1e-3) / 1e12 / BF16_PEAK_TFLOPS,
                        "useful_tflops": useful / (ms_tc * 1e-3) / 1e12,
                        "useful_frac": useful / (ms_tc * 1e-3) / 1e12 / BF16_PEAK_TFLOPS,
                        "speedup_vs_fp32": ms / ms_tc, "rel_l2_vs_fp32_path": rel,
                        "note": "claim table, BF16 image of A, tcgen05 kernel"}
            if sigma == 0.05 and fp == 16:
                def transform():
                    fmmgb.fgt_bin_points(g, fxd, st["sperm"], st["sstart"], st["swork"])
                    fmmgb.fgt_p2h_binned(g, fp, sigma, fxd, fqd, st["sperm"], st["A"])
                    fmmgb.fgt_bin_points(g, fyd, st["tperm"], st["tstart"], st["twork"])
                    fmmgb.fgt_h2p(g, ncut, fp, sigma, st["A"], fyd, st["tperm"], st["tstart"], st["G"])

                ms_all = statistics.median(_timed(torch, _graph(torch, transform), args.steps, stream, flush))
                rows["fgt_hermite_transform_sigma0.05_p16"] = {
                    "ms": ms_all, "sources": int(fcfg["n"]), "targets": int(fcfg["n"]),
                    "points_per_s": fcfg["n"] / (ms_all * 1e-3), "launches": 8,
                    "note": "fgt_bin_points (3 kernels) x 2, fgt_p2h_binned, fgt_h2p; mixture targets"}
            del st
    fmmgb.fmm_sync_status()
    return rows


SUMMARY_ROWS = ("m2l_adjoint_fp32_levels_2_8", "m2l_tc_bf16x3_levels_2_8", "m2l_tc_tf32x3_levels_2_8",
                "m2l_fp32_p24_levels_2_8",
                "m2l_tc_bf16x3_p24_levels_2_8", "m2l_adaptive_gmm_levels_2_9", "m2l_tc_bf16x3_adaptive_gmm_levels_2_9",
                "m2l_batched_256_problems",
                "m2l_paper_design_levels_2_8", "fgt_h2t_sigma0.05_p16", "fgt_h2t_tc_bf16x3_sigma0.05_p16",
                "fgt_h2t_sigma0.1_p16", "fgt_h2t_sigma0.2_p16", "fgt_h2p_sigma0.05_p16", "fgt_h2p_tc_bf16x3_sigma0.05_p16",
                "fmm_p2p_level8", "fmm_potential_level8_p16", "far_field_gradient_gmm")


def summarise(rows: dict) -> dict:
    """The main rows in short (time and a headline fraction), 4 significant digits: the end of the
    printed line, so a reader of its last few kilobytes sees them."""
    keep = ("ms", "alu_frac", "sfu_frac", "tensor_frac", "tensor_frac_of_measured_bf16", "useful_frac",
            "speedup_vs_fp32", "fused_speedup")
    out = {}
    for name in SUMMARY_ROWS:
        r = rows.get(name)
        if r:
            out[name] = {k: float(f"{r[k]:.4g}") for k in keep if isinstance(r.get(k), (int, float))}
    return out


def _traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, or None if the kernel source changed since."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            rec = json.load(f)[kernel]
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        return rec["dram_bytes_per_launch"] if h.hexdigest().startswith(rec["sources_sha256_prefix"]) else None
    except Exception:
        return None


def _graph(torch, fn):
    """fn() (library calls on the current stream) captured once as a CUDA graph after a warm
    call; returns the replay, so that the device time between events excludes host enqueue."""
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        fn()
    torch.cuda.synchronize()
    _graph.keep.append(g)
    return g.replay


_graph.keep = []


def _timed(torch, fn, steps, stream, flush):
    """Per-step CUDA-event durations (ms) of fn() on `stream`, L2 flushed between steps."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        evs[i][0].record(stream)
        fn()
        evs[i][1].record(stream)
        flush.zero_()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def _batched_setup(torch, fmmgb, dev, autotune=True, nprob=None):
    """The 256-problem batch (or its first nprob problems): particles -> device
    P2M/M2M per problem (untimed), one plan over every problem's levels 2..depth."""
    cfg = workloads.CONFIGS["m2l_batched"]
    rng = workloads.rng_for("m2l_batched")
    shapes = workloads.batched_problems(cfg["nprob"], rng, depths=cfg["depths"], orders=cfg["orders"],
                                        n_range=cfg["n_range"])[:nprob]
    trees, ps, Ms, Ls = [], [], [], []
    flops = 0
    for sh in shapes:
        L, p = sh["max_level"], sh["p"]
        xy, c = workloads.uniform_particles(sh["n"], rng)
        xyd = torch.from_numpy(xy).to(dev)
        cd = torch.from_numpy(c).to(dev)
        M = {l: torch.empty((4 ** l, p), dtype=torch.complex64, device=dev) for l in range(2, L + 1)}
        fmmgb.fmm_p2m(L, p, xyd, cd, M[L])
        for l in range(L, 2, -1):
            fmmgb.fmm_m2m(l, p, M[l], M[l - 1])
        tree = fmmgb.fmm_build_lists(None, L)
        trees.append(tree)
        ps.append(p)
        Ms.append([M[l] for l in range(2, L + 1)])
        Ls.append([torch.empty_like(M[l]) for l in range(2, L + 1)])
        flops += sum(tree.translations(l) for l in range(2, L + 1)) * metrics.m2l_flops_per_translation(p)
    torch.cuda.synchronize()
    plan = fmmgb.fmm_batch_create(trees, ps, Ms, Ls, autotune=autotune)
    return dict(plan=plan, trees=trees, ps=ps, Ms=Ms, Ls=Ls, flops=flops, info=plan.info())


def run_ours(args):
    import torch

    from paper_1009_3457_gb300 import dist as fdist
    from paper_1009_3457_gb300 import fmmgb

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fmmgb.load()
    fmmgb.fmm_prepare(P)
    stream = torch.cuda.current_stream()
    peaks = device_peaks(torch, dev)

    # --- inputs: particles -> device P2M/M2M (untimed) ---
    xy, c = workloads.uniform_particles(CFG["n"], workloads.rng_for(WORKLOAD))
    xyd = torch.from_numpy(xy).to(dev)
    cd = torch.from_numpy(c).to(dev)
    tree = fmmgb.fmm_build_lists(None, MAXL)
    M = {l: torch.empty((4 ** l, P), dtype=torch.complex64, device=dev) for l in LEVELS}
    Lx = {l: torch.empty((4 ** l, P), dtype=torch.complex64, device=dev) for l in LEVELS}
    G = {l: torch.empty((4 ** l, P), dtype=torch.complex64, device=dev) for l in LEVELS}
    fmmgb.fmm_p2m(MAXL, P, xyd, cd, M[MAXL])
    for l in range(MAXL, LEVELS[0], -1):
        fmmgb.fmm_m2m(l, P, M[l], M[l - 1])
    torch.cuda.synchronize()
    del xyd, cd
    Ms = [M[l] for l in LEVELS]
    Ls = [Lx[l] for l in LEVELS]
    Gs = [G[l] for l in LEVELS]

    def step():  # the whole hot path: every translation of levels 2..8, reduction fused, one launch
        fmmgb.fmm_m2l_levels(tree, LEVELS[0], P, Ms, Ls, stream=stream)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(max(3, args.warmup)):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    fmmgb.fmm_sync_status()
    if args.mode == "kernels" and args.prec == "batched":
        # profiling case: the 256-problem batched launch only
        bt = _batched_setup(torch, fmmgb, dev, autotune=False, nprob=args.nprob)
        for _ in range(args.steps):
            bt["plan"].run(stream)
        torch.cuda.synchronize()
        fmmgb.fmm_sync_status()
        if rank == 0:
            print(json.dumps({"mode": "kernels", "steps": args.steps, "launches_per_step": 1, "batch": bt["info"]}))
        return 0
    if args.mode == "kernels" and args.prec in ("fgt", "fgt_tc"):
        # profiling case: the FGT H2T of the sigma (default 0.05), p = 16 workload (fgt_tc: tensor cores)
        fcfg = workloads.CONFIGS["fgt"]
        fx, fq = workloads.gmm_particles(fcfg["n"], workloads.rng_for("fgt"))
        sigma, fp = args.sigma, 16
        g = workloads.fgt_grid_log2(sigma)
        A = torch.empty((4 ** g, fp, fp), dtype=torch.float32, device=dev)
        Cf = torch.empty_like(A)
        W = torch.empty_like(A)
        fmmgb.fgt_p2h(g, fp, sigma, torch.from_numpy(fx).to(dev), torch.from_numpy(fq).to(dev), A)
        tc = args.prec == "fgt_tc"
        for _ in range(args.steps):
            fmmgb.fgt_h2t(g, fcfg["ncut"], fp, sigma, A, Cf, work=W,
                          prec=fmmgb.FMM_TC_BF16X3 if tc else fmmgb.FMM_FP32)
        torch.cuda.synchronize()
        fmmgb.fmm_sync_status()
        if rank == 0:
            print(json.dumps({"mode": "kernels", "steps": args.steps,
                              "launches_per_step": 1 if tc else fgt_h2t_launches(g)}))
        return 0
    if args.mode == "kernels" and args.prec == "p2p":
        # profiling case: the near field at level 8 of the 2^22-point headline workload
        from paper_1009_3457_gb300 import farfield

        xy, c = workloads.uniform_particles(CFG["n"], workloads.rng_for(WORKLOAD))
        xyd, cd = torch.from_numpy(xy).to(dev), torch.from_numpy(c).to(dev)
        pot = farfield.FmmPotential(fmmgb.fmm_build_lists(None, MAXL), P, xyd, cd, xyd)
        for _ in range(args.steps):
            fmmgb.fmm_p2p(MAXL, xyd, cd, pot.sperm, pot.sstart, xyd, pot.tperm, pot.tstart, pot.phi)
        torch.cuda.synchronize()
        fmmgb.fmm_sync_status()
        if rank == 0:
            print(json.dumps({"mode": "kernels", "steps": args.steps, "launches_per_step": 2}))
        return 0
    if args.mode == "kernels" and args.prec == "h2p":
        # profiling case: FGT Hermite evaluation, sigma = 0.05, p = 16, 2^20 mixture targets
        fcfg = workloads.CONFIGS["fgt"]
        fx, fq = workloads.gmm_particles(fcfg["n"], workloads.rng_for("fgt"))
        fy, _ = workloads.gmm_particles(fcfg["n"], workloads.rng_for("fgt_targets"))
        fyd = torch.from_numpy(fy).to(dev)
        st = _fgt_hermite_setup(torch, fmmgb, dev, torch.from_numpy(fx).to(dev), torch.from_numpy(fq).to(dev),
                                fyd, 0.05, 16)
        hprec = fmmgb.FMM_TC_BF16X3 if args.tc else fmmgb.FMM_FP32
        for _ in range(args.steps):
            fmmgb.fgt_h2p(st["g"], fcfg["ncut"], 16, 0.05, st["A"], fyd, st["tperm"], st["tstart"], st["G"],
                          prec=hprec)
        torch.cuda.synchronize()
        fmmgb.fmm_sync_status()
        if rank == 0:
            print(json.dumps({"mode": "kernels", "steps": args.steps, "launches_per_step": 1,
                              "box_pairs": st["pairs"]}))
        return 0
    if args.mode == "kernels":
        # profiling case: the step's launch only (no e2e copies, no CPU baseline, no other rows)
        prec = {"fp32": fmmgb.FMM_FP32, "tc3": fmmgb.FMM_TC_BF16X3, "tc1": fmmgb.FMM_TC_BF16,
                "tf3": fmmgb.FMM_TC_TF32X3}[args.prec]
        for _ in range(args.steps):
            fmmgb.fmm_m2l_levels(tree, LEVELS[0], P, Ms, Ls, prec=prec, stream=stream)
        torch.cuda.synchronize()
        fmmgb.fmm_sync_status()
        if rank == 0:
            print(json.dumps({"mode": "kernels", "steps": args.steps, "launches_per_step": 1}))
        return 0

    # --- timed region: device-resident inputs; the step (the same public call) is
    # captured once as a CUDA graph and replayed, so the device time between the
    # events is the step's own, not the host's enqueue of the call ---
    step_graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(step_graph, capture_error_mode="thread_local"):
        fmmgb.fmm_m2l_levels(tree, LEVELS[0], P, Ms, Ls)  # on the capture stream
    torch.cuda.synchronize()
    ref_L = [torch.empty_like(x) for x in Ls]
    fmmgb.fmm_m2l_levels(tree, LEVELS[0], P, Ms, ref_L, stream=stream)
    step_graph.replay()
    torch.cuda.synchronize()
    graph_matches = all(bool((a == b).all()) for a, b in zip(ref_L, Ls))
    del ref_L
    clk = ClockSampler(local)
    if rank == 0:
        clk.start()
        time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = _timed(torch, step_graph.replay, args.steps, stream, flush)
    if ws > 1:
        dist.barrier()
    # whole job: every rank's translations over the slowest rank's time (replicas, weak scaling)
    tot_ms = fdist.max_over_ranks(sum(step_ms))
    value = fdist.job_rate(NTR * args.steps, sum(step_ms) * 1e-3)

    # --- e2e: host buffers through the library's C entry point fmm_host_stream_submit (wrapped by
    # pipeline.HostStreamM2L): every step copies its MEs in from pinned host memory and its LEs
    # back out; consecutive steps overlap on the library's three streams, the way a stream of
    # problems is served ---
    from paper_1009_3457_gb300 import pipeline

    pipe = pipeline.HostStreamM2L(tree, LEVELS[0], LEVELS[-1], P)
    Mh = torch.empty(pipe.flat_size(), dtype=torch.complex64).pin_memory()  # the levels back to back
    for v, l in zip(pipe.level_views(Mh), LEVELS):
        v.copy_(M[l])
    Lh = [torch.empty_like(Mh).pin_memory() for _ in range(2)]
    h2d = sum(M[l].numel() * 8 for l in LEVELS)
    d2h = sum(Lx[l].numel() * 8 for l in LEVELS)
    pipe.run([Mh] * max(3, args.warmup), [Lh[i % 2] for i in range(max(3, args.warmup))])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(pipe.h2d)
    pipe.run([Mh] * args.steps, [Lh[i % 2] for i in range(args.steps)])
    e1.record(pipe.d2h)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_matches = all(bool((v == Lx[l].cpu()).all()) for v, l in zip(pipe.level_views(Lh[(args.steps - 1) % 2]), LEVELS))
    e2e_value = fdist.job_rate(NTR * args.steps, e2e_ms * 1e-3)
    clocks = clk.stop() if rank == 0 else None

    # --- the other rows of the hot path, same device-resident protocol ---
    rows = {}
    if rank == 0 and not args.no_rows:
        def per_level():
            for l in sorted(LEVELS, reverse=True):
                fmmgb.fmm_m2l(tree, l, P, M[l], Lx[l])

        def adjoint():
            fmmgb.fmm_m2l_adjoint_levels(tree, LEVELS[0], P, Ls, Gs, conj=True)

        def tc_x3():
            fmmgb.fmm_m2l_levels(tree, LEVELS[0], P, Ms, Ls, prec=fmmgb.FMM_TC_BF16X3)

        def tc_x1():
            fmmgb.fmm_m2l_levels(tree, LEVELS[0], P, Ms, Ls, prec=fmmgb.FMM_TC_BF16)

        def tc_adjoint():
            fmmgb.fmm_m2l_adjoint_levels(tree, LEVELS[0], P, Ls, Gs, prec=fmmgb.FMM_TC_BF16X3, conj=True)

        def tc_tf32():
            fmmgb.fmm_m2l_levels(tree, LEVELS[0], P, Ms, Ls, prec=fmmgb.FMM_TC_TF32X3)

        # every row below times a CUDA-graph replay of its library calls (as the headline step does)
        for name, fn, launches in (("m2l_fp32_one_launch_per_level", per_level, len(LEVELS)),
                                   ("m2l_adjoint_fp32_levels_2_8", adjoint, 1),
                                   ("m2l_tc_bf16x3_levels_2_8", tc_x3, 1),
                                   ("m2l_tc_bf16_levels_2_8", tc_x1, 1),
                                   ("m2l_tc_bf16x3_adjoint_levels_2_8", tc_adjoint, 1),
                                   ("m2l_tc_tf32x3_levels_2_8", tc_tf32, 1)):
            ms = statistics.median(_timed(torch, _graph(torch, fn), args.steps, stream, flush))
            gf = NTR * metrics.m2l_flops_per_translation(P) / (ms * 1e-3) / 1e9
            rows[name] = {"translations_per_s": NTR / (ms * 1e-3), "ms": ms, "launches": launches, "gflops": gf}
            if "fp32" in name:
                rows[name]["alu_frac"] = gf / 1e3 / alu_peak_tflops()
            else:  # tensor cores: issued MMA work against the measured peak of the operand type
                # (TF32: the measured BF16 peak x the nominal dense ratio 1.1 / 2.25), and the useful part
                prods = 1 if name == "m2l_tc_bf16_levels_2_8" else 3
                peak = BF16_PEAK_TFLOPS * (TF32_PER_BF16 if "tf32" in name else 1.0)
                tt = metrics.m2l_tc_mma_flops(LEVELS, P, prods) / (ms * 1e-3) / 1e12
                rows[name].update({"tensor_tflops": tt, "tensor_frac": tt / peak,
                                   "useful_tflops": gf / 1e3 * prods,
                                   "useful_frac": gf / 1e3 * prods / peak})
                if "tf32" in name:
                    rows[name]["peak_note"] = "TF32 peak = measured BF16 peak x 1.1 / 2.25 (nominal dense ratio)"
        # precision study at p = 24 on the same tree: FP32 kernel vs tensor cores (BF16x3)
        p24 = workloads.CONFIGS["m2l_tc"]["p"]
        xyd = torch.from_numpy(xy).to(dev)
        cd = torch.from_numpy(c).to(dev)
        M24 = {l: torch.empty((4 ** l, p24), dtype=torch.complex64, device=dev) for l in LEVELS}
        L24 = {l: torch.empty((4 ** l, p24), dtype=torch.complex64, device=dev) for l in LEVELS}
        fmmgb.fmm_p2m(MAXL, p24, xyd, cd, M24[MAXL])
        for l in range(MAXL, LEVELS[0], -1):
            fmmgb.fmm_m2m(l, p24, M24[l], M24[l - 1])
        del xyd, cd
        M24s, L24s = [M24[l] for l in LEVELS], [L24[l] for l in LEVELS]
        t24 = {}
        for name, prec in (("m2l_fp32_p24_levels_2_8", fmmgb.FMM_FP32), ("m2l_tc_bf16x3_p24_levels_2_8",
                                                                         fmmgb.FMM_TC_BF16X3)):
            def run24(prec=prec):
                fmmgb.fmm_m2l_levels(tree, LEVELS[0], p24, M24s, L24s, prec=prec)

            ms = statistics.median(_timed(torch, _graph(torch, run24), args.steps, stream, flush))
            t24[prec] = ms
            gf = NTR * metrics.m2l_flops_per_translation(p24) / (ms * 1e-3) / 1e9
            rows[name] = {"translations_per_s": NTR / (ms * 1e-3), "ms": ms, "launches": 1, "gflops": gf}
            if prec == fmmgb.FMM_FP32:
                rows[name]["alu_frac"] = gf / 1e3 / alu_peak_tflops()
            else:
                tt = metrics.m2l_tc_mma_flops(LEVELS, p24, 3) / (ms * 1e-3) / 1e12
                rows[name].update({"tensor_tflops": tt, "tensor_frac": tt / BF16_PEAK_TFLOPS,
                                   "useful_tflops": gf / 1e3 * 3, "useful_frac": gf / 1e3 * 3 / BF16_PEAK_TFLOPS})
        rows["tc_vs_fp32_speedup_p24"] = {"speedup": t24[fmmgb.FMM_FP32] / t24[fmmgb.FMM_TC_BF16X3],
                                          "note": "both meet the tensor-core bar (truncation + 1e-4); "
                                                  "measured coefficient errors in tests/test_m2l_tc_gpu.py"}
        rows["tc_vs_fp32_speedup_p16"] = {"speedup": statistics.median(step_ms) / rows["m2l_tc_bf16x3_levels_2_8"]["ms"]}
        rows["tc_tf32x3_vs_fp32_speedup_p16"] = {
            "speedup": statistics.median(step_ms) / rows["m2l_tc_tf32x3_levels_2_8"]["ms"],
            "note": "TF32x3 is held to the FP32 bar (1e-5) in tests/test_m2l_tc_tf32_gpu.py"}
        del M24, L24, M24s, L24s
        # the paper's two-kernel data flow (per-translation LEs written to HBM, then a separate
        # reduction) on the headline workload, against the fused stencil
        work = torch.empty((4 ** MAXL, 27, P), dtype=torch.complex64, device=dev)
        Lpd = [torch.empty_like(m) for m in Ms]

        def paper_design():
            for i, l in enumerate(LEVELS):
                fmmgb.fmm_m2l_paper_design(tree, l, P, Ms[i], Lpd[i], work)

        ms_pd = statistics.median(_timed(torch, _graph(torch, paper_design), args.steps, stream, flush))
        rows["m2l_paper_design_levels_2_8"] = {
            "translations_per_s": NTR / (ms_pd * 1e-3), "ms": ms_pd, "launches": 2 * len(LEVELS),
            "le_bytes_through_hbm": 2 * NTR * P * 8,
            "fused_speedup": ms_pd / statistics.median(step_ms),
            "note": "block per source ME, thread per LE row, one LE per translation to HBM, then a reduction "
                    "kernel per level (Sec. 4.1.1-4.1.2); the same operator tables"}
        del work, Lpd
        # paper-shape periodic runs (27 translations per box, levels 2..8, Tables m2ltesla and
        # m2lfermi): p = 8, 12, 16; the C1060 rates of the largest size printed in Table m2ltesla
        # go beside them as context
        paper_c1060 = {8: 163.31e6, 12: 80.05e6, 16: 51.14e6}
        ptree = fmmgb.fmm_build_lists(None, MAXL, periodic=True)
        xyd = torch.from_numpy(xy).to(dev)
        cd = torch.from_numpy(c).to(dev)
        for pp in (8, 12, 16):
            Mq = {l: torch.empty((4 ** l, pp), dtype=torch.complex64, device=dev) for l in LEVELS}
            fmmgb.fmm_p2m(MAXL, pp, xyd, cd, Mq[MAXL])
            for l in range(MAXL, LEVELS[0], -1):
                fmmgb.fmm_m2m(l, pp, Mq[l], Mq[l - 1])
            Mqs = [Mq[l] for l in LEVELS]
            Lqs = [torch.empty_like(m) for m in Mqs]

            def shape_run(pp=pp, Mqs=Mqs, Lqs=Lqs):
                fmmgb.fmm_m2l_levels(ptree, LEVELS[0], pp, Mqs, Lqs)

            ms = statistics.median(_timed(torch, _graph(torch, shape_run), args.steps, stream, flush))
            ntr_p = sum(ptree.translations(l) for l in LEVELS)
            rows[f"m2l_fp32_paper_shape_p{pp}"] = {
                "translations_per_s": ntr_p / (ms * 1e-3), "ms": ms, "launches": 1, "translations": ntr_p,
                "paper_gops": ntr_p * metrics.paper_ops_per_translation(pp) / (ms * 1e-3) / 1e9,
                "gflops": ntr_p * metrics.m2l_flops_per_translation(pp) / (ms * 1e-3) / 1e9,
                "paper_tesla_c1060_translations_per_s": paper_c1060[pp],
                "ratio_to_paper_c1060": ntr_p / (ms * 1e-3) / paper_c1060[pp]}
            del Mq, Mqs, Lqs

        # near field at level 8 (2^22 uniform points, targets = sources) and the whole FMM on the
        # device: P2M, M2M, M2L (levels 2..8), L2L, L2P and P2P, every stage a library kernel
        from paper_1009_3457_gb300 import farfield

        tree8 = fmmgb.fmm_build_lists(None, MAXL)
        pot = farfield.FmmPotential(tree8, P, xyd, cd, xyd)

        def near():
            fmmgb.fmm_p2p(MAXL, xyd, cd, pot.sperm, pot.sstart, xyd, pot.tperm, pot.tstart, pot.phi)

        ms_p2p = statistics.median(_timed(torch, _graph(torch, near), args.steps, stream, flush))
        counts = torch.diff(pot.sstart).cpu().numpy()
        pairs = metrics.p2p_pairs(MAXL, counts, counts, self_pairs=int(CFG["n"]))
        sfu_peak = SM_COUNT * 16 * SM_MAX_MHZ * 1e6  # one reciprocal per pair, 16 per SM per cycle
        rows["fmm_p2p_level8"] = {
            "ms": ms_p2p, "points": int(CFG["n"]), "pairs": pairs, "pairs_per_s": pairs / (ms_p2p * 1e-3),
            "sfu_frac": pairs / (ms_p2p * 1e-3) / sfu_peak, "launches": 2,
            "note": "claim table + kernel; targets = sources (each point skips itself)"}
        ms_fmm = statistics.median(_timed(torch, _graph(torch, pot), args.steps, stream, flush))
        rows["fmm_potential_level8_p16"] = {
            "ms": ms_fmm, "points": int(CFG["n"]), "points_per_s": CFG["n"] / (ms_fmm * 1e-3),
            "m2l_translations": NTR, "near_pairs": pairs,
            "note": "P2M, M2M, M2L (levels 2-8, one launch), L2L, L2P, P2P: the potential at all 2^22 points; "
                    "the near field on a second stream beside the far field up to L2L (FMM_P2P_SHARE_SM)"}
        del pot, tree8, xyd, cd

        # adaptive tree: 2^20 Gaussian-mixture points, q = 64, levels 2..9, p = 16: V-list M2L,
        # its adjoint, and one gradient of the far-field objective (forward + backward)
        gcfg = workloads.CONFIGS["m2l_gmm"]
        gx, gc = workloads.gmm_particles(gcfg["n"], workloads.rng_for("m2l_gmm"))
        gtree = fmmgb.fmm_build_lists(gx, gcfg["max_level"], leaf_cap=gcfg["leaf_cap"])
        glev = list(range(2, gcfg["max_level"] + 1))
        gp = gcfg["p"]
        gxd = torch.from_numpy(gx).to(dev)
        gcd = torch.from_numpy(gc).to(dev)
        gM = [torch.empty((4 ** l, gp), dtype=torch.complex64, device=dev) for l in glev]
        for l, m in zip(glev, gM):
            fmmgb.fmm_p2m(l, gp, gxd, gcd, m)
        gL = [torch.zeros_like(m) for m in gM]
        gG = [torch.zeros_like(m) for m in gM]
        gntr = sum(gtree.translations(l) for l in glev)
        gLt = [torch.zeros_like(m) for m in gM]
        for name, fn in (("m2l_adaptive_gmm_levels_2_9",
                          lambda: fmmgb.fmm_m2l_levels(gtree, 2, gp, gM, gL)),
                         ("m2l_adjoint_adaptive_gmm_levels_2_9",
                          lambda: fmmgb.fmm_m2l_adjoint_levels(gtree, 2, gp, gL, gG, conj=True)),
                         ("m2l_tc_bf16x3_adaptive_gmm_levels_2_9",
                          lambda: fmmgb.fmm_m2l_levels(gtree, 2, gp, gM, gLt, prec=fmmgb.FMM_TC_BF16X3))):
            ms = statistics.median(_timed(torch, _graph(torch, fn), args.steps, stream, flush))
            rows[name] = {"translations_per_s": gntr / (ms * 1e-3), "ms": ms, "launches": 1, "translations": gntr,
                          "gflops": gntr * metrics.m2l_flops_per_translation(gp) / (ms * 1e-3) / 1e9,
                          "boxes": {l: int(gtree.level_info(l).nexist) for l in glev}}
            if "tc" in name:
                rows[name]["speedup_vs_fp32"] = rows["m2l_adaptive_gmm_levels_2_9"]["ms"] / ms
                rows[name]["rel_l2_vs_fp32_path"] = float(
                    sum(torch.linalg.vector_norm((a - b).to(torch.complex128)) ** 2 for a, b in zip(gLt, gL)) ** 0.5
                    / sum(torch.linalg.vector_norm(b.to(torch.complex128)) ** 2 for b in gL) ** 0.5)
            else:
                rows[name]["alu_frac"] = (gntr * metrics.m2l_flops_per_translation(gp) / (ms * 1e-3) / 1e12
                                          / alu_peak_tflops())
        from paper_1009_3457_gb300 import farfield

        zr = np.random.default_rng(workloads.SEED_BASE + 5)
        zz = zr.random(4096) + 1j * zr.random(4096)
        zw = torch.from_numpy(zr.uniform(-1, 1, 4096)).to(dev)
        gxr = gxd.clone().requires_grad_(True)
        gleaf = farfield.leaf_boxes(gtree, gxd)
        gzl = farfield.leaf_boxes(gtree, torch.from_numpy(np.stack([zz.real, zz.imag], 1)).to(dev))
        zzd = torch.from_numpy(zz).to(dev)

        def grad_step():
            gxr.grad = None
            J = farfield.far_field_objective(gtree, gp, gxr, gcd, gleaf, zzd, gzl, zw)
            J.backward()

        grad_step()
        torch.cuda.synchronize()
        ms = statistics.median(_timed(torch, grad_step, max(3, args.steps // 4), stream, flush))
        rows["far_field_gradient_gmm"] = {"ms": ms, "points": int(gcfg["n"]),
                                          "note": "forward J + backward to all 2^20 source positions: "
                                                  "P2M, M2L, L2L, L2P and their adjoints, all library kernels"}
        del gM, gL, gG, gxd, gcd, gxr
        fmmgb.fmm_sync_status()

        # batched persistent launch: 256 independent problems (depth 4..9, p in {6, 8, 12, 16})
        bt = _batched_setup(torch, fmmgb, dev)
        bplan = bt["plan"]
        ms = statistics.median(_timed(torch, _graph(torch, lambda: bplan.run()), args.steps, stream, flush))

        def per_problem():
            for tr, p_, m_, l_ in zip(bt["trees"], bt["ps"], bt["Ms"], bt["Ls"]):
                fmmgb.fmm_m2l_levels(tr, 2, p_, m_, l_)

        ms_seq = statistics.median(_timed(torch, _graph(torch, per_problem), args.steps, stream, flush))
        ntr_b = bt["info"]["translations"]
        rows["m2l_batched_256_problems"] = {
            "translations_per_s": ntr_b / (ms * 1e-3), "ms": ms, "launches": 1, "translations": ntr_b,
            "gflops": bt["flops"] / (ms * 1e-3) / 1e9,
            "alu_frac": bt["flops"] / (ms * 1e-3) / 1e12 / alu_peak_tflops(),
            "plan": bt["info"], "one_launch_per_problem_ms": ms_seq,
            "speedup_vs_one_launch_per_problem": ms_seq / ms}
        del bt, bplan
        fmmgb.fmm_sync_status()
        fcfg = workloads.CONFIGS["fgt"]
        fx, fq = workloads.gmm_particles(fcfg["n"], workloads.rng_for("fgt"))
        fxd = torch.from_numpy(fx).to(dev)
        fqd = torch.from_numpy(fq).to(dev)
        for sigma in fcfg["sigmas"]:
            for fp in fcfg["orders"]:
                g = workloads.fgt_grid_log2(sigma)
                A = torch.empty((4 ** g, fp, fp), dtype=torch.float32, device=dev)
                Cf = torch.empty_like(A)
                W = torch.empty_like(A)
                sperm = torch.empty(fcfg["n"], dtype=torch.int32, device=dev)
                sstart = torch.empty(4 ** g + 1, dtype=torch.int32, device=dev)
                swork = torch.empty(4 ** g, dtype=torch.int32, device=dev)
                fmmgb.fgt_bin_points(g, fxd, sperm, sstart, swork)
                fmmgb.fgt_p2h_binned(g, fp, sigma, fxd, fqd, sperm, A)

                def fgt():
                    fmmgb.fgt_h2t(g, fcfg["ncut"], fp, sigma, A, Cf, work=W)

                ms = statistics.median(_timed(torch, _graph(torch, fgt), args.steps, stream, flush))
                ntr = metrics.fgt_translations(g, fcfg["ncut"])
                taps = 2 * fcfg["ncut"] + 1
                if sigma == 0.05 and fp == 16:
                    # the whole transform: 2^20 sources -> bin -> P2H -> H2T -> T2P at 2^20 targets
                    fy = torch.rand((fcfg["n"], 2), dtype=torch.float64, device=dev,
                                    generator=torch.Generator(device=dev).manual_seed(workloads.SEED_BASE + 5))
                    Gy = torch.empty(fcfg["n"], dtype=torch.float32, device=dev)
                    tperm = torch.empty(fcfg["n"], dtype=torch.int32, device=dev)
                    tstart = torch.empty(4 ** g + 1, dtype=torch.int32, device=dev)

                    def fgt_all():
                        fmmgb.fgt_bin_points(g, fxd, sperm, sstart, swork)
                        fmmgb.fgt_p2h_binned(g, fp, sigma, fxd, fqd, sperm, A)
                        fmmgb.fgt_h2t(g, fcfg["ncut"], fp, sigma, A, Cf, work=W)
                        fmmgb.fgt_bin_points(g, fy, tperm, tstart, swork)
                        fmmgb.fgt_t2p_binned(g, fp, sigma, Cf, fy, tperm, tstart, Gy)

                    ms_all = statistics.median(_timed(torch, _graph(torch, fgt_all), args.steps, stream, flush))
                    rows["fgt_transform_sigma0.05_p16"] = {
                        "ms": ms_all, "sources": int(fcfg["n"]), "targets": int(fcfg["n"]),
                        "points_per_s": fcfg["n"] / (ms_all * 1e-3), "launches": 8 + fgt_h2t_launches(g),
                        "note": "fgt_bin_points of the sources (3 kernels), fgt_p2h_binned, fgt_h2t, "
                                "fgt_bin_points of the targets (3 kernels), fgt_t2p_binned; uniform targets"}
                gfs = (4 ** g) * metrics.fgt_flops_per_box_separable(fp, taps, taps) / (ms * 1e-3) / 1e9
                rows[f"fgt_h2t_sigma{sigma}_p{fp}"] = {
                    "translations_per_s": ntr / (ms * 1e-3), "ms": ms, "launches": fgt_h2t_launches(g),
                    "grid": f"{1 << g}^2", "gflops_separable": gfs, "alu_frac": gfs / 1e3 / alu_peak_tflops()}
                if fp == 16:
                    # the same translation on the tensor cores (one cooperative launch, both passes)
                    Ct = torch.empty_like(A)

                    def fgt_tc():
                        fmmgb.fgt_h2t(g, fcfg["ncut"], fp, sigma, A, Ct, work=W, prec=fmmgb.FMM_TC_BF16X3)

                    ms_tc = statistics.median(_timed(torch, _graph(torch, fgt_tc), args.steps, stream, flush))
                    mma = metrics.fgt_h2t_tc_mma_flops(g, fcfg["ncut"]) / (ms_tc * 1e-3) / 1e12
                    rel = float(torch.linalg.vector_norm((Ct - Cf).double()) / torch.linalg.vector_norm(Cf.double()))
                    rows[f"fgt_h2t_tc_bf16x3_sigma{sigma}_p16"] = {
                        "ms": ms_tc, "translations_per_s": ntr / (ms_tc * 1e-3), "launches": 1,
                        "tensor_tflops": mma, "tensor_frac": mma / BF16_PEAK_TFLOPS,
                        "speedup_vs_fp32": ms / ms_tc, "rel_l2_vs_fp32_path": rel,
                        "note": "one cooperative launch: both separable passes, grid barrier between"}
        rows.update(_fgt_hermite_rows(torch, fmmgb, dev, fxd, fqd, args, stream, flush))
        fmmgb.fmm_sync_status()

    if rank == 0:
        flops = NTR * metrics.m2l_flops_per_translation(P)
        k_avg_s = statistics.mean(step_ms) * 1e-3
        achieved = flops / k_avg_s / 1e12
        peak = alu_peak_tflops()
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": CONFIG,
            "paper_gops": value * metrics.paper_ops_per_translation(P) / 1e9,
            "executed_gflops": value * metrics.m2l_flops_per_translation(P) / 1e9,
            "roofline": {
                "bound": "alu", "kernel": "m2l_fp32_kernel<16> (levels 2-8, one launch)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": _traffic(f"m2l_fp32_kernel<{P}>"),
                "peak_source": f"{SM_COUNT} SMs (device attribute) x 128 FP32 lanes x 2 flop x {SM_MAX_MHZ:.0f} MHz "
                               f"({peaks['clock_source']})",
                "measured_sgemm_fp32_tflops": peaks["sgemm_fp32_tflops"],
                "frac_of_measured_sgemm": achieved / peaks["sgemm_fp32_tflops"],
                "flops_per_launch": flops, "launch_ms": statistics.mean(step_ms),
                "frac_at_sampled_clock": (achieved / (peak * clocks["sm_mhz"] / SM_MAX_MHZ))
                if clocks and clocks.get("sm_mhz") else None,
            },
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "matches_device_result": e2e_matches,
                    "how": "K consecutive fmm_host_stream_submit calls (the C ABI's host-buffer entry point, "
                           "through pipeline.HostStreamM2L): each copies its MEs from pinned host memory and its "
                           "LEs back; copies in, translation and copies out of neighbouring steps overlap on the "
                           "library's three streams; CUDA events around all K steps"},
            "gpu_launches": args.steps,
            "graph_replay_matches_direct_call": graph_matches,
            "clocks": clocks,
            "device": peaks,
            "rows": rows,
        }
        if rows:
            out["summary"] = summarise(rows)
            out["tc_vs_fp32"] = {
                "p24_levels_2_8": {"fp32_ms": rows["m2l_fp32_p24_levels_2_8"]["ms"],
                                   "bf16x3_ms": rows["m2l_tc_bf16x3_p24_levels_2_8"]["ms"],
                                   "speedup": rows["tc_vs_fp32_speedup_p24"]["speedup"]},
                "p16_levels_2_8": {"fp32_ms": statistics.median(step_ms),
                                   "bf16x3_ms": rows["m2l_tc_bf16x3_levels_2_8"]["ms"],
                                   "speedup": rows["tc_vs_fp32_speedup_p16"]["speedup"],
                                   "tf32x3_ms": rows["m2l_tc_tf32x3_levels_2_8"]["ms"],
                                   "tf32x3_speedup": rows["tc_tf32x3_vs_fp32_speedup_p16"]["speedup"]},
                "workload": "2^22 points, uniform to level 8, levels 2-8 (2,316,900 translations)"}
        if not args.no_cpu_baseline and ws == 1:
            if rows:
                out["tc_vs_fp32"]["accuracy"] = tc_accuracy_vs_oracle(torch, fmmgb, dev)
            ksteps = 3
            v, times, ntr, cores = cpu_baseline_all_cores(steps=ksteps, warmup=1)
            v1, dt1, _ = cpu_baseline_run()
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                   "sample": f"the whole step ({ntr} translations, levels 2-8): 1 untimed + "
                                             f"{ksteps} timed steps ({sum(times):.2f} s), FP64 oracle in {cores} "
                                             f"processes over disjoint target slices (as --impl reference)",
                                   "single_thread": {"value": v1, "cores": 1, "seconds": dt1}}
        print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true", help="skip the adjoint / per-level / FGT rows")
    ap.add_argument("--mode", default="full", choices=["full", "kernels"],
                    help="kernels: only the timed step's launches (for ncu captures)")
    ap.add_argument("--tc", action="store_true", help="with --prec h2p: the tensor-core (BF16x3) form")
    ap.add_argument("--prec", default="fp32",
                    choices=["fp32", "tc3", "tc1", "tf3", "batched", "fgt", "fgt_tc", "h2p", "p2p"],
                    help="launches of --mode kernels: the step at this precision, or the 256-problem batch, "
                         "or the FGT H2T at sigma 0.05, p 16")
    ap.add_argument("--sigma", type=float, default=0.05, help="--mode kernels --prec fgt: the FGT bandwidth")
    ap.add_argument("--nprob", type=int, default=None,
                    help="--mode kernels --prec batched: the first N problems of the batch (profiling case)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
