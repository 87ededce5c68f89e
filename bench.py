"""Benchmark: box-evaluations per second of the CSF subdivision hot path on one GB300.

A step is one whole enclosure (Algorithm 3, levels 0..depth: CSF level evaluation with C0,
compaction, 2^k split and rebuild) of the workload

    two trivariate Kostlan polynomials of total degree 100 (a curve), domain [-1,1]^3,
    depth 10 (finest grid 1024^3)

with the polynomials already resident in device memory.  The headline path is binary32
interval arithmetic with binary64-certified decisions (mode VX_FP32: every level's kept set
equals the binary64 one); the plain binary64 path is timed beside it.
box-evals/s = (sum over levels of the boxes tested) / time.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

For N = 2^s > 1 (torchrun, one rank per GPU) rank r runs Algorithm 3 from level s on the boxes
with x_1 index r (no data exchange; paper_2406_09857_gb300/shard.py), which yields exactly its
share of the single-GPU result; the value is the boxes evaluated by all ranks over the slowest
rank's time.  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "box-evals/s & enclosure wall time: FP32-midrad+batched vs FP64 on 1 GB300"
UNIT = "box-evals/s"
WORKLOAD = ("curve: 2 trivariate Kostlan polynomials of total degree 100 on [-1,1]^3, "
            "subdivision depth 10 (1024^3 finest grid)")

# Roofline denominators of the plain-ALU evaluation kernels, from unit counts: 128 binary32
# FMA lanes and 2 binary64 lanes per SM per clock, times the device's SM count and the median
# SM clock sampled under load in the timed region (its maximum clock when no sample was taken).
FP32_LANES_PER_SM, FP64_LANES_PER_SM = 128, 2
NOMINAL_SM_MHZ = 2070.0  # the part's maximum SM clock, used only when no clock was read


def alu_peaks(sms: int, mhz: float):
    """(binary32 FMA, binary64) lane-operation peaks in T/s."""
    return (sms * FP32_LANES_PER_SM * mhz * 1e6 / 1e12, sms * FP64_LANES_PER_SM * mhz * 1e6 / 1e12)
# FMA-pipe lane operations of one interval multiply-add: binary32 certified = 2 directed FMAs
# for the endpoints (one paired instruction) + 2 for the error bound; binary64 = 2 directed
# multiplies + 2 directed adds.
OPS_PER_MADD = {"fp32": 4, "fp64": 4}
L2_FLUSH_BYTES = 512 << 20  # > 129 MB of L2
# certified binary32 runs of the small workloads (the paper's random family, its two systems)
# take levels below this many interval multiply-adds in binary64 (the same decisions, fewer
# launches); the headline curve runs every level in binary32
SMALL_LEVEL_MADDS = 1 << 24
# the headline enclosure starts from the full grid of this level (opts.first_level): the curve
# keeps nearly every box of levels 0..6, whose launches cost more than their few boxes, and
# pruning them changes no final box
FIRST_LEVEL = 6
# dram__bytes_read.sum + dram__bytes_write.sum of the certified binary32 leaf kernel
# (k_leaf_tma_q<4>) on the curve's level 9 (ncu --set full): 1561.9 MB + 172.4 MB for
# 1.784e10 interval multiply-adds (Algorithm 2's count)
LEAF32_DRAM_B_PER_MADD = (1561.9e6 + 172.4e6) / 1.78408304e10


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


PEAKS = load_peaks()


def log(*a):
    print(*a, file=sys.stderr, flush=True)


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons, sampled every 200 ms while active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.4)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, power, reasons = [], [], [], set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(self.NAMES, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power), "reasons": sorted(reasons)}


def oracle_lineage(polys, domain, depth: int, x1: int) -> int:
    """The CPU oracle's Algorithm 3 on the lineage of finest x_1-slab ``x1``: at level l only
    the boxes whose x_1 index is x1's ancestor (x1 >> (depth - l)) are evaluated and
    subdivided.  These are exactly the boxes the full run evaluates in that lineage (each box
    is decided on its own), so the sample keeps the run's mix of levels and the sharing of
    partial evaluations along the CSF.  Returns the number of box evaluations."""
    import oracle

    k = len(domain) // 2
    S = np.zeros((1, k - 1), dtype=np.int32)  # indices along x_2..x_k
    bits = np.array([[(b >> (k - 2 - c)) & 1 for c in range(k - 1)] for b in range(1 << (k - 1))],
                    dtype=np.int32)
    evals = 0
    for l in range(depth + 1):
        full = np.empty((S.shape[0], k), dtype=np.int32)
        full[:, 0] = x1 >> (depth - l)
        full[:, 1:] = S
        _, _, keep, _ = oracle.eval_csf(polys, domain, l, full)
        evals += full.shape[0]
        S = S[keep == 1]
        if l == depth or S.shape[0] == 0:
            break
        S = (2 * S[:, None, :] + bits[None, :, :]).reshape(-1, k - 1)
        S = S[np.lexsort(S.T[::-1])]
    return evals


def oracle_sample(polys, domain, depth, budget_s: float, seed: int, min_lineages: int = 1):
    """Times oracle_lineage on random finest slabs until ``budget_s`` seconds have passed."""
    from paper_2406_09857_gb300 import synth

    st = synth.Stream(seed)
    side = 1 << depth
    boxes, secs, n = 0, 0.0, 0
    while (secs < budget_s or n < min_lineages) and n < 256:
        x1 = int(st.uniform_int(0, side - 1, 1)[0])
        t0 = time.perf_counter()
        boxes += oracle_lineage(polys, domain, depth, x1)
        secs += time.perf_counter() - t0
        n += 1
    desc = ("CPU oracle (plain C, binary64 directed rounding, 1 thread): Algorithm 3 along the "
            "lineage of %d random finest x1-slabs (every level's boxes of each slab), %d box "
            "evaluations in %.1f s" % (n, boxes, secs))
    return boxes / secs, boxes, secs, desc


def config_dict(world: int, mode: str):
    return {"workload": WORKLOAD, "k": 3, "npoly": 2, "degree": 100, "depth": 10,
            "domain": "[-1,1]^3", "coefficients": "Kostlan: N(0,1) * sqrt(multinomial)",
            "mode": mode,
            "l2": "512 MB written between steps, outside the per-step CUDA events",
            "parallelism": ("x1-slab shards: rank r starts at level log2(N) from the boxes "
                            "with x1 index r" if world > 1 else "single GPU")}


def bench_dense(vx, synth, torch, stream, flush, d=128, level=10, reps=2):
    """One complete level of a degree-(d,d,d) tensor on [-1,1]^3 (config 5's largest cell):
    every box of the 2^level-per-axis grid evaluated by the staged (mode-by-mode) partial
    evaluation, in each arithmetic; the certified binary32 kept set must equal binary64's."""
    s = synth.dense_sweep(d)
    sysv = vx.System(s.polys)
    c = vx.csf_full_grid(3, level)
    n = 1 << (3 * level)
    out = {"workload": "dense level: degree %d per variable ((d+1)^3 = %d coefficients, iid "
                       "N(0,1)), every box of the %d^3 grid of [-1,1]^3" % (d, (d + 1) ** 3, 1 << level)}
    keeps = {}
    for name, mode in (("fp32", vx.FP32), ("midrad", vx.FP32_MIDRAD), ("fp64", vx.FP64)):
        vx.csf_eval_level(sysv, c, s.domain, mode, stream=stream)
        ms = []
        for r in range(reps):
            flush.fill_(float(r))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            k = vx.csf_eval_level(sysv, c, s.domain, mode, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        keeps[name] = k
        out[name] = {"value": n / (min(ms) * 1e-3), "unit": UNIT, "ms": min(ms),
                     "kept": int(k.sum().item())}
    out["fp32_equals_fp64"] = bool(torch.equal(keeps["fp32"], keeps["fp64"]))
    out["midrad_superset"] = bool(torch.all(keeps["midrad"] >= keeps["fp64"]).item())
    out["speedup_fp32_vs_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    c.free()
    out["tensor_core"] = bench_dense_tc(vx, torch, stream, flush, sysv, s, d, level, reps,
                                        keeps["fp64"], min(out["fp32"]["ms"], out["fp64"]["ms"]))
    return out


def bench_dense_sweep(vx, synth, torch, stream, flush):
    """Config 5's sweep: degree d in {32, 64, 128} per variable, N in {256, 512, 1024} boxes per
    axis; per cell the full-grid level in certified binary32 and binary64 (interval path) and
    on the tensor cores (prefilter, then the survivors decided exactly); kept sets compared."""
    out = {}

    def timed(fn):
        fn()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), r

    for d in (32, 64, 128):
        s = synth.dense_sweep(d)
        sysv = vx.System(s.polys, stream=stream)
        for level in (8, 9, 10):
            n = 1 << (3 * level)
            c = vx.csf_full_grid(3, level)
            ms32, k32 = timed(lambda: vx.csf_eval_level(sysv, c, s.domain, vx.FP32, stream=stream))
            ms64, k64 = timed(lambda: vx.csf_eval_level(sysv, c, s.domain, vx.FP64, stream=stream))
            c.free()
            plan = vx.DensePlan(sysv, level, s.domain, stream=stream)
            keep = torch.empty(n, dtype=torch.uint8, device="cuda")
            mstc, (_, surv) = timed(lambda: plan.level_keep(vx.make_opts(vx.FP32), keep=keep,
                                                            stream=stream))
            mask = torch.empty(n // 32, dtype=torch.int32, device="cuda")
            mspre, _ = timed(lambda: plan.prefilter(mask, stream=stream))
            plan.free()
            out["d%d-N%d" % (d, 1 << level)] = {
                "boxes": n, "kept": int(k64.sum().item()),
                "fp32_ms": round(ms32, 3), "fp64_ms": round(ms64, 3),
                "tc_prefilter_ms": round(mspre, 3), "tc_exact_ms": round(mstc, 3),
                "tc_survivors": int(surv),
                "tc_exact_box_evals_per_s": n / (mstc * 1e-3),
                "fp32_equals_fp64": bool(torch.equal(k32, k64)),
                "tc_exact_equals_fp64": bool(torch.equal(keep, k64))}
        sysv.free()
    return out


def bench_dense_tc(vx, torch, stream, flush, sysv, s, d, level, reps, keep64, best_ms):
    """The same level on the tensor cores: the power-form prefilter (TF32 contractions, a
    superset of the kept boxes) alone, and the level decided exactly (prefilter, then the
    survivors through the certified binary32 path), which must equal binary64's keep."""
    n = 1 << (3 * level)
    N = 1 << level
    t0 = time.perf_counter()
    plan = vx.DensePlan(sysv, level, s.domain, stream=stream)
    plan_s = time.perf_counter() - t0
    mask = torch.empty(n // 32, dtype=torch.int32, device="cuda")

    def timed(fn):
        fn()
        ms = []
        for r in range(reps):
            flush.fill_(float(r))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return min(ms)

    with torch.cuda.stream(stream):
        pre_ms = timed(lambda: plan.prefilter(mask, stream=stream, check=False))
        vx.lib().vx_dense_check_status(vx._stream(stream))
        pre = vx.mask_to_bool(mask, n)
        keep = torch.empty(n, dtype=torch.uint8, device="cuda")
        surv = [0]

        def exact():
            surv[0] = plan.level_keep(vx.make_opts(vx.FP32), keep=keep, stream=stream)[1]

        ex_ms = timed(exact)
    # executed TF32 flops of the three contractions (padding included) and the algorithmic
    # flops of the midpoints alone (Property 1's contractions on the unpadded tensor)
    Kp = (d + 1 + 7) // 8 * 8
    N2p = (d + 1 + 15) // 16 * 16
    ncols1 = ((d + 1) ** 2 + 127) // 128 * 128
    executed = 2.0 * (N * ncols1 * 2 * Kp + N * N * N2p * 3 * Kp + N * N * N * 3 * Kp)
    algorithmic = 2.0 * (N * (d + 1) ** 3 + N * N * (d + 1) ** 2 + N ** 3 * (d + 1))
    tf32_peak = PEAKS.get("bf16_tflops", 1900.0) / 2.0  # TF32 dense rate = bf16's / 2 (nominal)
    res = {
        "plan_s": plan_s, "plan_bytes": plan.device_bytes(),
        "prefilter": {"value": n / (pre_ms * 1e-3), "unit": UNIT, "ms": pre_ms,
                      "kept": int(pre.sum().item()),
                      "superset_of_fp64": bool(torch.all(pre | (keep64 == 0)).item()),
                      "tf32_executed_tflops": executed / (pre_ms * 1e-3) / 1e12,
                      "tf32_algorithmic_mid_tflops": algorithmic / (pre_ms * 1e-3) / 1e12,
                      "tf32_peak_tflops": tf32_peak,
                      "frac_executed": executed / (pre_ms * 1e-3) / 1e12 / tf32_peak},
        "exact_fp32": {"value": n / (ex_ms * 1e-3), "unit": UNIT, "ms": ex_ms,
                       "survivors": surv[0], "kept": int(keep.sum().item()),
                       "equals_fp64": bool(torch.equal(keep, keep64))},
        "speedup_exact_vs_best_interval_path": best_ms / ex_ms,
    }
    plan.free()
    return res


def _lineage_job(args):
    """One oracle lineage in a worker process (spawned): (box evaluations, seconds)."""
    polys, domain, depth, x1 = args
    t0 = time.perf_counter()
    n = oracle_lineage(polys, domain, depth, x1)
    return n, time.perf_counter() - t0


def oracle_parallel(polys, domain, depth, nlineages: int, seed: int, procs: int):
    """The oracle on ``nlineages`` random finest x1-slab lineages spread over ``procs`` spawned
    worker processes (the x1 slabs are independent, the parallel form of the oracle run over
    depth-1 nodes): box evaluations per second of wall time, and the processes used."""
    import multiprocessing as mp

    from paper_2406_09857_gb300 import synth

    st = synth.Stream(seed)
    side = 1 << depth
    jobs = [(polys, domain, depth, int(x)) for x in st.uniform_int(0, side - 1, nlineages)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_lineage_job, jobs[:procs])  # workers started and the oracle loaded
        t0 = time.perf_counter()
        res = pool.map(_lineage_job, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    boxes = sum(r[0] for r in res)
    return boxes / wall, boxes, wall


def bench_configs(vx, synth, torch, stream, cpu: bool, cpu_budget: float):
    """Configs 1-3 (plain, surface, curve) end to end with the system resident: box-evals/s
    and enclosure ms in certified binary32 (band re-decided at the last level) and binary64
    (median of 3 after a warm-up), beside the CPU oracle on random finest x1-slab lineages,
    one process and one per core (a reported baseline)."""
    out = {}
    ncores = os.cpu_count() or 1
    for name, make in (("plain", synth.plain), ("surface", synth.surface), ("curve", synth.curve)):
        s = make()
        sysv = vx.System(s.polys)
        e = {"workload": s.name, "depth": s.depth}
        for mode_name, mode, rl in (("fp32", vx.FP32, True), ("fp64", vx.FP64, False)):
            o = vx.make_opts(mode, recheck_last=rl)
            vx.enclose_system(sysv, s.domain, s.depth, o, stream).free()
            ms, evals = [], 0
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = vx.enclose_system(sysv, s.domain, s.depth, o, stream)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
                st = r.stats()
                evals = int(st["tested"].sum()) if mode == vx.FP64 else evals
                if mode == vx.FP64:
                    e["boxes"] = int(st["kept"][-1])
                r.free()
            e[mode_name] = {"ms_median": statistics.median(ms), "ms_min": min(ms)}
        # box evaluations of the exact subdivision (binary64's levels)
        e["box_evals"] = evals
        for mode_name in ("fp32", "fp64"):
            e[mode_name]["box_evals_per_s"] = evals / (e[mode_name]["ms_median"] * 1e-3)
        e["fp32_speedup_vs_fp64"] = e["fp64"]["ms_median"] / e["fp32"]["ms_median"]
        if cpu:
            v1, b1, t1, d1 = oracle_sample(s.polys, s.domain, s.depth, cpu_budget / 3, seed=13)
            nl = 4 * ncores
            vp, bp, tp = oracle_parallel(s.polys, s.domain, s.depth, nl, seed=17, procs=ncores)
            e["cpu_oracle"] = {
                "one_process": {"box_evals_per_s": v1, "box_evals": b1, "s": t1, "cores": 1},
                "all_cores": {"box_evals_per_s": vp, "box_evals": bp, "s": tp, "cores": ncores,
                              "lineages": nl},
                "sample": "Algorithm 3 along random finest x1-slab lineages (every level's boxes "
                          "of each slab), binary64 directed rounding; the all-cores run spreads "
                          "the lineages over spawned processes, one per core",
                "gpu_fp32_over_all_cores": e["fp32"]["box_evals_per_s"] / vp,
            }
        sysv.free()
        out[name] = e
    return out


def bench_precision(vx, synth, torch):
    """Per config (plain, surface, curve): excess boxes of binary32 midpoint-radius over
    binary64 at every level (no binary64 final level), and the radius inflation on the
    binary64 survivors of the last level: per box and polynomial, the midpoint-radius width
    2r over the binary64 width hi - lo (a seeded sample of at most 200 000 boxes)."""
    out = {}
    for name, make in (("plain", synth.plain), ("surface", synth.surface), ("curve", synth.curve)):
        s = make()
        sysv = vx.System(s.polys)
        r64 = vx.enclose_system(sysv, s.domain, s.depth, vx.make_opts(vx.FP64))
        rmr = vx.enclose_system(sysv, s.domain, s.depth, vx.make_opts(vx.FP32_MIDRAD))
        r32 = vx.enclose_system(sysv, s.domain, s.depth, vx.make_opts(vx.FP32))
        k64 = r64.stats()["kept"].astype(np.float64)
        kmr = rmr.stats()["kept"].astype(np.float64)
        excess = (kmr / np.maximum(k64, 1) - 1.0).tolist()
        t = r64.csf().tuples()
        n = int(t.shape[0])
        if n > 200000:
            sel = torch.from_numpy(np.unique(synth.Stream(11).uniform_int(0, n - 1, 200000))).cuda()
            t = t[sel].contiguous()
        c = vx.csf_build(s.k, s.depth, t)
        _, lo, hi = vx.csf_eval_level(sysv, c, s.domain, vx.FP64, values=True)
        _, mlo, mhi = vx.csf_eval_level(sysv, c, s.domain, vx.FP32_MIDRAD, values=True)
        ratio = ((mhi - mlo) / torch.clamp(hi - lo, min=1e-300)).flatten()
        q = torch.quantile(ratio.float(), torch.tensor([0.5, 0.9, 0.99], device=ratio.device))
        out[name] = {
            "midrad_excess_per_level": [round(x, 4) for x in excess],
            "midrad_excess_max_intermediate": round(max(excess[:-1]) if len(excess) > 1 else 0.0, 4),
            "midrad_excess_final": round(excess[-1], 4),
            "certified_fp32_excess": 0.0 if np.array_equal(r32.stats()["kept"], r64.stats()["kept"]) else None,
            "radius_inflation_median": round(float(q[0]), 4),
            "radius_inflation_p90": round(float(q[1]), 4),
            "radius_inflation_p99": round(float(q[2]), 4),
            "boxes_sampled": int(t.shape[0]),
        }
        c.free()
        for r in (r64, rmr, r32):
            r.free()
    return out


# Table 1 of the paper (single thread, the paper's laptop, Taylor-form C0 and C1 for single
# equations): seconds per cell, for context next to ours (different criteria, other hardware)
PAPER_TABLE1_S = {
    (2, 20): {"points": 0.006, "curves": 0.062, "hypersurfaces": 0.062},
    (2, 100): {"points": 0.32, "curves": 0.31, "hypersurfaces": 0.31},
    (3, 20): {"points": 0.5, "curves": 1.3, "hypersurfaces": 1.1},
    (3, 100): {"points": 273.0, "curves": 270.0, "hypersurfaces": 412.0},
    (4, 20): {"points": 56.0, "curves": 91.0, "hypersurfaces": 373.0},
}


def bench_table1(vx, synth, torch, stream, taylor=True):
    """The random-polynomial family of the experiments (Sec. 4.1, Table 1): k = 2, 3, 4,
    total degree 20 or 100 (20 for k = 4), coefficients U[-10, 10], [-2,2]^k; points (k
    equations) and curves (k-1) to boxes of size 2^-8 (depth 10), hypersurfaces to 2^-5
    (depth 7) with exclusion only.  Certified binary32 enclosure time (system resident, CUDA
    events, best of 2 after a warm-up) and boxes; the paper's seconds as context.  With
    `taylor`, the same cells with C0 on the order-2 Taylor form in certified binary32 and in
    binary64 (one timed run each), and the hypersurfaces with C1 too."""
    out = {}
    for (k, d), paper in PAPER_TABLE1_S.items():
        for kind in ("points", "curves", "hypersurfaces"):
            s = synth.table1(k, d, kind)
            sysv = vx.System(s.polys, stream=stream)
            # levels whose next level would exceed 2^29 boxes run in x1-slab ranges
            opts = vx.make_opts(vx.FP32, small_level_madds=SMALL_LEVEL_MADDS,
                                max_level_boxes=1 << 29)
            # the largest depth <= the paper's that runs (a single x1 slab whose next level
            # exceeds the range's limit cannot be split further)
            depth, note = s.depth, None
            while True:
                try:
                    vx.enclose_system(sysv, s.domain, depth, opts, stream=stream).free()
                    break
                except vx.VxError as e:
                    if e.code != vx.EOVERFLOW or depth <= 1:
                        raise
                    note = "depth %d exceeds one x1 slab's limit (%s)" % (s.depth, e)
                    depth -= 1
            best, r = None, None
            for _ in range(2):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rr = vx.enclose_system(sysv, s.domain, depth, opts, stream=stream)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                if best is None or ms < best:
                    best = ms
                    if r is not None:
                        r.free()
                    r = rr
                else:
                    rr.free()
            st = r.stats()
            cell = {
                "ms": round(best, 3), "depth": depth, "paper_depth": s.depth, "note": note,
                "boxes": int(st["kept"][-1]),
                "box_evals": int(st["tested"].sum()),
                "box_evals_per_s": float(st["tested"].sum()) / (best * 1e-3),
                "paper_voxelize_s": paper[kind]}
            r.free()
            if taylor:
                # C0 on the Taylor form of order 2 (Def. 3) at the same depth, in certified
                # binary32 (the decisions of binary64) and in binary64
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                for tag, mode in (("fp32", vx.FP32), ("fp64", vx.FP64)):
                    to = vx.make_opts(mode, taylor_order=2, small_level_madds=SMALL_LEVEL_MADDS,
                                      max_level_boxes=1 << 29)
                    vx.enclose_system(sysv, s.domain, min(depth, 3), to, stream=stream).free()
                    e0.record(stream)
                    rt = vx.enclose_system(sysv, s.domain, depth, to, stream=stream)
                    e1.record(stream)
                    e1.synchronize()
                    tst = rt.stats()
                    cell["taylor2_" + tag] = {"ms": round(e0.elapsed_time(e1), 3),
                                              "boxes": int(tst["kept"][-1]),
                                              "box_evals": int(tst["tested"].sum()),
                                              "binary64_rechecks": int(tst["recheck"].sum())}
                    rt.free()
                if kind == "hypersurfaces":
                    # as the paper's hypersurface row: C0 and C1 on the Taylor form, C1 from
                    # the size threshold (level 7) on, until no box is left (cap: level 14)
                    cap = 14
                    for tag, mode in (("fp32", vx.FP32), ("fp64", vx.FP64)):
                        to = vx.make_opts(mode, taylor_order=2, c1=vx.C1_TAYLOR, c1_level=depth,
                                          small_level_madds=SMALL_LEVEL_MADDS)
                        e0.record(stream)
                        rt = vx.enclose_system(sysv, s.domain, cap, to, stream=stream)
                        e1.record(stream)
                        e1.synchronize()
                        tst = rt.stats()
                        lev, _ = rt.included()
                        cell["taylor2_c1_" + tag] = {
                            "ms": round(e0.elapsed_time(e1), 3), "c1_level": depth,
                            "level_cap": cap, "certified": int(lev.shape[0]),
                            "certified_per_level": np.bincount(lev, minlength=cap + 1)[depth:].tolist(),
                            "undecided_at_cap": int(tst["kept"][-1] - np.sum(lev == cap)),
                            "box_evals": int(tst["tested"].sum()),
                            "binary64_rechecks": int(tst["recheck"].sum())}
                        rt.free()
            out["k%d-d%d-%s" % (k, d, kind)] = cell
            sysv.free()
    return out


PAPER_APPLICATIONS = {"robotics-R": {"voxelize_s": 0.1, "voxelize_boxes": 7228},
                      "automatic-A": {"voxelize_s": 1.2, "voxelize_boxes": 0}}


def bench_applications(vx, synth, torch, stream):
    """The systems of Sec. 4.2 (equations, inequalities, sqrt(3) coefficients as intervals):
    (R) to boxes of width 2^-4 and 2^-5 (depths 5 and 6 on [-1,1]^4), (A) until no box is left
    (depth 6 on [-1,1]^6).  System resident; CUDA events; best of 3 after a warm-up."""
    out = {}
    for s, depths in ((synth.robotics(), (5, 6)), (synth.automatic(), (6,))):
        sysv = vx.System(s.polys, stream=stream, his=s.his, rel=s.rel)
        cell = {"k": s.k, "polys": len(s.polys),
                "inequalities": int(sum(1 for r in s.rel if r != synth.REL_EQ)),
                "paper": PAPER_APPLICATIONS[s.name]}
        for depth in depths:
            runs = [("fp32", vx.make_opts(vx.FP32, small_level_madds=SMALL_LEVEL_MADDS)),
                    ("fp64", vx.make_opts(vx.FP64))]
            if math.comb(2 + s.k, s.k) <= vx.MAXPOLY:  # the order-2 form's derivatives
                runs.append(("taylor2_fp32", vx.make_opts(vx.FP32, taylor_order=2,
                                                          small_level_madds=SMALL_LEVEL_MADDS)))
                runs.append(("taylor2_fp64", vx.make_opts(vx.FP64, taylor_order=2)))
            for name, opts in runs:
                vx.enclose_system(sysv, s.domain, depth, opts, stream=stream).free()
                best, st = None, None
                for _ in range(3):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    r = vx.enclose_system(sysv, s.domain, depth, opts, stream=stream)
                    e1.record(stream)
                    e1.synchronize()
                    ms = e0.elapsed_time(e1)
                    if best is None or ms < best:
                        best, st = ms, r.stats()
                    r.free()
                cell["depth%d_%s" % (depth, name)] = {
                    "ms": round(best, 3), "boxes": int(st["kept"][-1]),
                    "box_evals": int(st["tested"].sum())}
        out[s.name] = cell
        sysv.free()
    return out


def oracle_batch_sample(systems, nlineages: int, seed: int, procs: int):
    """The oracle on random (system, finest x1-slab) lineages of a batch, spread over
    ``procs`` spawned worker processes: box evaluations per second of wall time."""
    import multiprocessing as mp

    from paper_2406_09857_gb300 import synth

    st = synth.Stream(seed)
    jobs = []
    for _ in range(nlineages):
        polys, domain, depth = systems[int(st.uniform_int(0, len(systems) - 1, 1)[0])]
        jobs.append((polys, domain, depth, int(st.uniform_int(0, (1 << depth) - 1, 1)[0])))
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_lineage_job, jobs[:procs])
        t0 = time.perf_counter()
        res = pool.map(_lineage_job, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    boxes = sum(r[0] for r in res)
    return boxes / wall, boxes, wall


def bench_batch(vx, synth, torch, workers=16, cpu=False):
    """Config 4: 256 independent systems (128 bivariate single equations of degree 10..60 and
    128 trivariate pairs of degree 10..40, depths 8..10) through vx_enclose_batch, from host
    polynomials to host boxes, in each arithmetic; every system's result must agree."""
    systems = [(x.polys, x.domain, x.depth) for x in synth.batch()]
    out = {"workload": "batch: 128 x (k=2, 1 Kostlan poly, d~U{10..60}) + 128 x (k=3, 2 "
                       "Kostlan polys, d~U{10..40}), depth ~U{8..10}, [-1,1]^k",
           "engine": "one CSF forest per k: one launch per depth per level for all systems",
           "timed": "vx_enclose_batch from host polynomials to device-resident results"}
    boxes, evals = {}, {}
    # binary64 first: its box evaluations (the exact subdivision's) are every rate's count
    for name, mode, last in (("fp64", vx.FP64, False), ("fp32", vx.FP32, False),
                             ("fp32_recheck_last", vx.FP32, True)):
        opts = vx.make_opts(mode, recheck_last=last)
        for r in vx.enclose_batch(systems[:16], opts, nworkers=workers):
            r.free()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = vx.enclose_batch(systems, opts, nworkers=workers)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        evals[name] = sum(int(r.stats()["tested"].sum()) for r in res)
        ev = evals["fp64"]
        boxes[name] = [r.boxes() for r in res]
        out[name] = {"value": ev / el, "unit": UNIT, "wall_s": el, "box_evals": ev,
                     "boxes": int(sum(b.shape[0] for b in boxes[name]))}
        if last:
            out[name]["box_evals_run"] = evals[name]
        for r in res:
            r.free()
    out["fp32_equals_fp64"] = all(np.array_equal(a, b) for a, b in zip(boxes["fp32"], boxes["fp64"]))
    out["fp32_recheck_last_equals_fp64"] = all(
        np.array_equal(a, b) for a, b in zip(boxes["fp32_recheck_last"], boxes["fp64"]))
    out["speedup_fp32_vs_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    if cpu:
        ncores = os.cpu_count() or 1
        v, b, t = oracle_batch_sample(systems, 8 * ncores, seed=23, procs=ncores)
        out["cpu_oracle"] = {"box_evals_per_s": v, "box_evals": b, "s": t, "cores": ncores,
                             "sample": "Algorithm 3 along %d random (system, finest x1-slab) "
                                       "lineages of the batch, binary64 directed rounding, in "
                                       "%d spawned processes" % (8 * ncores, ncores),
                             "gpu_fp32_over_all_cores": out["fp32"]["value"] / v}
    return out


def run_reference(args):
    """The CPU oracle as the reference arm: each step runs Algorithm 3 along one random finest
    x1-slab lineage per host core, the lineages spread over spawned worker processes (one per
    core); value = box evaluations / wall time of the steps."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    import multiprocessing as mp

    import oracle
    from paper_2406_09857_gb300 import synth

    oracle.build()
    s = synth.curve()
    ncores = os.cpu_count() or 1
    st = synth.Stream(1000)
    side = 1 << s.depth
    total_boxes, total_s = 0, 0.0
    with mp.get_context("spawn").Pool(ncores) as pool:
        for i in range(args.warmup + args.steps):
            jobs = [(s.polys, s.domain, s.depth, int(x))
                    for x in st.uniform_int(0, side - 1, ncores)]
            t0 = time.perf_counter()
            res = pool.map(_lineage_job, jobs, chunksize=1)
            t = time.perf_counter() - t0
            if i >= args.warmup:
                total_boxes += sum(r[0] for r in res)
                total_s += t
    value = total_boxes / total_s
    sample = ("each step: Algorithm 3 along %d random finest x1-slab lineages (every level's boxes "
              "of each slab), one per host core, in %d spawned processes" % (ncores, ncores))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(1, "CPU oracle, binary64 directed rounding"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def reduce(x, op):
        if world == 1:
            return x
        t = torch.tensor([float(x)], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=op)
        return float(t.item())

    from paper_2406_09857_gb300 import build, shard, synth, vx

    if rank == 0:
        build.build()
    barrier()
    vx.lib()
    s = synth.curve()
    dom, depth = s.domain, s.depth
    torch.cuda.synchronize()
    pk0 = time.perf_counter()
    sysv = vx.System(s.polys)  # packing and upload, once
    torch.cuda.synchronize()
    pack_ms = (time.perf_counter() - pk0) * 1e3
    start = None
    if world > 1:
        lvl0, t0 = shard.rank_start(s.k, depth, rank, world)
        start = vx.csf_build(s.k, lvl0, torch.from_numpy(t0).cuda())

    def enclose_once(mode, timing, recheck_last=True):
        # binary32: the error band re-decided in binary64 at the last level only (the final
        # boxes are binary64's either way; recheck_last=False re-decides it at every level)
        o = vx.make_opts(mode, timing=timing, recheck_last=recheck_last and mode == vx.FP32,
                         first_level=FIRST_LEVEL if mode == vx.FP32 else 0)
        if start is None:
            return vx.enclose_system(sysv, dom, depth, o, stream)
        return vx.enclose_from(sysv, start, dom, depth, o, stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def run_steps(mode, nsteps, timing, recheck_last=True):
        """nsteps enclosures; returns per-step ms, total box-evals, results' stats/timing."""
        ms, evals, tims, last = [], 0, [], None
        for i in range(nsteps):
            flush.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = enclose_once(mode, timing, recheck_last)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            st = r.stats()
            evals += int(st["tested"].sum())
            if timing:
                tims.append(r.timing())
            if last is not None:
                last.free()
            last = r
        return ms, evals, tims, last

    def result_digest(r):
        t = r.csf().tuples()
        if t.shape[0] == 0:
            return 0, 0
        t = t.long()
        h = ((t[:, 0] * 1048583 + t[:, 1]) * 1048589 + t[:, 2]) % 2305843009213693951
        return int(t.shape[0]), int(h.sum().item())

    # ---- headline: binary32 certified, K timed steps -------------------------------------
    log("[bench] warmup %d x fp32" % args.warmup)
    # the first enclosure of the process times the autotuner's variants of every launch shape
    cold_ms, _, _, rc0 = run_steps(vx.FP32, 1, False)
    rc0.free()
    if args.warmup > 1:
        run_steps(vx.FP32, args.warmup - 1, False)[3].free()
    barrier()
    torch.cuda.synchronize()
    launches0 = vx.kernel_launches()
    with ClockSampler(local) as clk:
        w0 = time.perf_counter()
        ms32, evals32, tims32, r32 = run_steps(vx.FP32, args.steps, True)
        torch.cuda.synchronize()
        barrier()
        wall32 = time.perf_counter() - w0
    launches = vx.kernel_launches() - launches0
    clocks = clk.summary()
    st32 = r32.stats()
    t32 = reduce(sum(ms32), torch.distributed.ReduceOp.MAX if world > 1 else None)
    digest32 = result_digest(r32)
    # the same enclosure re-deciding the band at every level (every level's boxes binary64's)
    log("[bench] fp32 with the band re-decided at every level")
    run_steps(vx.FP32, 1, False, recheck_last=False)[3].free()
    msev, evalsev, _, rev = run_steps(vx.FP32, max(1, min(args.steps, 3)), False,
                                      recheck_last=False)
    digest_ev = result_digest(rev)
    rev.free()

    # ---- binary64 beside it ------------------------------------------------------------------
    n64 = max(1, min(args.steps, 2))
    log("[bench] fp64: 1 warmup + %d timed" % n64)
    run_steps(vx.FP64, 1, False)[3].free()
    ms64, evals64, tims64, r64 = run_steps(vx.FP64, n64, True)
    t64 = reduce(sum(ms64), torch.distributed.ReduceOp.MAX if world > 1 else None)
    ev64 = reduce(evals64, torch.distributed.ReduceOp.SUM if world > 1 else None)
    value64 = ev64 / (t64 * 1e-3)
    digest64 = result_digest(r64)
    st64 = r64.stats()
    same = digest32 == digest64 and digest_ev == digest64 and st32["kept"][-1] == st64["kept"][-1]
    # the workload's box evaluations are those of the exact subdivision (binary64's levels)
    # from the level the binary32 run starts at, whose whole grid it tests; the extra
    # evaluations of band boxes kept below the last level are not counted
    if world == 1:
        ev_exact_step = float(st64["tested"][FIRST_LEVEL + 1:].sum()) + float(1 << (s.k * FIRST_LEVEL))
    else:
        ev_exact_step = ev64 / n64
    value = ev_exact_step * args.steps / (t32 * 1e-3)

    def roofline(tims, arith, peak_t):
        tot = {}
        for tm in tims:
            for name, v in tm.items():
                a = tot.setdefault(name, {"ms": 0.0, "launches": 0, "work": 0})
                a["ms"] += v["ms"]
                a["launches"] += v["launches"]
                a["work"] += v["work"]
        evalk = {n: v for n, v in tot.items() if v["launches"] and n.startswith(("stage", "leaf"))}
        top = max(evalk, key=lambda n: evalk[n]["ms"])
        v = evalk[top]
        per_launch_ms = v["ms"] / v["launches"]
        ops_per_launch = v["work"] / v["launches"] * OPS_PER_MADD[arith]
        achieved = ops_per_launch / (per_launch_ms * 1e-3) / 1e12
        share = {n: round(x["ms"] / sum(y["ms"] for y in tot.values()), 4) for n, x in tot.items()
                 if x["launches"]}
        traffic = None
        if arith == "fp32" and top == "leaf_fp32":
            # DRAM bytes per multiply-add of the leaf kernel from one ncu capture of a smaller
            # launch of the same kernel, scaled by the multiply-adds of an average launch
            traffic = LEAF32_DRAM_B_PER_MADD * v["work"] / v["launches"]
        return {"kernel": top, "bound": "alu", "achieved": achieved, "peak": peak_t,
                "unit": "T FMA-pipe lane-ops/s", "frac": achieved / peak_t, "traffic": traffic,
                "traffic_unit": "bytes per launch (DRAM read + write)",
                "launches": v["launches"], "avg_launch_ms": per_launch_ms,
                "madds_per_launch": v["work"] / v["launches"], "time_share": share}

    def roofline_by_kind(tims, fp32_peak, fp64_peak):
        """Every kernel kind of a step with its fraction of the roofline that bounds it: the
        evaluation kinds against the FMA-pipe (binary32) or FP64 (binary64) lane rate (4 lane
        operations per interval multiply-add: both endpoint products of both ends), the integer
        kinds (prune, split, compact, recheck selection, tree builds) against the measured HBM
        copy bandwidth, with their algorithmic bytes (inputs read once, outputs written once)."""
        tot = {}
        for tm in tims:
            for name, v in tm.items():
                a = tot.setdefault(name, {"ms": 0.0, "launches": 0, "work": 0})
                a["ms"] += v["ms"]
                a["launches"] += v["launches"]
                a["work"] += v["work"]
        step_ms = sum(v["ms"] for v in tot.values())
        hbm = PEAKS.get("hbm_gbs")
        out = {}
        for name, v in tot.items():
            if not v["launches"] or v["ms"] <= 0:
                continue
            e = {"ms_per_step": v["ms"] / len(tims), "time_share": v["ms"] / step_ms}
            if name.startswith(("stage", "leaf")):
                peak = fp64_peak if name.endswith("fp64") else fp32_peak
                ach = v["work"] * OPS_PER_MADD["fp32"] / (v["ms"] * 1e-3) / 1e12
                e.update({"bound": "alu", "unit": "T lane-ops/s", "achieved": ach, "peak": peak,
                          "frac": ach / peak, "madds_per_step": v["work"] / len(tims)})
            else:
                ach = v["work"] / (v["ms"] * 1e-3) / 1e9
                e.update({"bound": "hbm", "unit": "GB/s", "achieved": ach, "peak": hbm,
                          "peak_what": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                          "frac": ach / hbm if hbm else None,
                          "bytes_per_step": v["work"] / len(tims)})
            out[name] = e
        return out

    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = int(props.multi_processor_count)
    peak_mhz = (clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or PEAKS.get("sm_max_mhz")
                or NOMINAL_SM_MHZ)
    fp32_peak, fp64_peak = alu_peaks(sms, float(peak_mhz))
    roof32 = roofline(tims32, "fp32", fp32_peak)
    roof64 = roofline(tims64, "fp64", fp64_peak)
    for r in (roof32, roof64):
        r["peak_basis"] = {"sms": sms, "sm_mhz": float(peak_mhz),
                           "lanes_per_sm": FP32_LANES_PER_SM if r is roof32 else FP64_LANES_PER_SM}
    by_kind32 = roofline_by_kind(tims32, fp32_peak, fp64_peak)

    # ---- end to end through the host API -----------------------------------------------------
    log("[bench] e2e")
    polys_host = s.polys

    def e2e_once():
        """Host polynomials in, host boxes out, through the public API."""
        # host_codes: the last compaction writes the boxes' codes into pinned host memory
        o = vx.make_opts(vx.FP32, recheck_last=True, first_level=FIRST_LEVEL, host_codes=True)
        if world == 1:
            r = vx.enclose(polys_host, dom, depth, o)
            return r, sysv.upload_bytes()  # vx_enclose packs and uploads the same system
        sv = vx.System(polys_host)
        st = vx.csf_build(s.k, lvl0, torch.from_numpy(t0).cuda())
        r = vx.enclose_from(sv, st, dom, depth, o)
        return r, sv.upload_bytes() + t0.nbytes

    r0 = e2e_once()[0]  # warm-up, and the pinned result buffer enters the pool
    r0.box_codes(copy=False)
    r0.free()
    ne2e = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    barrier()
    # no collector pauses of the Python harness inside the timed calls (as timeit does)
    import gc

    gc.collect()
    gc.disable()
    w0 = time.perf_counter()
    e2e_evals, d2h, h2d, e2e_ms = 0, 0, 0, []
    for _ in range(ne2e):
        s0 = time.perf_counter()
        r, hb = e2e_once()
        b = r.box_codes(copy=False)  # the result to the host: one grid-index code per box
        e2e_ms.append((time.perf_counter() - s0) * 1e3)
        e2e_evals += ev_exact_step / max(world, 1)
        d2h += b.nbytes
        h2d += hb
        r.free()
    torch.cuda.synchronize()
    e2e_wall = time.perf_counter() - w0
    gc.enable()
    e2e_s = reduce(e2e_wall, torch.distributed.ReduceOp.MAX if world > 1 else None)
    e2e_evals = reduce(e2e_evals, torch.distributed.ReduceOp.SUM if world > 1 else None)
    e2e = {"value": e2e_evals / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d // ne2e,
           "d2h_bytes_per_step": d2h // ne2e, "steps": ne2e,
           "ms_each": [round(x, 2) for x in e2e_ms],
           "what": "vx_enclose from host polynomials (pack + upload) to the host's boxes (one uint32 grid-index code per box, written into pinned host memory by the last level's compaction: host_codes; vx_result_box_codes)"}

    # ---- config 5: one complete level (Property 1's dense grid), and config 4: the batch ----
    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        log("[bench] dense level and batch")
        extra["dense_level"] = bench_dense(vx, synth, torch, stream, flush)
        extra["dense_sweep"] = bench_dense_sweep(vx, synth, torch, stream, flush)
        extra["batch"] = bench_batch(vx, synth, torch, cpu=not args.no_cpu)
        extra["precision"] = bench_precision(vx, synth, torch)
        extra["configs"] = bench_configs(vx, synth, torch, stream, not args.no_cpu,
                                         args.cpu_budget)
        extra["table1"] = bench_table1(vx, synth, torch, stream)
        extra["applications"] = bench_applications(vx, synth, torch, stream)

    # ---- CPU oracle on a bounded sample ------------------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        log("[bench] cpu baseline (%.0f s budget)" % args.cpu_budget)
        import oracle

        oracle.build()
        v, b, t, desc = oracle_sample(s.polys, s.domain, s.depth, args.cpu_budget, seed=7)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}

    if rank == 0:
        peaks = PEAKS
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t32 / args.steps, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
            "dtype": "f32 (float pairs, then f64, on the error band)", "data": "synthetic",
            "config": config_dict(world, "binary32 intervals from the full level-%d grid; the "
                                         "error band re-decided at the last level (recheck_last) "
                                         "by float pairs, then binary64" % FIRST_LEVEL),
            "boxes_final": int(st32["kept"][-1]), "box_evals_per_step": int(ev_exact_step),
            "box_evals_run_per_step": evals32 // args.steps,
            "every_level_recheck": {"ms_median": statistics.median(msev),
                                    "value": evalsev / (sum(msev) * 1e-3),
                                    "what": "the band re-decided at every level: every "
                                            "level's boxes are binary64's"},
            "wall_s_timed_region": wall32,
            "enclosure_ms": {"median": statistics.median(ms32), "min": min(ms32),
                             "max": max(ms32),
                             "cold": {"pack_and_upload_ms": pack_ms,
                                      "first_enclosure_ms": cold_ms[0],
                                      "note": "the process's first enclosure, autotuning "
                                              "every launch shape on the way"}},
            "fp64": {"value": value64, "ms_per_step": t64 / n64, "steps": n64,
                     "roofline": roof64},
            "speedup_vs_fp64": value / value64,
            "same_result_as_fp64": bool(same),
            "excess_boxes": 0.0 if same else None,
            "recheck_boxes_per_step": int(st32["recheck"].sum()),
            "binary64_recheck_boxes_per_step": int(st32["recheck64"].sum()),
            "roofline": roof32,
            "roofline_by_kind": by_kind32,
            "cpu_baseline": cpu,
            **extra,
            "e2e": e2e,
            "gpu_launches": launches,
            "gpu_launches_per_step": launches / args.steps,
            "clocks": clocks,
            "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")} if peaks else None,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_profile_case(args):
    """One enclosure of the workload to --profile-case DEPTH (a small case for ncu captures)."""
    import torch

    from paper_2406_09857_gb300 import synth, vx

    torch.cuda.set_device(0)
    s = synth.curve()
    mode = {"fp32": vx.FP32, "fp64": vx.FP64, "midrad": vx.FP32_MIDRAD}[args.mode]
    if args.variant is not None:  # one launch per kernel and level: variant V everywhere
        vx.autotune(2 + args.variant)
    r = vx.enclose_system(vx.System(s.polys), s.domain, args.profile_case, vx.make_opts(mode))
    torch.cuda.synchronize()
    st = r.stats()
    print(json.dumps({"profile_case_depth": args.profile_case, "mode": args.mode,
                      "boxes": int(st["kept"][-1]), "tested": st["tested"].tolist(),
                      "kept": st["kept"].tolist(), "nodes": st["nodes"].tolist(),
                      "madds": st["madds"].tolist(), "ms": r.elapsed_ms()}))
    return 0


def run_profile_dense(args):
    """One tensor-core prefilter of the degree-128 dense tensor at --profile-dense LEVEL (a
    small case for ncu captures: 3 tensor-core launches after the plan's 9 factor launches)."""
    import torch

    from paper_2406_09857_gb300 import synth, vx

    torch.cuda.set_device(0)
    s = synth.dense_sweep(128)
    plan = vx.DensePlan(vx.System(s.polys), args.profile_dense, s.domain)
    mask = plan.prefilter()
    torch.cuda.synchronize()
    n = 1 << (3 * args.profile_dense)
    print(json.dumps({"profile_dense_level": args.profile_dense, "plan_bytes": plan.device_bytes(),
                      "prefilter_kept": int(vx.mask_to_bool(mask, n).sum().item())}))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["vx", "reference"], default="vx")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of CPU oracle work for the cpu_baseline sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline sample")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the dense-level and batch sub-reports")
    ap.add_argument("--profile-case", type=int, default=None, metavar="DEPTH",
                    help="run one enclosure of the workload to DEPTH and exit (for ncu)")
    ap.add_argument("--profile-dense", type=int, default=None, metavar="LEVEL",
                    help="run one tensor-core prefilter of the degree-128 dense tensor at LEVEL "
                         "and exit (for ncu)")
    ap.add_argument("--mode", choices=["fp32", "fp64", "midrad"], default="fp32",
                    help="arithmetic of --profile-case")
    ap.add_argument("--variant", type=int, default=None, metavar="V",
                    help="--profile-case: launch variant V of every kernel that has one, no "
                         "autotuning (0 two boxes per thread, 2 leaves from shared memory)")
    args = ap.parse_args()
    if args.profile_case is not None:
        return run_profile_case(args)
    if args.profile_dense is not None:
        return run_profile_dense(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
