#!/usr/bin/env python
"""Demag evaluations per second of the tetrahedral FMM (Palmesi et al.) on GB300.

One step = one demag_eval of the whole hot path (P2M, M2M, M2L, L2L, L2P, P2P,
lumped H) over a batch of B magnetisation states of the workload mesh, inputs
resident in HBM.  The metric counts (mesh, state) evaluations per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--precision fp64|fp32|tf32|bf16x3] [--batch B]

Default workload: the ball of 559,564 quasi-uniform Delaunay tets with 256
magnetisation states (unit vectors smoothed over 3 mesh-neighbour passes),
p = 8, theta = 0.5, split-BF16, leaf size picked by the library's leaf tuner.
The accuracy gate of the metric (rel-L2 of u and H against the FP64 GPU FMM of
the same plan settings, <= 1e-4) is checked on every state.

--impl reference times the CPU oracle (the plain FP64 FMM of oracle/) on the
host cores, on a fixed sample of the same workload (the full upward pass plus
4 target leaves per thread, extrapolated to all target leaves) -- the same
sample as the cpu_baseline of our own line.
Multi-GPU (torchrun): every rank evaluates its own batch on its own GPU
(replicas, no data-path collective); value = all ranks' evals / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "demag evals/sec at rel-L2 1e-4 vs FP64: mixed+batched vs FP64 GPU FMM"
UNIT = "evals/s"

# Workloads.  sphere500k is the batched configuration the metric is quoted
# on: many magnetisation states on one ~500k-tet ball (seeded unit vectors
# smoothed over 3 mesh-neighbour passes), leaf size from the leaf tuner.
# batch / autotune are the defaults of each workload (--batch / --autotune
# override them).
WORKLOADS = {
    "sphere500k": dict(mesh="sphere", h="SPHERE_500K_H", p=8, theta=0.5, leaf=128, M="smoothed", batch=256,
                       autotune=3),
    # the ~200k-tet ball with Gaussian unit states
    "sphere200k": dict(mesh="sphere", h="SPHERE_200K_H", p=8, theta=0.5, leaf=128, batch=128, autotune=1),
    "cube8": dict(mesh="cube", n=8, p=4, theta=0.5, leaf=32, batch=128, autotune=1),
    "sphere30k": dict(mesh="sphere", h=0.095, p=6, theta=0.5, leaf=32, batch=128, autotune=1),
    # 64 meshes of uneven size (10k-300k tets: cubes, balls, ellipsoids) in one submission
    "multi64": dict(mesh="multi", n=64, p=8, theta=0.5, leaf=128, M="smoothed", batch=1, autotune=1),
}


def aggregate_ranks(total_ms, evals_per_rank, world, device):
    """Whole-job throughput of replicas: every rank evaluated `evals_per_rank`
    (mesh, state) pairs in `total_ms`; the job time is the maximum over ranks
    and the value is all ranks' evaluations over that time.  Returns
    (max_ms, evals/s).  With world > 1 the process group must be initialised."""
    if world > 1:
        import torch

        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
        torch.distributed.barrier()
    return total_ms, world * evals_per_rank / (total_ms * 1e-3)


def workload(args):
    """The named workload with any --p / --leaf / --theta / --batch / --autotune
    overrides; also fills args.batch and args.autotune from the workload's
    defaults when they are not given."""
    w = dict(WORKLOADS[args.workload])
    for k in ("p", "leaf", "theta"):
        v = getattr(args, k, None)
        if v:
            w[k] = v
    if getattr(args, "batch", 0) in (0, None):
        args.batch = w["batch"]
    if getattr(args, "autotune", -1) in (-1, None):
        args.autotune = w["autotune"]
    if getattr(args, "leaf", 0):
        args.autotune = int(args.autotune) & ~2  # a given leaf size is not tuned
    w["cpu_leaf"] = w["leaf"]  # the CPU legs use the requested leaf (the GPU leaf tuner does not run there)
    return w


def make_mesh(w):
    from paper_1606_00247_gb300 import inputs

    if w["mesh"] == "cube":
        return inputs.unit_cube(w["n"])
    h = getattr(inputs, w["h"]) if isinstance(w["h"], str) else w["h"]
    return inputs.sphere(h=h)


def make_M(nn, B, seed_offset=0, tets=None, w=None):
    from paper_1606_00247_gb300 import inputs

    if w is not None and w.get("M") == "smoothed":
        return inputs.smoothed_unit_m(tets, nn, batch=B, seed=inputs.MAG_SEED + 3 + seed_offset)
    return inputs.gaussian_unit_m(nn, seed=inputs.MAG_SEED + 1 + seed_offset, batch=B)


def data_note(w):
    shape = "seeded Delaunay ball" if w["mesh"] == "sphere" else w["mesh"]
    mag = "unit nodal M smoothed over 3 neighbour passes" if w.get("M") == "smoothed" else "Gaussian unit nodal M"
    return f"synthetic ({shape}, {mag})"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def live_peaks():
    """MEASURED_PEAKS.json (HBM copy, cuBLAS BF16) plus this run's own FMA and
    tcgen05 microbenchmarks (keys <kind>_measured)."""
    peaks = dict(measured_peaks())
    try:
        for k, v in measure_peaks().items():
            peaks[k + "_measured"] = v
    except Exception as e:  # the line still reports the unit-count peaks
        peaks["peaks_error"] = str(e)
    return peaks


# FP64 operations of the on-the-fly near field per (target node, source tet)
# pair, counted from the source (p2p.cuh, p2p.cu); sqrt, log1p, divisions and
# atan2 are not counted.
#  batches of fewer than P2P_AT_MIN_B states, pair_contract per pair and state:
#   12 subtractions, 4 norms (5 each), 6 edges x 4, 4 faces x (h 5, triple
#   product 14, 3 dots 15, denominator 7, 3 edges x 14, face combination 12),
#   M(r) 18  -> 48+24+4*95+18 = 470 per state;
#  larger batches, pair_at once per pair (12 + 20 + 24 + 1, then 4 faces x
#   (h 5, triple product 14, 3 dots 15, denominator 8, Om and I 2, 3 edges x 69,
#   a 12, T 87) = 1457) and 44 per state (M(r) 18, T:J 14, M(r).a + T:J/2 7,
#   the warp's shuffle sum 5).
P2P_AT_MIN_B = 2
P2P_PAIR_FLOPS, P2P_STATE_FLOPS, P2P_PERSTATE_FLOPS = 1457, 44, 470


def p2p_fp64_flops(B):
    """FP64 flops of one (target node, source tet) pair for a batch of B states."""
    return P2P_PERSTATE_FLOPS * B if B < P2P_AT_MIN_B else P2P_PAIR_FLOPS + P2P_STATE_FLOPS * B


def m2l_macs(p):
    """Multiply-adds of one M2L pair for one state: #{(n, m): |n| + |m| <= p} = C(p+6, 6)."""
    from math import comb

    return comb(p + 6, 6)


def m2l_split_degree(p):
    """The library's default split degree of the tensor-core M2L: the products
    with the second BF16 limb only for terms |m| + |n| <= p - 4 (p - 3 below
    order 8)."""
    return p - 4 if p >= 8 else p - 3


def m2l_tile_flops(p, precision, split_all=False):
    """Flops the tensor-core M2L issues per pair and state: every k-step
    (16 BF16 or 8 TF32 values of n) is one M = 128 MMA over the rows m still
    needed at that k-step (rows of degree t need |n| < C(p - t + 3, 3)),
    padded to 16.  Split BF16 adds the hi x lo and lo x hi MMAs over the rows
    whose terms take the second limb (degree <= split degree - the k-step's
    lowest |n|; every row with split_all)."""
    cnc = lambda t: 0 if t < 0 else (t + 1) * (t + 2) * (t + 3) // 6
    pad = lambda x, m: (x + m - 1) // m * m
    deg = lambda m: next(t for t in range(p + 1) if cnc(t) > m)
    kw = 16 if precision == "bf16x3" else 8
    sd = m2l_split_degree(p)
    total = 0
    for ks in range(pad(cnc(p), kw) // kw):
        rows = pad(max([cnc(t) for t in range(p + 1) if cnc(p - t) > ks * kw] or [0]), 16)
        total += rows * kw
        if precision == "bf16x3":
            r = sd - deg(ks * kw)
            rows2 = rows if split_all else min(pad(cnc(r), 16) if r >= 0 else 0, rows)
            total += 2 * rows2 * kw
    return 2.0 * total


def alu_peak_tflops(kind, sm_mhz):
    """Peak from unit counts x clock: 152 SMs x 128 FP32 lanes (FMA = 2 flops);
    FP64 is 1/64 of that on GB300 (nominal 1.25 TFLOP/s at 2.07 GHz).  Used only
    when the live measurement (demag_measure_peak) is not available."""
    lanes = 152 * 128 * 2 * (sm_mhz or 2070.0) * 1e6
    return lanes / 1e12 if kind == "fp32" else lanes / 64 / 1e12


def measure_peaks(kinds=("fp64_fma", "fp32_fma", "tf32_mma", "bf16_mma")):
    """Arithmetic peaks of this GPU measured by the library's own microbenchmarks
    (demag_measure_peak): TFLOP/s per kind, None where the probe failed."""
    from paper_1606_00247_gb300 import _lib as L

    out = {}
    for k in kinds:
        st, v = L.demag_measure_peak(L.PEAK_KINDS[k])
        out[k] = v if st == L.DEMAG_OK else None
    return out


def _alu_peak(kind, peaks, sm_mhz):
    """(peak TFLOP/s, source) of the FP64 or FP32 CUDA-core path."""
    v = peaks.get(f"{kind}_fma_measured")
    if v:
        return v, f"measured {kind.upper()} FMA (demag_measure_peak, this run)"
    return alu_peak_tflops(kind, sm_mhz), (f"derived: 152 SMs x 128 FP32 lanes x 2 x {sm_mhz or 2070:.0f} MHz"
                                           + (" / 64 (FP64)" if kind == "fp64" else ""))


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of a
# kernel, from one ncu capture on GB300 of this exact configuration and kernel
# version; any other configuration reports null
NCU_TRAFFIC = {
    # (stage, precision, p, leaf, batch, n_tets): bytes
    # ball of 559,564 tets, 256 states, leaf 512 (the headline workload): one launch of k_m2l_tc
    # (22.457 GB read + 0.469 GB written), ncu --metrics
    # gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum on
    # python bench.py --workload sphere500k --leaf 512 --autotune 1 --steps 1 --warmup 3
    # --no-cpu-baseline --no-fp64-ref.  The same capture measured k_near_tc at 16.648 GB, but
    # that kernel has changed since (the M of a column group copied per run of consecutive
    # node ids), so its traffic is reported as unknown until it is captured again.
    ("m2l", "bf16x3", 8, 512, 256, 559564): 22.926e9,
}


def m2l_on_tensor_cores(precision, B, table_batch):
    """The tensor-core precisions run the FP32 table M2L on CUDA cores up to
    m2l_table_batch states (0: the library default of 8; < 0: never)."""
    limit = 8 if table_batch == 0 else max(table_batch, 0)
    return precision in ("tf32", "bf16x3", "bf16x6") and B > limit


def _peak_bf16(peaks):
    sus = peaks.get("bf16_tflops_sustained")
    return (sus, "measured bf16 sustained (MEASURED_PEAKS.json)") if sus else (
        peaks.get("bf16_tflops", 1900.0), "measured bf16 burst (MEASURED_PEAKS.json)")


def stage_roofline(stage, stats, steps_profiled, precision, peaks, sm_mhz, tensor_m2l=True):
    """Roofline record of one stage from its live per-stage CUDA-event time
    (summed over the profiled evaluations, divided by its launches)."""
    ms = stats["stage_ms"][stage]
    launches = max(1, stats["stage_launches"][stage])
    per_launch_s = ms / launches * 1e-3
    launches_per_eval = launches / max(1, steps_profiled)
    B, p, nn = stats["_batch"], stats["p"], stats["n_nodes"]
    out = {"kernel": stage, "ms_per_step": ms / max(1, steps_profiled), "launches_per_step": launches_per_eval}
    key = (stage, precision, p, stats["leaf_size"], B, stats["n_tets"])
    kind = "fp64" if precision == "fp64" else "fp32"
    if stage == "m2l":
        work = 2.0 * stats["n_m2l"] * m2l_macs(p) * B / launches_per_eval
        if precision in ("tf32", "bf16x3") and tensor_m2l:
            # tcgen05 M2L timed inside a long step: the sustained measured BF16 rate is
            # the denominator (TF32: x the nominal TF32/BF16 ratio 1.1 / 2.25 PFLOP/s)
            base, src = _peak_bf16(peaks)
            peak = base
            if precision == "tf32":
                peak = peaks.get("tf32_mma_measured") or base * (1.1 / 2.25)
                src = ("measured TF32 tcgen05.mma (demag_measure_peak, this run)" if peaks.get("tf32_mma_measured")
                       else src + " x 1.1/2.25 nominal TF32 ratio")
            tile_flops = (m2l_tile_flops(p, precision, split_all=stats.get("_split_all", False)) * stats["n_m2l"] * B
                          / launches_per_eval)
            achieved = work / per_launch_s / 1e12
            out.update({"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": NCU_TRAFFIC.get(key),
                        "executed_tflops": tile_flops / per_launch_s / 1e12,
                        "peak_source": src,
                        "note": "achieved counts algorithmic flops 2*C(p+6,6) per pair per state; executed_tflops "
                                "counts the padded per-k-step row prefixes issued to the tensor pipe "
                                + ("(hi x hi everywhere, hi x lo and lo x hi on the rows whose terms take the "
                                   "second limb)" if precision == "bf16x3" else "(1 TF32 MMA per tile)")})
            return out
        achieved = work / per_launch_s / 1e12
        peak, src = _alu_peak(kind, peaks, sm_mhz)
        out.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": NCU_TRAFFIC.get(key), "peak_source": src,
                    "note": f"algorithmic flops 2*C(p+6,6) per pair per state, {kind} CUDA cores"})
        return out
    if stage == "p2p" and stats["near_mode"] == 0:
        work = stats["n_p2p_pairs"] * p2p_fp64_flops(B) / launches_per_eval
        achieved = work / per_launch_s / 1e12
        peak, src = _alu_peak("fp64", peaks, sm_mhz)
        out.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": NCU_TRAFFIC.get(key), "peak_source": src,
                    "note": (f"FP64 pipe, {p2p_fp64_flops(B)} FP64 flops per (node, tet) pair for {B} states "
                             "(pair geometry once per pair from 2 states on); transcendentals not counted")})
        return out
    if stage == "p2p":
        # stored near field: every (target node, source node) coefficient triple read once per
        # launch in the stored format, M of every node and u of every node once per state
        pairs = stats["n_near_cols"]
        tc = stats.get("n_near_tiles", 0) > 0
        w_bytes = 12 if tc else (16 if kind == "fp32" else 24)
        alg = (pairs * w_bytes + nn * B * (12 if kind == "fp32" else 24) + nn * B * 2 * (4 if kind == "fp32" else 8))
        alg /= launches_per_eval
        achieved = alg / per_launch_s / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        flops = 2.0 * 3 * pairs * B / launches_per_eval
        out.update({"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": NCU_TRAFFIC.get(key), "algorithmic_bytes": alg,
                    "stored_bytes": stats.get("near_bytes"),
                    "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)" if "hbm_gbs" in peaks
                                   else "fallback 6800 GB/s",
                    "note": (f"{w_bytes} B of stored coefficients per (target node, source node) pair "
                             "(3 components"
                             + (" x 2 BF16 limbs" if tc else "") + ") read once, M and u of every node once "
                             "per state; tiles of the tensor-core near field also store zeros where a column is "
                             "outside a row's near set (stored_bytes)")})
        if tc:
            base, src = _peak_bf16(peaks)
            ach_t = flops / per_launch_s / 1e12
            out["tensor_view"] = {"achieved": ach_t, "peak": base, "unit": "TFLOP/s", "frac": ach_t / base,
                                  "peak_source": src,
                                  "note": "2 flops per coefficient component and state (3 BF16 MMAs issue 3x this)"}
        return out
    out.update({"bound": "hbm", "achieved": None, "peak": peaks.get("hbm_gbs", 6800.0), "unit": "GB/s",
                "frac": None, "traffic": None})
    return out


def roofline_for(stats, steps_profiled, precision, peaks, sm_mhz, tensor_m2l=True):
    """Roofline of the dominant stage, plus the M2L and near-field records."""
    ms = stats["stage_ms"]
    dom = max(ms, key=lambda k: ms[k])
    out = stage_roofline(dom, stats, steps_profiled, precision, peaks, sm_mhz, tensor_m2l)
    out["stage_ms_per_step"] = {k: round(v / max(1, steps_profiled), 4) for k, v in ms.items()}
    out["stages"] = {st: stage_roofline(st, stats, steps_profiled, precision, peaks, sm_mhz, tensor_m2l)
                     for st in ("m2l", "p2p") if ms.get(st, 0) > 0}
    return out


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
class OracleSampler:
    """The oracle FMM (plain CPU FP64, one state) timed on a fixed sample of the
    workload: the full upward pass (P2M, M2M) plus n target leaves spread
    evenly over all target leaves (default 4 per thread), the downward time
    extrapolated to every target leaf.  The leaf size is the workload's
    requested one (the GPU leaf tuner does not run on the CPU legs), so the
    cpu_baseline of our line and the --impl reference line time the same
    sample."""

    def __init__(self, nodes, tets, w):
        import oracle

        oracle.build()
        self.oracle = oracle
        self.w = w
        self.leaf = w.get("cpu_leaf", w["leaf"])
        self.tree = oracle.Tree(nodes, tets, self.leaf, w["theta"])
        ex = self.tree.export()
        self.leaves = np.where((ex["cell_child"][:, 1] == 0) & (ex["cell_ranges"][:, 3] > ex["cell_ranges"][:, 2]))[0]

    def run(self, M1, nthreads=0, n_leaves=None):
        threads = nthreads if nthreads > 0 else self.oracle.max_threads()
        n = int(min(len(self.leaves), n_leaves or 4 * threads))
        sample = self.leaves[np.linspace(0, len(self.leaves) - 1, n).astype(np.int64)]
        p = self.w["p"]
        t0 = time.perf_counter()
        self.tree.fmm(M1, p, target_leaves=np.zeros(0, np.int64), nthreads=nthreads)
        t_up = time.perf_counter() - t0
        t0 = time.perf_counter()
        self.tree.fmm(M1, p, target_leaves=sample, nthreads=nthreads)
        t_tot = time.perf_counter() - t0
        t_down = max(0.0, t_tot - t_up)
        t_eval = t_up + t_down * len(self.leaves) / n
        return {"value": 1.0 / t_eval, "unit": UNIT, "cores": threads, "kind": "oracle",
                "sample": f"plain CPU FMM, p={p}, leaf {self.leaf}, 1 state, {threads} thread(s): full upward pass "
                          f"({t_up:.2f} s) + {n}/{len(self.leaves)} target leaves ({t_down:.2f} s), "
                          f"extrapolated to all target leaves",
                "seconds": t_up + t_tot}


def direct_sample(nodes, tets, M1, u_fmm64=None, n=64, seed=1606):
    """The oracle's direct sum (the plain definition of u, Eq. (2), every tet at
    every target in closed form) at n seeded target nodes on all host cores: its
    time extrapolated to every node, and, given the FP64 GPU FMM's u of the same
    state, the FMM's truncation error at those nodes."""
    import oracle

    nn = nodes.shape[0]
    tg = np.sort(np.random.default_rng(seed).choice(nn, size=min(n, nn), replace=False))
    t0 = time.perf_counter()
    ud = oracle.direct(nodes, tets, M1, targets=tg)
    t = time.perf_counter() - t0
    out = {"kind": "oracle_direct", "value": len(tg) / (t * nn), "unit": UNIT, "cores": oracle.max_threads(),
           "sample": f"direct sum over all {tets.shape[0]} tets at {len(tg)} seeded target nodes ({t:.2f} s), "
                     f"extrapolated to all {nn} nodes", "seconds": t}
    if u_fmm64 is not None:
        out["fp64_gpu_fmm_vs_direct_rel_l2"] = float(np.linalg.norm(u_fmm64[tg] - ud) / np.linalg.norm(ud))
    return out


def cpu_baseline(nodes, tets, w, M1, single_core=True):
    """All-thread oracle sample, plus a single-thread one (upward pass + 4 leaves)."""
    smp = OracleSampler(nodes, tets, w)
    out = smp.run(M1)
    if single_core:
        one = smp.run(M1, nthreads=1, n_leaves=4)
        out["single_core"] = {k: one[k] for k in ("value", "unit", "cores", "sample", "seconds")}
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1606_00247_gb300 import build
    from paper_1606_00247_gb300.api import Plan

    build()
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    w = workload(args)
    w["name"] = args.workload
    if w["mesh"] == "multi":
        return run_multi(args, rank, world, local_rank, w)
    if args.llg_steps:
        return run_llg(args, rank, local_rank, w)
    nodes, tets = make_mesh(w)
    B = args.batch
    plan = Plan(nodes, tets, p=w["p"], leaf_size=w["leaf"], theta=w["theta"], precision=args.precision,
                near_mode=args.near_mode, max_batch=B, device=dev, autotune=int(args.autotune),
                m2l_table_batch=args.m2l_table_batch, m2l_split_degree=args.m2l_split_degree, sources=args.sources)
    st0 = plan.stats()
    w["leaf"] = st0["leaf_size"]  # the leaf kept by the leaf-size tuner (autotune bit 1), else the requested one
    w["p"] = st0["p"]  # the order kept by the order tuner (autotune bit 2), else the requested one
    M = torch.as_tensor(make_M(nodes.shape[0], B, seed_offset=rank, tets=tets, w=w), device=dev)
    u = torch.empty((B, nodes.shape[0]), dtype=torch.float64, device=dev)
    H = torch.empty((B, nodes.shape[0], 3), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        plan.eval(M, u, H)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # L2 flushed between timed steps (outside the events)
        ev[k][0].record(stream)
        plan.eval(M, u, H)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    launches = plan.stats()["eval_launches"] * args.steps
    u_acc, H_acc = u.clone(), H.clone()  # the timed evaluation's outputs, for the accuracy gate
    from paper_1606_00247_gb300 import _lib as L

    device_status = L.demag_status_string(L.demag_eval_status(plan.handle, stream.cuda_stream))
    total_ms, value = aggregate_ranks(total_ms, B * args.steps, world, dev)

    # end to end through the C ABI with host buffers (H2D of M, D2H of u and H inside the
    # call), in pinned host memory
    Mh = torch.empty((B, nodes.shape[0], 3), dtype=torch.float64).pin_memory().numpy()
    Mh[:] = make_M(nodes.shape[0], B, seed_offset=rank, tets=tets, w=w)
    uh = torch.empty((B, nodes.shape[0]), dtype=torch.float64).pin_memory().numpy()
    Hh = torch.empty((B, nodes.shape[0], 3), dtype=torch.float64).pin_memory().numpy()
    plan.eval_host(Mh, u=uh, H=Hh)
    t_e2e = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        plan.eval_host(Mh, u=uh, H=Hh)
        t_e2e.append(time.perf_counter() - t0)
    e2e_value = world * B * args.steps / sum(t_e2e)

    # live per-stage timing pass (CUDA events on the eval stream, inside the library)
    prof = Plan(nodes, tets, p=w["p"], leaf_size=w["leaf"], theta=w["theta"], precision=args.precision,
                near_mode=args.near_mode, max_batch=B, device=dev, profile=True, autotune=int(args.autotune) & 1,
                m2l_table_batch=args.m2l_table_batch, m2l_split_degree=args.m2l_split_degree, sources=args.sources)
    for _ in range(2):
        prof.eval(M, u, H)
    prof.reset_timers()
    nprof = max(2, min(args.steps, 5))
    for _ in range(nprof):
        flush.zero_()
        prof.eval(M, u, H)
    prof_status = L.demag_status_string(L.demag_eval_status(prof.handle, stream.cuda_stream))
    pst = prof.stats()
    pst["_batch"] = B
    pst["near_mode"] = args.near_mode
    pst["_split_all"] = args.m2l_split_degree < 0
    peaks = live_peaks()
    roof = roofline_for(pst, nprof, args.precision, peaks, clk.get("sm_mhz"),
                        m2l_on_tensor_cores(args.precision, B, args.m2l_table_batch))
    roof["peaks_measured_live"] = {k: peaks.get(k + "_measured") for k in ("fp64_fma", "fp32_fma", "tf32_mma",
                                                                             "bf16_mma")}
    prof.close()

    # FP64 GPU FMM of the same plan settings: throughput, and the accuracy gate
    # of the metric (rel-L2 of u and of H vs FP64, per state, every state)
    ref_info = None
    u0_64 = u_acc[0].cpu().numpy() if args.precision == "fp64" else None
    if args.precision != "fp64" and not args.no_fp64_ref:
        nb = min(B, 16)
        p64 = Plan(nodes, tets, p=w["p"], leaf_size=w["leaf"], theta=w["theta"], precision="fp64",
                   near_mode=1, max_batch=nb, device=dev, sources=args.sources)
        eu, eh = [], []
        for k0 in range(0, B, nb):
            kb = min(nb, B - k0)
            u64, H64 = p64.eval(M[k0:k0 + kb])
            if k0 == 0:
                u0_64 = u64[0].cpu().numpy()  # state 0 in FP64, for the direct-sum sample
            eu += (torch.linalg.norm(u_acc[k0:k0 + kb] - u64, dim=1) / torch.linalg.norm(u64, dim=1)).tolist()
            dh = (H_acc[k0:k0 + kb] - H64).reshape(kb, -1)
            eh += (torch.linalg.norm(dh, dim=1) / torch.linalg.norm(H64.reshape(kb, -1), dim=1)).tolist()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p64.eval(M[:1])
        ev0.record(stream)
        for _ in range(2):
            p64.eval(M[:1])
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        t64 = ev0.elapsed_time(ev1) / 2
        ev0.record(stream)
        for _ in range(2):
            p64.eval(M[:nb])
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        t64b = ev0.elapsed_time(ev1) / 2
        p64.close()
        ref_info = {"fp64_gpu_fmm_evals_per_s": 1e3 / t64, "fp64_ms_per_eval": t64, "fp64_near_mode": 1,
                    "fp64_batched_evals_per_s": nb * 1e3 / t64b, "fp64_batch": nb,
                    "rel_l2_u_vs_fp64": max(eu), "rel_l2_H_vs_fp64": max(eh),
                    "rel_l2_u_median": float(np.median(eu)), "rel_l2_H_median": float(np.median(eh)),
                    "states_checked": len(eu), "meets_1e-4": bool(max(eu) <= 1e-4 and max(eh) <= 1e-4),
                    "speedup_vs_fp64_gpu_fmm": value / (1e3 / t64),
                    "speedup_vs_fp64_batched": value / (nb * 1e3 / t64b)}

    if rank != 0:
        return None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": data_note(w),
        "config": {"workload": args.workload, "n_tets": st0["n_tets"], "n_nodes": st0["n_nodes"],
                   "p": w["p"], "theta": w["theta"], "leaf_size": w["leaf"], "batch_per_gpu": B,
                   "precision": args.precision, "near_mode": args.near_mode, "l2": "flushed between steps",
                   "sources": args.sources, "m2l_split_degree": ("default" if args.m2l_split_degree == 0 else "all"),
                   "parallelism": f"replicas x{world}", "n_cells": st0["n_cells"], "n_m2l": st0["n_m2l"],
                   "n_p2p_leaf_pairs": st0["n_p2p"], "n_p2p_pairs": st0["n_p2p_pairs"],
                   "plan_ms": st0["plan_ms"], "m2l_operators": st0["n_m2l_ops"],
                   "m2l_ring": {"targets_per_cta": st0["m2l_targets_per_cta"], "kps": st0["m2l_kps"],
                                "bytes": st0["m2l_ring_bytes"],
                                "autotuned": bool(args.autotune & 1)},
                   "leaf_tuned": bool(args.autotune & 2), "p_tuned": bool(args.autotune & 4)},
        "roofline": roof,
        "fp64_reference": ref_info,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(Mh.nbytes),
                "d2h_bytes_per_step": int(uh.nbytes + Hh.nbytes), "host_buffers": "pinned"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "wall_s_timed": wall,
        "device_status": {"timed": device_status, "profiled": prof_status},
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(nodes, tets, w, make_M(nodes.shape[0], 1, tets=tets, w=w)[0],
                                           single_core=not args.no_single_core)
        try:  # a reference row; a failure here is recorded, it does not void the measured line
            out["cpu_baseline"]["direct_sample"] = direct_sample(nodes, tets, M[0].cpu().numpy(), u0_64)
        except Exception as e:  # noqa: BLE001
            out["cpu_baseline"]["direct_sample"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def run_llg(args, rank, local_rank, w):
    """LLG stepping of B states (demag_llg_rk4): classical RK4, each stage one
    batched evaluation of the B stage states; reports steps/s and the
    evaluations/s inside them."""
    import torch

    from paper_1606_00247_gb300 import inputs
    from paper_1606_00247_gb300.api import Plan

    dev = torch.device(f"cuda:{local_rank}")
    nodes, tets = make_mesh(w)
    B = args.batch
    pl = Plan(nodes, tets, p=w["p"], leaf_size=w["leaf"], theta=w["theta"], precision=args.precision,
              near_mode=args.near_mode, max_batch=B, device=dev, autotune=int(args.autotune) & 1,
              m2l_table_batch=args.m2l_table_batch, m2l_split_degree=args.m2l_split_degree)
    m = torch.as_tensor(inputs.smoothed_unit_m(tets, nodes.shape[0], batch=B, seed=inputs.MAG_SEED + 9), device=dev)
    pl.llg_rk4(m, Ms=1.0, alpha=0.1, dt=0.02, steps=max(1, args.warmup))
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local_rank)
    clocks.start()
    t0 = time.perf_counter()
    pl.llg_rk4(m, Ms=1.0, alpha=0.1, dt=0.02, steps=args.llg_steps)  # synchronous
    dt_s = time.perf_counter() - t0
    clk = clocks.stop()
    if rank != 0:
        return None
    return {"metric": "LLG RK4 steps/s (B states, 4 batched demag evaluations per step)",
            "value": args.llg_steps / dt_s, "unit": "steps/s", "higher_is_better": True,
            "ms_per_step": 1e3 * dt_s / args.llg_steps, "evals_per_s": 4 * B * args.llg_steps / dt_s,
            "steps": args.llg_steps, "warmup": args.warmup, "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": data_note(w), "config": {"workload": args.workload, "batch": B, "precision": args.precision,
                                             "p": w["p"], "theta": w["theta"], "leaf_size": w["leaf"],
                                             "alpha": 0.1, "dt": 0.02},
            "clocks": clk}


def multi_meshes(w):
    from paper_1606_00247_gb300 import inputs

    return inputs.batch_meshes(n=w["n"])


def run_multi(args, rank, world, local_rank, w):
    """Meshes of uneven size, each with B states, through one submission
    (demag_eval_multi: run once, recorded as a CUDA graph, replayed per step).
    One evaluation = one state on one mesh."""
    import torch

    from paper_1606_00247_gb300.api import Plan, eval_multi_into

    dev = torch.device(f"cuda:{local_rank}")
    meshes = multi_meshes(w)
    B = args.batch
    kw = dict(p=w["p"], leaf_size=w["leaf"], theta=w["theta"], precision=args.precision, near_mode=args.near_mode,
              max_batch=B, device=dev, autotune=int(args.autotune) & 1, m2l_table_batch=args.m2l_table_batch, m2l_split_degree=args.m2l_split_degree)
    t0 = time.perf_counter()
    plans = [Plan(n, t, **kw) for n, t in meshes]
    plan_s = time.perf_counter() - t0
    Mh = [make_M(n.shape[0], B, seed_offset=rank + 17 * k, tets=t, w=w) for k, (n, t) in enumerate(meshes)]
    Ms = [torch.as_tensor(m, device=dev) for m in Mh]
    us = [torch.empty((B, n.shape[0]), dtype=torch.float64, device=dev) for n, _ in meshes]
    Hs = [torch.empty((B, n.shape[0], 3), dtype=torch.float64, device=dev) for n, _ in meshes]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        eval_multi_into(plans, Ms, us, Hs)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        eval_multi_into(plans, Ms, us, Hs)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    total_ms = float(sum(a.elapsed_time(b) for a, b in ev))
    per_sub = sum(pl.stats()["eval_launches"] for pl in plans)
    total_ms, value = aggregate_ranks(total_ms, len(plans) * B * args.steps, world, dev)
    # end to end: pinned host M in, u and H out, around the same submission
    Mp = [torch.as_tensor(m).pin_memory() for m in Mh]
    up = [torch.empty(u.shape, dtype=u.dtype).pin_memory() for u in us]
    Hp = [torch.empty(H.shape, dtype=H.dtype).pin_memory() for H in Hs]
    t_e2e = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        for d, h in zip(Ms, Mp):
            d.copy_(h, non_blocking=True)
        eval_multi_into(plans, Ms, us, Hs)
        for h, d in zip(up + Hp, us + Hs):
            h.copy_(d, non_blocking=True)
        torch.cuda.synchronize(dev)
        t_e2e.append(time.perf_counter() - t1)
    e2e_value = world * len(plans) * B * args.steps / sum(t_e2e)
    # accuracy gate on the smallest, a median and the largest mesh: state 0 vs FP64
    order = sorted(range(len(meshes)), key=lambda k: meshes[k][1].shape[0])
    errs = []
    if args.precision != "fp64" and not args.no_fp64_ref:
        for k in (order[0], order[len(order) // 2], order[-1]):
            n, t = meshes[k]
            u64, H64 = Plan(n, t, p=w["p"], leaf_size=w["leaf"], theta=w["theta"], precision="fp64", near_mode=1,
                            max_batch=1, device=dev).eval(Ms[k][:1])
            errs.append({"n_tets": int(t.shape[0]),
                         "rel_l2_u": float(torch.linalg.norm(us[k][0] - u64[0]) / torch.linalg.norm(u64[0])),
                         "rel_l2_H": float(torch.linalg.norm(Hs[k][0] - H64[0]) / torch.linalg.norm(H64[0]))})
    # roofline of the dominant stage on the largest mesh, evaluated alone with stage timers
    big = order[-1]
    prof = Plan(meshes[big][0], meshes[big][1], profile=True, **kw)
    prof.reset_timers()
    nprof = max(2, min(args.steps, 5))
    for _ in range(nprof):
        flush.zero_()
        prof.eval(Ms[big], us[big], Hs[big])
    pst = prof.stats()
    pst["_batch"] = B
    pst["near_mode"] = args.near_mode
    pst["_split_all"] = args.m2l_split_degree < 0
    roof = roofline_for(pst, nprof, args.precision, measured_peaks(), clk.get("sm_mhz"),
                        m2l_on_tensor_cores(args.precision, B, args.m2l_table_batch))
    roof["scope"] = f"largest mesh of the submission ({meshes[big][1].shape[0]} tets), evaluated alone"
    prof.close()
    if rank != 0:
        return None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": f"synthetic ({len(meshes)} meshes: Kuhn cubes, Delaunay balls and ellipsoids; "
                "unit nodal M smoothed over 3 neighbour passes)",
        "config": {"workload": args.workload, "n_meshes": len(meshes),
                   "n_tets_total": int(sum(t.shape[0] for _, t in meshes)),
                   "n_tets_min": int(meshes[order[0]][1].shape[0]), "n_tets_max": int(meshes[big][1].shape[0]),
                   "p": w["p"], "theta": w["theta"], "leaf_size": w["leaf"], "batch_per_mesh": B,
                   "precision": args.precision, "near_mode": args.near_mode, "l2": "flushed between steps",
                   "parallelism": f"replicas x{world}", "submission": "demag_eval_multi, replayed CUDA graph",
                   "plan_s_total": plan_s},
        "roofline": roof,
        "accuracy_vs_fp64": errs,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(sum(m.nbytes for m in Mh)),
                "d2h_bytes_per_step": int(sum(u.numel() * 8 + H.numel() * 8 for u, H in zip(us, Hs)))},
        "gpu_launches": int(per_sub * args.steps),
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        n, t = meshes[big]
        out["cpu_baseline"] = cpu_baseline(n, t, w, make_M(n.shape[0], 1, tets=t, w=w)[0],
                                           single_core=not args.no_single_core)
    return out


def run_reference(args, rank):
    """The oracle on the host cores, each step one fixed sample of the workload
    (the same sample as our line's cpu_baseline)."""
    if rank != 0:
        return None
    w = workload(args)
    w["name"] = args.workload
    if w["mesh"] == "multi":
        nodes, tets = max(multi_meshes(w), key=lambda m: m[1].shape[0])
    else:
        nodes, tets = make_mesh(w)
    M1 = make_M(nodes.shape[0], 1, tets=tets, w=w)[0]
    smp = OracleSampler(nodes, tets, w)
    vals, first = [], None
    for k in range(args.warmup + args.steps):
        r = smp.run(M1)
        first = first or r
        if k >= args.warmup:
            vals.append(r["value"])
    value = float(np.mean(vals))
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": data_note(w),
            "config": {"workload": args.workload, "p": w["p"], "theta": w["theta"], "leaf_size": smp.leaf,
                       "batch_per_gpu": 1},
            "cpu_baseline": {"kind": "oracle", "cores": first["cores"], "sample": first["sample"], "value": value,
                             "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def accuracy_sweep(args):
    """FMM truncation error against the direct sum on the same mesh, per (p, theta):
    the direct sum is the library itself with theta -> 0 (every pair in the
    analytic FP64 near field), one state; each FMM is run in FP64 and in the
    mixed split-BF16 mode.  One JSON line."""
    import torch

    from paper_1606_00247_gb300 import build
    from paper_1606_00247_gb300.api import Plan

    build()
    w = workload(args)
    nodes, tets = make_mesh(w)
    M = torch.as_tensor(make_M(nodes.shape[0], 1), device="cuda")
    t0 = time.perf_counter()
    direct = Plan(nodes, tets, p=2, leaf_size=w["leaf"], theta=1e-6, precision="fp64", near_mode=0, max_batch=1)
    ud, Hd = direct.eval(M)
    torch.cuda.synchronize()
    t_direct = time.perf_counter() - t0
    n_pairs_direct = direct.stats()["n_p2p_pairs"]
    direct.close()

    def rel(a, b):
        return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))

    rows = []
    for theta in (0.3, 0.5, 0.8):
        for p in (4, 6, 8, 10):
            for prec in ("fp64", "bf16x3"):
                pl = Plan(nodes, tets, p=p, leaf_size=w["leaf"], theta=theta, precision=prec, near_mode=1, max_batch=1)
                u, H = pl.eval(M)
                st = pl.stats()
                rows.append({"theta": theta, "p": p, "precision": prec, "rel_l2_u": rel(u, ud), "rel_l2_H": rel(H, Hd),
                             "n_m2l": st["n_m2l"], "n_p2p_pairs": st["n_p2p_pairs"]})
                pl.close()
    return {"accuracy_sweep": rows, "workload": args.workload, "n_tets": int(tets.shape[0]), "leaf": w["leaf"],
            "direct": {"pairs": n_pairs_direct, "seconds_incl_plan": t_direct}, "state": "seeded Gaussian unit M"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere500k", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="bf16x3", choices=["fp64", "fp32", "tf32", "bf16x3", "bf16x6"])
    ap.add_argument("--near-mode", type=int, default=1)
    ap.add_argument("--batch", type=int, default=0, help="states per evaluation (0: the workload's default)")
    ap.add_argument("--no-fp64-ref", action="store_true")
    ap.add_argument("--autotune", type=int, default=-1,
                    help="bit 0: time the M2L launch shapes at plan time; bit 1: tune the leaf size; "
                         "bit 2: pick the smallest p meeting 5e-5 against FP64 p = 10 (-1: the workload's default)")
    ap.add_argument("--m2l-table-batch", type=int, default=0,
                    help="largest batch run by the FP32 table M2L in the tensor-core precisions (0: default, -1: never)")
    ap.add_argument("--m2l-split-degree", type=int, default=0,
                    help="split BF16 tensor-core M2L: 0 = second-limb products up to term degree p - 4 "
                         "(default), < 0 = on every term")
    ap.add_argument("--p", type=int, default=0)
    ap.add_argument("--leaf", type=int, default=0)
    ap.add_argument("--theta", type=float, default=0.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-single-core", action="store_true", help="skip the single-thread oracle sample")
    ap.add_argument("--sources", default="tets", choices=["tets", "dipoles"],
                    help="P1 tetrahedra (the method) or point dipoles at the nodes (the comparison model)")
    ap.add_argument("--llg-steps", type=int, default=0,
                    help="time this many LLG RK4 steps of --batch states instead of the evaluation benchmark")
    ap.add_argument("--accuracy-sweep", action="store_true",
                    help="print the FMM-vs-direct error table over p and theta instead of timing")
    ap.add_argument("--peaks", action="store_true",
                    help="print the measured FP64 / FP32 FMA and BF16 / TF32 tcgen05 peaks with the SM clock")
    args = ap.parse_args()
    if args.accuracy_sweep:
        print(json.dumps(accuracy_sweep(args)), flush=True)
        return
    if args.peaks:
        import torch

        from paper_1606_00247_gb300 import build

        build()
        torch.cuda.init()
        clocks = ClockSampler(0)
        clocks.start()
        vals = measure_peaks()
        clk = clocks.stop()
        print(json.dumps({"peaks_tflops": vals, "clocks": clk, "how": "demag_measure_peak: register FMA chains on "
                          "every SM (FP64, FP32); one CTA per SM issuing M=128 N=256 tcgen05.mma on shared-memory "
                          "operands (BF16 K=16, TF32 K=8); best of 3 after a warm-up"}), flush=True)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        out = run_reference(args, rank)
    else:
        out = run_ours(args, rank, world, local_rank)
    if out is not None:
        print(json.dumps(out), flush=True)
    if world > 1 and args.impl == "ours":
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
