"""Host-side logic of bench.py that needs no GPU: workload overrides, the choice
of M2L path behind the roofline line, the issued-tile flop model of the
tensor-core M2L, and the roofline record built from per-stage timers."""
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_workload_overrides():
    a = types.SimpleNamespace(workload="sphere200k", p=6, leaf=0, theta=0.0)
    w = bench.workload(a)
    assert (w["p"], w["leaf"], w["theta"]) == (6, 128, 0.5)
    assert bench.WORKLOADS["sphere200k"]["p"] == 8  # the table itself is not modified


def test_m2l_path_choice():
    assert not bench.m2l_on_tensor_cores("bf16x3", 8, 0)  # table M2L up to 8 states by default
    assert bench.m2l_on_tensor_cores("bf16x3", 9, 0)
    assert bench.m2l_on_tensor_cores("bf16x3", 4, -1)  # never the table
    assert not bench.m2l_on_tensor_cores("bf16x3", 32, 32)
    assert not bench.m2l_on_tensor_cores("fp32", 128, 0)


def test_m2l_counts():
    assert bench.m2l_macs(8) == 3003 and bench.m2l_macs(4) == 210  # C(p + 6, 6)
    # split BF16, p = 8: k-step row prefixes 176, 64, 48, 32 and seven of 16, K = 16
    rows = [176, 64, 48, 32] + [16] * 7
    assert bench.m2l_tile_flops(8, "bf16x3", split_all=True) == 2.0 * sum(r * 16 for r in rows) * 3
    # default split degree p - 4 = 4: the second-limb rows are those of degree <= 4 - (lowest |n| of
    # the k-step) -- 35 (pad 48), 4 (16), 1 (16) for k-steps 0-2 (lowest |n| 0, 3, 4), none after
    rows2 = [48, 16, 16] + [0] * 8
    assert bench.m2l_tile_flops(8, "bf16x3") == 2.0 * 16 * (sum(rows) + 2 * sum(rows2))
    assert bench.m2l_split_degree(8) == 4 and bench.m2l_split_degree(6) == 3


def test_roofline_record_tensor_and_alu():
    stats = {"stage_ms": {"m2l": 80.0, "p2p": 30.0}, "stage_launches": {"m2l": 10, "p2p": 10}, "_batch": 128,
             "p": 8, "n_m2l": 866523, "near_mode": 1, "n_near_cols": 107e6, "leaf_size": 128, "n_tets": 223668,
             "n_nodes": 35840, "m2l_targets_per_cta": 1, "m2l_kps": 2}
    peaks = {"bf16_tflops_sustained": 1744.5, "hbm_gbs": 6689.8}
    r = bench.roofline_for(stats, 10, "bf16x3", peaks, 2070.0, tensor_m2l=True)
    assert r["kernel"] == "m2l" and r["bound"] == "tensor" and r["peak"] == 1744.5
    achieved = 2.0 * 866523 * 3003 * 128 / 8e-3 / 1e12
    assert abs(r["achieved"] - achieved) < 1e-9 * achieved and abs(r["frac"] - achieved / 1744.5) < 1e-12
    r2 = bench.roofline_for(stats, 10, "bf16x3", peaks, 2070.0, tensor_m2l=False)
    assert r2["bound"] == "alu" and abs(r2["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9


def test_roofline_near_field_record():
    """The stored near field on the tensor cores is held against HBM: 12 B of
    split-BF16 coefficients per (target, source node) pair, M and u of every
    node once per state; its tensor-pipe view counts 2 flops per component."""
    stats = {"stage_ms": {"m2l": 10.0, "p2p": 30.0}, "stage_launches": {"m2l": 10, "p2p": 10}, "_batch": 256,
             "p": 8, "n_m2l": 1000, "near_mode": 1, "n_near_cols": 583e6, "n_near_tiles": 700, "near_bytes": 10e9,
             "leaf_size": 512, "n_tets": 559564, "n_nodes": 87443}
    peaks = {"bf16_tflops_sustained": 1705.4, "hbm_gbs": 6766.0}
    r = bench.roofline_for(stats, 10, "bf16x3", peaks, 2070.0)
    assert r["kernel"] == "p2p" and r["bound"] == "hbm" and r["peak"] == 6766.0
    alg = 583e6 * 12 + 87443 * 256 * 12 + 87443 * 256 * 8
    assert abs(r["algorithmic_bytes"] - alg) < 1e-9 * alg
    assert abs(r["achieved"] - alg / 3e-3 / 1e9) < 1e-9 * r["achieved"]
    tv = r["tensor_view"]
    assert abs(tv["achieved"] - 2.0 * 3 * 583e6 * 256 / 3e-3 / 1e12) < 1e-9 * tv["achieved"]
    assert r["stages"]["m2l"]["bound"] == "tensor" and r["stages"]["p2p"]["bound"] == "hbm"


def test_workload_defaults_fill_batch_and_autotune():
    a = types.SimpleNamespace(workload="sphere500k", p=0, leaf=0, theta=0.0, batch=0, autotune=-1)
    w = bench.workload(a)
    assert a.batch == 256 and a.autotune == 3 and w["cpu_leaf"] == 128
    b = types.SimpleNamespace(workload="sphere500k", p=0, leaf=512, theta=0.0, batch=0, autotune=-1)
    w = bench.workload(b)
    assert b.autotune == 1 and w["leaf"] == 512 and w["cpu_leaf"] == 512  # a given leaf is not tuned


def test_direct_sample_times_the_oracle_and_measures_truncation():
    """The direct-sum reference row: the oracle's direct sum at seeded sample
    nodes, extrapolated to all nodes; against a u that is the direct sum itself
    the measured 'truncation' is zero, against a perturbed u it is the
    perturbation."""
    import numpy as np

    import oracle
    from paper_1606_00247_gb300 import inputs

    nodes, tets = inputs.kuhn_box((4, 4, 4))
    M1 = inputs.gaussian_unit_m(nodes.shape[0], batch=1)[0]
    u = oracle.direct(nodes, tets, M1)
    r = bench.direct_sample(nodes, tets, M1, u, n=16)
    assert r["kind"] == "oracle_direct" and r["value"] > 0 and r["cores"] >= 1
    assert r["fp64_gpu_fmm_vs_direct_rel_l2"] == 0.0
    r2 = bench.direct_sample(nodes, tets, M1, u * (1 + 1e-6), n=16)
    assert abs(r2["fp64_gpu_fmm_vs_direct_rel_l2"] - 1e-6) < 1e-12
    assert "fp64_gpu_fmm_vs_direct_rel_l2" not in bench.direct_sample(nodes, tets, M1, None, n=4)


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle on the host cores) on the small
    cube: exactly one JSON line with the contract's keys, the reference's own
    cpu_baseline record and an e2e object that moves no bytes."""
    import json
    import subprocess

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "cube8",
                        "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (2, 3, 1) and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "cube8"


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 runs the oracle and prints; another rank exits 0 silently."""
    import subprocess

    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "cube8",
                        "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT,
                       env=env)
    assert r.returncode == 0 and r.stdout.strip() == "", (r.stdout[-500:], r.stderr[-1000:])
