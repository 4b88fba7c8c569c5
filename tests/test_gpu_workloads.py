"""Full-size configurations other than the benchmark's (parity cases, not
bench lines):

* the thin film 2000 x 1000 x 10 (1,990,656 tets, 500,259 nodes) with a Landau
  flux-closure magnetisation plus 5 % random tilt, p = 8, theta = 0.5: the FP64
  GPU FMM against the oracle FMM on sampled target leaves computed one by one,
  and the split-BF16 tensor-core path against FP64 per state;
* the 224k-tet ball (223,668 tets) with a uniform magnetisation -- smooth M
  makes the far field a sum of large cancelling dipole terms, the hardest case
  for the tensor-core M2L's accumulation.

Both check the effect of promoting the leading M2L accumulator rows to FP32
registers (the default): without it the film misses the 1e-4 bar.

Batched serving (many states on one mesh, many meshes in one submission):

* the ball of 559,564 tets with 256 smoothed unit states (two 128-state
  tensor-core tiles): sampled states of both tiles against FP64, and against
  the same states evaluated as a batch of 2 (table-driven FP32 M2L);
* the graded unit cube (22.1M tets, 3.27M nodes, 50 inclusions refined 8x), up to 32
  iid unit states: the mixed path (split BF16, table-driven FP32 M2L at this
  batch, leaf 64, batch chosen to fit 180 GB) against the FP64 GPU FMM (near field on the fly)
  on state 0, and the FP64 GPU FMM against the oracle's direct sum on 16
  sampled nodes (inside inclusions, in shells and outside) within the
  truncation error;
* 64 meshes of 10k-280k tets (cubes, balls, ellipsoids up to 1:4) with one state
  each through one demag_eval_multi submission: every mesh bit-identical to its
  own demag_eval, and the smallest, a median and the largest mesh against FP64."""
import numpy as np
import pytest
import torch

from paper_1606_00247_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_film_full_size(orc):
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.thin_film()
    assert tets.shape[0] == 1990656 and nodes.shape[0] == 500259
    M = np.stack([inputs.landau_m(nodes), inputs.landau_m(nodes, seed=inputs.MAG_SEED + 7)])
    Md = torch.as_tensor(M, device="cuda")
    p64 = Plan(nodes, tets, p=8, leaf_size=128, theta=0.5, precision="fp64", near_mode=1, max_batch=2)
    u64, H64 = p64.eval(Md)
    ex = p64.export_tree()
    del p64
    # FP64 GPU vs the oracle FMM on 12 sampled target leaves (state 0)
    tr = orc.Tree(nodes, tets, 128, 0.5)
    leaves = np.where((ex["cell_child"][:, 1] == 0) & (ex["cell_ranges"][:, 3] > ex["cell_ranges"][:, 2]))[0]
    pick = leaves[np.linspace(0, len(leaves) - 1, 12).astype(int)]
    ref = tr.fmm(M[0], 8, target_leaves=pick)
    sel = np.concatenate([ex["node_perm"][ex["cell_ranges"][c, 2]:ex["cell_ranges"][c, 3]] for c in pick])
    g = u64[0].cpu().numpy()[sel]
    assert np.linalg.norm(g - ref[sel]) / np.linalg.norm(ref[sel]) < 1e-10
    # split BF16 (promotion on by default) vs FP64, per state; and without promotion
    errs = {}
    for promote in (0, -1):  # tensor-core M2L forced at this batch of 2
        pl = Plan(nodes, tets, p=8, leaf_size=128, theta=0.5, precision="bf16x3", near_mode=1, max_batch=2,
                  m2l_promote=promote, m2l_table_batch=-1)
        u, H = pl.eval(Md)
        errs[promote] = max(max(rel(u[k], u64[k]), rel(H[k], H64[k])) for k in range(2))
        del pl
    assert errs[0] <= 1e-4, errs
    assert errs[0] < errs[-1] / 3, errs  # promotion is what brings the film under the bar
    # default at a batch of 2: the table-driven FP32 M2L on CUDA cores
    pl = Plan(nodes, tets, p=8, leaf_size=128, theta=0.5, precision="bf16x3", near_mode=1, max_batch=2)
    u, H = pl.eval(Md)
    err = max(max(rel(u[k], u64[k]), rel(H[k], H64[k])) for k in range(2))
    assert err <= 1e-4, err


def test_ball_uniform_m_tensor_core():
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.sphere(h=inputs.SPHERE_200K_H)
    M = torch.as_tensor(np.stack([inputs.uniform_m(nodes.shape[0], d) for d in ((0, 0, 1), (1, 0, 0))]),
                        device="cuda")
    u64, H64 = Plan(nodes, tets, p=8, leaf_size=128, theta=0.5, near_mode=1, max_batch=2).eval(M)
    for prec, bar, tb in (("bf16x3", 1e-5, -1), ("bf16x6", 1e-5, -1), ("fp32", 1e-5, 0)):
        u, H = Plan(nodes, tets, p=8, leaf_size=128, theta=0.5, precision=prec, near_mode=1, max_batch=2,
                    m2l_table_batch=tb).eval(M)
        for k in range(2):
            assert rel(u[k], u64[k]) <= bar and rel(H[k], H64[k]) <= bar, (prec, k)


def test_ball500k_256_states():
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.sphere(h=inputs.SPHERE_500K_H)
    assert tets.shape[0] == 559564
    M = torch.as_tensor(inputs.smoothed_unit_m(tets, nodes.shape[0], batch=256), device="cuda")
    u, H = Plan(nodes, tets, p=8, leaf_size=128, theta=0.5, precision="bf16x3", near_mode=1, max_batch=256).eval(M)
    pick = [0, 127, 128, 255]
    Mp = M[pick].contiguous()
    u64, H64 = Plan(nodes, tets, p=8, leaf_size=128, theta=0.5, near_mode=1, max_batch=4).eval(Mp)
    for k, b in enumerate(pick):
        assert rel(u[b], u64[k]) < 1e-5 and rel(H[b], H64[k]) < 1e-5, b
    u2, H2 = Plan(nodes, tets, p=8, leaf_size=128, theta=0.5, precision="bf16x3", near_mode=1,
                  max_batch=2).eval(M[[0, 255]].contiguous())
    for k, b in enumerate((0, 255)):
        assert rel(u2[k], u[b]) < 1e-5 and rel(H2[k], H[b]) < 1e-5, b


def test_multi64_one_submission():
    from paper_1606_00247_gb300.api import Plan, eval_multi_into

    meshes = inputs.batch_meshes()
    assert len(meshes) == 64
    sizes = [t.shape[0] for _, t in meshes]
    assert min(sizes) >= 10000 and max(sizes) <= 300000
    plans = [Plan(n, t, p=8, leaf_size=128, theta=0.5, precision="bf16x3", near_mode=1, max_batch=1)
             for n, t in meshes]
    Ms = [torch.as_tensor(inputs.smoothed_unit_m(t, n.shape[0], seed=900 + k), device="cuda")
          for k, (n, t) in enumerate(meshes)]
    us = [torch.full((1, n.shape[0]), np.nan, dtype=torch.float64, device="cuda") for n, _ in meshes]
    Hs = [torch.full((1, n.shape[0], 3), np.nan, dtype=torch.float64, device="cuda") for n, _ in meshes]
    eval_multi_into(plans, Ms, us, Hs)  # direct run + graph recording
    eval_multi_into(plans, Ms, us, Hs)  # replay
    torch.cuda.synchronize()
    for pl, M, u, H in zip(plans, Ms, us, Hs):
        u1, H1 = pl.eval(M)
        assert torch.equal(u, u1) and torch.equal(H, H1)
    order = np.argsort(sizes)
    for k in (order[0], order[len(order) // 2], order[-1]):
        n, t = meshes[k]
        u64, H64 = Plan(n, t, p=8, leaf_size=128, theta=0.5, near_mode=1, max_batch=1).eval(Ms[k])
        assert rel(us[k][0], u64[0]) < 1e-4 and rel(Hs[k][0], H64[0]) < 1e-4, sizes[k]


def test_graded_20m(orc):
    import time

    from paper_1606_00247_gb300.api import Plan

    t0 = time.perf_counter()
    nodes, tets, cen, rad = inputs.graded_cube()
    t_mesh = time.perf_counter() - t0
    nn = nodes.shape[0]
    assert 20e6 < tets.shape[0] < 24e6 and 3.0e6 < nn < 3.6e6
    M = inputs.gaussian_unit_m(nn, batch=32, seed=inputs.MAG_SEED + 5)
    # FP64 reference on state 0 first (near field integrated on the fly: no stored coefficients)
    p64 = Plan(nodes, tets, p=8, leaf_size=64, theta=0.5, precision="fp64", near_mode=0, max_batch=1)
    u64, H64 = p64.eval(torch.as_tensor(M[:1], device="cuda"))
    u64, H64 = u64.cpu(), H64.cpu()
    p64.close()
    del p64
    torch.cuda.empty_cache()
    # the per-leaf FP32 near field (near_tc = -1): with ~2 target nodes per 64-tet leaf a
    # 128-node tile spans ~60 leaves, whose column union would store the coefficients
    # several times over and leave no room for the batch within 180 GB
    pl = Plan(nodes, tets, p=8, leaf_size=64, theta=0.5, precision="bf16x3", near_mode=1, max_batch=32,
              m2l_table_batch=32, near_tc=-1)
    st = pl.stats()
    # the batch: the largest power of two (at most 32) whose workspace and inputs/outputs fit in
    # 180 GB with the plan (FP32 moments and locals per cell, FP32 and FP64 node arrays per state)
    per_state = st["n_cells"] * 165 * 4 * 2 + nn * (3 * 4 + 4) + nn * (3 * 8 + 8 + 3 * 8)
    B = 32
    while B > 1 and st["device_bytes"] + B * per_state > 175e9:
        B //= 2
    Md = torch.as_tensor(M[:B], device="cuda")
    t1 = time.perf_counter()
    u, H = pl.eval(Md)
    torch.cuda.synchronize()
    t_eval = time.perf_counter() - t1
    free, total = torch.cuda.mem_get_info()
    print(f"graded: mesh {t_mesh:.0f} s, plan {st['plan_ms'] / 1e3:.0f} s, plan {st['device_bytes'] / 1e9:.1f} GB, "
          f"B = {B}, device in use {(total - free) / 1e9:.1f} GB, first eval {t_eval:.2f} s, "
          f"cells {st['n_cells']}, M2L pairs {st['n_m2l']}")
    assert B >= 8
    assert total - free < 180e9  # plan, workspace for B states, inputs and outputs
    u0, H0 = u[0].cpu(), H[0].cpu()
    assert rel(u0, u64[0]) < 1e-4 and rel(H0, H64[0]) < 1e-4
    # FP64 FMM vs the direct sum on sampled nodes: 6 inside inclusions, 5 in shells, 5 outside
    d = np.full(nn, np.inf)
    for c, r in zip(cen, rad):
        d = np.minimum(d, np.linalg.norm(nodes - c, axis=1) - r)
    rng = np.random.default_rng(7)
    pick = np.concatenate([rng.choice(np.where(d < -0.005)[0], 6, replace=False),
                           rng.choice(np.where((d > 0.001) & (d < 0.02))[0], 5, replace=False),
                           rng.choice(np.where(d > 0.05)[0], 5, replace=False)])
    ref = orc.direct(nodes, tets, M[0], targets=pick)
    g = u64[0].numpy()[pick]
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-4
