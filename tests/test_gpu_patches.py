"""Vertex-patch sources on the GPU (the paper's own clustering, Sec. 2.1
"vertex interaction" and Sec. 3.1-3.2): node i carries lambda_i M over every
tet around it, is binned by its own key, and a cell's source radius reaches
the farthest vertex of the tets around its nodes.

* tree, radii and both interaction lists bit for bit against the oracle's
  patch tree;
* theta -> 0: every pair in the analytic near field, the patches partition the
  same integrand as the tets, so u is the oracle's direct sum to rounding;
* theta = 0.5: the FP64 patch FMM against the oracle's patch FMM;
* split BF16 (tensor-core M2L and near field) against the FP64 patch FMM."""
import numpy as np
import pytest

from paper_1606_00247_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _plan(nodes, tets, **kw):
    from paper_1606_00247_gb300.api import Plan

    return Plan(nodes, tets, sources="patches", near_mode=1, **kw)


@pytest.mark.parametrize("mesh,leaf,theta", [("sphere", 32, 0.5), ("cube", 16, 0.3), ("sphere", 64, 0.8)])
def test_patch_tree_and_lists_bit_exact(orc, mesh, leaf, theta):
    nodes, tets = inputs.sphere(h=0.2) if mesh == "sphere" else inputs.unit_cube(8)
    ref = orc.Tree(nodes, tets, leaf, theta, sources="patches")
    g, o = _plan(nodes, tets, p=2, leaf_size=leaf, theta=theta).export_tree(), ref.export()
    for k in ("cell_ranges", "cell_child", "m2l_off", "m2l_src", "p2p_off", "p2p_src"):
        assert np.array_equal(g[k], o[k]), k
    assert np.array_equal(g["cell_radius"].view(np.uint64), o["cell_radius"].view(np.uint64))


def test_patch_theta_zero_is_direct_sum(orc):
    nodes, tets = inputs.sphere(h=0.2)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=2, seed=71)
    u, H = _plan(nodes, tets, p=2, leaf_size=32, theta=1e-9, max_batch=2).eval(M)
    ref = orc.direct(nodes, tets, M)
    assert rel_l2(u.cpu().numpy(), ref) < 1e-12
    assert rel_l2(H.cpu().numpy(), orc.lumped_H(nodes, tets, ref)) < 1e-12


@pytest.mark.parametrize("p", [4, 8])
def test_patch_fmm_vs_oracle_patch_fmm(orc, p):
    nodes, tets = inputs.sphere(h=0.15)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=2, seed=72)
    u, _ = _plan(nodes, tets, p=p, leaf_size=32, theta=0.5, max_batch=2).eval(M)
    ref = orc.Tree(nodes, tets, 32, 0.5, sources="patches").fmm(M, p)
    assert rel_l2(u.cpu().numpy(), ref) < 1e-10
    # the truncation against the direct sum falls with p (the same integrand as the tets)
    d = orc.direct(nodes, tets, M)
    assert rel_l2(u.cpu().numpy(), d) < (2e-3 if p == 4 else 1e-4)


def test_patch_mixed_vs_fp64():
    nodes, tets = inputs.sphere(h=0.13)
    B = 128
    M = inputs.smoothed_unit_m(tets, nodes.shape[0], batch=B, seed=73)
    kw = dict(p=8, leaf_size=64, theta=0.5, max_batch=B)
    u64, H64 = _plan(nodes, tets, **kw).eval(M)
    pm = _plan(nodes, tets, precision="bf16x3", **kw)
    assert pm.stats()["n_near_tiles"] > 0
    u, H = pm.eval(M)
    eu = max(rel_l2(u[k].cpu().numpy(), u64[k].cpu().numpy()) for k in range(B))
    eh = max(rel_l2(H[k].cpu().numpy(), H64[k].cpu().numpy()) for k in range(B))
    assert eu <= 1e-4 and eh <= 1e-4, (eu, eh)
