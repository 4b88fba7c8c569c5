"""FP64 on-the-fly near field (near_mode = 0, Sec. 2.1).

Two kernels compute the same analytic pair sums: for one state pair by pair
(pair_contract on per-tet records), from 2 states on the state-independent
vector a and tensor T of each (target node, source tet) pair are computed once
and contracted with every state of a slice of 16.
With theta -> 0 every interaction is near field, so the evaluation is the
near-field kernel alone: held against the oracle's direct sum per state, at
batches that fill state slices partly and exactly, and at leaves of more
target nodes than one pass of the kernel holds (64).
"""
import numpy as np
import pytest
import torch

from paper_1606_00247_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _plan(nodes, tets, **kw):
    from paper_1606_00247_gb300.api import Plan

    return Plan(nodes, tets, precision="fp64", near_mode=0, **kw)


@pytest.mark.parametrize("B", [1, 2, 3, 16, 17, 33])
def test_theta_zero_every_state_is_the_direct_sum(orc, B):
    nodes, tets = inputs.sphere(h=0.25)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=B, seed=500 + B)
    u, H = _plan(nodes, tets, p=2, leaf_size=16, theta=1e-9, max_batch=B).eval(M)
    u = u.cpu().numpy()
    for k in sorted({0, B // 2, B - 1}):
        assert rel_l2(u[k], orc.direct(nodes, tets, M[k])) < 1e-12, k


def test_batched_kernel_equals_per_state_kernel():
    """Each of three states through the per-state kernel (a batch of 1) and
    through the batched one (a batch of 3 that holds them): the same sums in
    another order, equal to rounding."""
    nodes, tets = inputs.sphere(h=0.14)
    M = inputs.smoothed_unit_m(tets, nodes.shape[0], batch=3, seed=510)
    kw = dict(p=6, leaf_size=32, theta=0.5)
    u3, H3 = _plan(nodes, tets, max_batch=3, **kw).eval(M)
    p1 = _plan(nodes, tets, max_batch=1, **kw)
    for k in range(3):
        u1, H1 = p1.eval(M[k:k + 1])
        assert rel_l2(u3[k].cpu(), u1[0].cpu()) < 1e-13
        assert rel_l2(H3[k].cpu(), H1[0].cpu()) < 1e-13


def test_large_leaves_take_several_passes(orc):
    """Leaves of more than 64 target nodes: the batched kernel covers them in
    passes of 64, each against every source tet of the P2P list."""
    nodes, tets = inputs.sphere(h=0.13)
    kw = dict(p=2, leaf_size=4096, theta=1e-9)
    ex = _plan(nodes, tets, **kw).export_tree()
    leaf = ex["cell_child"][:, 1] == 0
    per_leaf = ex["cell_ranges"][:, 3] - ex["cell_ranges"][:, 2]
    assert per_leaf[leaf].max() > 64
    B = 5
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=B, seed=511)
    u, _ = _plan(nodes, tets, max_batch=B, **kw).eval(M)
    for k in (0, B - 1):
        assert rel_l2(u[k].cpu().numpy(), orc.direct(nodes, tets, M[k])) < 1e-12


def test_batched_kernel_is_deterministic():
    """Each target's sum is formed in a fixed order (lane shuffle tree, then
    the owning warp): repeated evaluations give the same bits."""
    nodes, tets = inputs.sphere(h=0.14)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=9, seed=512)
    pl = _plan(nodes, tets, p=4, leaf_size=32, theta=0.5, max_batch=9)
    ua, Ha = pl.eval(M)
    ub, Hb = pl.eval(M)
    assert torch.equal(ua, ub) and torch.equal(Ha, Hb)
