"""Near field on the tensor cores (split-BF16 precisions, near_mode = 1).

The stored near-field coefficients (Sec. 3.4) are applied per tile of up to
128 target nodes as a dense BF16x3 product accumulated in tensor memory.
With theta -> 0 every interaction is near field, so the evaluation is the
near-field kernel alone: it is held against the oracle's direct sum and
against the FP64 path of the library, at batches that fill one or two
128-state blocks per CTA, partly or exactly.  The plan build adds the
per-tet contributions to the coefficients as exact integer sums, so two
builds give the same bits.
"""
import numpy as np
import pytest
import torch

from paper_1606_00247_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def per_state(a, b):
    return max(rel_l2(a[k], b[k]) for k in range(a.shape[0]))


def _plan(nodes, tets, **kw):
    from paper_1606_00247_gb300.api import Plan

    return Plan(nodes, tets, **kw)


@pytest.mark.parametrize("B", [1, 3, 128, 160, 256])
def test_near_tc_theta_zero_vs_fp64_and_direct(orc, B):
    """Every pair in the near field: the split-BF16 tensor-core product against
    the FP64 coefficients applied in FP64, per state, and state 0 against the
    oracle's direct sum.  Two BF16 limbs keep 16 significant bits of each
    operand: hi x hi + hi x lo + lo x hi leaves up to 3 * 2^-18 ~ 1.1e-5 of
    each product, so the bar is 3e-5 (the mixed-path bar is 1e-4)."""
    nodes, tets = inputs.sphere(h=0.2)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=B, seed=300 + B)
    kw = dict(p=2, leaf_size=32, theta=1e-9, near_mode=1, max_batch=B)
    ptc = _plan(nodes, tets, precision="bf16x3", **kw)
    st = ptc.stats()
    assert st["n_near_tiles"] > 0 and st["n_m2l"] == 0
    u, H = ptc.eval(M)
    u64, H64 = _plan(nodes, tets, precision="fp64", **kw).eval(M)
    eu = per_state(u.cpu().numpy(), u64.cpu().numpy())
    eh = per_state(H.cpu().numpy(), H64.cpu().numpy())
    assert eu < 3e-5 and eh < 3e-5, (eu, eh)
    ref = orc.direct(nodes, tets, M[0])
    assert rel_l2(u[0].cpu().numpy(), ref) < 3e-5


def test_near_tc_vs_cuda_core_near_field():
    """The tensor-core near field and the FP32 CUDA-core one apply the same
    coefficients: they agree to the split-BF16 rounding."""
    nodes, tets = inputs.sphere(h=0.13)
    B = 128
    M = inputs.smoothed_unit_m(tets, nodes.shape[0], batch=B, seed=401)
    kw = dict(p=8, leaf_size=64, theta=0.5, near_mode=1, max_batch=B, precision="bf16x3")
    a = _plan(nodes, tets, **kw)
    b = _plan(nodes, tets, near_tc=-1, **kw)
    assert a.stats()["n_near_tiles"] > 0 and b.stats()["n_near_tiles"] == 0
    ua, Ha = a.eval(M)
    ub, Hb = b.eval(M)
    assert per_state(ua.cpu().numpy(), ub.cpu().numpy()) < 3e-5
    assert per_state(Ha.cpu().numpy(), Hb.cpu().numpy()) < 3e-5
    u64, H64 = _plan(nodes, tets, p=8, leaf_size=64, theta=0.5, near_mode=1, max_batch=B).eval(M)
    assert per_state(ua.cpu().numpy(), u64.cpu().numpy()) < 1e-4
    assert per_state(Ha.cpu().numpy(), H64.cpu().numpy()) < 1e-4


def test_near_tc_split_tiles_of_a_large_leaf(orc):
    """Leaves with more than 128 target nodes get tiles of their own (128 rows
    each, the leaf's columns in every one)."""
    nodes, tets = inputs.sphere(h=0.13)
    kw = dict(p=4, leaf_size=4096, theta=0.5, near_mode=1, max_batch=2)
    ex = _plan(nodes, tets, **kw).export_tree()
    leaf = ex["cell_child"][:, 1] == 0
    nodes_per_leaf = ex["cell_ranges"][:, 3] - ex["cell_ranges"][:, 2]
    assert nodes_per_leaf[leaf].max() > 128
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=2, seed=402)
    ptc = _plan(nodes, tets, precision="bf16x3", **kw)
    u, H = ptc.eval(M)
    u64, H64 = _plan(nodes, tets, precision="fp64", **kw).eval(M)
    assert per_state(u.cpu().numpy(), u64.cpu().numpy()) < 3e-5
    assert per_state(H.cpu().numpy(), H64.cpu().numpy()) < 3e-5


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "fp32"])
def test_plan_build_is_deterministic(prec):
    """Two builds of the same plan give bit-identical stored coefficients, so
    bit-identical results (the near-field contributions are summed as exact
    integers, independent of the order in which threads add them)."""
    nodes, tets = inputs.sphere(h=0.13)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=4, seed=403)
    kw = dict(p=6, leaf_size=32, theta=0.5, near_mode=1, max_batch=4, precision=prec)
    ua, Ha = _plan(nodes, tets, **kw).eval(M)
    ub, Hb = _plan(nodes, tets, **kw).eval(M)
    assert torch.equal(ua, ub) and torch.equal(Ha, Hb)


def test_near_tc_dipole_sources(orc):
    """The point-dipole comparison model through the tensor-core near field:
    theta -> 0 against the direct dipole sum."""
    nodes, tets = inputs.sphere(h=0.2)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=2, seed=404)
    kw = dict(p=2, leaf_size=32, theta=1e-9, near_mode=1, max_batch=2, sources="dipoles")
    u, _ = _plan(nodes, tets, precision="bf16x3", **kw).eval(M)
    ref = orc.dipole_direct(nodes, tets, M[0])
    assert rel_l2(u[0].cpu().numpy(), ref) < 3e-5


@pytest.mark.parametrize("B", [2, 160])
def test_near_tc_repeated_evaluations_are_identical(B):
    """One plan evaluated five times: every evaluation gives the same bits and
    no device wait expires.  The state warps take part in every column group,
    so each waits for every use of each shared-memory stage in order (a
    skipped use lets a phase parity alias an older phase).  A thin film with
    smooth domains (long tiles) and a ball with one full and one partial
    state block."""
    from paper_1606_00247_gb300 import _lib

    if B == 2:
        nodes, tets = inputs.thin_film(nx=288, ny=144, nz=2, size=(1000.0, 500.0, 10.0))
        M = np.stack([inputs.landau_m(nodes, size=(1000.0, 500.0)),
                      inputs.landau_m(nodes, size=(1000.0, 500.0), seed=inputs.MAG_SEED + 7)])
        kw = dict(p=8, leaf_size=128)
    else:
        nodes, tets = inputs.sphere(h=0.06)
        M = inputs.smoothed_unit_m(tets, nodes.shape[0], batch=B, seed=405)
        kw = dict(p=6, leaf_size=64)
    pl = _plan(nodes, tets, theta=0.5, near_mode=1, max_batch=B, precision="bf16x3", **kw)
    assert pl.stats()["n_near_tiles"] > 0
    Md = torch.as_tensor(M, device="cuda")
    u0, H0 = pl.eval(Md)
    for _ in range(4):
        u, H = pl.eval(Md)
        st = _lib.demag_eval_status(pl.handle, torch.cuda.current_stream().cuda_stream)
        assert st == _lib.DEMAG_OK
        assert torch.equal(u, u0) and torch.equal(H, H0)
