"""Pointwise field H = -grad u at the interior nodes (demag_eval_field; the
remark of Sec. 4.1-4.2 that computing H directly gives lower errors than the
mass-lumped H):
* theta -> 0 (every pair in the near field): the closed-form field of the near
  tets' face and volume charges against the oracle's whole-mesh charge route,
  to rounding;
* theta = 0.5: far field by the gradient of the local expansions; the
  difference to the oracle falls with p (FMM truncation);
* boundary nodes keep the mass-lumped H of demag_eval, u equals demag_eval's;
* uniformly magnetised ball: the pointwise field at interior nodes is closer
  to -M/3 than the mass-lumped one."""
import numpy as np
import pytest
import torch

from paper_1606_00247_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _plan(nodes, tets, **kw):
    from paper_1606_00247_gb300.api import Plan

    return Plan(nodes, tets, precision="fp64", **kw)


@pytest.mark.parametrize("mesh", ["sphere", "cube"])
@pytest.mark.parametrize("near_mode", [0, 1])
def test_field_theta_zero_equals_oracle(orc, mesh, near_mode):
    nodes, tets = inputs.sphere(h=0.25) if mesh == "sphere" else inputs.unit_cube(5)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=3, seed=91)
    pl = _plan(nodes, tets, p=2, leaf_size=32, theta=1e-9, near_mode=near_mode, max_batch=3)
    u, H = pl.eval_field(M)
    ii = orc.interior_nodes(tets, nodes.shape[0])
    ref = orc.field_charges(nodes, tets, M, nodes[ii])
    assert rel(H.cpu().numpy()[:, ii], ref) < 1e-11
    u0, H0 = pl.eval(M)
    assert torch.equal(u, u0)
    bnd = np.setdiff1d(np.arange(nodes.shape[0]), ii)
    assert np.array_equal(H.cpu().numpy()[:, bnd], H0.cpu().numpy()[:, bnd])


def test_field_truncation_falls_with_p(orc):
    nodes, tets = inputs.sphere(h=0.15)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=2, seed=92)
    ii = orc.interior_nodes(tets, nodes.shape[0])
    ref = orc.field_charges(nodes, tets, M, nodes[ii])
    errs = []
    for p in (4, 6, 8):
        _, H = _plan(nodes, tets, p=p, leaf_size=32, theta=0.5, near_mode=1, max_batch=2).eval_field(M)
        errs.append(rel(H.cpu().numpy()[:, ii], ref))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 1e-4, errs


def test_pointwise_field_beats_lumping_on_the_ball(orc):
    nodes, tets = inputs.sphere(h=0.15)
    M = inputs.uniform_m(nodes.shape[0], (0.0, 0.0, 1.0))
    pl = _plan(nodes, tets, p=8, leaf_size=32, theta=0.5, near_mode=1)
    _, Hp = pl.eval_field(M)
    _, Hl = pl.eval(M)
    ii = orc.interior_nodes(tets, nodes.shape[0])
    ii = ii[np.linalg.norm(nodes[ii], axis=1) < 0.7]
    want = np.tile([0.0, 0.0, -1.0 / 3.0], (len(ii), 1))
    ep = rel(Hp.cpu().numpy()[ii], want)
    el = rel(Hl.cpu().numpy()[ii], want)
    assert ep < el, (ep, el)
