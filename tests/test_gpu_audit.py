"""Bounds audit of the plan's index lists (demag_plan_audit).

demag_plan_create audits every plan before returning it, so every plan of the
suite passes through it; here it is run again on plans of each kind (FP64 on
the fly, stored FP64, FP32, split BF16 with both tensor-core stages, two-target
M2L groups, point dipoles and vertex patches), and its error path is taken by
auditing a scratch copy of the M2L source list with one entry out of range
(demag_plan_debug bit 1): only the audit kernel reads that copy, so nothing
follows the bad index, and the plan's own lists stay as they were."""
import pytest
import torch

from paper_1606_00247_gb300 import inputs

pytestmark = pytest.mark.gpu

KINDS = [
    dict(precision="fp64", near_mode=0),
    dict(precision="fp64", near_mode=1),
    dict(precision="fp32", near_mode=1, max_batch=4),
    dict(precision="bf16x3", near_mode=1, max_batch=128),
    dict(precision="bf16x3", near_mode=1, max_batch=128, m2l_targets_per_cta=2, m2l_promote=-1),
    dict(precision="fp32", near_mode=1, sources="dipoles"),
    dict(precision="fp64", near_mode=1, sources="patches"),
]


def _plan(nodes, tets, **kw):
    from paper_1606_00247_gb300.api import Plan

    return Plan(nodes, tets, **kw)


@pytest.mark.parametrize("kw", KINDS, ids=lambda k: "-".join(str(v) for v in k.values()))
def test_every_plan_kind_passes_the_audit(kw):
    from paper_1606_00247_gb300 import _lib

    nodes, tets = inputs.sphere(h=0.13)
    pl = _plan(nodes, tets, p=8 if kw["precision"] == "bf16x3" else 6, leaf_size=32, **kw)
    assert _lib.demag_plan_audit(pl.handle) == _lib.DEMAG_OK, _lib.demag_last_error()
    pl.close()


def test_audit_reports_an_index_out_of_range_and_the_plan_stays_usable():
    from paper_1606_00247_gb300 import _lib

    nodes, tets = inputs.sphere(h=0.2)
    M = torch.as_tensor(inputs.gaussian_unit_m(nodes.shape[0], batch=2, seed=503), device="cuda")
    pl = _plan(nodes, tets, p=6, leaf_size=16, max_batch=2, precision="fp32", near_mode=1)
    st = pl.stats()
    assert st["n_m2l"] > 0
    u0, H0 = pl.eval(M)
    assert _lib.demag_plan_debug(pl.handle, 2) == _lib.DEMAG_OK
    assert _lib.demag_plan_audit(pl.handle) == _lib.DEMAG_ERR_INTERNAL
    msg = _lib.demag_last_error()
    assert f"m2l_src (planted copy)[{st['n_m2l'] - 1}] = {st['n_cells']}" in msg and "(1 entries)" in msg
    assert _lib.demag_plan_debug(pl.handle, 0) == _lib.DEMAG_OK
    assert _lib.demag_plan_audit(pl.handle) == _lib.DEMAG_OK
    u1, H1 = pl.eval(M)
    assert torch.equal(u0, u1) and torch.equal(H0, H1)
    assert _lib.demag_plan_debug(pl.handle, 4) == _lib.DEMAG_ERR_INVALID_ARG
