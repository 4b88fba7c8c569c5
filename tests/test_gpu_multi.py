"""demag_eval_multi: several meshes (different sizes, orders and precisions)
in one submission, first call direct + graph recording, later calls graph
replay.  Every result is bit-identical to the plan's own demag_eval."""
import numpy as np
import pytest
import torch

from paper_1606_00247_gb300 import inputs

pytestmark = pytest.mark.gpu


def _meshes():
    return [
        (inputs.unit_cube(4), dict(p=4, leaf_size=16, near_mode=1, precision="fp64"), 3),
        (inputs.sphere(h=0.15), dict(p=6, leaf_size=32, near_mode=1, precision="fp32"), 5),
        (inputs.sphere(h=0.13), dict(p=8, leaf_size=32, near_mode=1, precision="bf16x3"), 128),
        (inputs.unit_cube(6), dict(p=4, leaf_size=16, near_mode=0, precision="fp32"), 2),
    ]


def test_multi_equals_separate_evals_and_replays():
    from paper_1606_00247_gb300.api import Plan, eval_multi_into

    plans, Ms, ref = [], [], []
    for k, ((nodes, tets), kw, B) in enumerate(_meshes()):
        pl = Plan(nodes, tets, max_batch=B, **kw)
        M = torch.as_tensor(inputs.gaussian_unit_m(nodes.shape[0], seed=300 + k, batch=B), device="cuda")
        plans.append(pl)
        Ms.append(M)
        ref.append(pl.eval(M))
    us = [torch.empty_like(r[0]) for r in ref]
    Hs = [torch.empty_like(r[1]) for r in ref]
    for call in range(3):  # direct + record, then two replays
        for u, H in zip(us, Hs):
            u.fill_(np.nan)
            H.fill_(np.nan)
        eval_multi_into(plans, Ms, us, Hs)
        torch.cuda.synchronize()
        for (u0, H0), u, H in zip(ref, us, Hs):
            assert torch.equal(u, u0) and torch.equal(H, H0), call
    # new inputs in the same tensors replay the graph with the new values
    for k, M in enumerate(Ms):
        M.copy_(torch.as_tensor(inputs.gaussian_unit_m(M.shape[1], seed=400 + k, batch=M.shape[0])))
    eval_multi_into(plans, Ms, us, Hs)
    for pl, M, u, H in zip(plans, Ms, us, Hs):
        u1, H1 = pl.eval(M)
        assert torch.equal(u, u1) and torch.equal(H, H1)


def test_multi_rejects_bad_arguments():
    from paper_1606_00247_gb300 import _lib as L
    from paper_1606_00247_gb300.api import Plan, eval_multi_into

    nodes, tets = inputs.unit_cube(3)
    pl = Plan(nodes, tets, p=3, leaf_size=8, max_batch=2)
    M = torch.as_tensor(inputs.gaussian_unit_m(nodes.shape[0], batch=2), device="cuda")
    u = torch.empty((2, nodes.shape[0]), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):  # the same plan twice
        eval_multi_into([pl, pl], [M, M], [u, u])
    with pytest.raises(RuntimeError):  # batch above max_batch
        M3 = torch.cat([M, M[:1]])
        eval_multi_into([pl], [M3], [torch.empty((3, nodes.shape[0]), dtype=torch.float64, device="cuda")])
    with pytest.raises(RuntimeError):  # host pointers
        eval_multi_into([pl], [M.cpu()], [u])


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_single_eval_graph_replay(prec):
    """graph = 1: demag_eval with device pointers records its first call as a
    CUDA graph and replays it; results equal a plan without graphs, bit for
    bit, on the first call and on replays with new values in the same
    tensors."""
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.sphere(h=0.15)
    B = 8 if prec == "fp64" else 128
    kw = dict(p=6, leaf_size=32, near_mode=1, max_batch=B, precision=prec)
    g = Plan(nodes, tets, graph=True, **kw)
    d = Plan(nodes, tets, **kw)
    M = torch.as_tensor(inputs.gaussian_unit_m(nodes.shape[0], batch=B, seed=61), device="cuda")
    u = torch.empty((B, nodes.shape[0]), dtype=torch.float64, device="cuda")
    H = torch.empty((B, nodes.shape[0], 3), dtype=torch.float64, device="cuda")
    for seed in (61, 62, 63):
        M.copy_(torch.as_tensor(inputs.gaussian_unit_m(nodes.shape[0], batch=B, seed=seed)))
        g.eval(M, u, H)
        ud, Hd = d.eval(M)
        torch.cuda.synchronize()
        assert torch.equal(u, ud) and torch.equal(H, Hd), seed
