"""Argument checks of the Python binding (no GPU needed): the library reads and
writes (B, N_n, 3) and (B, N_n) doubles through bare pointers, so arrays of
another shape, type or layout are rejected in Python before any call."""
import numpy as np
import pytest
import torch


def _plan(nn):
    from paper_1606_00247_gb300.api import Plan

    pl = object.__new__(Plan)  # a plan object without a library plan behind it
    pl._h = None
    pl.device = torch.device("cpu")
    pl.n_nodes, pl.n_tets, pl.p, pl.max_batch = nn, 1, 4, 2
    return pl


def test_mesh_arrays_must_be_n_by_3_and_n_by_4():
    from paper_1606_00247_gb300.api import Plan

    tets = np.array([[0, 1, 2, 3]])
    with pytest.raises(ValueError):
        Plan(np.zeros((4, 2)), tets, device="cpu")
    with pytest.raises(ValueError):
        Plan(np.eye(4, 3), tets[:, :3], device="cpu")


def test_eval_rejects_mis_shaped_inputs_and_outputs():
    nn = 7
    pl = _plan(nn)
    M = torch.zeros(2, nn, 3, dtype=torch.float64)
    with pytest.raises(ValueError):
        pl.eval(torch.zeros(2, nn + 1, 3))
    with pytest.raises(ValueError):
        pl.eval(torch.zeros(2, nn * 3))
    with pytest.raises(ValueError):
        pl.eval(M, u=torch.zeros(2, nn, dtype=torch.float32))
    with pytest.raises(ValueError):
        pl.eval(M, u=torch.zeros(2, nn + 1, dtype=torch.float64))
    with pytest.raises(ValueError):
        pl.eval(M, u=torch.zeros(nn, 2, dtype=torch.float64).t())  # not contiguous
    with pytest.raises(ValueError):
        pl.eval(M, u=torch.zeros(2, nn, dtype=torch.float64), H=torch.zeros(2, nn, 2, dtype=torch.float64))
    with pytest.raises(ValueError):
        pl.eval_field(torch.zeros(1, nn - 1, 3))
    with pytest.raises(ValueError):
        pl.energy(M, torch.zeros(1, nn, 3, dtype=torch.float64))
    with pytest.raises(ValueError):
        pl.llg_rk4(torch.zeros(2, nn, 4, dtype=torch.float64))


def test_eval_host_rejects_mis_shaped_arrays():
    nn = 5
    pl = _plan(nn)
    with pytest.raises(ValueError):
        pl.eval_host(np.zeros((2, nn, 2)))
    with pytest.raises(ValueError):
        pl.eval_host(np.zeros((2, nn, 3)), u=np.zeros((2, nn), dtype=np.float32))
    with pytest.raises(ValueError):
        pl.eval_host(np.zeros((2, nn, 3)), u=np.zeros((2, nn)), H=np.zeros((2, nn, 3))[:, ::-1])
    with pytest.raises(ValueError):
        pl.eval_host(np.zeros((2, nn, 3)), u=np.zeros((2, nn + 1)))


def test_eval_multi_into_rejects_mis_shaped_arrays():
    from paper_1606_00247_gb300.api import eval_multi_into

    a, b = _plan(5), _plan(6)
    Ms = [torch.zeros(2, 5, 3, dtype=torch.float64), torch.zeros(1, 6, 3, dtype=torch.float64)]
    us = [torch.zeros(2, 5, dtype=torch.float64), torch.zeros(1, 6, dtype=torch.float64)]
    with pytest.raises(ValueError):  # counts differ
        eval_multi_into([a, b], Ms[:1], us)
    with pytest.raises(ValueError):  # a 2-D magnetisation has no batch extent
        eval_multi_into([a], [torch.zeros(5, 3, dtype=torch.float64)], [torch.zeros(1, 5, dtype=torch.float64)])
    with pytest.raises(ValueError):  # another mesh's node count
        eval_multi_into([a, b], [Ms[1], Ms[0]], us)
    with pytest.raises(ValueError):  # output of the wrong size
        eval_multi_into([a, b], Ms, [us[0], torch.zeros(2, 6, dtype=torch.float64)])
    with pytest.raises(ValueError):  # H of the wrong size
        eval_multi_into([a, b], Ms, us, [torch.zeros(2, 5, 3, dtype=torch.float64), torch.zeros(1, 6, dtype=torch.float64)])
    with pytest.raises(ValueError):  # single precision
        eval_multi_into([a], [Ms[0].float()], us[:1])
