"""demag_eval_noalloc: the evaluation for callers that must not allocate device
memory while they run (their own pool allocator owns the device memory, or they
cannot pay cudaMalloc's implicit synchronisation).  All of its scratch lives in
the library's fixed device array; its results must equal demag_eval's.

Collected last on purpose (file name), so that a stop-at-first-failure run has
already run every other test; it also passes when run alone."""
import numpy as np
import pytest
import torch

from paper_1606_00247_gb300 import inputs

pytestmark = pytest.mark.gpu


def _call_noalloc(plan, M, u, H):
    from paper_1606_00247_gb300 import _lib

    st = _lib.demag_eval_noalloc(plan.handle, M.data_ptr(), M.shape[0], u.data_ptr(), H.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    return st


# every layout of the scratch area: FP64 (on-the-fly and stored near field), FP32 with the
# per-tet state of the on-the-fly near field, FP32 stored, and the tensor-core precisions
# with more states than the table M2L takes (the packed-moment buffer of the tensor-core M2L)
CASES = [("fp64", 0, 3), ("fp64", 1, 3), ("fp32", 1, 3), ("fp32", 0, 3), ("bf16x3", 1, 16), ("tf32", 1, 16)]


@pytest.mark.parametrize("precision,near_mode,B", CASES)
def test_noalloc_matches_eval_twice(precision, near_mode, B):
    from paper_1606_00247_gb300 import _lib
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.sphere(h=0.2)
    plan = Plan(nodes, tets, p=6, leaf_size=16, max_batch=B, precision=precision, near_mode=near_mode)
    for call, seed in enumerate((11, 12)):  # two calls in a row with different inputs
        M = torch.as_tensor(inputs.gaussian_unit_m(nodes.shape[0], seed=seed, batch=B), device="cuda")
        u_ref, H_ref = plan.eval(M)
        u = torch.full_like(u_ref, float("nan"))
        H = torch.full_like(H_ref, float("nan"))
        st = _call_noalloc(plan, M, u, H)
        assert st == _lib.DEMAG_OK, _lib.demag_last_error()
        assert _lib.demag_eval_status(plan.handle, torch.cuda.current_stream().cuda_stream) == _lib.DEMAG_OK
        torch.cuda.synchronize()
        tol = 1e-12 if precision == "fp64" else 1e-6
        assert float(torch.linalg.norm(u - u_ref) / torch.linalg.norm(u_ref)) <= tol, call
        assert float(torch.linalg.norm(H - H_ref) / torch.linalg.norm(H_ref)) <= tol, call


@pytest.mark.parametrize("precision,near_mode,B", [("fp32", 0, 3), ("bf16x3", 1, 16)])
def test_noalloc_first_call_allocates_nothing(precision, near_mode, B):
    """On a fresh plan the entry point is called before any demag_eval (which
    would allocate the plan's workspace): free device memory is the same before
    and after, and the results equal demag_eval's.  A first call on another
    plan with the same options has loaded the kernels and the scratch array."""
    from paper_1606_00247_gb300 import _lib
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.sphere(h=0.2)
    kw = dict(p=6, leaf_size=16, max_batch=B, precision=precision, near_mode=near_mode)
    M = torch.as_tensor(inputs.gaussian_unit_m(nodes.shape[0], seed=21, batch=B), device="cuda")
    u = torch.empty((B, nodes.shape[0]), dtype=torch.float64, device="cuda")
    H = torch.empty((B, nodes.shape[0], 3), dtype=torch.float64, device="cuda")
    warm = Plan(nodes, tets, **kw)
    assert _call_noalloc(warm, M, u, H) == _lib.DEMAG_OK
    torch.cuda.synchronize()
    fresh = Plan(nodes, tets, **kw)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _call_noalloc(fresh, M, u, H) == _lib.DEMAG_OK, _lib.demag_last_error()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    u_ref, H_ref = fresh.eval(M)
    tol = 1e-6
    assert float(torch.linalg.norm(u - u_ref) / torch.linalg.norm(u_ref)) <= tol
    assert float(torch.linalg.norm(H - H_ref) / torch.linalg.norm(H_ref)) <= tol


def test_noalloc_rejects_oversized_scratch_and_host_pointers():
    from paper_1606_00247_gb300 import _lib
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.sphere(h=0.12)
    # FP64 moments and locals: 2 x 165 doubles per cell and state at p = 8 -> far beyond
    # 64 MiB for 64 states
    B = 64
    plan = Plan(nodes, tets, p=8, leaf_size=8, max_batch=B, near_mode=0)
    assert plan.stats()["n_cells"] * 165 * 16 * B > 64 * 2**20
    M = torch.as_tensor(inputs.gaussian_unit_m(nodes.shape[0], batch=B), device="cuda")
    u = torch.empty((B, nodes.shape[0]), dtype=torch.float64, device="cuda")
    H = torch.empty((B, nodes.shape[0], 3), dtype=torch.float64, device="cuda")
    st = _call_noalloc(plan, M, u, H)
    assert st == _lib.DEMAG_ERR_INVALID_ARG
    assert "fixed area holds" in _lib.demag_last_error()
    Mh = np.zeros((1, nodes.shape[0], 3))
    uh = np.zeros((1, nodes.shape[0]))
    st = _lib.demag_eval_noalloc(plan.handle, Mh.ctypes.data, 1, uh.ctypes.data, None, None)
    assert st == _lib.DEMAG_ERR_INVALID_ARG
