"""The error path of a bounded device wait, made to run out on purpose in the
safe form: the tensor-core near field's coefficient producer issues no copy
(demag_plan_debug bit 0), so the MMA issuer's wait for the first stage
expires with no copy and no MMA in flight.  The kernel records
DEMAG_ERR_TIMEOUT, frees its tensor memory and returns; the host learns it
from demag_eval (host pointers) or demag_eval_status (device pointers), and
the same plan then evaluates correctly."""
import numpy as np
import pytest
import torch

from paper_1606_00247_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_and_the_plan_recovers():
    from paper_1606_00247_gb300 import _lib
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.sphere(h=0.2)
    B = 4
    M = torch.as_tensor(inputs.gaussian_unit_m(nodes.shape[0], batch=B, seed=501), device="cuda")
    plan = Plan(nodes, tets, p=6, leaf_size=32, max_batch=B, precision="bf16x3", near_mode=1)
    assert plan.stats()["n_near_tiles"] > 0
    u_ok, H_ok = plan.eval(M)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    assert _lib.demag_eval_status(plan.handle, stream) == _lib.DEMAG_OK

    assert _lib.demag_plan_debug(plan.handle, 1) == _lib.DEMAG_OK
    # device pointers: the call is asynchronous and returns OK; the status query sees the expiry
    u = torch.empty_like(u_ok)
    H = torch.empty_like(H_ok)
    st = _lib.demag_eval(plan.handle, M.data_ptr(), B, u.data_ptr(), H.data_ptr(), stream)
    assert st == _lib.DEMAG_OK
    assert _lib.demag_eval_status(plan.handle, stream) == _lib.DEMAG_ERR_TIMEOUT
    assert "bounded device wait" in _lib.demag_last_error()
    # host pointers: the call itself reports it
    Mh = M.cpu().numpy()
    uh = np.empty((B, nodes.shape[0]))
    with torch.cuda.device(0):
        st = _lib.demag_eval(plan.handle, Mh.ctypes.data, B, uh.ctypes.data, None, None)
    assert st == _lib.DEMAG_ERR_TIMEOUT

    # normal operation again on the same plan and context
    assert _lib.demag_plan_debug(plan.handle, 0) == _lib.DEMAG_OK
    u2, H2 = plan.eval(M)
    assert _lib.demag_eval_status(plan.handle, stream) == _lib.DEMAG_OK
    assert torch.equal(u2, u_ok) and torch.equal(H2, H_ok)
    assert _lib.demag_plan_debug(plan.handle, 4) == _lib.DEMAG_ERR_INVALID_ARG  # bits 0 and 1 are the hooks
