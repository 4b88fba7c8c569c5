"""Argument validation of the C ABI, on the host (no GPU needed): every bad
argument is reported as a status, with a message, before any device work."""
import ctypes as C

import numpy as np
import pytest

from paper_1606_00247_gb300 import _lib as L
from paper_1606_00247_gb300 import inputs

INVALID, UNSUPPORTED = 1, 6


@pytest.fixture(scope="module")
def mesh():
    from paper_1606_00247_gb300 import build

    build()
    nodes, tets = inputs.unit_cube(2)
    return np.ascontiguousarray(nodes), np.ascontiguousarray(tets, dtype=np.int32)


def _create(mesh, p=4, leaf=8, theta=0.5, **opts):
    nodes, tets = mesh
    o = L.demag_options_default()
    for k, v in opts.items():
        setattr(o, k, v)
    st, h = L.demag_plan_create(nodes.ctypes.data, nodes.shape[0], tets.ctypes.data, tets.shape[0], p, leaf, theta,
                                o)
    if st == 0:
        L.demag_plan_destroy(h)
    return st


@pytest.mark.parametrize("kw, status", [
    (dict(p=0), INVALID), (dict(p=13), INVALID), (dict(leaf=0), INVALID), (dict(theta=0.0), INVALID),
    (dict(theta=float("nan")), INVALID), (dict(max_batch=0), INVALID), (dict(autotune=8), INVALID),
    (dict(near_mode=2), INVALID), (dict(precision=5), INVALID), (dict(m2l_targets_per_cta=3), INVALID),
    (dict(m2l_kps=9), INVALID), (dict(m2l_promote_rows=65), INVALID), (dict(sources=3), INVALID),
    (dict(sources=1, near_mode=0), UNSUPPORTED), (dict(sources=2, near_mode=0), UNSUPPORTED),
    (dict(graph=2), INVALID), (dict(m2l_split_degree=1), INVALID),
])
def test_plan_create_rejects(mesh, kw, status):
    assert _create(mesh, **kw) == status
    assert L.demag_last_error()  # a message says which argument


def test_null_arguments(mesh):
    nodes, tets = mesh
    h = C.c_void_p()
    lib = L.load()
    assert lib.demag_plan_create(None, nodes.shape[0], tets.ctypes.data, tets.shape[0], 4, 8, 0.5, None,
                                 C.byref(h)) == INVALID
    assert lib.demag_eval(None, None, 1, None, None, None) == INVALID
    assert lib.demag_energy(None, None, None, 1, None, None) == INVALID
    assert lib.demag_llg_rk4(None, None, 1, 1.0, 0.1, None, 0.01, 1, None) == INVALID
    assert lib.demag_plan_destroy(None) == INVALID
    assert L.demag_status_string(INVALID) and L.demag_status_string(UNSUPPORTED)
