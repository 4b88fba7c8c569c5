"""ctypes binding of libdemag.so (include/demag.h): same names, argument
marshalling only.  Every computation runs in the CUDA library; there is no
Python or CPU fallback -- if the library cannot be loaded, this raises."""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdemag.so")

DEMAG_OK = 0
DEMAG_ERR_INVALID_ARG = 1
DEMAG_ERR_DEGENERATE_TET = 2
DEMAG_ERR_OUT_OF_MEMORY = 3
DEMAG_ERR_CUDA = 4
DEMAG_ERR_TIMEOUT = 5
DEMAG_ERR_UNSUPPORTED = 6
DEMAG_ERR_INTERNAL = 7

DEMAG_FP64 = 0
DEMAG_MIXED_FP32 = 1
DEMAG_MIXED_TF32 = 2
DEMAG_MIXED_BF16X3 = 3
DEMAG_MIXED_BF16X6 = 4


class demag_options(C.Structure):
    _fields_ = [("p", C.c_int), ("leaf_size", C.c_int), ("theta", C.c_double), ("precision", C.c_int),
                ("near_mode", C.c_int), ("max_batch", C.c_int), ("autotune", C.c_int), ("profile", C.c_int),
                ("m2l_targets_per_cta", C.c_int), ("m2l_kps", C.c_int),
                ("m2l_promote", C.c_int), ("m2l_promote_rows", C.c_int),
                ("m2l_table_batch", C.c_int), ("sources", C.c_int), ("near_tc", C.c_int),
                ("graph", C.c_int), ("m2l_split_degree", C.c_int)]


DEMAG_N_STAGES = 9
STAGES = ["gather", "p2m", "m2m", "m2l", "l2l", "l2p", "near_prep", "p2p", "h"]


class demag_stats(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tets", C.c_int64), ("n_cells", C.c_int64), ("n_leaves", C.c_int64),
                ("n_levels", C.c_int64), ("n_m2l", C.c_int64), ("n_p2p", C.c_int64), ("n_p2p_pairs", C.c_int64),
                ("n_near_cols", C.c_int64), ("device_bytes", C.c_int64), ("lo", C.c_double * 3),
                ("side", C.c_double), ("scale", C.c_double), ("plan_ms", C.c_double), ("p", C.c_int),
                ("leaf_size", C.c_int), ("precision", C.c_int), ("near_mode", C.c_int), ("max_batch", C.c_int),
                ("theta", C.c_double), ("eval_launches", C.c_int64), ("n_evals_profiled", C.c_int64),
                ("stage_ms", C.c_double * DEMAG_N_STAGES), ("stage_launches", C.c_int64 * DEMAG_N_STAGES),
                ("n_m2l_ops", C.c_int64), ("m2l_kps", C.c_int), ("m2l_ring_bytes", C.c_int),
                ("m2l_targets_per_cta", C.c_int), ("n_near_tiles", C.c_int64), ("near_tile_cols", C.c_int64),
                ("near_bytes", C.c_int64), ("tune_source", C.c_int)]


class demag_tree_export(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in (
        "node_key", "tet_key", "node_perm", "tet_perm", "cell_level", "cell_prefix", "cell_ranges", "cell_parent",
        "cell_child", "cell_centre", "cell_radius", "m2l_off", "m2l_src", "p2p_off", "p2p_src")]


_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True):
    """Load libdemag.so (building it with nvcc if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH) and build_if_missing:
            from .build import build  # the package exports the function under the module's name

            build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libdemag.so is not built (run paper_1606_00247_gb300/build.py)")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int, C.c_double
        L.demag_options_default.restype = None
        L.demag_options_default.argtypes = [C.POINTER(demag_options)]
        L.demag_plan_create.restype = i32
        L.demag_plan_create.argtypes = [vp, i64, vp, i64, i32, i32, d, C.POINTER(demag_options), C.POINTER(vp)]
        L.demag_eval.restype = i32
        L.demag_eval.argtypes = [vp, vp, i32, vp, vp, vp]
        L.demag_eval_field.restype = i32
        L.demag_eval_field.argtypes = [vp, vp, i32, vp, vp, vp]
        L.demag_plan_debug.restype = i32
        L.demag_plan_debug.argtypes = [vp, i32]
        L.demag_plan_audit.restype = i32
        L.demag_plan_audit.argtypes = [vp]
        L.demag_eval_status.restype = i32
        L.demag_eval_status.argtypes = [vp, vp]
        L.demag_eval_noalloc.restype = i32
        L.demag_eval_noalloc.argtypes = [vp, vp, i32, vp, vp, vp]
        L.demag_eval_multi.restype = i32
        L.demag_eval_multi.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.demag_energy.restype = i32
        L.demag_energy.argtypes = [vp, vp, vp, i32, vp, vp]
        L.demag_llg_rk4.restype = i32
        L.demag_llg_rk4.argtypes = [vp, vp, i32, d, d, vp, d, i32, vp]
        L.demag_plan_destroy.restype = i32
        L.demag_plan_destroy.argtypes = [vp]
        L.demag_plan_stats.restype = i32
        L.demag_plan_stats.argtypes = [vp, C.POINTER(demag_stats)]
        L.demag_plan_reset_timers.restype = i32
        L.demag_plan_reset_timers.argtypes = [vp]
        L.demag_plan_export_tree.restype = i32
        L.demag_plan_export_tree.argtypes = [vp, C.POINTER(demag_tree_export)]
        L.demag_measure_peak.restype = i32
        L.demag_measure_peak.argtypes = [i32, C.POINTER(C.c_double)]
        L.demag_status_string.restype = C.c_char_p
        L.demag_status_string.argtypes = [i32]
        L.demag_last_error.restype = C.c_char_p
        L.demag_last_error.argtypes = []
        _lib = L
        return L


def demag_options_default() -> demag_options:
    o = demag_options()
    load().demag_options_default(C.byref(o))
    return o


def demag_plan_create(nodes_ptr, n_nodes, tets_ptr, n_tets, p, leaf_size, theta, opt: demag_options | None):
    h = C.c_void_p()
    st = load().demag_plan_create(nodes_ptr, n_nodes, tets_ptr, n_tets, p, leaf_size, theta,
                                  C.byref(opt) if opt is not None else None, C.byref(h))
    return st, h


def demag_eval(plan, M_ptr, batch, u_ptr, H_ptr, stream_ptr):
    return load().demag_eval(plan, M_ptr, batch, u_ptr, H_ptr, stream_ptr)


def demag_eval_status(plan, stream_ptr):
    """DEMAG_ERR_TIMEOUT if a bounded device wait expired in the plan's last evaluation (synchronises)."""
    return load().demag_eval_status(plan, stream_ptr)


def demag_eval_field(plan, M_ptr, batch, u_ptr, H_ptr, stream_ptr):
    """u and the pointwise field -grad u at the interior nodes (mass-lumped H at boundary nodes)."""
    return load().demag_eval_field(plan, M_ptr, batch, u_ptr, H_ptr, stream_ptr)


def demag_plan_debug(plan, flags):
    """Test hooks: bit 0 stalls the tensor-core near field so that its bounded wait
    expires; bit 1 makes demag_plan_audit also audit a copy of the M2L list with one
    entry out of range."""
    return load().demag_plan_debug(plan, flags)


def demag_plan_audit(plan):
    """Bounds audit of the plan's index lists (run by demag_plan_create on every plan)."""
    return load().demag_plan_audit(plan)


def demag_eval_noalloc(plan, M_ptr, batch, u_ptr, H_ptr, stream_ptr):
    """demag_eval with its scratch in the library's fixed device array (no allocation)."""
    return load().demag_eval_noalloc(plan, M_ptr, batch, u_ptr, H_ptr, stream_ptr)


def demag_eval_multi(plans_ptr, n_plans, M_ptrs, batch_ptr, u_ptrs, H_ptrs, stream_ptr):
    """Several plans in one submission; every argument but n_plans is a pointer to an array."""
    return load().demag_eval_multi(plans_ptr, n_plans, M_ptrs, batch_ptr, u_ptrs, H_ptrs, stream_ptr)


def demag_energy(plan, M_ptr, H_ptr, batch, e_ptr, stream_ptr):
    return load().demag_energy(plan, M_ptr, H_ptr, batch, e_ptr, stream_ptr)


def demag_llg_rk4(plan, m_ptr, batch, Ms, alpha, h_ext_ptr, dt, steps, stream_ptr):
    return load().demag_llg_rk4(plan, m_ptr, batch, Ms, alpha, h_ext_ptr, dt, steps, stream_ptr)


def demag_plan_destroy(plan):
    return load().demag_plan_destroy(plan)


def demag_plan_stats(plan) -> tuple[int, demag_stats]:
    s = demag_stats()
    st = load().demag_plan_stats(plan, C.byref(s))
    return st, s


def demag_plan_reset_timers(plan):
    return load().demag_plan_reset_timers(plan)


def demag_plan_export_tree(plan, out: demag_tree_export):
    return load().demag_plan_export_tree(plan, C.byref(out))


PEAK_KINDS = {"fp64_fma": 0, "fp32_fma": 1, "bf16_mma": 2, "tf32_mma": 3}


def demag_measure_peak(kind: int) -> tuple[int, float]:
    """Measured TFLOP/s of one arithmetic path of the current device (see include/demag.h)."""
    v = C.c_double(0.0)
    st = load().demag_measure_peak(int(kind), C.byref(v))
    return st, float(v.value)


def demag_status_string(status: int) -> str:
    return load().demag_status_string(status).decode()


def demag_last_error() -> str:
    return load().demag_last_error().decode()


class DemagError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {demag_status_string(status)} ({demag_last_error()})")


def check(status: int, where: str):
    if status != DEMAG_OK:
        raise DemagError(status, where)
