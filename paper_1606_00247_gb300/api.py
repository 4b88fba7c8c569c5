"""Python face of the C ABI: a Plan object over demag_plan_create / demag_eval.

PyTorch supplies device memory and streams; every stage runs in libdemag.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L

_PREC = {"fp64": L.DEMAG_FP64, "fp32": L.DEMAG_MIXED_FP32, "tf32": L.DEMAG_MIXED_TF32,
         "bf16x3": L.DEMAG_MIXED_BF16X3, "bf16x6": L.DEMAG_MIXED_BF16X6}
_SOURCES = {"tets": 0, "dipoles": 1, "patches": 2}  # DEMAG_SOURCES_TETS, _DIPOLES, _PATCHES


def _as_f64(x, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.float64).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device=device)


def _same_device(t, device):
    return t.device.type == device.type and (device.index is None or t.device.index == device.index)


def _check_rows(name, t, n_nodes, width):
    """The library reads and writes (B, n_nodes[, width]) doubles through a bare
    pointer, so a tensor of another shape is rejected here, before the call."""
    tail = (n_nodes,) if width is None else (n_nodes, width)
    if tuple(t.shape[-len(tail):]) != tail or t.dim() > len(tail) + 1:
        raise ValueError(f"{name} must have shape (B, {', '.join(map(str, tail))}) or {tail}, not {tuple(t.shape)}")


def _check_out(name, t, numel, device=None):
    """A caller-given output tensor: contiguous float64 (on the plan's device when
    given) with room for exactly the result (the library writes doubles into it)."""
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous() \
            or t.numel() != numel or (device is not None and not _same_device(t, device)):
        raise ValueError(f"{name} must be a contiguous float64 tensor of {numel} elements"
                         + (f" on {device}" if device is not None else ""))


def _check_host_out(name, a, numel):
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != numel:
        raise ValueError(f"{name} must be a C-contiguous float64 array of {numel} elements")


def _as_i32(x, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.int32).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.int32), device=device)


class Plan:
    """Tree, lists and operators of one mesh (demag_plan_create)."""

    def __init__(self, nodes, tets, p=4, leaf_size=32, theta=0.5, precision="fp64", near_mode=0, max_batch=1,
                 device="cuda", profile=False, autotune=False, m2l_targets_per_cta=0, m2l_kps=0,
                 m2l_promote=0, m2l_promote_rows=0, m2l_table_batch=0, sources="tets", near_tc=0, graph=False,
                 m2l_split_degree=0):
        self.device = torch.device(device)
        nodes_t = _as_f64(nodes, self.device)
        tets_t = _as_i32(tets, self.device)
        if nodes_t.dim() != 2 or nodes_t.shape[1] != 3 or tets_t.dim() != 2 or tets_t.shape[1] != 4:
            raise ValueError(f"nodes must be (N_n, 3) and tets (N_t, 4), not {tuple(nodes_t.shape)} and "
                             f"{tuple(tets_t.shape)}")
        self.n_nodes, self.n_tets = int(nodes_t.shape[0]), int(tets_t.shape[0])
        opt = L.demag_options_default()
        opt.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        opt.near_mode = int(near_mode)
        opt.max_batch = int(max_batch)
        opt.profile = int(bool(profile))
        opt.autotune = int(autotune)  # bit 0: M2L launch shape, bit 1: leaf size
        opt.m2l_targets_per_cta = int(m2l_targets_per_cta)
        opt.m2l_kps = int(m2l_kps)
        opt.m2l_promote = int(m2l_promote)
        opt.m2l_promote_rows = int(m2l_promote_rows)
        opt.m2l_table_batch = int(m2l_table_batch)
        opt.sources = _SOURCES[sources] if isinstance(sources, str) else int(sources)
        opt.near_tc = int(near_tc)
        opt.m2l_split_degree = int(m2l_split_degree)
        opt.graph = int(bool(graph))  # demag_eval with device pointers: record once, replay as a CUDA graph
        with torch.cuda.device(self.device):
            st, h = L.demag_plan_create(nodes_t.data_ptr(), self.n_nodes, tets_t.data_ptr(), self.n_tets, int(p),
                                        int(leaf_size), float(theta), opt)
        L.check(st, "demag_plan_create")
        self._h = h
        self.p, self.max_batch = int(p), int(max_batch)

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            L.demag_plan_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def eval(self, M, u=None, H=None, with_H=True, stream=None):
        """u (B, N_n) and H (B, N_n, 3) for M (B, N_n, 3) or (N_n, 3) on the device."""
        M = _as_f64(M, self.device)
        _check_rows("M", M, self.n_nodes, 3)
        squeeze = M.dim() == 2
        if squeeze:
            M = M.unsqueeze(0)
        B = int(M.shape[0])
        if u is None:
            u = torch.empty((B, self.n_nodes), dtype=torch.float64, device=self.device)
        else:
            _check_out("u", u, B * self.n_nodes, self.device)
        if with_H and H is None:
            H = torch.empty((B, self.n_nodes, 3), dtype=torch.float64, device=self.device)
        elif with_H:
            _check_out("H", H, B * self.n_nodes * 3, self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        st = L.demag_eval(self._h, M.data_ptr(), B, u.data_ptr(), H.data_ptr() if with_H else None, s.cuda_stream)
        L.check(st, "demag_eval")
        if squeeze:
            return u[0], (H[0] if with_H else None)
        return u, (H if with_H else None)

    def eval_field(self, M, stream=None):
        """u (B, N_n) and the pointwise field H = -grad u (B, N_n, 3) at the interior
        nodes (mass-lumped H at the boundary nodes); FP64 plans with tet sources."""
        M = _as_f64(M, self.device)
        _check_rows("M", M, self.n_nodes, 3)
        squeeze = M.dim() == 2
        if squeeze:
            M = M.unsqueeze(0)
        B = int(M.shape[0])
        u = torch.empty((B, self.n_nodes), dtype=torch.float64, device=self.device)
        H = torch.empty((B, self.n_nodes, 3), dtype=torch.float64, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        L.check(L.demag_eval_field(self._h, M.data_ptr(), B, u.data_ptr(), H.data_ptr(), s.cuda_stream),
                "demag_eval_field")
        return (u[0], H[0]) if squeeze else (u, H)

    def energy(self, M, H, stream=None):
        """e[b] = -(1/2) sum_i V_i M_b,i . H_b,i (demag_energy; E = mu0 e), device tensors (B, N_n, 3)."""
        if M.dim() == 2:
            M, H = M.unsqueeze(0), H.unsqueeze(0)
        if M.dtype != torch.float64 or H.dtype != torch.float64 or not M.is_contiguous() or not H.is_contiguous():
            raise ValueError("M and H must be contiguous float64 device tensors")
        _check_rows("M", M, self.n_nodes, 3)
        if H.shape != M.shape:
            raise ValueError(f"H must have M's shape {tuple(M.shape)}, not {tuple(H.shape)}")
        e = torch.empty(M.shape[0], dtype=torch.float64, device=M.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        L.check(L.demag_energy(self._h, M.data_ptr(), H.data_ptr(), M.shape[0], e.data_ptr(), s.cuda_stream),
                "demag_energy")
        return e

    def llg_rk4(self, m, Ms=1.0, alpha=0.0, h_ext=None, dt=0.01, steps=1, stream=None):
        """Advance the unit states m (B, N_n, 3), in place, by `steps` RK4 steps of the
        LLG equation with the demagnetising field (demag_llg_rk4, reduced units)."""
        if m.dtype != torch.float64 or not m.is_contiguous() or not m.is_cuda:
            raise ValueError("m must be a contiguous float64 device tensor")
        _check_rows("m", m, self.n_nodes, 3)
        if m.dim() == 2:
            m = m.unsqueeze(0)
        hx = None
        if h_ext is not None:
            hx = (C.c_double * 3)(*[float(v) for v in h_ext])
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        L.check(L.demag_llg_rk4(self._h, m.data_ptr(), m.shape[0], float(Ms), float(alpha),
                                C.cast(hx, C.c_void_p) if hx is not None else None, float(dt), int(steps),
                                s.cuda_stream), "demag_llg_rk4")
        return m

    def eval_host(self, M: np.ndarray, with_H=True, u=None, H=None):
        """Same call with host (numpy) buffers: the library copies in and out.
        u and H may be given (e.g. views of pinned host memory, for fast copies)."""
        M = np.ascontiguousarray(M, dtype=np.float64)
        if M.shape[-2:] != (self.n_nodes, 3) or M.ndim > 3:
            raise ValueError(f"M must have shape (B, {self.n_nodes}, 3) or ({self.n_nodes}, 3), not {M.shape}")
        squeeze = M.ndim == 2
        if squeeze:
            M = M[None]
        B = M.shape[0]
        if u is None:
            u = np.empty((B, self.n_nodes))
        else:
            _check_host_out("u", u, B * self.n_nodes)
        if with_H and H is None:
            H = np.empty((B, self.n_nodes, 3))
        elif with_H:
            _check_host_out("H", H, B * self.n_nodes * 3)
        if not with_H:
            H = None
        with torch.cuda.device(self.device):
            st = L.demag_eval(self._h, M.ctypes.data, B, u.ctypes.data, H.ctypes.data if with_H else None, None)
        L.check(st, "demag_eval")
        if squeeze:
            return u[0], (H[0] if with_H else None)
        return u, H

    def stats(self) -> dict:
        st, s = L.demag_plan_stats(self._h)
        L.check(st, "demag_plan_stats")
        out = {f: getattr(s, f) for f, _ in s._fields_}
        out["lo"] = list(s.lo)
        out["stage_ms"] = dict(zip(L.STAGES, list(s.stage_ms)))
        out["stage_launches"] = dict(zip(L.STAGES, list(s.stage_launches)))
        return out

    def reset_timers(self):
        L.check(L.demag_plan_reset_timers(self._h), "demag_plan_reset_timers")

    def export_tree(self) -> dict:
        s = self.stats()
        nn, nt, nc = s["n_nodes"], s["n_tets"], s["n_cells"]
        arrs = dict(
            node_key=np.zeros(nn, np.uint64), tet_key=np.zeros(nt, np.uint64), node_perm=np.zeros(nn, np.int64),
            tet_perm=np.zeros(nt, np.int64), cell_level=np.zeros(nc, np.int32), cell_prefix=np.zeros(nc, np.uint64),
            cell_ranges=np.zeros((nc, 4), np.int64), cell_parent=np.zeros(nc, np.int64),
            cell_child=np.zeros((nc, 2), np.int64), cell_centre=np.zeros((nc, 3)), cell_radius=np.zeros((nc, 2)),
            m2l_off=np.zeros(nc + 1, np.int64), m2l_src=np.zeros(max(s["n_m2l"], 1), np.int64),
            p2p_off=np.zeros(nc + 1, np.int64), p2p_src=np.zeros(max(s["n_p2p"], 1), np.int64))
        ex = L.demag_tree_export()
        for k, a in arrs.items():
            setattr(ex, k, a.ctypes.data)
        L.check(L.demag_plan_export_tree(self._h, ex), "demag_plan_export_tree")
        arrs["m2l_src"] = arrs["m2l_src"][: s["n_m2l"]]
        arrs["p2p_src"] = arrs["p2p_src"][: s["n_p2p"]]
        return arrs


def eval_multi(plans, Ms, stream=None, with_H=True):
    """Evaluate several plans through one submission (demag_eval_multi):
    Ms[i] is (B_i, N_n_i, 3) on plans[i]'s device.  Returns lists of u and H.
    The first call with given tensors runs directly and records a CUDA graph;
    later calls with the same tensors replay it."""
    import ctypes as C

    n = len(plans)
    if n != len(Ms) or n < 1:
        raise ValueError("one magnetisation tensor per plan")
    dev = plans[0].device
    Ms = [_as_f64(M, dev) for M in Ms]
    Ms = [M.unsqueeze(0) if M.dim() == 2 else M for M in Ms]
    us = [torch.empty((int(M.shape[0]), pl.n_nodes), dtype=torch.float64, device=dev) for M, pl in zip(Ms, plans)]
    Hs = [torch.empty((int(M.shape[0]), pl.n_nodes, 3), dtype=torch.float64, device=dev) for M, pl in zip(Ms, plans)]
    return eval_multi_into(plans, Ms, us, Hs if with_H else None, stream=stream)


def eval_multi_into(plans, Ms, us, Hs=None, stream=None):
    """demag_eval_multi with caller-provided outputs (same tensors -> graph replay)."""
    import ctypes as C

    n = len(plans)
    if n < 1 or len(Ms) != n or len(us) != n or (Hs is not None and len(Hs) != n):
        raise ValueError("one magnetisation and one output tensor per plan")
    for i, (pl, M) in enumerate(zip(plans, Ms)):  # shapes here; devices and batch limits in the library
        _check_rows(f"Ms[{i}]", M, pl.n_nodes, 3)
        if M.dim() != 3:
            raise ValueError(f"Ms[{i}] must be (B, {pl.n_nodes}, 3): the batch is its first extent")
        B = int(M.shape[0])
        _check_out(f"Ms[{i}]", M, B * pl.n_nodes * 3)
        _check_out(f"us[{i}]", us[i], B * pl.n_nodes)
        if Hs is not None:
            _check_out(f"Hs[{i}]", Hs[i], B * pl.n_nodes * 3)
    P = (C.c_void_p * n)(*[pl.handle for pl in plans])
    Mp = (C.c_void_p * n)(*[M.data_ptr() for M in Ms])
    up = (C.c_void_p * n)(*[u.data_ptr() for u in us])
    Hp = (C.c_void_p * n)(*[H.data_ptr() for H in Hs]) if Hs is not None else None
    bt = (C.c_int * n)(*[int(M.shape[0]) for M in Ms])
    s = stream if stream is not None else torch.cuda.current_stream(plans[0].device)
    st = L.demag_eval_multi(C.cast(P, C.c_void_p), n, C.cast(Mp, C.c_void_p), C.cast(bt, C.c_void_p),
                            C.cast(up, C.c_void_p), C.cast(Hp, C.c_void_p) if Hp is not None else None, s.cuda_stream)
    L.check(st, "demag_eval_multi")
    return us, Hs

