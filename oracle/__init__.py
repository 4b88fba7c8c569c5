"""CPU FP64 oracle for the tetrahedral-FMM demagnetisation potential.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product path (the CUDA library behind ``include/demag.h``) shares no code with
it and never calls it.

The C sources (``oracle_direct.c``, ``oracle_fmm.c``) implement, from the paper
(Palmesi et al., Sec. 1 Eq. (1)-(2), Sec. 2, Sec. 3, Sec. 4.1):
  * the closed-form integral of M.grad'(1/R) over one P1-magnetised tet,
  * the same integral by the paper's target-apex cone decomposition with
    adaptive quadrature (Sec. 2.1 / Sec. 4 check), and by a 3-D product rule,
  * the direct O(N_nodes N_tets) sum and the mass-lumped H (Sec. 4.1),
  * exact tet moments (Eq. expCoeffs), M2M / M2L / L2L / L2P (Sec. 2, 2.3),
  * the octree, radii, MAC and dual tree traversal (Sec. 3.1-3.3),
  * the plain CPU FMM.
This module is ctypes marshalling around them, plus two plain numpy routines:
the lumped nodal volumes and the direct sum of the point-dipole comparison
model (dipole_direct).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRCS = ["oracle_direct.c", "oracle_fmm.c"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so in place (gcc, FP64, no FMA contraction, OpenMP)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_t for s in srcs):
            return _SO
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", _SO + ".tmp"] + [os.path.join(_HERE, s) for s in _SRCS] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int, C.c_double
            L.oracle_tet_potential.restype = d
            L.oracle_tet_potential.argtypes = [vp, vp, vp]
            L.oracle_tet_potential_cone_quad.restype = d
            L.oracle_tet_potential_cone_quad.argtypes = [vp, vp, vp, d]
            L.oracle_tet_potential_gauss3d.restype = d
            L.oracle_tet_potential_gauss3d.argtypes = [vp, vp, vp, i32]
            L.oracle_direct.restype = i32
            L.oracle_direct.argtypes = [vp, i64, vp, i64, vp, i32, vp, i64, vp, i32]
            L.oracle_direct_charges.restype = i32
            L.oracle_direct_charges.argtypes = [vp, i64, vp, i64, vp, i64, vp, i32, vp, i64, vp, i32]
            L.oracle_field_charges.restype = i32
            L.oracle_field_charges.argtypes = [vp, i64, vp, i64, vp, i64, vp, i32, vp, i64, vp, i32]
            L.oracle_lumped_H.restype = i32
            L.oracle_lumped_H.argtypes = [vp, i64, vp, i64, vp, i32, vp]
            L.oracle_tet_volumes.restype = None
            L.oracle_tet_volumes.argtypes = [vp, vp, i64, vp]
            L.oracle_ncoef.restype = i32
            L.oracle_ncoef.argtypes = [i32]
            L.oracle_multi_indices.restype = None
            L.oracle_multi_indices.argtypes = [i32, vp]
            L.oracle_laplace_derivs.restype = None
            L.oracle_laplace_derivs.argtypes = [vp, i32, vp]
            L.oracle_tet_moments.restype = None
            L.oracle_tet_moments.argtypes = [vp, vp, vp, i32, vp]
            L.oracle_tet_lambda_monomial_exact.restype = d
            L.oracle_tet_lambda_monomial_exact.argtypes = [vp, vp, i32, i32, i32, i32]
            for fn in ("oracle_m2m", "oracle_m2l", "oracle_l2l"):
                getattr(L, fn).restype = None
                getattr(L, fn).argtypes = [i32, vp, vp, vp]
            L.oracle_l2p.restype = d
            L.oracle_l2p.argtypes = [i32, vp, vp]
            L.oracle_multipole_eval.restype = d
            L.oracle_multipole_eval.argtypes = [i32, vp, vp, vp]
            L.oracle_tree_build.restype = vp
            L.oracle_tree_build.argtypes = [vp, i64, vp, i64, i32, d, C.POINTER(C.c_int)]
            L.oracle_tree_build_sources.restype = vp
            L.oracle_tree_build_sources.argtypes = [vp, i64, vp, i64, i32, d, i32, C.POINTER(C.c_int)]
            L.oracle_tree_free.restype = None
            L.oracle_tree_free.argtypes = [vp]
            L.oracle_tree_info.restype = None
            L.oracle_tree_info.argtypes = [vp, vp]
            L.oracle_tree_box.restype = None
            L.oracle_tree_box.argtypes = [vp, vp]
            L.oracle_tree_export.restype = None
            L.oracle_tree_export.argtypes = [vp] + [vp] * 15
            L.oracle_fmm_eval.restype = i32
            L.oracle_fmm_eval.argtypes = [vp, i32, vp, i32, vp, vp, i64, i32]
            L.oracle_max_threads.restype = i32
            L.oracle_max_threads.argtypes = []
            _lib = L
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def max_threads() -> int:
    return int(lib().oracle_max_threads())


# ---- single tet -----------------------------------------------------------
def tet_potential(r, v, M) -> float:
    """int_tet M.grad'(1/|r-r'|) dV' (no 1/4pi), closed form."""
    r, v, M = _f64(r, 3), _f64(v, 12), _f64(M, 12)
    return lib().oracle_tet_potential(_p(r), _p(v), _p(M))


def tet_potential_cone_quad(r, v, M, rel_tol=1e-13) -> float:
    r, v, M = _f64(r, 3), _f64(v, 12), _f64(M, 12)
    return lib().oracle_tet_potential_cone_quad(_p(r), _p(v), _p(M), rel_tol)


def tet_potential_gauss3d(r, v, M, q=24) -> float:
    r, v, M = _f64(r, 3), _f64(v, 12), _f64(M, 12)
    return lib().oracle_tet_potential_gauss3d(_p(r), _p(v), _p(M), q)


# ---- whole mesh -------------------------------------------------------------
def direct(nodes, tets, M, targets=None, nthreads=0):
    """u (B, n_targets) by the direct sum (Eq. (2)); M is (B, N_n, 3) or (N_n, 3)."""
    nodes, tets = _f64(nodes), _i32(tets)
    M = _f64(M)
    squeeze = M.ndim == 2
    if squeeze:
        M = M[None]
    B = M.shape[0]
    nn, nt = nodes.shape[0], tets.shape[0]
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    ntg = nn if tg is None else tg.shape[0]
    u = np.zeros((B, ntg))
    rc = lib().oracle_direct(_p(nodes), nn, _p(tets), nt, _p(M), B, _p(tg), ntg, _p(u), nthreads)
    if rc:
        raise RuntimeError("oracle_direct failed")
    return u[0] if squeeze else u


def boundary_faces(tets):
    """(tet, local face) pairs of the faces that belong to one tet only (face f
    is opposite vertex f)."""
    t = np.asarray(tets, dtype=np.int64)
    faces = np.concatenate([np.delete(t, f, axis=1) for f in range(4)])  # (4 N_t, 3), face f of tet j at f N_t + j
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    one = np.where(cnt[inv.ravel()] == 1)[0]
    return np.stack([one % len(t), one // len(t)], axis=1).astype(np.int32)


def direct_charges(nodes, tets, M, targets=None, nthreads=0):
    """u by the whole-mesh charge route (boundary-face charges + volume charges),
    the same shape conventions as direct()."""
    nodes, tets = _f64(nodes), _i32(tets)
    M = _f64(M)
    squeeze = M.ndim == 2
    if squeeze:
        M = M[None]
    B = M.shape[0]
    nn, nt = nodes.shape[0], tets.shape[0]
    bf = np.ascontiguousarray(boundary_faces(tets))
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    ntg = nn if tg is None else tg.shape[0]
    u = np.zeros((B, ntg))
    rc = lib().oracle_direct_charges(_p(nodes), nn, _p(tets), nt, _p(bf), bf.shape[0], _p(M), B, _p(tg), ntg, _p(u),
                                     nthreads)
    if rc:
        raise RuntimeError("oracle_direct_charges failed")
    return u[0] if squeeze else u


def field_charges(nodes, tets, M, points, nthreads=0):
    """Pointwise field H = -grad u (B, n_pts, 3) at points (n_pts, 3) that lie on
    no boundary face, by the whole-mesh charge route in closed form: the field
    of the boundary faces' affine surface charges n.M plus every tet's constant
    volume charge -div M (the remark of Sec. 4.1-4.2 on computing H directly)."""
    nodes, tets = _f64(nodes), _i32(tets)
    M = _f64(M)
    squeeze = M.ndim == 2
    if squeeze:
        M = M[None]
    B = M.shape[0]
    pts = _f64(points).reshape(-1, 3)
    bf = np.ascontiguousarray(boundary_faces(tets))
    H = np.zeros((B, pts.shape[0], 3))
    rc = lib().oracle_field_charges(_p(nodes), nodes.shape[0], _p(tets), tets.shape[0], _p(bf), bf.shape[0], _p(M), B,
                                    _p(pts), pts.shape[0], _p(H), nthreads)
    if rc:
        raise RuntimeError("oracle_field_charges failed")
    return H[0] if squeeze else H


def interior_nodes(tets, n_nodes):
    """Indices of the nodes that lie on no boundary face (where the pointwise field is defined)."""
    t = np.asarray(tets, dtype=np.int64)
    bf = boundary_faces(t)
    on = np.zeros(n_nodes, bool)
    for f in range(4):
        sel = bf[bf[:, 1] == f, 0]
        on[np.delete(t[sel], f, axis=1).ravel()] = True
    return np.where(~on)[0]


def lumped_volumes(nodes, tets):
    """Lumped nodal volumes V_i = sum over the tets t containing node i of |Omega_t| / 4."""
    vol = np.abs(tet_volumes(nodes, tets))  # tet_volumes is signed by orientation
    V = np.zeros(np.asarray(nodes).shape[0])
    np.add.at(V, np.asarray(tets, dtype=np.int64).ravel(), np.repeat(vol / 4.0, 4))
    return V


def dipole_direct(nodes, tets, M, targets=None, points=None, chunk=512):
    """Point-dipole comparison model (the node-dipole treatment the paper compares
    with, Sec. 4): every node j carries the dipole V_j M_j and
        u(r) = 1/(4 pi) sum_j V_j M_j . (r - r_j) / |r - r_j|^3,
    the self term j = i left out at a node.  Evaluated at the nodes `targets`
    (all by default) or at the off-mesh `points` (n, 3).  M is (N_n, 3) or
    (B, N_n, 3); plain O(N^2) numpy."""
    nodes = np.asarray(nodes, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    squeeze = M.ndim == 2
    if squeeze:
        M = M[None]
    m = lumped_volumes(nodes, tets)[None, :, None] * M  # (B, N_n, 3) dipole moments
    if points is not None:
        R = np.asarray(points, dtype=np.float64)
        self_idx = None
    else:
        idx = np.arange(nodes.shape[0]) if targets is None else np.asarray(targets, dtype=np.int64)
        R = nodes[idx]
        self_idx = idx
    u = np.zeros((M.shape[0], R.shape[0]))
    for a in range(0, R.shape[0], chunk):
        d = R[a:a + chunk, None, :] - nodes[None, :, :]  # (n, N_n, 3)
        r2 = np.einsum("ijk,ijk->ij", d, d)
        if self_idx is not None:
            r2[np.arange(d.shape[0]), self_idx[a:a + chunk]] = np.inf
        w = d / (r2 * np.sqrt(r2))[:, :, None]
        u[:, a:a + chunk] = np.einsum("ijk,bjk->bi", w, m) / (4.0 * np.pi)
    return u[0] if squeeze else u


def lumped_H(nodes, tets, u):
    nodes, tets, u = _f64(nodes), _i32(tets), _f64(u)
    squeeze = u.ndim == 1
    if squeeze:
        u = u[None]
    B = u.shape[0]
    H = np.zeros((B, nodes.shape[0], 3))
    rc = lib().oracle_lumped_H(_p(nodes), nodes.shape[0], _p(tets), tets.shape[0], _p(u), B, _p(H))
    if rc:
        raise RuntimeError("oracle_lumped_H failed")
    return H[0] if squeeze else H


def tet_volumes(nodes, tets):
    nodes, tets = _f64(nodes), _i32(tets)
    vol = np.zeros(tets.shape[0])
    lib().oracle_tet_volumes(_p(nodes), _p(tets), tets.shape[0], _p(vol))
    return vol


# ---- expansions -------------------------------------------------------------
def ncoef(p: int) -> int:
    return int(lib().oracle_ncoef(p))


def multi_indices(p: int) -> np.ndarray:
    out = np.zeros((ncoef(p), 3), dtype=np.int32)
    lib().oracle_multi_indices(p, _p(out))
    return out


def laplace_derivs(x, p):
    x = _f64(x, 3)
    D = np.zeros(ncoef(p))
    lib().oracle_laplace_derivs(_p(x), p, _p(D))
    return D


def tet_moments(v, M, c, p):
    v, M, c = _f64(v, 12), _f64(M, 12), _f64(c, 3)
    Q = np.zeros(ncoef(p))
    lib().oracle_tet_moments(_p(v), _p(M), _p(c), p, _p(Q))
    return Q


def tet_lambda_monomial_exact(v, c, k, m):
    v, c = _f64(v, 12), _f64(c, 3)
    return lib().oracle_tet_lambda_monomial_exact(_p(v), _p(c), k, int(m[0]), int(m[1]), int(m[2]))


def m2m(p, d, Qc):
    d, Qc = _f64(d, 3), _f64(Qc)
    Qp = np.zeros(ncoef(p))
    lib().oracle_m2m(p, _p(d), _p(Qc), _p(Qp))
    return Qp


def m2l(p, R, Q):
    R, Q = _f64(R, 3), _f64(Q)
    L = np.zeros(ncoef(p))
    lib().oracle_m2l(p, _p(R), _p(Q), _p(L))
    return L


def l2l(p, d, Lp):
    d, Lp = _f64(d, 3), _f64(Lp)
    Lc = np.zeros(ncoef(p))
    lib().oracle_l2l(p, _p(d), _p(Lp), _p(Lc))
    return Lc


def l2p(p, z, L):
    z, L = _f64(z, 3), _f64(L)
    return lib().oracle_l2p(p, _p(z), _p(L))


def multipole_eval(p, c, Q, r):
    c, Q, r = _f64(c, 3), _f64(Q), _f64(r, 3)
    return lib().oracle_multipole_eval(p, _p(c), _p(Q), _p(r))


# ---- tree + FMM ---------------------------------------------------------------
class Tree:
    """Octree, radii and interaction lists of Sec. 3.1-3.3 (see oracle_fmm.c)."""

    def __init__(self, nodes, tets, leaf_size=32, theta=0.5, sources="tets"):
        """sources: "tets" (the method), "dipoles" (point dipoles V_i M_i at the nodes) or
        "patches" (vertex patches lambda_i M_i binned by node, the paper's clustering)."""
        self.nodes, self.tets = _f64(nodes), _i32(tets)
        st = C.c_int(0)
        h = lib().oracle_tree_build_sources(_p(self.nodes), self.nodes.shape[0], _p(self.tets),
                                            self.tets.shape[0], leaf_size, theta,
                                            {"tets": 0, "dipoles": 1, "patches": 2}[sources], C.byref(st))
        if not h or st.value:
            raise ValueError("oracle_tree_build rejected the input")
        self._h = h
        info = np.zeros(5, dtype=np.int64)
        lib().oracle_tree_info(h, _p(info))
        self.n_cells, self.n_m2l, self.n_p2p, self.n_levels, self.n_leaves = (int(x) for x in info)
        box = np.zeros(5)
        lib().oracle_tree_box(h, _p(box))
        self.lo, self.side, self.scale = box[:3].copy(), float(box[3]), float(box[4])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_tree_free(h)
            self._h = None

    def export(self) -> dict:
        nn, nt, nc = self.nodes.shape[0], self.tets.shape[0], self.n_cells
        out = dict(
            node_key=np.zeros(nn, np.uint64), tet_key=np.zeros(nt, np.uint64),
            node_perm=np.zeros(nn, np.int64), tet_perm=np.zeros(nt, np.int64),
            cell_level=np.zeros(nc, np.int32), cell_prefix=np.zeros(nc, np.uint64),
            cell_ranges=np.zeros((nc, 4), np.int64), cell_parent=np.zeros(nc, np.int64),
            cell_child=np.zeros((nc, 2), np.int64), cell_centre=np.zeros((nc, 3)),
            cell_radius=np.zeros((nc, 2)), m2l_off=np.zeros(nc + 1, np.int64),
            m2l_src=np.zeros(max(self.n_m2l, 1), np.int64), p2p_off=np.zeros(nc + 1, np.int64),
            p2p_src=np.zeros(max(self.n_p2p, 1), np.int64))
        keys = ["node_key", "tet_key", "node_perm", "tet_perm", "cell_level", "cell_prefix", "cell_ranges",
                "cell_parent", "cell_child", "cell_centre", "cell_radius", "m2l_off", "m2l_src", "p2p_off",
                "p2p_src"]
        lib().oracle_tree_export(self._h, *[_p(out[k]) for k in keys])
        out["m2l_src"] = out["m2l_src"][: self.n_m2l]
        out["p2p_src"] = out["p2p_src"][: self.n_p2p]
        return out

    def fmm(self, M, p, target_leaves=None, nthreads=0):
        """u (B, N_n) by the plain CPU FMM; with target_leaves only their nodes are filled (NaN elsewhere)."""
        M = _f64(M)
        squeeze = M.ndim == 2
        if squeeze:
            M = M[None]
        B = M.shape[0]
        u = np.full((B, self.nodes.shape[0]), np.nan)
        tl = None if target_leaves is None else np.ascontiguousarray(target_leaves, dtype=np.int64)
        rc = lib().oracle_fmm_eval(self._h, p, _p(M), B, _p(u), _p(tl), 0 if tl is None else tl.shape[0],
                                   nthreads)
        if rc:
            raise RuntimeError("oracle_fmm_eval failed")
        return u[0] if squeeze else u


# ---- energy and LLG stepping (uses of H next to the potential, Sec. 4.1-4.2) -----
def energy(nodes, tets, M, H):
    """Magnetostatic self-energy per state, e = -(1/2) sum_i V_i M_i . H_i with the
    lumped nodal volumes V_i of the mass-lumped H (E = mu0 e).  M, H: (N_n, 3) or
    (B, N_n, 3); plain numpy."""
    V = lumped_volumes(nodes, tets)
    M, H = np.asarray(M, dtype=np.float64), np.asarray(H, dtype=np.float64)
    return -0.5 * np.einsum("i,...ik,...ik->...", V, M, H)


def llg_rhs(m, h, alpha):
    """Landau-Lifshitz-Gilbert right-hand side in reduced units,
    dm/dt = -1/(1 + alpha^2) [ m x h + alpha m x (m x h) ], row by row (..., 3)."""
    mxh = np.cross(m, h)
    return -(mxh + alpha * np.cross(m, mxh)) / (1.0 + alpha * alpha)


def rk4_step(f, y, dt):
    """One classical fourth-order Runge-Kutta step of dy/dt = f(y)."""
    k1 = f(y)
    k2 = f(y + 0.5 * dt * k1)
    k3 = f(y + 0.5 * dt * k2)
    k4 = f(y + dt * k3)
    return y + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def llg_rk4(m, field, Ms, alpha, h_ext, dt, steps):
    """`steps` RK4 steps of the reduced LLG equation for unit states m (B, N_n, 3):
    h = field(Ms y) / Ms + h_ext at every stage state y, where field(M) returns the
    demagnetising field H (B, N_n, 3) of the magnetisation M; m renormalised to
    unit length after each step.  Returns the new m."""
    m = np.array(m, dtype=np.float64)
    hx = np.zeros(3) if h_ext is None else np.asarray(h_ext, dtype=np.float64)
    for _ in range(steps):
        m = rk4_step(lambda y: llg_rhs(y, field(Ms * y) / Ms + hx, alpha), m, dt)
        m /= np.linalg.norm(m, axis=-1, keepdims=True)
    return m
