"""Seeded synthetic inputs: tetrahedral meshes and nodal magnetisations.

This module holds no arithmetic of the method itself: it only produces meshes
(node coordinates + tet connectivity) and nodal magnetisation fields with the
shapes and structure of the paper's workloads.  The paper's own meshes are not
available, so these stand in for them.  It is the one module shared by the
CUDA path's tests/benchmarks and the CPU oracle's tests.

Recipes (seeds: mesh 1606, magnetisation 247, per-workload offsets +0..+4):
  * Kuhn box: an nx x ny x nz grid of sub-cubes, each split into the 6
    tetrahedra [v, v+e_a, v+e_a+e_b, v+(1,1,1)] over the 6 axis orders (a,b,c);
    conforming across sub-cubes.  Unit cube 8^3 -> 3072 tets / 729 nodes; thin
    film 2000x1000x10 on 576x288x2 -> 1,990,656 tets / 500,259 nodes.
  * Sphere: jittered cubic lattice (spacing h, uniform jitter +-0.2h) inside
    r < R - h/2 plus Fibonacci points on r = R at spacing ~h, Delaunay
    tetrahedralised (scipy), tets with volume < 1e-6 h^3 dropped.
  * Ellipsoid: the sphere recipe scaled by (1, a, b).
  * Magnetisations: uniform; iid Gaussian vectors normalised per node; a
    Landau flux-closure pattern plus seeded tilt; random unit vectors smoothed
    over mesh-edge neighbours.
"""
from __future__ import annotations

import itertools

import numpy as np

MESH_SEED = 1606
MAG_SEED = 247


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------
def kuhn_box(n=(8, 8, 8), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Structured Kuhn (Freudenthal) tetrahedralisation of a box."""
    nx, ny, nz = (int(v) for v in n)
    xs = np.linspace(lo[0], hi[0], nx + 1)
    ys = np.linspace(lo[1], hi[1], ny + 1)
    zs = np.linspace(lo[2], hi[2], nz + 1)
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    nodes = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def idx(i, j, k):
        return (i * (ny + 1) + j) * (nz + 1) + k

    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    tets = []
    for perm in itertools.permutations(range(3)):
        e = np.eye(3, dtype=np.int64)
        p0 = np.stack([I, J, K], 1)
        p1 = p0 + e[perm[0]]
        p2 = p1 + e[perm[1]]
        p3 = p0 + 1
        tets.append(np.stack([idx(*q.T) for q in (p0, p1, p2, p3)], 1))
    tets = np.stack(tets, 1).reshape(-1, 4)
    return nodes.astype(np.float64), tets.astype(np.int32)


def unit_cube(n=8):
    return kuhn_box((n, n, n))


def thin_film(nx=576, ny=288, nz=2, size=(2000.0, 1000.0, 10.0)):
    return kuhn_box((nx, ny, nz), (0.0, 0.0, 0.0), size)


def _fibonacci_sphere(n, radius):
    i = np.arange(n) + 0.5
    phi = np.arccos(1.0 - 2.0 * i / n)
    golden = np.pi * (3.0 - np.sqrt(5.0))
    th = golden * i
    return radius * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)


def sphere(h=0.05, radius=1.0, seed=MESH_SEED + 1, scale=(1.0, 1.0, 1.0)):
    """Quasi-uniform Delaunay tet mesh of a ball (optionally scaled to an ellipsoid)."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    m = int(np.ceil(radius / h)) + 1
    g = np.arange(-m, m + 1) * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    pts = pts + rng.uniform(-0.2 * h, 0.2 * h, size=pts.shape)
    pts = pts[np.linalg.norm(pts, axis=1) < radius - 0.5 * h]
    n_surf = int(round(4.0 * np.pi * radius ** 2 / (h * h * np.sqrt(3.0) / 2.0)))
    pts = np.concatenate([pts, _fibonacci_sphere(n_surf, radius)], 0)
    tri = Delaunay(pts)
    tets = tri.simplices.astype(np.int64)
    a, b, c, d = (pts[tets[:, k]] for k in range(4))
    vol = np.einsum("ij,ij->i", b - a, np.cross(c - a, d - a)) / 6.0
    tets = tets[np.abs(vol) >= 1e-6 * h ** 3]
    used = np.unique(tets)
    remap = -np.ones(pts.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.shape[0])
    nodes = pts[used] * np.asarray(scale, dtype=np.float64)[None, :]
    return np.ascontiguousarray(nodes, dtype=np.float64), remap[tets].astype(np.int32)


def ellipsoid(h=0.05, a=2.0, b=3.0, seed=MESH_SEED + 3):
    return sphere(h=h, radius=1.0, seed=seed, scale=(1.0, a, b))


# Mesh spacings that give the tet counts of the named workloads (found once by
# running the generator; Delaunay counts vary by well under 1% with the seed).
SPHERE_200K_H = 0.0505
SPHERE_500K_H = 0.0372


def batch_meshes(n=64, min_tets=1e4, max_tets=3e5, seed=MESH_SEED + 4):
    """Meshes of uneven size for many-mesh submissions: target sizes
    log-uniform in [min_tets, max_tets], types round-robin Kuhn cube, ball,
    ellipsoid with axis ratios (1, a, b), a, b ~ U[1, 4] (a ball mesh stretched
    by those factors).  Ball spacings are scaled from the ball of 223,668 tets
    at SPHERE_200K_H."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(min_tets), np.log(max_tets), n))
    out = []
    for i, size in enumerate(sizes):
        kind = i % 3
        if kind == 0:
            k = max(2, int(round((size / 6.0) ** (1.0 / 3.0))))
            out.append(kuhn_box((k, k, k)))
        elif kind == 1:
            out.append(sphere(h=SPHERE_200K_H * (223668.0 / size) ** (1.0 / 3.0), seed=seed + i))
        else:
            a, b = rng.uniform(1.0, 4.0, 2)  # the ball's mesh stretched: same tet count, elongated tets
            h = SPHERE_200K_H * (223668.0 / size) ** (1.0 / 3.0)
            out.append(sphere(h=h, seed=seed + i, scale=(1.0, a, b)))
    return out


# ---------------------------------------------------------------------------
# magnetisations (nodal, shape (N_n, 3) or (B, N_n, 3))
# ---------------------------------------------------------------------------
def uniform_m(n_nodes, direction=(0.0, 0.0, 1.0)):
    return np.tile(np.asarray(direction, dtype=np.float64)[None, :], (n_nodes, 1))


def gaussian_unit_m(n_nodes, seed=MAG_SEED + 1, batch=None):
    rng = np.random.default_rng(seed)
    shape = (n_nodes, 3) if batch is None else (batch, n_nodes, 3)
    m = rng.standard_normal(shape)
    return m / np.linalg.norm(m, axis=-1, keepdims=True)


def affine_m(nodes, A, b):
    """M(r) = A r + b sampled at the nodes (P1-exact)."""
    return nodes @ np.asarray(A, dtype=np.float64).T + np.asarray(b, dtype=np.float64)[None, :]


def landau_m(nodes, size=(2000.0, 1000.0), tilt=0.05, seed=MAG_SEED + 2):
    """Flux-closure pattern: nearest film edge (ties: bottom, right, top, left)
    gives +x, +y, -x, -y; then normalise(M0 + tilt * N(0,1)^3)."""
    x, y = nodes[:, 0], nodes[:, 1]
    d = np.stack([y, size[0] - x, size[1] - y, x], 1)  # bottom, right, top, left
    which = np.argmin(d, axis=1)
    dirs = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0]], dtype=np.float64)
    m = dirs[which]
    rng = np.random.default_rng(seed)
    m = m + tilt * rng.standard_normal(m.shape)
    return m / np.linalg.norm(m, axis=1, keepdims=True)


def smoothed_unit_m(tets, n_nodes, batch=1, passes=3, seed=MAG_SEED + 3):
    """iid unit vectors, then `passes` times M_i <- normalise(M_i + sum_{j~i} M_j)
    over mesh-edge neighbours."""
    import scipy.sparse as sp

    rng = np.random.default_rng(seed)
    m = rng.standard_normal((batch, n_nodes, 3))
    m /= np.linalg.norm(m, axis=-1, keepdims=True)
    t = np.asarray(tets, dtype=np.int64)
    e = np.concatenate([t[:, [a, b]] for a in range(4) for b in range(a + 1, 4)], 0)
    e = np.unique(np.sort(e, axis=1), axis=0)
    # I + adjacency of the mesh edges (each edge once, both directions)
    A = sp.coo_matrix((np.ones(2 * len(e)), (np.r_[e[:, 0], e[:, 1]], np.r_[e[:, 1], e[:, 0]])),
                      shape=(n_nodes, n_nodes)).tocsr() + sp.identity(n_nodes, format="csr")
    for _ in range(passes):
        acc = (A @ m.transpose(1, 0, 2).reshape(n_nodes, -1)).reshape(n_nodes, batch, 3).transpose(1, 0, 2)
        m = acc / np.linalg.norm(acc, axis=-1, keepdims=True)
    return np.ascontiguousarray(m)


def random_tet(rng, scale=1.0, min_quality=0.05):
    """A random non-degenerate tet (4x3) for the single-tet checks."""
    while True:
        v = rng.uniform(-scale, scale, size=(4, 3))
        a, b, c, d = v
        vol = abs(np.dot(b - a, np.cross(c - a, d - a))) / 6.0
        edges = [np.linalg.norm(v[i] - v[j]) for i in range(4) for j in range(i + 1, 4)]
        if vol / max(edges) ** 3 > min_quality / 6.0 * 0.1:
            return v


INCLUSION_SEED = 603
GRADED_20M_H0 = 1.0 / 80.0


def _lattice(lo, hi, h, rng, jitter=0.2):
    """Jittered cubic lattice of spacing h over the box [lo, hi] (points inside it)."""
    axes = [np.arange(lo[a] + 0.5 * h, hi[a], h) for a in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    p = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    return p + rng.uniform(-jitter * h, jitter * h, size=p.shape)


def graded_cube(h0=GRADED_20M_H0, n_incl=50, seed=INCLUSION_SEED):
    """Unit cube with n_incl spherical inclusions refined 8x: point spacing h0
    outside, h0/2 and h0/4 in two transition shells (1.5 h0 and 0.75 h0
    thick), h0/8 inside each ball.  Centres U[0.1, 0.9]^3, radii U[0.02, 0.05],
    rejection so balls plus shells are disjoint.  Jittered lattices per region,
    the cube's boundary sampled on an unjittered face lattice of spacing h0,
    Delaunay (scipy); tets with volume below 1e-6 (h0/8)^3 dropped.  Returns
    (nodes, tets, centres, radii)."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    sa, sb = 0.75 * h0, 1.5 * h0
    cen, rad = [], []
    for _ in range(1000 * n_incl):
        if len(cen) == n_incl:
            break
        c, r = rng.uniform(0.1, 0.9, 3), rng.uniform(0.02, 0.05)
        if all(np.linalg.norm(c - c2) > r + r2 + 2 * (sa + sb) for c2, r2 in zip(cen, rad)):
            cen.append(c)
            rad.append(r)
    if len(cen) < n_incl:
        raise ValueError(f"{n_incl} inclusions with their shells do not fit at h0 = {h0}")
    cen, rad = np.array(cen), np.array(rad)
    outer = rad + sa + sb
    pts = []
    # outside: spacing h0, away from every ball's outer shell and from the cube faces
    p = _lattice((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), h0, rng)
    p = p[np.all((p > 0.25 * h0) & (p < 1.0 - 0.25 * h0), axis=1)]
    d = np.min(np.linalg.norm(p[:, None, :] - cen[None, :, :], axis=2) - outer[None, :], axis=1)
    pts.append(p[d > 0.0])
    # cube faces: unjittered lattice of spacing h0 on each face (the hull is the cube)
    g = np.linspace(0.0, 1.0, int(round(1.0 / h0)) + 1)
    U, V = np.meshgrid(g, g, indexing="ij")
    for a in range(3):
        for v in (0.0, 1.0):
            f = np.zeros((U.size, 3))
            f[:, a] = v
            f[:, (a + 1) % 3] = U.ravel()
            f[:, (a + 2) % 3] = V.ravel()
            pts.append(f)
    # per inclusion: ball at h0/8, shells at h0/4 and h0/2
    for c, r in zip(cen, rad):
        for h, r0, r1 in ((h0 / 8, 0.0, r), (h0 / 4, r, r + sa), (h0 / 2, r + sa, r + sa + sb)):
            q = _lattice(c - r1, c + r1, h, rng)
            dq = np.linalg.norm(q - c, axis=1)
            keep = (dq >= r0) & (dq < r1) & np.all((q > 0.25 * h) & (q < 1.0 - 0.25 * h), axis=1)  # inside the cube
            pts.append(q[keep])
    pts = np.unique(np.concatenate(pts, 0), axis=0)
    tri = Delaunay(pts)
    tets = tri.simplices.astype(np.int64)
    a, b, c4, d4 = (pts[tets[:, k]] for k in range(4))
    vol = np.einsum("ij,ij->i", b - a, np.cross(c4 - a, d4 - a)) / 6.0
    tets = tets[np.abs(vol) >= 1e-6 * (h0 / 8) ** 3]
    used = np.unique(tets)
    remap = -np.ones(pts.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.shape[0])
    return np.ascontiguousarray(pts[used]), remap[tets].astype(np.int32), cen, rad
