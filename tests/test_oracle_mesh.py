"""Whole-mesh pins of the oracle (Sec. 1 Eq. (2), Sec. 4.1).

  * Uniformly magnetised cube: the discrete sum over the Kuhn tets must equal
    the closed-form potential of the two charged faces z=0, z=1 (sigma = -1, +1)
    exactly, because interior face charges cancel and div M = 0.  The face
    potential is the classical rectangle antiderivative
        F(X,Y) = X ln(Y+R) + Y ln(X+R) - Z atan(XY/(ZR)).
  * Cube demagnetising factor 1/3 and energy mu0 Ms^2/6 (Sec. 4.1), reached by
    the mass-lumped H as the mesh is refined.
  * Symmetries: mirror z -> 1-z flips u; rotating mesh and M leaves u unchanged.
  * Mass lumping reproduces -grad u exactly for a linear u.
"""
import os

import numpy as np
import pytest

from paper_1606_00247_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cube_demag.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def _rect_potential(x, y, z, x1, x2, y1, y2, z0):
    """int_{x1}^{x2} int_{y1}^{y2} dx' dy' / |(x',y',z0) - (x,y,z)|."""

    def F(X, Y, Z):
        R = np.sqrt(X * X + Y * Y + Z * Z)
        t1 = np.where(X == 0, 0.0, X * np.log(np.where(X == 0, 1.0, Y + R)))
        t2 = np.where(Y == 0, 0.0, Y * np.log(np.where(Y == 0, 1.0, X + R)))
        safe = (Z != 0) & (R > 0)
        t3 = np.where(safe, Z * np.arctan(np.where(safe, X * Y / np.where(safe, Z * R, 1.0), 0.0)), 0.0)
        return t1 + t2 - t3

    Z = z0 - z
    return (F(x2 - x, y2 - y, Z) - F(x1 - x, y2 - y, Z) - F(x2 - x, y1 - y, Z) + F(x1 - x, y1 - y, Z))


def cube_closed_form_u(nodes):
    x, y, z = nodes.T
    top = _rect_potential(x, y, z, 0.0, 1.0, 0.0, 1.0, 1.0)
    bot = _rect_potential(x, y, z, 0.0, 1.0, 0.0, 1.0, 0.0)
    return (top - bot) / (4.0 * np.pi)


@pytest.mark.parametrize("n", [2, 4])
def test_cube_direct_equals_closed_form(orc, n):
    nodes, tets = inputs.unit_cube(n)
    M = inputs.uniform_m(nodes.shape[0])
    u = orc.direct(nodes, tets, M)
    ref = cube_closed_form_u(nodes)
    assert np.max(np.abs(u - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_cube_closed_form_sanity():
    """The closed form itself: at the centre u = 0 by symmetry; on the top face
    centre the potential equals that of the top plate minus the bottom plate."""
    c = np.array([[0.5, 0.5, 0.5]])
    assert abs(cube_closed_form_u(c)[0]) < 1e-15
    # plate self-potential at its centre: 4 * int_0^{1/2}int_0^{1/2} 1/r = 4 ln(1+sqrt2)
    v = _rect_potential(np.array([0.5]), np.array([0.5]), np.array([1.0]), 0, 1, 0, 1, 1.0)[0]
    assert abs(v - 4.0 * np.log(1.0 + np.sqrt(2.0))) < 1e-14


def test_cube_mirror_symmetry(orc):
    nodes, tets = inputs.unit_cube(4)
    M = inputs.uniform_m(nodes.shape[0])
    u = orc.direct(nodes, tets, M)
    key = {tuple(np.round(p, 9)): i for i, p in enumerate(nodes)}
    mirror = np.array([key[(round(p[0], 9), round(p[1], 9), round(1.0 - p[2], 9))] for p in nodes])
    assert np.max(np.abs(u + u[mirror])) <= 1e-13 * np.max(np.abs(u))


def test_cube_demag_factor_and_energy(orc):
    """<H_z> -> -N Ms with N = 1/3 and E = -(mu0/2) sum V_i M.H_i -> mu0 Ms^2/6."""
    g = _golden()
    errs = []
    for n in (4, 8):
        nodes, tets = inputs.unit_cube(n)
        M = inputs.uniform_m(nodes.shape[0])
        u = cube_closed_form_u(nodes)  # exact nodal potential (pinned above)
        H = orc.lumped_H(nodes, tets, u)
        vol = np.abs(orc.tet_volumes(nodes, tets))
        V = np.zeros(nodes.shape[0])
        np.add.at(V, tets.ravel(), np.repeat(vol / 4.0, 4))
        E = -0.5 * np.sum(V * np.einsum("ij,ij->i", M, H))
        Hz = np.sum(V * H[:, 2]) / np.sum(V)
        errs.append((abs(E - g["energy_over_mu0_Ms2_V"]), abs(-Hz - g["demag_factor"])))
    # P1 interpolation error on the faces decays under refinement
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1]
    assert errs[1][0] < 5e-3 and errs[1][1] < 1e-2


def test_lumped_H_exact_for_linear_u(orc):
    nodes, tets = inputs.sphere(h=0.25)
    g = np.array([0.3, -1.2, 0.7])
    u = nodes @ g + 0.4
    H = orc.lumped_H(nodes, tets, u)
    assert np.max(np.abs(H + g[None, :])) < 1e-12


def test_direct_linear_and_batched(orc):
    nodes, tets = inputs.unit_cube(2)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=3)
    u = orc.direct(nodes, tets, M)
    for b in range(3):
        assert np.allclose(u[b], orc.direct(nodes, tets, M[b]), rtol=0, atol=1e-15)
    u_comb = orc.direct(nodes, tets, 2.0 * M[0] - M[1])
    assert np.max(np.abs(u_comb - (2.0 * u[0] - u[1]))) < 1e-13


def test_direct_rotation_invariant(orc):
    nodes, tets = inputs.sphere(h=0.3)
    M = inputs.gaussian_unit_m(nodes.shape[0])
    th = 0.7
    Q = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    ax = np.array([1.0, 2.0, 2.0]) / 3.0
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Q = Q @ (np.eye(3) + np.sin(0.4) * K + (1 - np.cos(0.4)) * K @ K)
    u0 = orc.direct(nodes, tets, M)
    u1 = orc.direct(nodes @ Q.T, tets, M @ Q.T)
    assert np.max(np.abs(u1 - u0)) <= 1e-12 * np.max(np.abs(u0))
    H0 = orc.lumped_H(nodes, tets, u0)
    H1 = orc.lumped_H(nodes @ Q.T, tets, u1)
    assert np.max(np.abs(H1 - H0 @ Q.T)) <= 1e-11 * np.max(np.abs(H0))


def test_sphere_uniform_interior_field(orc):
    """Uniformly magnetised ball: u = M.r/3 inside, H = -M/3 (convergence only,
    the Delaunay ball is a polyhedron)."""
    errs = []
    for h in (0.35, 0.22):
        nodes, tets = inputs.sphere(h=h)
        M = inputs.uniform_m(nodes.shape[0], (0.0, 0.0, 1.0))
        u = orc.direct(nodes, tets, M)
        inner = np.linalg.norm(nodes, axis=1) < 0.5
        errs.append(np.max(np.abs(u[inner] - nodes[inner, 2] / 3.0)))
    assert errs[1] < errs[0] and errs[1] < 0.02


def test_whole_mesh_charge_route(orc):
    """For continuous P1 M the interior face charges cancel, so the boundary-face
    charges plus the volume charges give the same u as the per-tet sum; the
    boundary faces found are exactly the cube's surface triangles."""
    for nodes, tets in (inputs.unit_cube(3), inputs.sphere(h=0.3)):
        M = inputs.gaussian_unit_m(nodes.shape[0], batch=2, seed=17)
        a = orc.direct(nodes, tets, M)
        b = orc.direct_charges(nodes, tets, M)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    nodes, tets = inputs.unit_cube(3)
    bf = orc.boundary_faces(tets)
    assert len(bf) == 6 * 2 * 3 * 3  # two triangles per boundary square
    faces = np.array([[tets[t][k] for k in range(4) if k != f] for t, f in bf])
    xyz = nodes[faces]  # (n_faces, 3 vertices, 3 coordinates)
    on_plane = np.any(np.all(np.isclose(xyz, 0.0), axis=1) | np.all(np.isclose(xyz, 1.0), axis=1), axis=1)
    assert np.all(on_plane)  # every boundary face lies in a face plane of the cube
