"""Pins of the oracle's single-tet integral (Sec. 2.1 near field, Eq. (2)).

The oracle integrates by parts (surface + volume charges).  It is checked
against two routes that share nothing with that derivation:
  * the paper's own validation protocol (Sec. 4): random tets, random linear
    M, numeric integration -- here the target-apex cone decomposition of
    Sec. 2.1 (Fig. 2) with globally adaptive quadrature over each face;
  * a plain 3-D product Gauss rule for targets well away from the tet;
and against exact invariants (linearity in M, constant-M reduces to the
surface charge of the faces, orientation independence).
"""
import numpy as np
import pytest

from paper_1606_00247_gb300 import inputs


def _targets(v, rng):
    c = v.mean(0)
    d = max(np.linalg.norm(v[i] - v[j]) for i in range(4) for j in range(i + 1, 4))
    n012 = np.cross(v[1] - v[0], v[2] - v[0])
    n012 /= np.linalg.norm(n012)
    return {
        "far": c + 3.0 * d * np.array([0.6, -0.64, 0.48]),
        "near": c + 0.7 * d * np.array([0.36, 0.48, -0.8]),
        "inside": c + 0.05 * d * rng.standard_normal(3),
        "vertex": v[0].copy(),
        "edge_interior": 0.3 * v[0] + 0.7 * v[1],
        "edge_line_beyond": v[1] + 0.4 * (v[1] - v[0]),
        "face_interior": (v[0] + v[1] + v[2]) / 3.0,
        "face_plane_outside": v[0] + 0.8 * (v[0] - v[2]) + 0.3 * (v[1] - v[0]),
        "near_face": (v[0] + v[1] + v[2]) / 3.0 + 1e-4 * d * n012,
        "near_edge": 0.5 * (v[0] + v[1]) + 1e-3 * d * n012,
    }


@pytest.mark.parametrize("seed", range(6))
def test_closed_form_vs_cone_quadrature(orc, seed):
    """Sec. 4: near field vs numeric integration, random tets and random linear M."""
    rng = np.random.default_rng(100 + seed)
    v = inputs.random_tet(rng)
    M = rng.standard_normal((4, 3))
    for name, r in _targets(v, rng).items():
        a = orc.tet_potential(r, v, M)
        q = orc.tet_potential_cone_quad(r, v, M, 1e-13)
        scale = orc.tet_potential_cone_quad(r, v, np.abs(M).max() * np.ones((4, 3)), 1e-10)
        err = abs(a - q) / max(abs(a), abs(scale), 1e-12)
        assert err < 1e-11, (name, a, q)


@pytest.mark.parametrize("seed", range(4))
def test_far_target_vs_product_gauss(orc, seed):
    rng = np.random.default_rng(200 + seed)
    v = inputs.random_tet(rng)
    M = rng.standard_normal((4, 3))
    c = v.mean(0)
    for k in range(4):
        r = c + (4.0 + k) * rng.standard_normal(3)
        a = orc.tet_potential(r, v, M)
        g = orc.tet_potential_gauss3d(r, v, M, 20)
        vol = abs(np.dot(v[1] - v[0], np.cross(v[2] - v[0], v[3] - v[0]))) / 6.0
        scale = vol * np.abs(M).max() / np.linalg.norm(r - c) ** 2  # size of the integrand x volume
        # the closed form cancels face terms of size |M| area/R down to a dipole
        # term of size |M| vol/R^2: far away it loses a few digits to that
        assert abs(a - g) <= 1e-9 * scale


def test_linear_in_M(orc):
    rng = np.random.default_rng(7)
    v = inputs.random_tet(rng)
    M1, M2 = rng.standard_normal((2, 4, 3))
    for r in (v.mean(0), v[2], v.mean(0) + 2.0, 0.5 * (v[1] + v[3])):
        lhs = orc.tet_potential(r, v, 2.5 * M1 - 1.5 * M2)
        rhs = 2.5 * orc.tet_potential(r, v, M1) - 1.5 * orc.tet_potential(r, v, M2)
        assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + abs(rhs) + 1e-12)


def test_vertex_order_and_orientation_independent(orc):
    rng = np.random.default_rng(8)
    v = inputs.random_tet(rng)
    M = rng.standard_normal((4, 3))
    r = v.mean(0) + np.array([0.3, -0.2, 0.1])
    ref = orc.tet_potential(r, v, M)
    for perm in ([1, 0, 2, 3], [3, 2, 1, 0], [2, 3, 0, 1]):
        assert abs(orc.tet_potential(r, v[perm], M[perm]) - ref) <= 1e-13 * abs(ref)


def test_constant_M_is_face_charge_only(orc):
    """Constant M: div M = 0, so only the face charges M.n remain.  A target far
    away sees a point dipole m = |tet| M:  u -> m.(r-c)/|r-c|^3 (x 4pi here)."""
    rng = np.random.default_rng(9)
    v = inputs.random_tet(rng)
    m0 = rng.standard_normal(3)
    M = np.tile(m0, (4, 1))
    vol = abs(np.dot(v[1] - v[0], np.cross(v[2] - v[0], v[3] - v[0]))) / 6.0
    c = v.mean(0)
    for R in (50.0, 200.0):
        r = c + R * np.array([0.48, 0.6, 0.64])
        a = orc.tet_potential(r, v, M)
        d = r - c
        dip = vol * np.dot(m0, d) / np.linalg.norm(d) ** 3
        # next term of the multipole series is O(diam/R) relative
        assert abs(a - dip) <= 4.0 / R * abs(dip)


@pytest.mark.parametrize("seed", range(4))
def test_poisson_equation(orc, seed):
    """u_t = (1/4 pi) int_t M . grad'(1/R) solves Poisson's equation: its Laplacian is
    div M inside the tet (-rho, the volume charge) and 0 outside.  The oracle returns
    4 pi u_t; a 7-point finite-difference Laplacian at interior and exterior points
    checks it, a relation the integration-by-parts derivation does not use."""
    rng = np.random.default_rng(100 + seed)
    v = inputs.random_tet(rng)
    A, b0 = rng.standard_normal((3, 3)), rng.standard_normal(3)
    M = np.array([A @ x + b0 for x in v])  # linear M: div M = trace A
    d = max(np.linalg.norm(v[i] - v[j]) for i in range(4) for j in range(i + 1, 4))
    h = 2e-3 * d
    f = lambda r: orc.tet_potential(r, v.ravel(), M.ravel())

    def lap(r):
        return sum(f(r + h * e) + f(r - h * e) - 2.0 * f(r) for e in np.eye(3)) / h ** 2

    lam = rng.dirichlet(np.ones(4) * 4.0)
    while lam.min() < 0.1:  # a point well inside: the stencil stays off the faces
        lam = rng.dirichlet(np.ones(4) * 4.0)
    inside = lam @ v
    assert abs(lap(inside) - 4.0 * np.pi * np.trace(A)) < 2e-3 * 4.0 * np.pi * max(1.0, abs(np.trace(A)))
    outside = v.mean(0) + 2.0 * d * np.array([0.48, 0.6, -0.64])
    scale = abs(f(outside)) / d ** 2
    assert abs(lap(outside)) < 1e-4 * scale
