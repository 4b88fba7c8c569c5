"""Pins of the oracle's energy and LLG stepping (plain numpy, used to check the
library's demag_energy and demag_llg_rk4):
* the right-hand side on hand-evaluated cross products, orthogonality to m and
  the sign of its projection on h (energy decreases when damped);
* the RK4 step on a linear system against the matrix exponential, with its
  fifth-order local error;
* a single moment in a uniform field (no demagnetising field) against the
  closed-form damped precession;
* the energy on a hand-built two-tet mesh."""
import numpy as np
import pytest

import oracle


def test_llg_rhs_by_hand():
    m = np.array([1.0, 0.0, 0.0])
    h = np.array([0.0, 0.0, 2.0])
    a = 0.3
    # m x h = -2 y; m x (m x h) = x x (-2 y) = -2 z
    want = -(np.array([0.0, -2.0, 0.0]) + a * np.array([0.0, 0.0, -2.0])) / (1 + a * a)
    assert np.allclose(oracle.llg_rhs(m, h, a), want, atol=1e-15)
    rng = np.random.default_rng(1)
    m = rng.normal(size=(50, 3))
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    h = rng.normal(size=(50, 3))
    r = oracle.llg_rhs(m, h, 0.2)
    assert np.max(np.abs(np.einsum("ik,ik->i", r, m))) < 1e-14
    assert np.all(np.einsum("ik,ik->i", r, h) >= -1e-14)  # d(-m.h)/dt <= 0 with damping


def test_rk4_linear_system_against_expm():
    from scipy.linalg import expm

    A = np.array([[0.0, 1.0, 0.2], [-1.0, -0.1, 0.0], [0.3, 0.0, -0.5]])
    y0 = np.array([1.0, 0.5, -0.2])
    errs = []
    for dt in (0.2, 0.1):
        y1 = oracle.rk4_step(lambda y: A @ y, y0, dt)
        errs.append(np.linalg.norm(y1 - expm(A * dt) @ y0))
    assert errs[0] < 1e-4 and 20 < errs[0] / errs[1] < 40  # local error O(dt^5): ratio ~32


def test_single_moment_damped_precession():
    """field = 0, uniform h = h0 z: the polar angle follows
    tan(theta/2) = tan(theta0/2) exp(-alpha h0 t / (1 + alpha^2)) and the
    azimuth turns at h0 / (1 + alpha^2) (reduced units)."""
    h0, a, th0, T = 1.5, 0.1, 1.0, 2.0
    m0 = np.array([[[np.sin(th0), 0.0, np.cos(th0)]]])
    nsteps = 400
    m = oracle.llg_rk4(m0, lambda M: np.zeros_like(M), 1.0, a, (0.0, 0.0, h0), T / nsteps, nsteps)[0, 0]
    th = 2 * np.arctan(np.tan(th0 / 2) * np.exp(-a * h0 * T / (1 + a * a)))
    ph = h0 * T / (1 + a * a)
    want = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    assert np.linalg.norm(m - want) < 1e-9


def test_energy_two_tets_by_hand():
    nodes = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], dtype=np.float64)
    tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], dtype=np.int32)
    V = oracle.lumped_volumes(nodes, tets)
    assert np.allclose(V, [1 / 24, 1 / 24 + 1 / 12, 1 / 24 + 1 / 12, 1 / 24 + 1 / 12, 1 / 12])  # |Omega| = 1/6, 1/3
    rng = np.random.default_rng(3)
    M = rng.normal(size=(2, 5, 3))
    H = rng.normal(size=(2, 5, 3))
    want = [-0.5 * sum(V[i] * M[b, i] @ H[b, i] for i in range(5)) for b in range(2)]
    assert np.allclose(oracle.energy(nodes, tets, M, H), want, rtol=1e-14)
