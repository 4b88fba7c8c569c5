"""Pins of the oracle's point-dipole model (oracle.dipole_direct), by routes
other than its own formula: a dipole is the limit of a +/- charge pair, and far
from the body the potential is that of the total moment (the quadrupole term of
a cube's uniform moments vanishes by the cube's centre symmetry of the node
lattice up to the lumped-volume pattern, so the next term is small)."""
import numpy as np

from paper_1606_00247_gb300 import inputs


def test_lumped_volumes_add_up_to_the_mesh(orc):
    nodes, tets = inputs.unit_cube(4)
    V = orc.lumped_volumes(nodes, tets)
    assert abs(V.sum() - 1.0) < 1e-13 and np.all(V > 0)


def test_dipole_is_the_limit_of_a_charge_pair(orc):
    """u(r) of the dipoles V_j M_j against sum_j V_j [1/|r - r_j - eps M_j / 2| - 1/|r - r_j + eps M_j / 2|]
    / (4 pi eps): central difference of monopole potentials, error O(eps^2)."""
    nodes, tets = inputs.unit_cube(3)
    rng = np.random.default_rng(3)
    M = inputs.gaussian_unit_m(nodes.shape[0], seed=4)
    pts = rng.uniform(-0.5, 1.5, (20, 3)) + np.array([0.0, 0.0, 2.0])
    u = orc.dipole_direct(nodes, tets, M, points=pts)
    V = orc.lumped_volumes(nodes, tets)
    eps = 1e-4
    ref = np.zeros(len(pts))
    for j in range(nodes.shape[0]):
        a = nodes[j] + 0.5 * eps * M[j]
        b = nodes[j] - 0.5 * eps * M[j]
        ref += V[j] * (1.0 / np.linalg.norm(pts - a, axis=1) - 1.0 / np.linalg.norm(pts - b, axis=1))
    ref /= 4.0 * np.pi * eps
    assert np.abs(u - ref).max() < 1e-6 * np.abs(ref).max()


def test_far_potential_is_that_of_the_total_moment(orc):
    nodes, tets = inputs.unit_cube(4)
    M = inputs.uniform_m(nodes.shape[0], (0.0, 0.0, 1.0))
    c = np.array([0.5, 0.5, 0.5])
    for Rr in (20.0, 80.0):
        pts = c + Rr * np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8], [0.0, 0.8, -0.6]])
        u = orc.dipole_direct(nodes, tets, M, points=pts)
        d = pts - c
        ref = d[:, 2] / (4.0 * np.pi * Rr ** 3)  # total moment (0, 0, 1) at the centre
        err = np.abs(u - ref).max() / np.abs(ref).max()
        assert err < 2.0 / Rr, (Rr, err)


def test_oracle_dipole_fmm(orc):
    """The oracle FMM with point-dipole sources (node radii, node moments, point-dipole near
    field): every pair near (theta -> 0) gives the direct dipole sum; at theta = 0.5 the
    truncation falls geometrically with p."""
    nodes, tets = inputs.sphere(h=0.15)
    M = inputs.gaussian_unit_m(nodes.shape[0], seed=9)
    ref = orc.dipole_direct(nodes, tets, M)
    u0 = orc.Tree(nodes, tets, 16, 1e-9, sources="dipoles").fmm(M, 4)
    assert np.linalg.norm(u0 - ref) / np.linalg.norm(ref) < 1e-12
    errs = [np.linalg.norm(orc.Tree(nodes, tets, 32, 0.5, sources="dipoles").fmm(M, p) - ref) / np.linalg.norm(ref)
            for p in (4, 6, 8)]
    assert errs[0] > 3 * errs[1] > 9 * errs[2] and errs[2] < 1e-3, errs
