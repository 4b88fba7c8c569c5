"""Pins of the oracle's pointwise field H = -grad u (the remark of Sec. 4.1-4.2
that computing H directly gives lower errors), from boundary-face and volume
charges in closed form:
* uniformly magnetised unit cube (Kuhn tets, M = z): the field of the two
  charged faces z = 0, 1 written independently here (derivatives of the
  rectangle antiderivative), at every interior node, to 1e-12;
* central differences of the per-tet potential (the oracle's other closed
  form) at interior nodes of a ball, for Gaussian and for affine M (which makes
  the in-plane gradient terms of the face charges and the volume charges
  non-zero);
* the uniformly magnetised ball: interior H -> -M/3 under refinement."""
import numpy as np
import pytest

from paper_1606_00247_gb300 import inputs


def _rect_field(p, x1, x2, y1, y2, z0):
    """int_{x1}^{x2} int_{y1}^{y2} (p - r') / |p - r'|^3 dx' dy', r' = (x', y', z0): the
    x, y components from the y- (x-) antiderivative ln(Y + R) of the x- (y-)
    integrated kernel, the z component from the solid-angle antiderivative
    atan(XY / (ZR))."""
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    Z = z0 - z
    out = np.zeros_like(p)
    for X, sx in ((x2 - x, 1.0), (x1 - x, -1.0)):
        for Y, sy in ((y2 - y, 1.0), (y1 - y, -1.0)):
            R = np.sqrt(X * X + Y * Y + Z * Z)
            s = sx * sy
            out[:, 0] += s * np.log(Y + R)  # int (x - x')/R^3 dx' = [1/R], then int dy'/R = ln(Y + R)
            out[:, 1] += s * np.log(X + R)
            out[:, 2] += -s * np.arctan(X * Y / (Z * R))
    return out


def test_cube_field_closed_form(orc):
    nodes, tets = inputs.unit_cube(6)
    M = inputs.uniform_m(nodes.shape[0], (0.0, 0.0, 1.0))
    ii = orc.interior_nodes(tets, nodes.shape[0])
    assert len(ii) == 5 ** 3
    p = nodes[ii]
    want = (_rect_field(p, 0, 1, 0, 1, 1.0) - _rect_field(p, 0, 1, 0, 1, 0.0)) / (4 * np.pi)
    got = orc.field_charges(nodes, tets, M, p)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    c = np.argmin(np.linalg.norm(p - 0.5, axis=1))  # the centre: -M/3 by symmetry
    assert np.allclose(got[c], [0, 0, -1 / 3], atol=1e-12)


def _u_points(orc, nodes, tets, M, pts):
    v = nodes[tets].reshape(-1, 12)
    m = M[tets].reshape(-1, 12)
    return np.array([sum(orc.tet_potential(q, v[t], m[t]) for t in range(len(tets))) for q in pts]) / (4 * np.pi)


@pytest.mark.parametrize("kind", ["gaussian", "affine"])
def test_field_matches_central_differences(orc, kind):
    """At generic interior points (inside tets, away from nodes and faces) the
    field equals the central differences of the summed per-tet potentials (to
    the O(d^2) of the differences); at an interior node, where the field is
    continuous but its gradient is log-singular (the volume charges jump between
    the tets around the node), the field is the limit of the field at points
    approaching the node."""
    nodes, tets = inputs.sphere(h=0.35)
    if kind == "gaussian":
        M = inputs.gaussian_unit_m(nodes.shape[0], seed=81)
    else:
        M = inputs.affine_m(nodes, np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.3], [-0.6, 0.2, 0.1]]),
                            np.array([0.2, -0.1, 1.0]))
    ii = orc.interior_nodes(tets, nodes.shape[0])
    inner = np.where(np.isin(tets, ii).all(axis=1))[0]
    pick = inner[np.linspace(0, len(inner) - 1, 4).astype(int)]
    lam = np.array([0.31, 0.27, 0.23, 0.19])
    pts = np.einsum("k,tka->ta", lam, nodes[tets[pick]])
    H = orc.field_charges(nodes, tets, M, pts)
    d = 1e-5
    for k, r in enumerate(pts):
        q = [r + s * d * e for e in np.eye(3) for s in (1.0, -1.0)]
        uu = _u_points(orc, nodes, tets, M, q).reshape(3, 2)
        fd = -(uu[:, 0] - uu[:, 1]) / (2 * d)
        assert np.linalg.norm(H[k] - fd) < 1e-7 * np.linalg.norm(fd), (k, H[k], fd)
    node = nodes[ii[len(ii) // 2]]
    h0 = orc.field_charges(nodes, tets, M, node[None])[0]
    dirn = np.array([0.48, -0.36, 0.8])
    gaps = [np.linalg.norm(orc.field_charges(nodes, tets, M, (node + eps * dirn)[None])[0] - h0)
            for eps in (1e-4, 1e-6, 1e-8)]
    assert gaps[2] < gaps[1] < gaps[0] and gaps[2] < 1e-6 * np.linalg.norm(h0), gaps


def test_ball_interior_field_tends_to_minus_third():
    import oracle as orc

    errs = []
    for h in (0.3, 0.2):
        nodes, tets = inputs.sphere(h=h)
        M = inputs.uniform_m(nodes.shape[0], (0.0, 0.0, 1.0))
        ii = orc.interior_nodes(tets, nodes.shape[0])
        ii = ii[np.linalg.norm(nodes[ii], axis=1) < 0.6]
        H = orc.field_charges(nodes, tets, M, nodes[ii])
        errs.append(np.abs(H - [0, 0, -1 / 3]).max() * 3)
    assert errs[1] < errs[0] < 0.1, errs
