"""Pins of the oracle's expansions, tree/lists and FMM (Sec. 2.2-2.3, Sec. 3).

  * D_n(x) = d^n(1/|x|): closed forms for |n| <= 2, the harmonic identity
    sum_i D_{n+2e_i} = 0 for every n, and central finite differences.
  * Exact moments (Eq. expCoeffs): quadrature vs the closed-form barycentric
    monomial integral; Q_0 = 0 (zero total charge); Q_{e_i} = int M_i dV.
  * M2M / L2L are exact for polynomials: M2M(child) = P2M about the parent;
    L2P(L2L(L)) = L2P(L).
  * M2L + L2P approaches the multipole sum with error decaying in p.
  * Lists: every (target node, source tet) pair is covered exactly once, by one
    P2P leaf pair or by one M2L pair of ancestors-or-self; every M2L pair passes
    the MAC; lists are sorted.
  * FMM: error vs the direct sum decays geometrically with p (Sec. 2.2,
    (alpha/2)^(p+1)); theta -> 0 turns every pair into P2P and the FMM into the
    direct sum; a batch equals single evaluations.
"""
import math

import numpy as np
import pytest

from paper_1606_00247_gb300 import inputs


def _idx(mi):
    return {tuple(int(x) for x in n): i for i, n in enumerate(mi)}


def test_multi_index_order(orc):
    mi = orc.multi_indices(4)
    assert mi.shape == (35, 3) and orc.ncoef(8) == 165 and orc.ncoef(10) == 286
    tot = mi.sum(1)
    assert np.all(np.diff(tot) >= 0) and len({tuple(n) for n in mi}) == 35


def test_laplace_derivs_closed_forms(orc):
    x = np.array([0.3, -0.7, 1.1])
    r = np.linalg.norm(x)
    D = orc.laplace_derivs(x, 2)
    ix = _idx(orc.multi_indices(2))
    assert abs(D[ix[(0, 0, 0)]] - 1 / r) < 1e-15
    for a in range(3):
        e = [0, 0, 0]
        e[a] = 1
        assert abs(D[ix[tuple(e)]] + x[a] / r ** 3) < 1e-15
        for b in range(3):
            e2 = [0, 0, 0]
            e2[a] += 1
            e2[b] += 1
            want = 3 * x[a] * x[b] / r ** 5 - (a == b) / r ** 3
            assert abs(D[ix[tuple(e2)]] - want) < 1e-14


def test_laplace_derivs_harmonic_and_fd(orc):
    p = 9
    x = np.array([0.8, 0.35, -0.5])
    D = orc.laplace_derivs(x, p)
    mi = orc.multi_indices(p)
    ix = _idx(mi)
    for n in mi:
        if n.sum() + 2 > p:
            continue
        s = 0.0
        for i in range(3):
            m = n.copy()
            m[i] += 2
            s += D[ix[tuple(m)]]
        assert abs(s) <= 1e-12 * max(abs(D[ix[tuple(n)]]), 1.0) * 10 ** n.sum()
    # finite difference of order-(p-1) derivatives in each axis
    h = 1e-5
    for n in mi:
        if n.sum() >= p:
            continue
        for i in range(3):
            e = np.zeros(3)
            e[i] = h
            Dp, Dm = orc.laplace_derivs(x + e, p - 1), orc.laplace_derivs(x - e, p - 1)
            sub = _idx(orc.multi_indices(p - 1))
            fd = (Dp[sub[tuple(n)]] - Dm[sub[tuple(n)]]) / (2 * h)
            m = n.copy()
            m[i] += 1
            ref = D[ix[tuple(m)]]
            assert abs(fd - ref) <= 1e-6 * max(1.0, abs(ref))


def test_moments_quadrature_vs_barycentric(orc):
    rng = np.random.default_rng(3)
    v = inputs.random_tet(rng)
    M = rng.standard_normal((4, 3))
    c = v.mean(0) + np.array([0.1, -0.2, 0.05])
    p = 5
    Q = orc.tet_moments(v, M, c, p)
    mi = orc.multi_indices(p)
    for i, n in enumerate(mi):
        want = 0.0
        for k in range(4):
            for a in range(3):
                if n[a] == 0:
                    continue
                m = n.copy()
                m[a] -= 1
                want += M[k, a] * n[a] * orc.tet_lambda_monomial_exact(v, c, k, m)
        assert abs(Q[i] - want) <= 1e-13 * max(1.0, np.abs(Q).max())


def test_moments_charge_and_dipole(orc):
    rng = np.random.default_rng(4)
    v = inputs.random_tet(rng)
    M = rng.standard_normal((4, 3))
    Q = orc.tet_moments(v, M, v.mean(0) + 0.3, 4)
    vol = abs(np.dot(v[1] - v[0], np.cross(v[2] - v[0], v[3] - v[0]))) / 6.0
    ix = _idx(orc.multi_indices(4))
    assert Q[0] == 0.0
    for a in range(3):
        e = [0, 0, 0]
        e[a] = 1
        assert abs(Q[ix[tuple(e)]] - vol * M[:, a].mean()) < 1e-14


def test_m2m_l2l_exact(orc):
    rng = np.random.default_rng(5)
    v = inputs.random_tet(rng)
    M = rng.standard_normal((4, 3))
    p = 6
    cc = v.mean(0) + np.array([0.05, 0.02, -0.03])
    cp = cc + np.array([0.4, -0.25, 0.3])
    Qc = orc.tet_moments(v, M, cc, p)
    Qp = orc.tet_moments(v, M, cp, p)
    Qs = orc.m2m(p, cc - cp, Qc)
    assert np.max(np.abs(Qs - Qp)) <= 1e-13 * np.max(np.abs(Qp))
    L = rng.standard_normal(orc.ncoef(p))
    d = np.array([0.2, -0.1, 0.15])
    Lc = orc.l2l(p, d, L)
    for _ in range(5):
        z = rng.uniform(-0.3, 0.3, 3)
        assert abs(orc.l2p(p, z, Lc) - orc.l2p(p, z + d, L)) <= 1e-13 * max(1.0, abs(orc.l2p(p, z + d, L)))


def test_m2l_converges_to_multipole(orc):
    rng = np.random.default_rng(6)
    v = inputs.random_tet(rng, scale=0.3)
    M = rng.standard_normal((4, 3))
    cs = v.mean(0)
    ct = cs + np.array([2.0, 1.5, -1.0])
    r = ct + np.array([0.15, -0.1, 0.2])
    errs = []
    exact = orc.tet_potential(r, v, M) / (4 * np.pi)
    for p in (2, 4, 6, 8, 10):
        Q = orc.tet_moments(v, M, cs, p)
        L = orc.m2l(p, ct - cs, Q)
        errs.append(abs(orc.l2p(p, r - ct, L) - exact))
        # the multipole series itself converges to the exact value
        assert abs(orc.multipole_eval(p, cs, Q, r) - exact) < 10 * 0.4 ** (p + 1) * abs(exact) + 1e-16
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))
    assert errs[-1] < 1e-6 * abs(exact)


def _ancestors(parent, c):
    out = []
    while c >= 0:
        out.append(c)
        c = parent[c]
    return out


@pytest.mark.parametrize("mesh,leaf,theta", [("cube4", 8, 0.5), ("sphere", 16, 0.6), ("cube4", 4, 0.3)])
def test_lists_cover_every_pair_once(orc, mesh, leaf, theta):
    if mesh == "cube4":
        nodes, tets = inputs.unit_cube(4)
    else:
        nodes, tets = inputs.sphere(h=0.3)
    tr = orc.Tree(nodes, tets, leaf, theta)
    ex = tr.export()
    nc = tr.n_cells
    parent = ex["cell_parent"]
    rng = ex["cell_ranges"]
    child = ex["cell_child"]
    leaf_of_node = np.full(nodes.shape[0], -1)
    leaf_of_tet = np.full(tets.shape[0], -1)
    for c in range(nc):
        if child[c, 1] == 0:
            leaf_of_tet[ex["tet_perm"][rng[c, 0]:rng[c, 1]]] = c
            leaf_of_node[ex["node_perm"][rng[c, 2]:rng[c, 3]]] = c
    assert np.all(leaf_of_node >= 0) and np.all(leaf_of_tet >= 0)
    # lists sorted and unique
    for off, src in ((ex["m2l_off"], ex["m2l_src"]), (ex["p2p_off"], ex["p2p_src"])):
        for c in range(nc):
            s = src[off[c]:off[c + 1]]
            assert np.all(np.diff(s) > 0)
    m2l = {(c, int(s)) for c in range(nc) for s in ex["m2l_src"][ex["m2l_off"][c]:ex["m2l_off"][c + 1]]}
    p2p = {(c, int(s)) for c in range(nc) for s in ex["p2p_src"][ex["p2p_off"][c]:ex["p2p_off"][c + 1]]}
    cen, rad = ex["cell_centre"], ex["cell_radius"]
    for (T, S) in m2l:
        assert rad[T, 1] + rad[S, 0] < theta * np.linalg.norm(cen[T] - cen[S])
    for (T, S) in p2p:
        assert child[T, 1] == 0 and child[S, 1] == 0
    anc_n = {c: _ancestors(parent, c) for c in set(leaf_of_node.tolist())}
    anc_t = {c: _ancestors(parent, c) for c in set(leaf_of_tet.tolist())}
    for ln in anc_n:
        for lt in anc_t:
            cnt = int((ln, lt) in p2p)
            for a in anc_n[ln]:
                for b in anc_t[lt]:
                    cnt += (a, b) in m2l
            assert cnt == 1, (ln, lt, cnt)


def test_morton_keys_and_centres(orc):
    nodes, tets = inputs.unit_cube(4)
    tr = orc.Tree(nodes, tets, 8, 0.5)
    ex = tr.export()
    assert np.all(np.diff(ex["node_key"][ex["node_perm"]].astype(np.float64)) >= 0)
    # the cube corner (0,0,0) has key 0, the opposite corner the largest key
    i0 = np.where(np.all(nodes == 0, axis=1))[0][0]
    assert ex["node_key"][i0] == 0
    # children tile their parent: centre offset is +-side/2^(l+2) per axis
    for c in range(1, tr.n_cells):
        p = ex["cell_parent"][c]
        l = ex["cell_level"][c]
        off = np.abs(ex["cell_centre"][c] - ex["cell_centre"][p])
        assert np.allclose(off, tr.side / 2 ** (l + 1), rtol=1e-14)


def test_fmm_error_decays_with_p(orc):
    nodes, tets = inputs.sphere(h=0.16)
    M = inputs.gaussian_unit_m(nodes.shape[0])
    ud = orc.direct(nodes, tets, M)
    tr = orc.Tree(nodes, tets, 16, 0.5)
    errs = []
    for p in (2, 4, 6, 8):
        uf = tr.fmm(M, p)
        errs.append(np.linalg.norm(uf - ud) / np.linalg.norm(ud))
    assert all(errs[i + 1] < 0.6 * errs[i] for i in range(3)), errs
    assert errs[-1] < 1e-4


def test_fmm_theta_zero_is_direct(orc):
    nodes, tets = inputs.unit_cube(4)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=2)
    tr = orc.Tree(nodes, tets, 8, 1e-9)
    assert tr.n_m2l == 0
    uf = tr.fmm(M, 3)
    ud = orc.direct(nodes, tets, M)
    assert np.max(np.abs(uf - ud)) <= 1e-14 * np.max(np.abs(ud))


def test_fmm_target_leaf_sample_matches_full(orc):
    nodes, tets = inputs.unit_cube(4)
    M = inputs.gaussian_unit_m(nodes.shape[0])
    tr = orc.Tree(nodes, tets, 8, 0.5)
    full = tr.fmm(M, 4)
    ex = tr.export()
    leaves = np.where(ex["cell_child"][:, 1] == 0)[0][::3]
    part = tr.fmm(M, 4, target_leaves=leaves)
    sel = np.concatenate([ex["node_perm"][ex["cell_ranges"][c, 2]:ex["cell_ranges"][c, 3]] for c in leaves])
    assert np.array_equal(part[sel], full[sel])


def test_vertex_patch_clustering(orc):
    """The paper's clustering (sources = vertex patches lambda_i M_i, binned by node,
    radius to the farthest vertex of the patch): the same u as the direct sum when
    every pair is near, and a truncation error that falls with p like the tet
    clustering's."""
    nodes, tets = inputs.sphere(h=0.2)
    M = inputs.gaussian_unit_m(nodes.shape[0], seed=9)
    ref = orc.direct(nodes, tets, M)
    u0 = orc.Tree(nodes, tets, 16, 1e-9, sources="patches").fmm(M, 4)
    assert np.linalg.norm(u0 - ref) / np.linalg.norm(ref) < 1e-12
    err = {}
    for src in ("tets", "patches"):
        err[src] = [np.linalg.norm(orc.Tree(nodes, tets, 16, 0.5, sources=src).fmm(M, p) - ref) / np.linalg.norm(ref)
                    for p in (4, 8)]
    assert err["patches"][0] > 10 * err["patches"][1]
    assert err["patches"][1] < 3 * err["tets"][1], err
