"""Magnetostatic energy and LLG stepping (demag_energy, demag_llg_rk4).

* energy = -(1/2) sum_i V_i M_i . H_i with the lumped nodal volumes, checked
  against the same sum formed on the host from the returned H, and the
  uniformly magnetised unit cube: demagnetising factor 1/3 gives e -> 1/6;
* LLG: unit length kept; with damping the energy never increases; without
  damping the integrator converges at fourth order and the energy stays
  constant up to the asymmetry of the discrete operator; a batch of states
  steps like the states one by one."""
import numpy as np
import pytest
import torch

from paper_1606_00247_gb300 import inputs

pytestmark = pytest.mark.gpu


def lumped_volumes(nodes, tets):
    v = nodes[tets]
    vol = np.abs(np.einsum("ij,ij->i", v[:, 1] - v[:, 0], np.cross(v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]))) / 6.0
    V = np.zeros(nodes.shape[0])
    np.add.at(V, tets.ravel(), np.repeat(vol / 4.0, 4))
    return V


def test_energy_host_sum_and_cube_factor():
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.unit_cube(8)
    M = np.stack([inputs.uniform_m(nodes.shape[0], (0, 0, 1)), inputs.gaussian_unit_m(nodes.shape[0], seed=5)])
    Md = torch.as_tensor(M, device="cuda")
    pl = Plan(nodes, tets, p=4, leaf_size=32, theta=0.5, max_batch=2)
    u, H = pl.eval(Md)
    e = pl.energy(Md, H).cpu().numpy()
    V = lumped_volumes(nodes, tets)
    ref = -0.5 * np.einsum("i,bij,bij->b", V, M, H.cpu().numpy())
    assert np.abs(e - ref).max() <= 1e-12 * np.abs(ref).max()
    assert abs(V.sum() - 1.0) < 1e-12
    assert abs(e[0] - 1.0 / 6.0) < 0.05 / 6.0, e[0]  # demagnetising factor 1/3, P1 on 8^3 sub-cubes


def _setup(B, precision="fp64"):
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.sphere(h=0.15)
    m = torch.as_tensor(inputs.smoothed_unit_m(tets, nodes.shape[0], batch=B, seed=41), device="cuda")
    pl = Plan(nodes, tets, p=6, leaf_size=32, theta=0.5, near_mode=1, max_batch=B, precision=precision)
    return pl, m


def _energy(pl, m):
    u, H = pl.eval(m)
    return pl.energy(m, H)


def test_llg_damped_energy_decreases_and_unit_length_kept():
    pl, m = _setup(3)
    e = [_energy(pl, m)]
    for _ in range(10):
        pl.llg_rk4(m, Ms=1.0, alpha=0.5, dt=0.05, steps=1)
        e.append(_energy(pl, m))
    e = torch.stack(e).cpu().numpy()
    assert np.all(np.diff(e, axis=0) <= 1e-10 * np.abs(e).max())
    assert e[-1].max() < e[0].min() or np.all(e[-1] < e[0])
    assert torch.allclose(torch.linalg.norm(m, dim=-1), torch.ones(m.shape[:2], dtype=m.dtype, device=m.device),
                          atol=1e-12, rtol=0)


def test_llg_rk4_is_fourth_order_and_undamped_energy_nearly_constant():
    """Precession only: the error of the final state against a fine-step run
    falls ~16x when dt halves (classical RK4).  The energy moves only by the
    asymmetry of the discrete demagnetising operator (u collocated at the
    nodes, H by the lumped gradient), well below 1e-3 over t = 0.2."""
    pl, m0 = _setup(1)
    runs = {}
    for dt in (0.04, 0.02, 0.005):
        m = m0.clone()
        pl.llg_rk4(m, Ms=1.0, alpha=0.0, dt=dt, steps=int(round(0.2 / dt)))
        runs[dt] = m
    e1 = float(torch.max(torch.abs(runs[0.04] - runs[0.005])))
    e2 = float(torch.max(torch.abs(runs[0.02] - runs[0.005])))
    assert e1 / e2 > 10.0, (e1, e2)
    E0, E1 = _energy(pl, m0), _energy(pl, runs[0.005])
    assert float(torch.abs(E1 - E0) / torch.abs(E0)) < 1e-3


def test_llg_batch_steps_like_single_states():
    pl, m = _setup(2)
    ms = [m[k:k + 1].clone() for k in range(2)]
    pl.llg_rk4(m, Ms=1.0, alpha=0.2, h_ext=(0.0, 0.0, 0.1), dt=0.02, steps=5)
    for k in range(2):
        pl.llg_rk4(ms[k], Ms=1.0, alpha=0.2, h_ext=(0.0, 0.0, 0.1), dt=0.02, steps=5)
        assert float(torch.max(torch.abs(ms[k][0] - m[k]))) < 1e-12


def test_energy_and_llg_rk4_against_the_oracle(orc):
    """demag_energy and demag_llg_rk4 (FP64 path) against the oracle's energy and
    RK4 stepping, whose field at every stage is the oracle's own FMM (same tree
    rules, p, leaf and theta) followed by its mass-lumped H: the library's FP64
    FMM agrees with the oracle FMM to rounding, so three steps agree to 1e-9."""
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.sphere(h=0.2)
    B, p, leaf, theta = 2, 6, 32, 0.5
    m0 = inputs.smoothed_unit_m(tets, nodes.shape[0], batch=B, seed=43)
    Ms, alpha, hext, dt, steps = 1.0, 0.2, (0.1, 0.0, 0.3), 0.05, 3
    pl = Plan(nodes, tets, p=p, leaf_size=leaf, theta=theta, near_mode=1, max_batch=B)
    md = torch.as_tensor(m0, device="cuda")
    u, H = pl.eval(md)
    e = pl.energy(md, H).cpu().numpy()
    tree = orc.Tree(nodes, tets, leaf, theta)
    Hor = orc.lumped_H(nodes, tets, tree.fmm(m0, p))
    assert np.abs(e - orc.energy(nodes, tets, m0, H.cpu().numpy())).max() <= 1e-13 * np.abs(e).max()
    assert np.abs(e - orc.energy(nodes, tets, m0, Hor)).max() <= 1e-10 * np.abs(e).max()
    pl.llg_rk4(md, Ms=Ms, alpha=alpha, h_ext=hext, dt=dt, steps=steps)
    torch.cuda.synchronize()
    field = lambda M: orc.lumped_H(nodes, tets, tree.fmm(M, p))
    mor = orc.llg_rk4(m0, field, Ms, alpha, hext, dt, steps)
    assert np.abs(md.cpu().numpy() - mor).max() < 1e-9
