"""The seeded input recipes (paper_1606_00247_gb300/inputs.py) hold the
properties the workloads state: the graded cube fills the unit cube with
disjoint refined inclusions, the mesh batch spans the stated size range, and
the smoothed states are unit vectors that vary less between neighbours than
the iid states they start from."""
import numpy as np

from paper_1606_00247_gb300 import inputs


def _volumes(nodes, tets):
    v = nodes[tets]
    return np.abs(np.einsum("ij,ij->i", v[:, 1] - v[:, 0], np.cross(v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]))) / 6.0


def test_graded_cube_small():
    h0 = 1.0 / 16.0
    nodes, tets, cen, rad = inputs.graded_cube(h0=h0, n_incl=4, seed=inputs.INCLUSION_SEED)
    assert len(cen) == 4 and np.all((rad >= 0.02) & (rad <= 0.05))
    assert nodes.min() >= -1e-12 and nodes.max() <= 1.0 + 1e-12
    assert abs(_volumes(nodes, tets).sum() - 1.0) < 1e-6  # the hull is the cube (faces unjittered)
    outer = rad + 0.75 * h0 + 1.5 * h0
    for i in range(4):
        for j in range(i):
            assert np.linalg.norm(cen[i] - cen[j]) > outer[i] + outer[j]
    # refinement: node density inside a ball ~ (8 / h0)^3, far above the outside (1 / h0)^3
    k = int(np.argmax(rad))
    inside = np.sum(np.linalg.norm(nodes - cen[k], axis=1) < rad[k])
    assert inside > 0.25 * (4.0 / 3.0) * np.pi * rad[k] ** 3 * (8.0 / h0) ** 3


def test_graded_cube_rejects_inclusions_that_do_not_fit():
    import pytest

    with pytest.raises(ValueError):
        inputs.graded_cube(h0=0.25, n_incl=50)


def test_batch_meshes_sizes_and_kinds():
    ms = inputs.batch_meshes(n=6, min_tets=2e3, max_tets=2e4)
    sizes = [t.shape[0] for _, t in ms]
    assert len(ms) == 6 and min(sizes) > 1e3 and max(sizes) < 4e4
    ext = [n.max(axis=0) - n.min(axis=0) for n, _ in ms]
    assert np.allclose(ext[0], ext[0][0])  # Kuhn cube
    assert max(ext[2]) / min(ext[2]) > 1.0 + 1e-6  # stretched ball


def test_smoothed_states():
    nodes, tets = inputs.sphere(h=0.2)
    m = inputs.smoothed_unit_m(tets, nodes.shape[0], batch=3, seed=5)
    assert m.shape == (3, nodes.shape[0], 3) and m.flags["C_CONTIGUOUS"]
    assert np.allclose(np.linalg.norm(m, axis=-1), 1.0)
    assert np.array_equal(m, inputs.smoothed_unit_m(tets, nodes.shape[0], batch=3, seed=5))
    e = np.unique(np.sort(np.concatenate([tets[:, [a, b]] for a in range(4) for b in range(a + 1, 4)]), axis=1),
                  axis=0)
    raw = inputs.smoothed_unit_m(tets, nodes.shape[0], batch=3, passes=0, seed=5)
    jump = lambda x: np.mean(np.linalg.norm(x[:, e[:, 0]] - x[:, e[:, 1]], axis=-1))
    assert jump(m) < 0.6 * jump(raw)


def test_benchmark_meshes_have_the_stated_sizes_and_fill_their_domains():
    """The seeded meshes the workloads and the bench are quoted on: the unit cube
    (8^3 cubes, 3072 tets), the 224k-tet ball and the 2M-tet film have the
    stated node and tet counts, positive volumes, and volumes that add up to
    the domain (the ball's up to the facets of its inscribed polyhedron)."""
    nodes, tets = inputs.kuhn_box((8, 8, 8))
    assert (nodes.shape[0], tets.shape[0]) == (729, 3072)
    assert abs(_volumes(nodes, tets).sum() - 1.0) < 1e-12

    nodes, tets = inputs.sphere(h=inputs.SPHERE_200K_H)
    assert (nodes.shape[0], tets.shape[0]) == (35840, 223668)
    vol = _volumes(nodes, tets)
    assert vol.min() > 0 and abs(vol.sum() - 4.0 / 3.0 * np.pi) < 0.01 * 4.0 / 3.0 * np.pi

    nodes, tets = inputs.thin_film()
    assert (nodes.shape[0], tets.shape[0]) == (500259, 1990656)
    assert abs(_volumes(nodes, tets).sum() / (2000.0 * 1000.0 * 10.0) - 1.0) < 1e-12
