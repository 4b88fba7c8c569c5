"""GPU plan build vs the oracle, bit for bit (Sec. 3.1-3.3): Morton keys,
sort permutations, cells, centres, radii and both interaction lists."""
import numpy as np
import pytest

from paper_1606_00247_gb300 import inputs

pytestmark = pytest.mark.gpu


def _meshes():
    yield "cube8", inputs.unit_cube(8)
    yield "sphere", inputs.sphere(h=0.2)
    yield "film", inputs.kuhn_box((24, 12, 2), (0, 0, 0), (2000.0 / 24 * 24, 1000.0, 10.0))
    yield "ellipsoid", inputs.ellipsoid(h=0.25, a=1.5, b=3.0)


MESHES = dict(_meshes())


@pytest.mark.parametrize("mesh", list(MESHES))
@pytest.mark.parametrize("leaf,theta", [(32, 0.5), (8, 0.3), (16, 0.8)])
def test_tree_and_lists_bit_exact(orc, mesh, leaf, theta):
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = MESHES[mesh]
    ref = orc.Tree(nodes, tets, leaf, theta)
    plan = Plan(nodes, tets, p=2, leaf_size=leaf, theta=theta)
    st = plan.stats()
    assert st["side"] == ref.side and st["scale"] == ref.scale and list(st["lo"]) == list(ref.lo)
    assert (st["n_cells"], st["n_m2l"], st["n_p2p"]) == (ref.n_cells, ref.n_m2l, ref.n_p2p)
    g, o = plan.export_tree(), ref.export()
    for k in ("node_key", "tet_key", "node_perm", "tet_perm", "cell_level", "cell_prefix", "cell_ranges",
              "cell_parent", "cell_child", "m2l_off", "m2l_src", "p2p_off", "p2p_src"):
        assert np.array_equal(g[k], o[k]), k
    # floating-point values that decide the lists: bit-identical
    assert np.array_equal(g["cell_centre"].view(np.uint64), o["cell_centre"].view(np.uint64))
    assert np.array_equal(g["cell_radius"].view(np.uint64), o["cell_radius"].view(np.uint64))


def test_single_leaf_mesh(orc):
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.unit_cube(1)  # 6 tets: the root is a leaf
    plan = Plan(nodes, tets, p=3, leaf_size=32, theta=0.5)
    g = plan.export_tree()
    assert plan.stats()["n_cells"] == 1 and list(g["p2p_src"]) == [0] and g["m2l_src"].size == 0


def test_invalid_inputs_are_rejected():
    from paper_1606_00247_gb300 import _lib
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.unit_cube(2)
    bad = tets.copy()
    bad[3, 2] = nodes.shape[0]
    with pytest.raises(_lib.DemagError) as e:
        Plan(nodes, bad)
    assert e.value.status == _lib.DEMAG_ERR_INVALID_ARG
    flat = tets.copy()
    n2 = nodes.copy()
    flat[0] = [0, 1, 2, 2]  # repeated vertex: zero volume
    with pytest.raises(_lib.DemagError) as e:
        Plan(n2, flat)
    assert e.value.status == _lib.DEMAG_ERR_DEGENERATE_TET
    for kw in (dict(p=0), dict(p=13), dict(leaf_size=0), dict(theta=0.0), dict(theta=float("nan"))):
        with pytest.raises(_lib.DemagError) as e:
            Plan(nodes, tets, **kw)
        assert e.value.status == _lib.DEMAG_ERR_INVALID_ARG
