"""Gmsh mesh and band-table readers (paper_2607_03226_b300.inputs)."""
import numpy as np
import pytest

import workloads as W
from paper_2607_03226_b300 import inputs

MESHES = {
    "quads": lambda: W.mesh.structured_quads(6, 4, 60e-9, 40e-9),
    "hexes": lambda: W.mesh.structured_hexes(3, 4, 2, 30e-9, 40e-9, 20e-9),
    "tris": lambda: W.mesh.finfet2d_tris(h=8e-9, seed=3),
    "tets": lambda: W.mesh.finfet3d_tets(h=12e-9, seed=4),
}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("version", ["2.2", "4.1"])
def test_gmsh_round_trip(tmp_path, name, version):
    m = MESHES[name]()
    path = tmp_path / f"{name}.msh"
    inputs.write_gmsh(path, m, version=version)
    r = inputs.read_gmsh(path)
    assert r.dim == m.dim and r.cell_type == m.cell_type
    assert np.array_equal(r.nodes, m.nodes)
    assert np.array_equal(r.cells, m.cells)
    # faces are grouped by tag in 4.1; compare as sets of (nodes, tag)
    key = lambda f, t: (tuple(int(x) for x in f), int(t))
    assert sorted(key(f, t) for f, t in zip(r.bfaces, r.btags)) == \
        sorted(key(f, t) for f, t in zip(m.bfaces, m.btags))


def test_gmsh_handwritten_v22(tmp_path):
    """Two triangles on the unit square, written by hand after the 2.2
    layout: the physical tag is the first element tag, node ids are 1-based,
    untagged lines and points are ignored."""
    text = """$MeshFormat
2.2 0 8
$EndMeshFormat
$Nodes
4
1 0 0 0
2 1 0 0
3 1 1 0
4 0 1 0
$EndNodes
$Elements
7
1 15 2 0 1 1
2 1 2 7 1 1 2
3 1 2 8 2 2 3
4 1 2 7 3 3 4
5 1 2 9 4 4 1
6 2 2 0 6 1 2 3
7 2 2 0 6 1 3 4
$EndElements
"""
    p = tmp_path / "sq.msh"
    p.write_text(text)
    r = inputs.read_gmsh(p)
    assert r.dim == 2 and r.cell_type == inputs.TRI
    assert r.cells.tolist() == [[0, 1, 2], [0, 2, 3]]
    assert r.bfaces.tolist() == [[0, 1], [1, 2], [2, 3], [3, 0]]
    assert r.btags.tolist() == [7, 8, 7, 9]
    assert np.array_equal(r.nodes, [[0, 0], [1, 0], [1, 1], [0, 1]])


def test_read_mesh_builds_in_library(tmp_path):
    from paper_2607_03226_b300 import build, nbte
    build.build()
    m = MESHES["tets"]()
    path = tmp_path / "t.msh"
    inputs.write_gmsh(path, m, version="4.1")
    r = inputs.read_gmsh(path)
    a = nbte.nbte_mesh_create(m.dim, m.nodes, m.cell_type, m.cells, m.bfaces, m.btags)
    b = nbte.nbte_mesh_create(r.dim, r.nodes, r.cell_type, r.cells, r.bfaces, r.btags)
    ia, ib = nbte.nbte_mesh_info(a), nbte.nbte_mesh_info(b)
    assert ia == ib
    nbte.nbte_mesh_destroy(a)
    nbte.nbte_mesh_destroy(b)


def test_band_table(tmp_path):
    p = tmp_path / "bands.txt"
    p.write_text("# C v tau\n1.0e5 6000 1e-11\n2.0e5 3000 5e-12\n")
    C, v, tau = inputs.read_band_table(p)
    assert C.tolist() == [1.0e5, 2.0e5] and v.tolist() == [6000, 3000] and tau.tolist() == [1e-11, 5e-12]
    p.write_text("1 2\n")
    with pytest.raises(ValueError):
        inputs.read_band_table(p)


def test_bands_from_modes_conserves_heat_capacity_and_conductivity():
    rng = np.random.default_rng(1)
    n = 5000
    C = rng.uniform(1.0, 2.0, n)
    v = rng.uniform(500.0, 8000.0, n)
    tau = np.exp(rng.uniform(np.log(1e-13), np.log(1e-9), n))
    Cb, vb, tb = inputs.bands_from_modes(C, v, tau, 15)
    assert len(Cb) == 15
    assert abs(Cb.sum() - C.sum()) <= 1e-12 * C.sum()
    kap = (C * v * v * tau).sum()
    assert abs((Cb * vb * vb * tb).sum() - kap) <= 1e-12 * kap
    assert abs((Cb * vb).sum() - (C * v).sum()) <= 1e-12 * (C * v).sum()
    # mean free paths of the bands are ordered like the bins
    assert np.all(np.diff(np.log(vb * tb)) > -1.0)


def test_bands_from_modes_single_modes_unchanged():
    C = np.array([1.0, 2.0, 3.0])
    v = np.array([1000.0, 2000.0, 3000.0])
    tau = np.array([1e-12, 1e-11, 1e-10])   # mean free paths 1e-9, 2e-8, 3e-7 m
    Cb, vb, tb = inputs.bands_from_modes(C, v, tau, 3)
    assert np.allclose(Cb, C) and np.allclose(vb, v) and np.allclose(tb, tau)
