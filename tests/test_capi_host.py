"""Host-side checks of the C ABI: the library loads, exports every symbol the
header declares, and rejects invalid input with the documented status codes
before any device work.  No GPU is needed (a solver created on a host without
a device still validates its set-up calls)."""
import os
import re

import numpy as np
import pytest

import workloads as W
from workloads.problems import Boundary
from paper_2607_03226_b300 import nbte

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_03226_b300 import build
    build.build()
    return nbte.load()


def test_exports_every_declared_symbol(lib):
    text = open(os.path.join(ROOT, "include", "nbte.h")).read()
    declared = set(re.findall(r"^(?:int|const char\*)\s+(nbte_\w+)\(", text, flags=re.M))
    assert declared, "no declarations parsed"
    assert declared == set(nbte.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
    assert "sm_103a" in nbte.nbte_version()


def _mesh(p):
    m = p.mesh
    return nbte.nbte_mesh_create(m.dim, m.nodes, m.cell_type, m.cells, m.bfaces, m.btags)


@pytest.mark.parametrize("maker,volume", [
    (lambda: W.problems.square_inplane(n=8), 1e-14),
    (lambda: W.problems.cube3d(n=4), (500e-9) ** 3),
    (lambda: W.problems.finfet2d(h=10e-9), 200e-9 * 100e-9 + 10e-9 * 40e-9),
    (lambda: W.problems.finfet3d(h=20e-9), 300e-9 * 100e-9 * 50e-9 + 7e-9 * 100e-9 * 50e-9),
])
def test_mesh_volume_and_count(lib, maker, volume):
    p = maker()
    h = _mesh(p)
    n, v = nbte.nbte_mesh_info(h)
    assert n == p.n_cells
    assert v == pytest.approx(volume, rel=1e-12)
    nbte.nbte_mesh_destroy(h)


def test_mesh_errors(lib):
    p = W.problems.square_inplane(n=4)
    m = p.mesh
    with pytest.raises(nbte.NbteError) as e:   # a boundary face missing
        nbte.nbte_mesh_create(2, m.nodes, m.cell_type, m.cells, m.bfaces[1:], m.btags[1:])
    assert e.value.code == nbte.NBTE_ERR_MESH
    with pytest.raises(nbte.NbteError) as e:   # an interior face listed as boundary
        bf = np.vstack([m.bfaces, [[6, 11]]])
        nbte.nbte_mesh_create(2, m.nodes, m.cell_type, m.cells, bf, np.append(m.btags, 9))
    assert e.value.code == nbte.NBTE_ERR_MESH
    with pytest.raises(nbte.NbteError) as e:   # node index out of range
        c = m.cells.copy()
        c[0, 0] = 10 ** 6
        nbte.nbte_mesh_create(2, m.nodes, m.cell_type, c, m.bfaces, m.btags)
    assert e.value.code == nbte.NBTE_ERR_MESH
    with pytest.raises(nbte.NbteError) as e:   # dim does not match the cell type
        nbte.nbte_mesh_create(3, m.nodes, m.cell_type, m.cells, m.bfaces, m.btags)
    assert e.value.code == nbte.NBTE_ERR_ARG
    with pytest.raises(nbte.NbteError) as e:   # degenerate (collapsed) cell
        nodes = m.nodes.copy()
        nodes[m.cells[0, 2]] = nodes[m.cells[0, 1]]
        nbte.nbte_mesh_create(2, nodes, m.cell_type, m.cells, m.bfaces, m.btags)
    assert e.value.code == nbte.NBTE_ERR_MESH
    with pytest.raises(nbte.NbteError) as e:   # NaN coordinate
        nodes = m.nodes.copy()
        nodes[3, 0] = np.nan
        nbte.nbte_mesh_create(2, nodes, m.cell_type, m.cells, m.bfaces, m.btags)
    assert e.value.code == nbte.NBTE_ERR_ARG


def test_setup_argument_errors(lib):
    p = W.problems.square_inplane(n=4)
    h = _mesh(p)
    s = nbte.nbte_solver_create(h, 300.0)

    def code(fn, *a):
        with pytest.raises(nbte.NbteError) as e:
            fn(*a)
        return e.value.code

    assert code(nbte.nbte_set_bands, s, [1e6], [-1.0], [1e-12]) == nbte.NBTE_ERR_ARG
    assert code(nbte.nbte_set_bands, s, [1e6], [6e3], [np.nan]) == nbte.NBTE_ERR_ARG
    assert code(nbte.nbte_set_bands, s, [0.0], [6e3], [1e-12]) == nbte.NBTE_ERR_ARG
    sq, w = W.quadrature.inplane(8)
    bad = sq.copy()
    bad[0] *= 1.01
    assert code(nbte.nbte_set_quadrature, s, bad, w) == nbte.NBTE_ERR_ARG
    assert code(nbte.nbte_set_quadrature, s, sq, -w) == nbte.NBTE_ERR_ARG
    # a tag without a condition, and a set without a thermalizing wall
    assert code(nbte.nbte_set_boundaries, s, p.boundaries[:3]) == nbte.NBTE_ERR_ARG
    assert code(nbte.nbte_set_boundaries, s, [Boundary(t, 1) for t in (1, 2, 3, 4)]) == nbte.NBTE_ERR_ARG
    assert code(nbte.nbte_set_boundaries, s, [Boundary(1, 0, 300.0), Boundary(2, 3, 0, 1.5),
                                              Boundary(3, 1), Boundary(4, 1)]) == nbte.NBTE_ERR_ARG
    for bad in (np.inf, -np.inf, np.nan):
        for at in (0, 2, p.n_cells - 1):
            q = np.zeros(p.n_cells)
            q[at] = bad
            assert code(nbte.nbte_set_heat_source, s, q) == nbte.NBTE_ERR_ARG
    nbte.nbte_set_heat_source(s, np.full(p.n_cells, 1e300))   # large but finite: accepted
    # solve before the set-up is complete
    st, _ = None, None
    with pytest.raises(nbte.NbteError) as e:
        nbte.nbte_solve_steady(s, nbte.make_opts())
    assert e.value.code == nbte.NBTE_ERR_STATE
    # valid set-up calls succeed without a device
    nbte.nbte_set_bands(s, p.C, p.v, p.tau)
    nbte.nbte_set_quadrature(s, p.s, p.w)
    nbte.nbte_set_boundaries(s, p.boundaries)
    nbte.nbte_set_heat_source(s, None)
    # results before any solve
    with pytest.raises(nbte.NbteError) as e:
        nbte.nbte_get_temperature(s, 0, p.n_cells)
    assert e.value.code == nbte.NBTE_ERR_STATE
    # option checks happen before device work
    with pytest.raises(nbte.NbteError) as e:
        nbte.nbte_solve_steady(s, nbte.make_opts(scheme=7))
    assert e.value.code == nbte.NBTE_ERR_ARG
    with pytest.raises(nbte.NbteError) as e:
        nbte.nbte_solve_steady(s, nbte.make_opts(tol=-1.0))
    assert e.value.code == nbte.NBTE_ERR_ARG
    with pytest.raises(nbte.NbteError) as e:
        nbte.nbte_solve_steady(s, nbte.make_opts(order=3))
    assert e.value.code == nbte.NBTE_ERR_ARG
    nbte.nbte_solver_destroy(s)
    nbte.nbte_mesh_destroy(h)


def test_result_buffer_checked_before_the_call(lib):
    """A caller's result array of the wrong dtype, shape or layout is
    refused by the binding before the library writes anything."""
    for bad in (np.empty(10, dtype=np.float32), np.empty(9), np.empty((10, 2))[:, 0]):
        with pytest.raises(ValueError):
            nbte.nbte_get_temperature(None, 0, 10, out=bad)
    with pytest.raises(ValueError):
        nbte.nbte_get_heat_flux(None, 10, 2, out=np.empty((2, 10)))


def test_struct_layout_matches_c_compiler(lib, tmp_path):
    """The binding's ctypes structs have the size and field offsets the C
    compiler gives the header's structs."""
    import ctypes
    import subprocess
    structs = {"nbte_solve_opts": nbte.nbte_solve_opts, "nbte_solve_info": nbte.nbte_solve_info,
               "nbte_boundary": nbte.nbte_boundary}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nbte.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"
