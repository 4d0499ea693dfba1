"""The input path a user of meshes and phonon data takes, solved on the GPU:
a seeded tetrahedral fin mesh written to a Gmsh 4.1 file and read back with
paper_2607_03226_b300.inputs.read_gmsh, bands from a seeded per-mode table
binned by mean free path (bands_from_modes) and passed through a band-table
file (read_band_table).  The library's solve on those arrays, converged in
FP64, matches the oracle solving the same arrays (T 1e-9, q 1e-8), and
the FP32 sweep (T 1e-6)."""
import numpy as np
import pytest

import workloads as W
from workloads.problems import Boundary, Problem, THERMALIZING, DIFFUSE, SPECULAR, PARTIAL
from oracle import OracleSolver
from cases import rel_T, rel_q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem(tmp_path_factory):
    from paper_2607_03226_b300 import inputs
    d = tmp_path_factory.mktemp("inputs")
    m = W.mesh.finfet3d_tets(h=16e-9, seed=31)
    path = d / "fin.msh"
    inputs.write_gmsh(path, m, version="4.1")
    mesh = inputs.read_gmsh(path)
    # per-mode data: 600 modes, speeds 1-8 km/s, relaxation times log-uniform
    # 1 ps - 1 ns, heat capacities summing to 1.66e6 J/m^3K
    rng = np.random.default_rng(2607)
    n = 600
    Cm = rng.uniform(0.5, 1.5, n)
    Cm *= 1.66e6 / Cm.sum()
    vm = rng.uniform(1e3, 8e3, n)
    taum = np.exp(rng.uniform(np.log(1e-12), np.log(1e-9), n))
    Cb, vb, tb = inputs.bands_from_modes(Cm, vm, taum, 6)
    table = d / "bands.txt"
    np.savetxt(table, np.stack([Cb, vb, tb], 1), header="C [J/m^3K]  v [m/s]  tau [s]")
    C, v, tau = inputs.read_band_table(table)
    s, w = W.quadrature.gl_azimuth(2, 8)
    bcs = [Boundary(1, THERMALIZING, 300.0), Boundary(2, SPECULAR, 0.0, 1.0), Boundary(3, DIFFUSE),
           Boundary(4, PARTIAL, 0.0, 0.5), Boundary(5, DIFFUSE), Boundary(6, THERMALIZING, 301.0)]
    xc = mesh.nodes[mesh.cells].mean(axis=1)
    Q = np.where(xc[:, 2] > 50e-9, 3e17, 0.0)
    return Problem("gmsh_fin", mesh, C, v, tau, s, w, bcs, Q, 300.0)


def test_gmsh_mesh_and_band_table_converged(gpu_lib, problem):
    from paper_2607_03226_b300 import nbte
    p = problem
    assert p.n_bands >= 4 and p.mesh.cell_type == W.mesh.TET
    ref = OracleSolver(p).solve(scheme="synthetic", tol=1e-14, max_iter=50000)
    assert ref["converged"]
    s = nbte.Solver(p)
    info = s.solve(scheme="sequential", precision="fp64", tol=1e-13, max_iter=50000)
    assert info["status"] == 0
    eT, eq = rel_T(s.temperature(0), ref["T"], p.T_ref), rel_q(s.heat_flux(), ref["q"])
    print(f"fp64: {info['iterations']} iterations, T {eT:.2e}, q {eq:.2e}")
    assert eT < 1e-9 and eq < 1e-8
    info = s.solve(scheme="synthetic", precision="fp32", tol=1e-9, max_iter=50000)
    assert info["status"] == 0
    eT = rel_T(s.temperature(0), ref["T"], p.T_ref)
    print(f"fp32 synthetic: {info['iterations']} iterations, T {eT:.2e}")
    assert eT < 1e-6
    s.close()
