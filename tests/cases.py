"""Small seeded problems shared by the GPU parity tests: every cell type and
every wall type, several bands, enough cells for several levels and ring-slot
reuse, and small enough that the oracle finishes in seconds."""
import numpy as np

import workloads as W
from workloads.problems import Boundary, THERMALIZING, DIFFUSE, SPECULAR, PARTIAL


def square_mixed():
    p = W.problems.square_inplane(n=12, ny=9, n_dirs=8, tau=8e-12)
    p.boundaries = [Boundary(1, THERMALIZING, 302.0), Boundary(2, THERMALIZING, 299.0),
                    Boundary(3, DIFFUSE), Boundary(4, SPECULAR, 0.0, 1.0)]
    p.Q = np.linspace(0.0, 4e17, p.n_cells)
    return p


def fin2d_mixed():
    p = W.problems.finfet2d(h=8e-9, B=3, n_pol_half=2, n_az=8, sigma=12e-9)
    p.boundaries = [Boundary(1, THERMALIZING, 300.5), Boundary(2, DIFFUSE), Boundary(3, SPECULAR, 0.0, 1.0),
                    Boundary(4, PARTIAL, 0.0, 0.5), Boundary(5, DIFFUSE)]
    return p


def fin3d_tets():
    return W.problems.finfet3d(h=20e-9, B=2, n_pol=2, n_az=8, q_fin=2e17)


def cube_hex():
    p = W.problems.cube3d(n=5, B=3, n_pol=2, n_az=8)
    p.boundaries = [Boundary(1, THERMALIZING, 310.0), Boundary(2, THERMALIZING, 300.0),
                    Boundary(3, DIFFUSE), Boundary(4, SPECULAR, 0.0, 1.0), Boundary(5, PARTIAL, 0.0, 0.3),
                    Boundary(6, DIFFUSE)]
    return p


def tets_cyclic():
    """A twisted annulus of tetrahedra (workloads.mesh.twisted_ring_tets):
    conforming and untangled, yet the upwind graph of many directions has
    cycles around the ring (checked on the CPU in test_oracle_tasks), so the
    sweep lags faces to break them.  Inner wall thermalizing at 302 K, outer
    at 299 K, diffuse bottom, partially specular top, a uniform heat source."""
    from workloads import mesh as M, quadrature as Qd, spectra as S
    from workloads.problems import Problem
    m = M.twisted_ring_tets()
    C, v, tau = S.silicon_like(2, 11)
    s, w = Qd.gl_azimuth(4, 8)
    bcs = [Boundary(1, THERMALIZING, 302.0), Boundary(2, THERMALIZING, 299.0), Boundary(3, DIFFUSE),
           Boundary(4, PARTIAL, 0.0, 0.5)]
    Q = np.full(m.n_cells, 1e17)
    return Problem("tets_cyclic", m, C, v, tau, s, w, bcs, Q, 300.0, scheme="sequential", tol=1e-10)


CASES = {"square_mixed": square_mixed, "fin2d_mixed": fin2d_mixed, "fin3d_tets": fin3d_tets,
         "cube_hex": cube_hex}


def rel_T(T, T_ref_field, T_ref):
    """C12 temperature metric: |T - T_oracle|_inf / |T_oracle - T_ref|_inf."""
    return float(np.abs(T - T_ref_field).max() / np.abs(T_ref_field - T_ref).max())


def rel_q(q, q_ref):
    return float(np.abs(q - q_ref).max() / np.abs(q_ref).max())
