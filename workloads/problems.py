"""Complete solve inputs for the five workload families.

A :class:`Problem` carries everything the solver's public calls take: the
mesh, the band table, the direction set, one boundary condition per tag, the
per-cell volumetric heat source and the reference temperature.

Families (full sizes by default; every builder takes smaller sizes for tests):

1. ``square_inplane``  - 100 nm square, 40x40 quads, gray band (v 6 km/s,
   tau 16.7 ps), 16 in-plane directions, thermalizing 301 K / 299 K left/right,
   specular top/bottom, no source, T_ref 300 K.
2. ``finfet2d``        - fin 10x40 nm on a 200x100 nm substrate, ~50k
   triangles, 20 silicon-like bands, 64 directions (4 half-range polar x 16
   azimuths), Gaussian hot spot (peak 1e18 W/m^3, sigma 5 nm) at the fin top,
   thermalizing bottom at 300 K, diffuse elsewhere.
3. ``cube3d``          - 500 nm cube, 64^3 hexes, 40 bands with mean free paths
   5-500 nm (Kn 0.01-1), 128 directions (8 GL x 16 azimuths), thermalizing
   310 K / 300 K on x=0 / x=L, diffuse elsewhere.
4. ``finfet3d``        - ~1.1M tetrahedra, fin 7 nm x 50 nm tall x 100 nm long
   on a 300x100x50 nm substrate, 40 bands, 200 directions (10 GL x 20
   azimuths); thermalizing bottom, specular substrate sides and y-ends,
   partially specular (p=0.5) fin sides, diffuse fin top and exposed substrate
   top; 5e17 W/m^3 uniform in the fin.
5. ``stream``          - see :mod:`workloads.stream`.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import mesh as M
from . import quadrature as Qd
from . import spectra as S

THERMALIZING, DIFFUSE, SPECULAR, PARTIAL = 0, 1, 2, 3


@dataclass
class Boundary:
    tag: int
    type: int
    T_wall: float = 0.0
    specularity: float = 0.0


@dataclass
class Problem:
    name: str
    mesh: M.Mesh
    C: np.ndarray
    v: np.ndarray
    tau: np.ndarray
    s: np.ndarray
    w: np.ndarray
    boundaries: list
    Q: np.ndarray | None
    T_ref: float = 300.0
    scheme: str = "sequential"
    tol: float = 1e-10
    max_iter: int = 5000
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self):
        return self.mesh.n_cells

    @property
    def n_bands(self):
        return int(self.C.size)

    @property
    def n_dirs(self):
        return int(self.w.size)

    @property
    def updates_per_iteration(self):
        return self.n_cells * self.n_bands * self.n_dirs


def square_inplane(n: int = 40, L: float = 100e-9, n_dirs: int = 16, v: float = 6000.0,
                   tau: float = 16.7e-12, C: float = S.C_SILICON, T_left: float = 301.0,
                   T_right: float = 299.0, T_ref: float = 300.0, ny: int | None = None,
                   top_bottom: int = SPECULAR) -> Problem:
    m = M.structured_quads(n, ny or n, L, L if ny is None else L * (ny / n))
    Cb, vb, tb = S.gray(C, v, tau)
    s, w = Qd.inplane(n_dirs)
    bcs = [Boundary(1, THERMALIZING, T_left), Boundary(2, THERMALIZING, T_right),
           Boundary(3, top_bottom, 0.0, 1.0 if top_bottom == SPECULAR else 0.0),
           Boundary(4, top_bottom, 0.0, 1.0 if top_bottom == SPECULAR else 0.0)]
    return Problem("square_inplane", m, Cb, vb, tb, s, w, bcs, None, T_ref,
                   scheme="sequential", tol=1e-10,
                   meta=dict(n=n, L=L, n_dirs=n_dirs, T_left=T_left, T_right=T_right))


def finfet2d(h: float = 0.9e-9, B: int = 20, n_pol_half: int = 4, n_az: int = 16,
             seed: int = 2607032262, q_peak: float = 1e18, sigma: float = 5e-9,
             T_ref: float = 300.0, jitter: float = 0.2, **geom) -> Problem:
    m = M.finfet2d_tris(h=h, seed=seed, jitter=jitter, **geom)
    C, v, tau = S.silicon_like(B, seed + 1)
    s, w = Qd.projected_3d_on_plane(n_pol_half, n_az)
    mm = m.meta
    x0 = np.array([0.5 * mm["sub_w"], mm["sub_h"] + mm["fin_h"]])
    xc = m.vertex_mean()
    Q = q_peak * np.exp(-np.sum((xc - x0) ** 2, axis=1) / (2.0 * sigma ** 2))
    bcs = [Boundary(1, THERMALIZING, 300.0)] + [Boundary(t, DIFFUSE) for t in (2, 3, 4, 5)]
    return Problem("finfet2d", m, C, v, tau, s, w, bcs, Q, T_ref, scheme="sequential", tol=1e-10,
                   meta=dict(h=h, B=B, n_pol_half=n_pol_half, n_az=n_az, seed=seed))


def cube3d(n: int = 64, L: float = 500e-9, B: int = 40, n_pol: int = 8, n_az: int = 16,
           seed: int = 2607032263, T_hot: float = 310.0, T_cold: float = 300.0,
           T_ref: float = 300.0) -> Problem:
    m = M.structured_hexes(n, n, n, L, L, L)
    C, v, tau = S.knudsen_spread(B, seed + 1)
    s, w = Qd.gl_azimuth(n_pol, n_az)
    bcs = [Boundary(1, THERMALIZING, T_hot), Boundary(2, THERMALIZING, T_cold)] + \
          [Boundary(t, DIFFUSE) for t in (3, 4, 5, 6)]
    return Problem("cube3d", m, C, v, tau, s, w, bcs, None, T_ref, scheme="synthetic", tol=1e-8,
                   meta=dict(n=n, L=L, B=B, n_pol=n_pol, n_az=n_az, seed=seed))


def finfet3d(h: float = 2e-9, B: int = 40, n_pol: int = 10, n_az: int = 20,
             seed: int = 2607032264, q_fin: float = 5e17, p_fin: float = 0.5,
             T_ref: float = 300.0, jitter: float = 0.1, **geom) -> Problem:
    m = M.finfet3d_tets(h=h, seed=seed, jitter=jitter, **geom)
    C, v, tau = S.silicon_like(B, seed + 1)
    s, w = Qd.gl_azimuth(n_pol, n_az)
    Q = np.where(m.meta["fin_cell"], q_fin, 0.0)
    bcs = [Boundary(1, THERMALIZING, 300.0), Boundary(2, SPECULAR, 0.0, 1.0),
           Boundary(3, SPECULAR, 0.0, 1.0), Boundary(4, PARTIAL, 0.0, p_fin),
           Boundary(5, DIFFUSE), Boundary(6, DIFFUSE)]
    return Problem("finfet3d", m, C, v, tau, s, w, bcs, Q, T_ref, scheme="synthetic", tol=1e-8,
                   meta=dict(h=h, B=B, n_pol=n_pol, n_az=n_az, seed=seed))
