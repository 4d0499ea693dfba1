"""Seeded request stream for the serving workload.

Each request is a steady solve of its own device geometry: a 2D triangle
fin-on-substrate, a 3D hexahedral box or a 3D tetrahedral fin, with
20k-500k cells (log-uniform), 10-40 bands, 32/64/128 directions, a heat load
of 1e16-1e18 W/m^3 (log-uniform) on a random box region and a boundary set
drawn from {thermalizing, diffuse, specular, partial p=0.5} with at least one
thermalizing wall.  Arrivals are a Poisson process of a chosen rate.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import mesh as M
from . import quadrature as Qd
from . import spectra as S
from .problems import Problem, Boundary, THERMALIZING, DIFFUSE, SPECULAR, PARTIAL


@dataclass
class Request:
    rid: int
    arrival: float
    kind: str          # "tri2d", "hex3d", "tet3d"
    n_cells_target: int
    B: int
    D: int
    q_load: float
    seed: int
    tol: float = 1e-8


def requests(n: int, rate: float, seed: int = 2607032265, n_range=(20_000, 500_000),
             b_range=(10, 40), d_choices=(32, 64, 128), kinds=("tri2d", "hex3d", "tet3d")):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for k in range(n):
        out.append(Request(
            rid=k, arrival=float(t[k]), kind=str(rng.choice(kinds)),
            n_cells_target=int(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))),
            B=int(rng.integers(b_range[0], b_range[1] + 1)), D=int(rng.choice(d_choices)),
            q_load=float(np.exp(rng.uniform(np.log(1e16), np.log(1e18)))),
            seed=int(seed * 1000 + k)))
    return out


def _bcs(rng, tags, first_thermalizing):
    kinds = [THERMALIZING, DIFFUSE, SPECULAR, PARTIAL]
    out = []
    for i, t in enumerate(tags):
        k = THERMALIZING if (i == 0 and first_thermalizing) else int(rng.choice(kinds))
        if k == THERMALIZING:
            out.append(Boundary(t, k, 300.0))
        elif k == SPECULAR:
            out.append(Boundary(t, k, 0.0, 1.0))
        elif k == PARTIAL:
            out.append(Boundary(t, k, 0.0, 0.5))
        else:
            out.append(Boundary(t, k))
    return out


def build(req: Request) -> Problem:
    """Materialise the problem a request describes (deterministic in ``req``)."""
    rng = np.random.default_rng(req.seed)
    N = req.n_cells_target
    if req.kind == "tri2d":
        area = 200e-9 * 100e-9 + 10e-9 * 40e-9
        h = float(np.sqrt(2.0 * area / N))
        m = M.finfet2d_tris(h=h, seed=req.seed)
        npol = {32: 2, 64: 4, 128: 8}[req.D]
        s, w = Qd.projected_3d_on_plane(npol, req.D // npol)
        tags = (1, 2, 3, 4, 5)
    elif req.kind == "hex3d":
        n = max(4, int(round(N ** (1.0 / 3.0))))
        L = 500e-9
        m = M.structured_hexes(n, n, n, L, L, L)
        npol = {32: 2, 64: 4, 128: 8}[req.D]
        s, w = Qd.gl_azimuth(npol, req.D // npol)
        tags = (1, 2, 3, 4, 5, 6)
    else:
        vol = 300e-9 * 100e-9 * 50e-9 + 7e-9 * 100e-9 * 50e-9
        h = float((6.0 * vol / N) ** (1.0 / 3.0))
        m = M.finfet3d_tets(h=h, seed=req.seed, hx_fin=min(h, 3.5e-9))
        npol = {32: 2, 64: 4, 128: 8}[req.D]
        s, w = Qd.gl_azimuth(npol, req.D // npol)
        tags = (1, 2, 3, 4, 5, 6)
    C, v, tau = S.silicon_like(req.B, req.seed + 7)
    bcs = _bcs(rng, tags, True)
    xc = m.vertex_mean()
    lo = xc.min(0)
    hi = xc.max(0)
    a = lo + rng.uniform(0.2, 0.5, size=lo.size) * (hi - lo)
    b = a + rng.uniform(0.1, 0.3, size=lo.size) * (hi - lo)
    inside = np.all((xc >= a) & (xc <= b), axis=1)
    Q = np.where(inside, req.q_load, 0.0)
    return Problem(f"req{req.rid}-{req.kind}", m, C, v, tau, s, w, bcs, Q, 300.0,
                   scheme="synthetic", tol=req.tol, meta=dict(rid=req.rid))
