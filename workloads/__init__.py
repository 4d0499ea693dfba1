"""Seeded synthetic inputs shaped like the paper's workloads.

This package only *generates inputs*: meshes (nodes, cells, tagged boundary
faces), band tables, discrete-ordinates sets, heat-source fields and request
streams.  It holds none of the solver's arithmetic (no face building, no
advection coefficients, no moments) and imports nothing from the CUDA
package or from the oracle, so both of those can consume it without sharing
code with each other.

The paper's own inputs (first-principles band tables, COMSOL/Gmsh device
meshes) are not available; the generators below stand in for them with the
shapes the paper describes: an in-plane square with thermalizing left/right
and specular top/bottom walls (Sec. III A), a fin-on-substrate device with a
hot spot near the fin top and mixed walls (Sec. III B, Table I), tens of
thousands to a million cells, 1-40 bands and 16-200 directions.
"""
from .mesh import Mesh, structured_quads, structured_hexes, finfet2d_tris, finfet3d_tets
from .quadrature import inplane, gl_azimuth, projected_3d_on_plane
from .spectra import gray, silicon_like, knudsen_spread
from .problems import Problem, Boundary, THERMALIZING, DIFFUSE, SPECULAR, PARTIAL
from . import problems, stream

__all__ = [
    "Mesh", "structured_quads", "structured_hexes", "finfet2d_tris", "finfet3d_tets",
    "inplane", "gl_azimuth", "projected_3d_on_plane",
    "gray", "silicon_like", "knudsen_spread",
    "Problem", "Boundary", "THERMALIZING", "DIFFUSE", "SPECULAR", "PARTIAL",
    "problems", "stream",
]
