"""Finite-volume geometry for the oracle (half-face form), FP64.

Definitions (the same ones the library documents, computed here with code of
the oracle's own):

* cell centroid ``x_c`` and face centroid ``x_f`` = vertex averages;
* face vector ``An_f`` = area times the unit normal pointing out of the cell
  that owns the half-face (2D edge p->q: length times the rotated tangent;
  3D triangle: half the cross product of two edges; 3D quadrilateral: half the
  cross product of its diagonals);
* cell volume (area in 2D): triangle 0.5|cross|, quadrilateral shoelace,
  tetrahedron |det|/6, hexahedron the sum of six tetrahedra around the 0-6
  diagonal.

Every cell face appears once per adjacent cell ("half-face"); a half-face with
no neighbouring cell must match exactly one tagged boundary face.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

TRI, QUAD, TET, HEX = 3, 4, 10, 12

LOCAL_FACES = {
    TRI: [(0, 1), (1, 2), (2, 0)],
    QUAD: [(0, 1), (1, 2), (2, 3), (3, 0)],
    TET: [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)],
    HEX: [(0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)],
}


@dataclass
class Geometry:
    dim: int
    n_cells: int
    V: np.ndarray        # (N,)
    xc: np.ndarray       # (N, dim)
    hf_cell: np.ndarray  # (H,) owner cell of each half-face
    hf_nb: np.ndarray    # (H,) neighbour cell, -1 on the boundary
    hf_An: np.ndarray    # (H, dim) outward face vector (area * unit normal)
    hf_xf: np.ndarray    # (H, dim) face centroid
    hf_tag: np.ndarray   # (H,) boundary tag, -1 for interior half-faces


def _volumes(nodes, cells, ctype):
    P = nodes[cells]
    if ctype == TRI:
        a = P[:, 1] - P[:, 0]
        b = P[:, 2] - P[:, 0]
        return 0.5 * np.abs(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    if ctype == QUAD:
        x, y = P[..., 0], P[..., 1]
        return 0.5 * np.abs(np.sum(x * np.roll(y, -1, axis=1) - np.roll(x, -1, axis=1) * y, axis=1))
    if ctype == TET:
        return np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6.0
    if ctype == HEX:
        vol = np.zeros(P.shape[0])
        for t in ((0, 1, 2, 6), (0, 2, 3, 6), (0, 3, 7, 6), (0, 7, 4, 6), (0, 4, 5, 6), (0, 5, 1, 6)):
            Q = P[:, list(t)]
            vol += np.abs(np.linalg.det(Q[:, 1:] - Q[:, :1])) / 6.0
        return vol
    raise ValueError(ctype)


def _face_vectors(FP, dim):
    """Unoriented area vectors of faces given their node coordinates."""
    if dim == 2:
        t = FP[:, 1] - FP[:, 0]
        return np.stack([t[:, 1], -t[:, 0]], axis=1)
    if FP.shape[1] == 3:
        return 0.5 * np.cross(FP[:, 1] - FP[:, 0], FP[:, 2] - FP[:, 0])
    return 0.5 * np.cross(FP[:, 2] - FP[:, 0], FP[:, 3] - FP[:, 1])


def build_geometry(mesh) -> Geometry:
    nodes = np.asarray(mesh.nodes, dtype=np.float64)
    cells = np.asarray(mesh.cells, dtype=np.int64)
    ctype = int(mesh.cell_type)
    dim = int(mesh.dim)
    N = cells.shape[0]
    lf = LOCAL_FACES[ctype]
    nf = len(lf)
    V = _volumes(nodes, cells, ctype)
    if np.any(V <= 0):
        raise ValueError("degenerate cell")
    xc = nodes[cells].mean(axis=1)

    # half-faces in (cell, local face) order
    hf_nodes = np.concatenate([cells[:, list(f)][:, None, :] for f in lf], axis=1).reshape(N * nf, -1)
    hf_cell = np.repeat(np.arange(N), nf)
    FP = nodes[hf_nodes]
    An = _face_vectors(FP, dim)
    xf = FP.mean(axis=1)
    flip = np.sum((xf - xc[hf_cell]) * An, axis=1) < 0
    An[flip] *= -1.0

    # match half-faces that share the same node set
    key = np.sort(hf_nodes, axis=1)
    order = np.lexsort(key.T[::-1])
    ks = key[order]
    same = np.all(ks[1:] == ks[:-1], axis=1)
    hf_nb = -np.ones(N * nf, dtype=np.int64)
    a = order[:-1][same]
    b = order[1:][same]
    if np.any(same[1:] & same[:-1]):
        raise ValueError("a face is shared by more than two cells")
    hf_nb[a] = hf_cell[b]
    hf_nb[b] = hf_cell[a]

    # boundary tags
    hf_tag = -np.ones(N * nf, dtype=np.int64)
    bnd = np.where(hf_nb < 0)[0]
    bkey = {tuple(k): i for i, k in enumerate(np.sort(np.asarray(mesh.bfaces), axis=1).tolist())}
    if len(bkey) != len(mesh.bfaces):
        raise ValueError("duplicate boundary face")
    seen = np.zeros(len(mesh.bfaces), dtype=bool)
    for h in bnd:
        k = tuple(key[h].tolist())
        j = bkey.get(k)
        if j is None:
            raise ValueError("untagged exterior face")
        seen[j] = True
        hf_tag[h] = int(mesh.btags[j])
    if not np.all(seen):
        raise ValueError("a tagged boundary face is not an exterior face")
    return Geometry(dim, N, V, xc, hf_cell, hf_nb, An, xf, hf_tag)
