"""Input readers: Gmsh meshes and phonon band tables, as the arrays the
library's calls take (``nbte_mesh_create``, ``nbte_set_bands``).

The paper's solver reads COMSOL and Gmsh meshes with boundary labels and
band-resolved phonon properties from a mean-free-path band discretisation of
per-mode data (Sec. II).  This module reads

* Gmsh ``.msh`` files, ASCII format 2.2 or 4.1: the highest-dimensional
  elements become the cells (triangles or quadrangles in 2D, tetrahedra or
  hexahedra in 3D), the elements one dimension lower that carry a physical
  tag become the tagged boundary faces;
* band tables: whitespace-separated text with one band per row,
  ``C [J/m^3K]  v [m/s]  tau [s]`` (``#`` starts a comment);
* per-mode tables (the same three columns, one phonon mode per row), binned
  into representative bands by mean free path (:func:`bands_from_modes`).

It also writes ``.msh`` 2.2 / 4.1 files (used to test the reader).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

TRI, QUAD, TET, HEX = 3, 4, 10, 12

# Gmsh element type -> (dimension, nodes, library cell type or None for faces)
_GMSH = {1: (1, 2, None), 2: (2, 3, TRI), 3: (2, 4, QUAD), 4: (3, 4, TET), 5: (3, 8, HEX)}
_TO_GMSH = {TRI: 2, QUAD: 3, TET: 4, HEX: 5}
_FACE_GMSH = {2: 1, 3: 2, 4: 3}   # face nodes -> Gmsh type (line, triangle, quadrangle)


@dataclass
class MeshArrays:
    dim: int
    nodes: np.ndarray      # (n_nodes, dim) float64
    cell_type: int
    cells: np.ndarray      # (n_cells, nodes per cell) int64, 0-based
    bfaces: np.ndarray     # (n_bfaces, nodes per face) int64, 0-based
    btags: np.ndarray      # (n_bfaces,) int32 physical tags


def _sections(text):
    out, cur, name = {}, None, None
    for line in text.splitlines():
        s = line.strip()
        if s.startswith("$End"):
            out[name] = cur
            cur = name = None
        elif s.startswith("$"):
            name, cur = s[1:], []
        elif cur is not None:
            cur.append(s)
    return out


def _finish(node_ids, xyz, elems):
    """elems: list of (gmsh type, physical tag, node ids)."""
    dims = [_GMSH[t][0] for t, _, _ in elems if t in _GMSH]
    if not dims:
        raise ValueError("no supported elements (triangle, quadrangle, tetrahedron, hexahedron)")
    dim = max(dims)
    index = {int(n): k for k, n in enumerate(node_ids)}
    cell_types = {_GMSH[t][2] for t, _, _ in elems if t in _GMSH and _GMSH[t][0] == dim}
    if len(cell_types) != 1:
        raise ValueError("mixed cell types in one mesh are not supported")
    ctype = cell_types.pop()
    cells = [[index[n] for n in ns] for t, _, ns in elems if t in _GMSH and _GMSH[t][0] == dim]
    faces = [([index[n] for n in ns], tag) for t, tag, ns in elems
             if t in _GMSH and _GMSH[t][0] == dim - 1 and tag > 0]
    nodes = np.asarray(xyz, dtype=np.float64)[:, :dim].copy()
    return MeshArrays(dim, nodes, ctype, np.asarray(cells, dtype=np.int64),
                      np.asarray([f for f, _ in faces], dtype=np.int64).reshape(len(faces), -1),
                      np.asarray([t for _, t in faces], dtype=np.int32))


def read_gmsh(path) -> MeshArrays:
    """Read a Gmsh ASCII mesh (format 2.2 or 4.1)."""
    text = open(path).read()
    sec = _sections(text)
    if "MeshFormat" not in sec:
        raise ValueError("not a Gmsh mesh: no $MeshFormat")
    fmt = sec["MeshFormat"][0].split()
    version, binary = float(fmt[0]), int(fmt[1])
    if binary:
        raise ValueError("binary Gmsh files are not supported")
    if version < 3:
        return _read_v2(sec)
    return _read_v4(sec)


def _read_v2(sec):
    lines = sec["Nodes"]
    n = int(lines[0])
    ids, xyz = [], []
    for s in lines[1:1 + n]:
        f = s.split()
        ids.append(int(f[0]))
        xyz.append([float(x) for x in f[1:4]])
    lines = sec["Elements"]
    m = int(lines[0])
    elems = []
    for s in lines[1:1 + m]:
        f = [int(x) for x in s.split()]
        t, ntags = f[1], f[2]
        tag = f[3] if ntags > 0 else 0          # first tag: the physical group
        elems.append((t, tag, f[3 + ntags:]))
    return _finish(ids, xyz, elems)


def _read_v4(sec):
    # entity (dim, tag) -> first physical tag
    phys = {}
    if "Entities" in sec:
        L = sec["Entities"]
        counts = [int(x) for x in L[0].split()]
        row = 1
        for dim, cnt in enumerate(counts):
            for _ in range(cnt):
                f = L[row].split()
                row += 1
                tag = int(f[0])
                at = 4 if dim == 0 else 7           # points: x y z; others: bounding box
                nphys = int(f[at])
                phys[(dim, tag)] = int(f[at + 1]) if nphys > 0 else 0
    L = sec["Nodes"]
    nblocks = int(L[0].split()[0])
    row = 1
    ids, xyz = [], []
    for _ in range(nblocks):
        _, _, param, nn = (int(x) for x in L[row].split())
        row += 1
        bids = [int(L[row + k]) for k in range(nn)]
        row += nn
        for k in range(nn):
            f = L[row + k].split()
            xyz.append([float(x) for x in f[:3]])
        row += nn
        if param:
            raise ValueError("parametric node blocks are not supported")
        ids += bids
    L = sec["Elements"]
    nblocks = int(L[0].split()[0])
    row = 1
    elems = []
    for _ in range(nblocks):
        edim, etag, etype, ne = (int(x) for x in L[row].split())
        row += 1
        tag = phys.get((edim, etag), 0)
        for k in range(ne):
            f = [int(x) for x in L[row + k].split()]
            elems.append((etype, tag, f[1:]))
        row += ne
    return _finish(ids, xyz, elems)


def write_gmsh(path, m, version="2.2"):
    """Write mesh arrays (fields dim, nodes, cell_type, cells, bfaces, btags)
    as a Gmsh ASCII file; boundary faces get their tag as physical group."""
    nodes3 = np.zeros((m.nodes.shape[0], 3))
    nodes3[:, :m.dim] = m.nodes
    ct, ft = _TO_GMSH[m.cell_type], _FACE_GMSH[m.bfaces.shape[1]]
    out = []
    if version == "2.2":
        out += ["$MeshFormat", "2.2 0 8", "$EndMeshFormat", "$Nodes", str(len(nodes3))]
        out += [f"{k + 1} {float(x)!r} {float(y)!r} {float(z)!r}" for k, (x, y, z) in enumerate(nodes3)]
        out += ["$EndNodes", "$Elements", str(len(m.bfaces) + len(m.cells))]
        e = 1
        for f, t in zip(m.bfaces, m.btags):
            out.append(f"{e} {ft} 2 {int(t)} {int(t)} " + " ".join(str(int(n) + 1) for n in f))
            e += 1
        for c in m.cells:
            out.append(f"{e} {ct} 2 0 1 " + " ".join(str(int(n) + 1) for n in c))
            e += 1
        out += ["$EndElements"]
    elif version == "4.1":
        tags = sorted({int(t) for t in m.btags})
        fd = m.dim - 1
        counts = [0, 0, 0, 0]
        counts[fd] = len(tags)
        counts[m.dim] += 1
        lo, hi = nodes3.min(0), nodes3.max(0)
        box = " ".join(repr(float(x)) for x in (*lo, *hi))
        out += ["$MeshFormat", "4.1 0 8", "$EndMeshFormat", "$Entities", " ".join(map(str, counts))]
        for d in range(4):
            if d == fd:
                for t in tags:
                    out.append(f"{t} {box} 1 {t} 0")
            if d == m.dim:
                out.append(f"1 {box} 0 0")
        out += ["$EndEntities", "$Nodes", f"1 {len(nodes3)} 1 {len(nodes3)}", f"{m.dim} 1 0 {len(nodes3)}"]
        out += [str(k + 1) for k in range(len(nodes3))]
        out += [f"{float(x)!r} {float(y)!r} {float(z)!r}" for x, y, z in nodes3]
        out += ["$EndNodes", "$Elements", f"{len(tags) + 1} {len(m.bfaces) + len(m.cells)} 1 "
                f"{len(m.bfaces) + len(m.cells)}"]
        e = 1
        for t in tags:
            sel = np.where(m.btags == t)[0]
            out.append(f"{fd} {t} {ft} {len(sel)}")
            for k in sel:
                out.append(f"{e} " + " ".join(str(int(n) + 1) for n in m.bfaces[k]))
                e += 1
        out.append(f"{m.dim} 1 {ct} {len(m.cells)}")
        for c in m.cells:
            out.append(f"{e} " + " ".join(str(int(n) + 1) for n in c))
            e += 1
        out += ["$EndElements"]
    else:
        raise ValueError("version must be '2.2' or '4.1'")
    with open(path, "w") as fh:
        fh.write("\n".join(out) + "\n")


def read_band_table(path):
    """(C, v, tau) arrays from a text table, one band per row."""
    a = np.loadtxt(path, comments="#", ndmin=2)
    if a.shape[1] != 3:
        raise ValueError("a band table has three columns: C v tau")
    C, v, tau = a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy()
    if np.any(C <= 0) or np.any(v <= 0) or np.any(tau <= 0):
        raise ValueError("C, v and tau must be positive")
    return C, v, tau


def bands_from_modes(C, v, tau, n_bands):
    """Representative bands from per-mode data by mean free path.

    Modes are grouped into ``n_bands`` bins of equal width in log(Lambda),
    Lambda = v tau, over the modes' range; empty bins are dropped.  A band
    keeps its modes' total heat capacity, C-weighted group speed and total
    conductivity kernel sum C v^2 tau:
        C_b = sum C,  v_b = sum C v / C_b,  tau_b = sum C v^2 tau / (C_b v_b^2).
    So the band set has the modes' heat capacity and bulk conductivity, and a
    band holding one mode is that mode."""
    C, v, tau = (np.asarray(x, dtype=np.float64) for x in (C, v, tau))
    if not (C.shape == v.shape == tau.shape) or C.ndim != 1 or C.size == 0:
        raise ValueError("C, v and tau must be 1-D arrays of one length")
    if np.any(C <= 0) or np.any(v <= 0) or np.any(tau <= 0):
        raise ValueError("C, v and tau must be positive")
    lam = np.log(v * tau)
    lo, hi = lam.min(), lam.max()
    if hi == lo:
        k = np.zeros(C.size, dtype=np.int64)
    else:
        k = np.minimum((n_bands * (lam - lo) / (hi - lo)).astype(np.int64), n_bands - 1)
    Cb = np.bincount(k, weights=C, minlength=n_bands)
    Cv = np.bincount(k, weights=C * v, minlength=n_bands)
    kap = np.bincount(k, weights=C * v * v * tau, minlength=n_bands)
    keep = Cb > 0
    Cb, Cv, kap = Cb[keep], Cv[keep], kap[keep]
    vb = Cv / Cb
    return Cb, vb, kap / (Cb * vb * vb)
