"""Seeded mesh generators (inputs only: nodes, cells, tagged boundary faces).

Cell-type codes and local node orderings are the library's input format:

* ``TRI = 3``  (2D) three nodes.
* ``QUAD = 4`` (2D) four nodes in cyclic order.
* ``TET = 10`` (3D) four nodes.
* ``HEX = 12`` (3D) eight nodes: bottom cycle 0-1-2-3, then top cycle 4-5-6-7
  with node 4 above node 0.

Boundary faces are given by their node lists (2 nodes in 2D; 3 for tet meshes,
4 for hex meshes) plus an integer tag.  Every exterior face of the mesh carries
exactly one tag.  Nothing here computes areas, normals or volumes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TRI, QUAD, TET, HEX = 3, 4, 10, 12


@dataclass
class Mesh:
    dim: int
    nodes: np.ndarray          # (n_nodes, dim) float64, metres
    cell_type: int
    cells: np.ndarray          # (n_cells, nodes_per_cell) int64
    bfaces: np.ndarray         # (n_bfaces, nodes_per_face) int64
    btags: np.ndarray          # (n_bfaces,) int32
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return int(self.cells.shape[0])

    @property
    def n_nodes(self) -> int:
        return int(self.nodes.shape[0])

    def vertex_mean(self) -> np.ndarray:
        """Vertex average of every cell (used by generators to place sources)."""
        return self.nodes[self.cells].mean(axis=1)


# --------------------------------------------------------------------------
# structured boxes
# --------------------------------------------------------------------------

def structured_quads(nx: int, ny: int, Lx: float, Ly: float) -> Mesh:
    """Axis-aligned ``nx x ny`` quads on ``[0,Lx] x [0,Ly]``.

    Tags: 1 left (x=0), 2 right (x=Lx), 3 bottom (y=0), 4 top (y=Ly).
    """
    xs = np.linspace(0.0, Lx, nx + 1)
    ys = np.linspace(0.0, Ly, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    nodes = np.stack([X.ravel(), Y.ravel()], axis=1)

    def nid(i, j):
        return j * (nx + 1) + i

    I, J = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    I, J = I.ravel(), J.ravel()
    cells = np.stack([nid(I, J), nid(I + 1, J), nid(I + 1, J + 1), nid(I, J + 1)], axis=1)

    bf, bt = [], []
    i = np.arange(nx)
    j = np.arange(ny)
    bf.append(np.stack([nid(0, j), nid(0, j + 1)], 1)); bt.append(np.full(ny, 1))
    bf.append(np.stack([nid(nx, j), nid(nx, j + 1)], 1)); bt.append(np.full(ny, 2))
    bf.append(np.stack([nid(i, 0), nid(i + 1, 0)], 1)); bt.append(np.full(nx, 3))
    bf.append(np.stack([nid(i, ny), nid(i + 1, ny)], 1)); bt.append(np.full(nx, 4))
    return Mesh(2, nodes, QUAD, cells.astype(np.int64), np.concatenate(bf).astype(np.int64),
                np.concatenate(bt).astype(np.int32),
                meta=dict(kind="structured_quads", nx=nx, ny=ny, Lx=Lx, Ly=Ly))


def structured_hexes(nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float) -> Mesh:
    """Axis-aligned ``nx x ny x nz`` hexahedra on a box.

    Tags: 1 x=0, 2 x=Lx, 3 y=0, 4 y=Ly, 5 z=0, 6 z=Lz.
    """
    xs = np.linspace(0.0, Lx, nx + 1)
    ys = np.linspace(0.0, Ly, ny + 1)
    zs = np.linspace(0.0, Lz, nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    nodes = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def nid(i, j, k):
        return (k * (ny + 1) + j) * (nx + 1) + i

    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    cells = np.stack([nid(I, J, K), nid(I + 1, J, K), nid(I + 1, J + 1, K), nid(I, J + 1, K),
                      nid(I, J, K + 1), nid(I + 1, J, K + 1), nid(I + 1, J + 1, K + 1),
                      nid(I, J + 1, K + 1)], axis=1)
    bf, bt = [], []
    # x faces
    B, A = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
    A, B = A.ravel(), B.ravel()
    for i0, tag in ((0, 1), (nx, 2)):
        bf.append(np.stack([nid(i0, A, B), nid(i0, A + 1, B), nid(i0, A + 1, B + 1), nid(i0, A, B + 1)], 1))
        bt.append(np.full(A.size, tag))
    # y faces
    B, A = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    A, B = A.ravel(), B.ravel()
    for j0, tag in ((0, 3), (ny, 4)):
        bf.append(np.stack([nid(A, j0, B), nid(A + 1, j0, B), nid(A + 1, j0, B + 1), nid(A, j0, B + 1)], 1))
        bt.append(np.full(A.size, tag))
    # z faces
    B, A = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    A, B = A.ravel(), B.ravel()
    for k0, tag in ((0, 5), (nz, 6)):
        bf.append(np.stack([nid(A, B, k0), nid(A + 1, B, k0), nid(A + 1, B + 1, k0), nid(A, B + 1, k0)], 1))
        bt.append(np.full(A.size, tag))
    return Mesh(3, nodes, HEX, cells.astype(np.int64), np.concatenate(bf).astype(np.int64),
                np.concatenate(bt).astype(np.int32),
                meta=dict(kind="structured_hexes", nx=nx, ny=ny, nz=nz, Lx=Lx, Ly=Ly, Lz=Lz))


# --------------------------------------------------------------------------
# helpers for fin-on-substrate background grids
# --------------------------------------------------------------------------

def _axis(breaks, h):
    """Grid lines through every break point with spacing close to ``h``."""
    pts = [breaks[0]]
    for a, b in zip(breaks[:-1], breaks[1:]):
        n = max(1, int(round((b - a) / h)))
        pts.extend(list(np.linspace(a, b, n + 1)[1:]))
    return np.asarray(pts, dtype=np.float64)


def _local_spacing(x):
    d = np.diff(x)
    out = np.empty_like(x)
    out[0] = d[0]
    out[-1] = d[-1]
    out[1:-1] = np.minimum(d[:-1], d[1:])
    return out


def finfet2d_tris(h: float = 0.9e-9, seed: int = 2607032262, jitter: float = 0.2,
                  sub_w: float = 200e-9, sub_h: float = 100e-9,
                  fin_w: float = 10e-9, fin_h: float = 40e-9) -> Mesh:
    """2D fin-on-substrate cross-section meshed with triangles.

    A background grid of near-``h`` quads covers the substrate
    ``[0,sub_w] x [0,sub_h]`` and a fin ``fin_w x fin_h`` centred on its top;
    each quad is cut into two triangles along a seeded diagonal and every
    interior node is moved by a seeded offset of at most ``jitter`` times the
    local grid spacing (per coordinate), which keeps every triangle valid.

    Tags: 1 substrate bottom, 2 substrate left/right sides, 3 exposed substrate
    top, 4 fin sides, 5 fin top.
    """
    rng = np.random.default_rng(seed)
    fx0 = 0.5 * (sub_w - fin_w)
    fx1 = fx0 + fin_w
    xs = _axis([0.0, fx0, fx1, sub_w], h)
    ys = _axis([0.0, sub_h, sub_h + fin_h], h)
    nx, ny = xs.size - 1, ys.size - 1
    ix0 = int(np.argmin(np.abs(xs - fx0)))
    ix1 = int(np.argmin(np.abs(xs - fx1)))
    jy_sub = int(np.argmin(np.abs(ys - sub_h)))

    I, J = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    active = (J < jy_sub) | ((I >= ix0) & (I < ix1))

    def nid(i, j):
        return j * (nx + 1) + i

    Xn, Yn = np.meshgrid(xs, ys, indexing="xy")
    nodes_all = np.stack([Xn.ravel(), Yn.ravel()], axis=1)

    ai, aj = I[active], J[active]
    a, b, c, d = nid(ai, aj), nid(ai + 1, aj), nid(ai + 1, aj + 1), nid(ai, aj + 1)
    diag = rng.integers(0, 2, size=ai.size).astype(bool)
    t1 = np.where(diag[:, None], np.stack([a, b, c], 1), np.stack([a, b, d], 1))
    t2 = np.where(diag[:, None], np.stack([a, c, d], 1), np.stack([b, c, d], 1))
    tris = np.empty((2 * ai.size, 3), dtype=np.int64)
    tris[0::2] = t1
    tris[1::2] = t2

    def is_active(i, j):
        ok = (i >= 0) & (i < nx) & (j >= 0) & (j < ny)
        res = np.zeros_like(ok)
        res[ok] = active[j[ok], i[ok]]
        return res

    bf, bt = [], []
    fin_col = (ai >= ix0) & (ai < ix1)
    # bottom side of each active quad
    m = ~is_active(ai, aj - 1)
    bf.append(np.stack([a[m], b[m]], 1))
    bt.append(np.where(aj[m] == 0, 1, 3))  # y=0 is the only exposed bottom
    # top side
    m = ~is_active(ai, aj + 1)
    bf.append(np.stack([d[m], c[m]], 1))
    bt.append(np.where(fin_col[m] & (aj[m] >= jy_sub), 5, 3))
    # left side
    m = ~is_active(ai - 1, aj)
    bf.append(np.stack([a[m], d[m]], 1))
    bt.append(np.where(aj[m] >= jy_sub, 4, 2))
    # right side
    m = ~is_active(ai + 1, aj)
    bf.append(np.stack([b[m], c[m]], 1))
    bt.append(np.where(aj[m] >= jy_sub, 4, 2))
    bfaces = np.concatenate(bf).astype(np.int64)
    btags = np.concatenate(bt).astype(np.int32)

    # compact nodes
    used = np.unique(tris)
    remap = -np.ones(nodes_all.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.size)
    nodes = nodes_all[used].copy()
    tris = remap[tris]
    bfaces = remap[bfaces]

    # seeded jitter of interior nodes
    on_bnd = np.zeros(nodes.shape[0], dtype=bool)
    on_bnd[bfaces.ravel()] = True
    gi = used % (nx + 1)
    gj = used // (nx + 1)
    hx = _local_spacing(xs)[gi]
    hy = _local_spacing(ys)[gj]
    off = rng.uniform(-jitter, jitter, size=nodes.shape)
    off[:, 0] *= hx
    off[:, 1] *= hy
    off[on_bnd] = 0.0
    nodes += off
    return Mesh(2, nodes, TRI, tris, bfaces, btags,
                meta=dict(kind="finfet2d_tris", h=h, seed=seed, jitter=jitter, sub_w=sub_w,
                          sub_h=sub_h, fin_w=fin_w, fin_h=fin_h))


# Kuhn (Freudenthal) split of a unit cube into 6 tetrahedra along 000-111.
_KUHN = []
for _p in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
    _v = [0, 0, 0]
    _path = [tuple(_v)]
    for _ax in _p:
        _v[_ax] = 1
        _path.append(tuple(_v))
    _KUHN.append(_path)


def finfet3d_tets(h: float = 2e-9, seed: int = 2607032264, jitter: float = 0.1,
                  sub_x: float = 300e-9, sub_y: float = 100e-9, sub_z: float = 50e-9,
                  fin_w: float = 7e-9, fin_h: float = 50e-9, hx_fin: float | None = None) -> Mesh:
    """3D fin-on-substrate device meshed with tetrahedra.

    A background grid of near-``h`` hexahedra covers the substrate
    ``sub_x x sub_y x sub_z`` and a fin ``fin_w`` wide (x), ``sub_y`` long (y)
    and ``fin_h`` tall (z) centred on the substrate top.  Each hexahedron is cut
    into the 6 Kuhn tetrahedra along its 000-111 diagonal (a conforming split);
    interior nodes then move by a seeded offset of at most ``jitter`` times the
    local spacing per coordinate.

    Tags: 1 substrate bottom (z=0), 2 substrate x-sides, 3 y-ends (substrate and
    fin), 4 fin x-sides, 5 fin top, 6 exposed substrate top.
    """
    rng = np.random.default_rng(seed)
    fx0 = 0.5 * (sub_x - fin_w)
    fx1 = fx0 + fin_w
    xs = _axis([0.0, fx0], h)
    xs = np.concatenate([xs, _axis([fx0, fx1], hx_fin or h)[1:], _axis([fx1, sub_x], h)[1:]])
    ys = _axis([0.0, sub_y], h)
    zs = _axis([0.0, sub_z, sub_z + fin_h], h)
    nx, ny, nz = xs.size - 1, ys.size - 1, zs.size - 1
    ix0 = int(np.argmin(np.abs(xs - fx0)))
    ix1 = int(np.argmin(np.abs(xs - fx1)))
    kz_sub = int(np.argmin(np.abs(zs - sub_z)))

    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    active = (K < kz_sub) | ((I >= ix0) & (I < ix1))
    ai, aj, ak = I[active], J[active], K[active]
    fin_cell_hex = ak >= kz_sub

    def nid(i, j, k):
        return (k * (ny + 1) + j) * (nx + 1) + i

    tets = []
    for path in _KUHN:
        tets.append(np.stack([nid(ai + p[0], aj + p[1], ak + p[2]) for p in path], 1))
    tets = np.stack(tets, 1).reshape(-1, 4).astype(np.int64)
    fin_cell = np.repeat(fin_cell_hex, 6)

    # boundary faces = tet faces seen once
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    faces = np.sort(tets[:, loc].reshape(-1, 3), axis=1)
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    key = (faces[:, 0] * nn + faces[:, 1]) * nn + faces[:, 2]
    uk, idx, cnt = np.unique(key, return_index=True, return_counts=True)
    bfaces = faces[idx[cnt == 1]]
    gi = bfaces % (nx + 1)
    gj = (bfaces // (nx + 1)) % (ny + 1)
    gk = bfaces // ((nx + 1) * (ny + 1))
    tags = np.zeros(bfaces.shape[0], dtype=np.int32)
    xpl = (gi[:, 0] == gi[:, 1]) & (gi[:, 1] == gi[:, 2])
    ypl = (gj[:, 0] == gj[:, 1]) & (gj[:, 1] == gj[:, 2])
    zpl = (gk[:, 0] == gk[:, 1]) & (gk[:, 1] == gk[:, 2])
    tags[xpl & ((gi[:, 0] == 0) | (gi[:, 0] == nx))] = 2
    tags[xpl & (gi[:, 0] != 0) & (gi[:, 0] != nx)] = 4
    tags[ypl] = 3
    tags[zpl & (gk[:, 0] == 0)] = 1
    tags[zpl & (gk[:, 0] == nz)] = 5
    tags[zpl & (gk[:, 0] == kz_sub)] = 6
    assert np.all(tags > 0), "untagged boundary face in generator"

    Zn, Yn, Xn = np.meshgrid(zs, ys, xs, indexing="ij")
    nodes_all = np.stack([Xn.ravel(), Yn.ravel(), Zn.ravel()], axis=1)
    used = np.unique(tets)
    remap = -np.ones(nn, dtype=np.int64)
    remap[used] = np.arange(used.size)
    nodes = nodes_all[used].copy()
    tets = remap[tets]
    bfaces = remap[bfaces]

    on_bnd = np.zeros(nodes.shape[0], dtype=bool)
    on_bnd[bfaces.ravel()] = True
    ui = used % (nx + 1)
    uj = (used // (nx + 1)) % (ny + 1)
    uk_ = used // ((nx + 1) * (ny + 1))
    hloc = np.stack([_local_spacing(xs)[ui], _local_spacing(ys)[uj], _local_spacing(zs)[uk_]], 1)
    off = rng.uniform(-jitter, jitter, size=nodes.shape) * hloc
    off[on_bnd] = 0.0
    nodes += off
    return Mesh(3, nodes, TET, tets, bfaces, tags,
                meta=dict(kind="finfet3d_tets", h=h, seed=seed, jitter=jitter, sub_x=sub_x,
                          sub_y=sub_y, sub_z=sub_z, fin_w=fin_w, fin_h=fin_h,
                          fin_cell=fin_cell))


def twisted_ring_tets(n_ring: int = 12, n_rad: int = 2, n_ax: int = 2, r0: float = 20e-9, r1: float = 40e-9,
                      H: float = 20e-9, twist: float = 0.5) -> Mesh:
    """An annulus ``r0 <= r <= r1``, ``0 <= z <= H`` whose node layers are
    turned about the z axis in proportion to height (``twist`` radians from
    bottom to top), meshed by the Kuhn split of its (ring, radius, height)
    index grid.  The faces between ring neighbours lean along the ring, so a
    direction with a z component crosses them all in the same turning sense:
    the upwind graph of such directions has cycles around the ring, while the
    mesh stays conforming and untangled.

    Tags: 1 inner wall (r = r0), 2 outer wall (r = r1), 3 bottom (z = 0),
    4 top (z = H).
    """
    def nid(i, j, k):
        return (k * (n_rad + 1) + j) * n_ring + (i % n_ring)

    kk, jj, ii = np.meshgrid(np.arange(n_ax + 1), np.arange(n_rad + 1), np.arange(n_ring), indexing="ij")
    th = 2.0 * np.pi * ii / n_ring + twist * kk / n_ax
    r = r0 + (r1 - r0) * jj / n_rad
    nodes = np.stack([(r * np.cos(th)).ravel(), (r * np.sin(th)).ravel(), (H * kk / n_ax).ravel()], axis=1)
    I, J, K = np.meshgrid(np.arange(n_ring), np.arange(n_rad), np.arange(n_ax), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    tets = np.stack([np.stack([nid(I + p[0], J + p[1], K + p[2]) for p in path], 1) for path in _KUHN], 1)
    tets = tets.reshape(-1, 4).astype(np.int64)
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    faces = np.sort(tets[:, loc].reshape(-1, 3), axis=1)
    _, idx, cnt = np.unique(faces, axis=0, return_index=True, return_counts=True)
    bfaces = faces[idx[cnt == 1]]
    gj = (bfaces // n_ring) % (n_rad + 1)
    gk = bfaces // (n_ring * (n_rad + 1))
    tags = np.zeros(bfaces.shape[0], dtype=np.int32)
    tags[np.all(gj == 0, axis=1)] = 1
    tags[np.all(gj == n_rad, axis=1)] = 2
    tags[np.all(gk == 0, axis=1)] = 3
    tags[np.all(gk == n_ax, axis=1)] = 4
    assert np.all(tags > 0), "untagged boundary face in generator"
    return Mesh(3, nodes, TET, tets, bfaces.astype(np.int64), tags,
                meta=dict(kind="twisted_ring_tets", n_ring=n_ring, n_rad=n_rad, n_ax=n_ax, r0=r0, r1=r1, H=H,
                          twist=twist))
