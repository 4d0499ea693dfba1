"""Independent dense assembly of the discrete fixed point (test helper).

For tiny inputs the steady problem the iteration converges to is one linear
system in the unknowns ``e'[c, l, i]``: the upwind finite-volume balance of
every (cell, band, direction) with the lattice temperature of the collision
moment substituted in, and every wall value written in terms of the *current*
distribution at its wall cell.  This module writes that system out with plain
loops and its own geometry (it shares no code with ``oracle/``) and solves it
with a dense LAPACK solve.
"""
from __future__ import annotations

import numpy as np

FACES = {
    3: [(0, 1), (1, 2), (2, 0)],
    4: [(0, 1), (1, 2), (2, 3), (3, 0)],
    10: [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)],
    12: [(0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)],
}


def _cell_volume(P, ctype):
    if ctype == 3:
        (x0, y0), (x1, y1), (x2, y2) = P
        return abs((x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)) / 2.0
    if ctype == 4:
        s = 0.0
        for k in range(4):
            s += P[k][0] * P[(k + 1) % 4][1] - P[(k + 1) % 4][0] * P[k][1]
        return abs(s) / 2.0
    if ctype == 10:
        a, b, c, d = (np.asarray(x) for x in P)
        return abs(np.dot(b - a, np.cross(c - a, d - a))) / 6.0
    if ctype == 12:
        # axis-aligned box (the only hexahedra used with this helper)
        P = np.asarray(P)
        ext = P.max(0) - P.min(0)
        return float(ext[0] * ext[1] * ext[2])
    raise ValueError(ctype)


def _face_vector(F, dim):
    F = [np.asarray(x, dtype=float) for x in F]
    if dim == 2:
        t = F[1] - F[0]
        return np.array([t[1], -t[0]])
    if len(F) == 3:
        return 0.5 * np.cross(F[1] - F[0], F[2] - F[0])
    # planar quad: split into two triangles
    return 0.5 * np.cross(F[1] - F[0], F[2] - F[0]) + 0.5 * np.cross(F[2] - F[0], F[3] - F[0])


def faces_of(mesh):
    """List of half-faces (cell, nb or None, An outward, tag or None, face
    centroid)."""
    nodes = mesh.nodes
    out = []
    table = {}
    for c, cell in enumerate(mesh.cells):
        for lf in FACES[mesh.cell_type]:
            key = tuple(sorted(int(cell[k]) for k in lf))
            table.setdefault(key, []).append((c, lf))
    btag = {tuple(sorted(int(x) for x in f)): int(t) for f, t in zip(mesh.bfaces, mesh.btags)}
    for key, owners in table.items():
        for (c, lf) in owners:
            cell = mesh.cells[c]
            F = [nodes[int(cell[k])] for k in lf]
            An = _face_vector(F, mesh.dim)
            xc = np.mean([nodes[int(k)] for k in cell], axis=0)
            xf = np.mean(F, axis=0)
            if np.dot(An, xf - xc) < 0:
                An = -An
            others = [o for o in owners if o[0] != c]
            nb = others[0][0] if others else None
            tag = None if others else btag[key]
            out.append((c, nb, An, tag, xf))
    return out


def lstsq_gradients(mesh, faces):
    """Per cell: (neighbour list, matrix G) with grad e_c = G (e_nb - e_c),
    the minimum-norm least-squares fit of a linear field to the face
    neighbours' values (LAPACK's least-squares solver on the offsets); none
    (G empty) for a cell with fewer than dim + 1 face neighbours."""
    xc = np.array([np.mean([mesh.nodes[int(k)] for k in cell], axis=0) for cell in mesh.cells])
    nbrs = [[] for _ in range(mesh.n_cells)]
    for (c, nb, An, tag, xf) in faces:
        if nb is not None:
            nbrs[c].append(nb)
    out = []
    for c in range(mesh.n_cells):
        if len(nbrs[c]) < mesh.dim + 1:
            out.append(([], np.zeros((mesh.dim, 0))))
            continue
        R = np.array([xc[m] - xc[c] for m in nbrs[c]])
        G = np.linalg.lstsq(R, np.eye(len(nbrs[c])), rcond=1e-6)[0]
        out.append((nbrs[c], G))
    return xc, out


def solve_fixed_point(problem, order=1):
    """Dense solve of the converged discrete problem.  Returns (T_L, q) with
    T_L absolute in K and q of shape (N, dim).  ``order=2``: on interior
    faces the upwind value is e_u + grad e_u . (x_f - x_u) with the
    least-squares gradient of :func:`lstsq_gradients` (at the fixed point the
    lagged gradient equals the current one); wall faces keep the cell value."""
    m = problem.mesh
    dim = m.dim
    N = m.n_cells
    B = problem.C.size
    D = problem.w.size
    s = np.asarray(problem.s, float)
    sd = s[:, :dim]
    w = np.asarray(problem.w, float)
    Wt = w.sum()
    C, v, tau = (np.asarray(x, float) for x in (problem.C, problem.v, problem.tau))
    beta = np.sum(C / tau)
    Ct = C.sum()
    Qd = np.zeros(N) if problem.Q is None else np.asarray(problem.Q, float)
    bcs = {b.tag: b for b in problem.boundaries}
    Vol = np.array([_cell_volume([m.nodes[int(k)] for k in cell], m.cell_type) for cell in m.cells])

    def idx(c, l, i):
        return (c * B + l) * D + i

    n = N * B * D
    A = np.zeros((n, n))
    rhs = np.zeros(n)
    for c in range(N):
        for l in range(B):
            for i in range(D):
                r = idx(c, l, i)
                A[r, r] += Vol[c] / tau[l]
                # - V C_l T'_c /(W tau_l), T'_c = sum_{l',j} w_j e/tau_l' / beta
                for l2 in range(B):
                    for j in range(D):
                        A[r, idx(c, l2, j)] -= Vol[c] * C[l] / (Wt * tau[l]) * w[j] / tau[l2] / beta
                rhs[r] += Vol[c] * Qd[c] * C[l] / (Ct * Wt)
    faces = faces_of(m)
    if order == 2:
        xc, grads = lstsq_gradients(m, faces)
    for (c, nb, An, tag, xf) in faces:
        nrm = An / np.linalg.norm(An)
        n3 = np.zeros(3)
        n3[:dim] = nrm
        for i in range(D):
            a = float(np.dot(sd[i], An))
            for l in range(B):
                r = idx(c, l, i)
                if order == 2 and nb is not None and a != 0:
                    # reconstruction increment grad e_u . (x_f - x_u)
                    u = c if a > 0 else nb
                    nbrs, G = grads[u]
                    wts = (xf - xc[u]) @ G
                    for mk, wk in zip(nbrs, wts):
                        A[r, idx(mk, l, i)] += v[l] * a * wk
                        A[r, idx(u, l, i)] -= v[l] * a * wk
                if a > 0:
                    A[r, r] += v[l] * a
                elif a < 0:
                    if nb is not None:
                        A[r, idx(nb, l, i)] += v[l] * a
                        continue
                    bc = bcs[tag]
                    sn = sd @ nrm
                    den = np.sum(w[sn < 0] * -sn[sn < 0])
                    mirror = s[i] - 2.0 * np.dot(s[i], n3) * n3
                    R = int(np.argmin(np.sum((s - mirror) ** 2, axis=1)))
                    if bc.type == 0:
                        rhs[r] -= v[l] * a * C[l] * (bc.T_wall - problem.T_ref) / Wt
                        continue
                    p = 1.0 if bc.type == 2 else (0.0 if bc.type == 1 else bc.specularity)
                    if p > 0:
                        A[r, idx(c, l, R)] += v[l] * a * p
                    if p < 1:
                        for j in range(D):
                            if sn[j] > 0:
                                A[r, idx(c, l, j)] += v[l] * a * (1 - p) * w[j] * sn[j] / den
    e = np.linalg.solve(A, rhs).reshape(N, B, D)
    TL = np.einsum("cld,d,l->c", e, w, 1.0 / tau) / beta
    q = np.einsum("cld,d,l,dk->ck", e, w, v, sd)
    return TL + problem.T_ref, q
