"""Plain FP64 reference of the steady non-gray BTE iteration (oracle; tests only).

All temperatures are carried as deviations ``T' = T - T_ref`` and all energy
densities as ``e' = e - C T_ref / W``; the equations are linear, so this is the
same problem written around the reference state of Sec. III A.

Per outer iteration ``n`` (Sec. II, Eq. (6) for the sequential scheme,
Eq. (12) for the synthetic one):

1. for every (band l, direction i) task solve the first-order upwind
   finite-volume form of Eq. (4),
   ``v_l sum_f (s_i . An_f) e~_f + V_c e_c / tau_l = V_c (C_l T'_c / (W tau_l) + S_cl)``
   with ``e~_f`` the upwind value (own cell on outflow faces, the neighbour or
   the wall's incoming value on inflow faces) and ``S_cl = Qdot_c C_l/(C_tot W)``
   (heat source as an equilibrium source, uniform over directions, split by
   heat capacity: Sec. III B).  The matrix ``I/tau_l + v_l K_i`` (Eq. (13))
   is factorised once and reused;
2. the moments ``N_L = sum_l (1/tau_l) sum_i w_i e'`` (Eq. (5)),
   ``E = sum_l sum_i w_i e'`` and ``q = sum_l sum_i w_i v_l s_i e'`` (Eq. (7));
3. sequential: ``T'^{n+1} = N_L / beta`` with ``beta = sum_l C_l / tau_l``;
   synthetic: ``T'^{n+1} = T'_L + delta`` with
   ``L delta = V beta (T'_L - T'^n)`` (Eqs. (8)-(10) with the gradient term of
   Eq. (9) taken at the kinetic temperature of the new distribution, i.e. the
   diffusion-synthetic form); the literal form ``T'^{n+1} = T'^n + delta`` is
   available as ``scheme="synthetic_literal"``.

Wall values for the next iteration come from the distribution at the wall
cell after this sweep (lagged coupling across directions); after a synthetic
update that distribution is shifted by the equilibrium part of the correction,
``C_l (T'^{n+1} - T'_L) / W``, so the lag does not re-inject the uncorrected
state (without this the diffusion correction diverges next to reflecting
walls):

* thermalizing: ``e'_in = C_l T'_w / W``;
* diffuse: ``e'_in = sum_{j: s_j.n>0} w_j (s_j.n) e'_j / sum_{k: s_k.n<0} w_k |s_k.n|``
  (zero net flux, isotropic re-emission);
* specular: ``e'_in(i) = e'(R(i))`` with ``R(i)`` the direction nearest to the
  mirror image ``s_i - 2 (s_i.n) n`` (lowest index on ties);
* partially specular with specularity ``p``: ``p * specular + (1 - p) * diffuse``.

At iteration 0 the "previous" distribution at the walls is the equilibrium
``C_l T'^0_c / W`` of the initial temperature.

Second-order upwind (``order=2``) adds to step 1 the linear reconstruction of
every interior face value from its upwind cell, with the least-squares
gradient of the previous sweep's distribution (none before the first sweep):
a right-hand-side correction of the same factorised system, the
deferred-correction form of the paper's precomputed gradient operators
(Sec. II).  Wall faces keep the cell value.
"""
from __future__ import annotations

import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .geometry import build_geometry

THERMALIZING, DIFFUSE, SPECULAR, PARTIAL = 0, 1, 2, 3


class _OrderedSystem:
    """``A = I/tau + v K`` of one (band, direction) task whose upwind graph is
    acyclic, held as the permutation ``order`` (a topological order of the
    graph) and ``Kp = K[order][:, order]`` (lower triangular).  ``solve``
    returns ``A^{-1} rhs`` in the original cell order."""

    def __init__(self, order, Kp, inv_tau, v):
        self.order, self.Kp, self.inv_tau, self.v = order, Kp, inv_tau, v

    def solve(self, rhs):
        n = self.order.size
        A = (sp.identity(n, format="csc") * self.inv_tau + self.Kp * self.v).tocsc()
        x = spla.spsolve_triangular(A, rhs[self.order], lower=True, overwrite_A=True)
        e = np.empty_like(x)
        e[self.order] = x
        return e


def quadrature_moments(s, w):
    """Zeroth, first and second moments of a direction set (pin: Eq. (11)'s W)."""
    s = np.asarray(s, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    return w.sum(), (w[:, None] * s).sum(0), np.einsum("i,ij,ik->jk", w, s, s)


class OracleSolver:
    """FP64 CPU reference solver for one problem (see module docstring)."""

    def __init__(self, problem):
        self.p = problem
        g = build_geometry(problem.mesh)
        self.g = g
        d = g.dim
        self.dim = d
        self.N = g.n_cells
        self.s3 = np.asarray(problem.s, dtype=np.float64)
        self.s = self.s3[:, :d]                      # in-domain components
        self.w = np.asarray(problem.w, dtype=np.float64)
        self.D = self.w.size
        self.W = float(self.w.sum())                 # W_Omega of Eq. (11)
        self.C = np.asarray(problem.C, dtype=np.float64)
        self.v = np.asarray(problem.v, dtype=np.float64)
        self.tau = np.asarray(problem.tau, dtype=np.float64)
        self.B = self.C.size
        self.beta = float(np.sum(self.C / self.tau))  # denominator of Eq. (5)
        self.Ctot = float(self.C.sum())
        self.T_ref = float(problem.T_ref)
        Q = problem.Q if problem.Q is not None else np.zeros(self.N)
        self.Qdot = np.asarray(Q, dtype=np.float64)

        # ---------------- boundary bookkeeping
        bcs = {b.tag: b for b in problem.boundaries}
        self.bhf = np.where(g.hf_nb < 0)[0]                 # boundary half-faces
        tags = g.hf_tag[self.bhf]
        for t in np.unique(tags):
            if int(t) not in bcs:
                raise ValueError(f"boundary tag {t} has no condition")
        self.btype = np.array([bcs[int(t)].type for t in tags], dtype=np.int64)
        self.bTw = np.array([bcs[int(t)].T_wall - self.T_ref for t in tags])
        self.bp = np.array([bcs[int(t)].specularity for t in tags])
        if not np.any(self.btype == THERMALIZING):
            raise ValueError("no thermalizing wall: the steady problem has no unique solution")
        self.bcell_of_hf = g.hf_cell[self.bhf]
        self.bcells, self.bidx = np.unique(self.bcell_of_hf, return_inverse=True)
        An_b = g.hf_An[self.bhf]
        self.bn = An_b / np.linalg.norm(An_b, axis=1, keepdims=True)   # unit normals
        sn = self.bn @ self.s.T                                           # (nb, D)
        self.b_sn = sn
        self.b_denom = np.sum(np.where(sn < 0, -sn, 0.0) * self.w[None, :], axis=1)
        # mirror map for every boundary half-face and direction
        n3 = np.zeros((self.bhf.size, 3))
        n3[:, :d] = self.bn
        self.R = np.zeros((self.bhf.size, self.D), dtype=np.int64)
        keyn = np.round(n3, 12)
        un, inv = np.unique(keyn, axis=0, return_inverse=True)
        for u in range(un.shape[0]):
            rows = np.where(inv.ravel() == u)[0]
            nn = n3[rows[0]]
            mirror = self.s3 - 2.0 * (self.s3 @ nn)[:, None] * nn[None, :]
            dist = np.sum((mirror[:, None, :] - self.s3[None, :, :]) ** 2, axis=2)
            self.R[rows] = np.argmin(dist, axis=1)[None, :]

        # per-direction unit advection operators K_i (Eq. (13)), built on
        # first use (see _direction)
        self._dir = {}
        self._lu = {}
        self._order = {}
        self._ordered = {}
        self._S = None
        self._lap = None

    def _direction(self, i):
        """K_i of Eq. (13) for direction i, and its inflow boundary half-faces
        with their coefficients |s_i . An| / V.  K_i e = sum over outflow faces
        (s.An/V) e_cell + sum over interior inflow faces (s.An/V) e_neighbour."""
        got = self._dir.get(i)
        if got is not None:
            return got
        g = self.g
        Vc = g.V[g.hf_cell]
        interior = g.hf_nb >= 0
        a = g.hf_An @ self.s[i]
        out = a > 0
        diag = np.bincount(g.hf_cell[out], weights=a[out] / Vc[out], minlength=self.N)
        m = (a < 0) & interior
        K = sp.coo_matrix((a[m] / Vc[m], (g.hf_cell[m], g.hf_nb[m])), shape=(self.N, self.N))
        K = (K + sp.diags(diag)).tocsc()
        ab = a[self.bhf]
        bi = np.where(ab < 0)[0]                 # inflow boundary half-faces
        got = (K, (bi, -ab[bi] / g.V[self.bcell_of_hf[bi]]))
        self._dir[i] = got
        return got

    # ------------------------------------------------------------------ pieces
    def source(self):
        """S_cl = Qdot_c C_l / (C_tot W) (Sec. III B)."""
        if self._S is None:
            self._S = self.Qdot[:, None] * (self.C / (self.Ctot * self.W))[None, :]
        return self._S

    def equilibrium_walls(self, Tdev):
        """Wall-cell distribution at equilibrium with ``Tdev`` (iteration-0 state)."""
        eb = np.empty((self.bcells.size, self.B, self.D))
        eb[:] = (Tdev[self.bcells][:, None] * self.C[None, :] / self.W)[:, :, None]
        return eb

    def incoming(self, eb_prev):
        """Incoming wall values e'_in[h, l, i] for every boundary half-face (all i;
        only inflow directions are used)."""
        nb = self.bhf.size
        e_cell = eb_prev[self.bidx]                               # (nb, B, D)
        sn = self.b_sn
        outw = np.where(sn > 0, sn, 0.0) * self.w[None, :]          # (nb, D)
        diff = np.einsum("hld,hd->hl", e_cell, outw) / self.b_denom[:, None]
        spec = np.take_along_axis(e_cell, self.R[:, None, :].repeat(self.B, axis=1), axis=2)
        therm = (self.bTw[:, None] * self.C[None, :] / self.W)
        e_in = np.empty((nb, self.B, self.D))
        t = self.btype
        e_in[t == THERMALIZING] = therm[t == THERMALIZING][:, :, None]
        e_in[t == DIFFUSE] = diff[t == DIFFUSE][:, :, None]
        e_in[t == SPECULAR] = spec[t == SPECULAR]
        pm = t == PARTIAL
        p = self.bp[pm][:, None, None]
        e_in[pm] = p * spec[pm] + (1.0 - p) * diff[pm][:, :, None]
        return e_in

    def incoming_band(self, eb_band, l):
        """The same incoming wall values as :meth:`incoming`, for band l only:
        ``eb_band`` is the wall-cell distribution of band l, shape (cells, D);
        returns (boundary half-faces, D).  Lets a single task be checked on a
        mesh whose full (cells, B, D) wall array would not fit in memory."""
        e_cell = eb_band[self.bidx]                                # (nb, D)
        sn = self.b_sn
        outw = np.where(sn > 0, sn, 0.0) * self.w[None, :]
        diff = np.sum(e_cell * outw, axis=1) / self.b_denom       # (nb,)
        spec = np.take_along_axis(e_cell, self.R, axis=1)         # (nb, D)
        t = self.btype
        e_in = np.empty((self.bhf.size, self.D))
        th = t == THERMALIZING
        e_in[th] = (self.bTw[th] * self.C[l] / self.W)[:, None]
        df = t == DIFFUSE
        e_in[df] = diff[df][:, None]
        e_in[t == SPECULAR] = spec[t == SPECULAR]
        pm = t == PARTIAL
        p = self.bp[pm][:, None]
        e_in[pm] = p * spec[pm] + (1.0 - p) * diff[pm][:, None]
        return e_in

    def solve_task(self, Tdev, e_in_band, i, l, e_prev=None):
        """e'_{l i} over all cells: the transport solve of one (band,
        direction) task of Eq. (4) from the temperature deviation ``Tdev`` and
        band l's incoming wall values (as returned by :meth:`incoming_band`).
        With ``e_prev`` (the task's previous distribution over all cells) the
        face values are second order (:meth:`second_order_source`)."""
        bi, coef = self._direction(i)[1]
        rhs = self.C[l] * Tdev / (self.W * self.tau[l]) + self.source()[:, l]
        rhs += self.v[l] * np.bincount(self.bcell_of_hf[bi], weights=coef * e_in_band[bi, i], minlength=self.N)
        if e_prev is not None:
            rhs += self.v[l] * self.second_order_source(e_prev, i)
        return self._factor(i, l).solve(rhs)

    # ------------------------------------------------------ second-order upwind
    def lsq_operator(self):
        """Per cell, the matrix P_c of the least-squares gradient over the
        cell's face neighbours: grad e_c = P_c sum_m r_m (e_m - e_c) with
        r_m = x_m - x_c.  P_c is the pseudo-inverse of M_c = sum_m r_m r_m^T
        (eigenvalues at or below 1e-9 of the largest are dropped, so
        neighbours spanning only a line or a plane give the gradient within
        that subspace).  A cell with fewer than dim + 1 face neighbours (a
        wall triangle or tetrahedron, a corner quadrilateral or hexahedron)
        gets no gradient: its stencil would be exactly determined, and such
        extrapolations make the lagged correction grow from one iteration to
        the next on coarse unstructured meshes in the ballistic limit."""
        if getattr(self, "_lsq_P", None) is not None:
            return self._lsq_P
        g = self.g
        m = g.hf_nb >= 0
        r = g.xc[g.hf_nb[m]] - g.xc[g.hf_cell[m]]
        M = np.zeros((self.N, self.dim, self.dim))
        np.add.at(M, g.hf_cell[m], r[:, :, None] * r[:, None, :])
        lam, U = np.linalg.eigh(M)
        keep = lam > 1e-9 * lam.max(axis=1, keepdims=True)
        inv = np.where(keep, 1.0 / np.where(keep, lam, 1.0), 0.0)
        P = np.einsum("cij,cj,ckj->cik", U, inv, U)
        P[np.bincount(g.hf_cell[m], minlength=self.N) < self.dim + 1] = 0.0
        self._lsq_P = P
        return self._lsq_P

    def gradient(self, e):
        """Least-squares cell gradients (N, dim) of a cell field e."""
        g = self.g
        m = g.hf_nb >= 0
        c, nb = g.hf_cell[m], g.hf_nb[m]
        b = np.zeros((self.N, self.dim))
        np.add.at(b, c, (g.xc[nb] - g.xc[c]) * (e[nb] - e[c])[:, None])
        return np.einsum("cij,cj->ci", self.lsq_operator(), b)

    def second_order_source(self, e, i):
        """Extra right-hand side of the second-order upwind balance for
        direction i, from the previous distribution e of the task.

        On every interior face the upwind value is reconstructed linearly
        from the upwind cell u: e~_f = e_u + grad e_u . (x_f - x_u), with the
        gradient of the previous iteration (deferred correction); wall faces
        keep the cell value, so the wall coupling and the energy balance are
        those of the first-order scheme.  The first-order part stays in the
        factorised operator of Eq. (13); the increment moves to the right:
        -sum_f (s_i . An_f / V_c) grad e_u . (x_f - x_u)."""
        g = self.g
        m = np.where(g.hf_nb >= 0)[0]
        a = g.hf_An[m] @ self.s[i]
        u = np.where(a > 0, g.hf_cell[m], g.hf_nb[m])
        grad = self.gradient(e)
        inc = np.sum(grad[u] * (g.hf_xf[m] - g.xc[u]), axis=1)
        return -np.bincount(g.hf_cell[m], weights=a * inc / g.V[g.hf_cell[m]], minlength=self.N)

    def upwind_order(self, i):
        """A topological order of direction i's upwind graph (every cell after
        the neighbours it receives from across an inflow face), or None when
        the graph has a cycle.  Kahn's algorithm: repeatedly take every cell
        whose upstream neighbours are all placed."""
        got = self._order.get(i)
        if got is not None or i in self._order:
            return got
        g = self.g
        a = g.hf_An @ self.s[i]
        m = (a < 0) & (g.hf_nb >= 0)
        dn, up = g.hf_cell[m], g.hf_nb[m]          # edge up -> dn
        indeg = np.bincount(dn, minlength=self.N)
        srt = np.argsort(up, kind="stable")
        dn_by_up = dn[srt]
        ptr = np.searchsorted(up[srt], np.arange(self.N + 1))
        placed = []
        front = np.flatnonzero(indeg == 0)
        while front.size:
            placed.append(front)
            lens = ptr[front + 1] - ptr[front]
            tot = int(lens.sum())
            if tot == 0:
                break
            first = np.repeat(ptr[front] - np.concatenate(([0], np.cumsum(lens)[:-1])), lens)
            reached, cnt = np.unique(dn_by_up[first + np.arange(tot)], return_counts=True)
            indeg[reached] -= cnt
            front = reached[indeg[reached] == 0]
        order = np.concatenate(placed) if placed else np.zeros(0, dtype=np.int64)
        got = order if order.size == self.N else None
        self._order[i] = got
        return got

    def forget_direction(self, i):
        """Drop what was cached for direction i (its advection operator,
        upwind order and factorisations); they are rebuilt on next use."""
        self._dir.pop(i, None)
        self._order.pop(i, None)
        self._ordered.pop(i, None)
        for key in [k for k in self._lu if k[0] == i]:
            del self._lu[key]

    def _factor(self, i, l):
        """The factorised system ``I/tau_l + v_l K_i`` of Eq. (13), as an object
        with ``solve(rhs)``.

        When direction i's upwind graph is acyclic, the system permuted to
        the graph's topological order is lower triangular, so its LU factors
        are read off with no fill (L the permuted matrix scaled to a unit
        diagonal, U its diagonal; SciPy's triangular solve); the permutation
        is only a fill-free ordering of the same unknowns.  Otherwise (an
        upwind cycle) the matrix is factorised by ``splu``."""
        key = (i, l)
        lu = self._lu.get(key)
        if lu is not None:
            return lu
        order = self.upwind_order(i)
        if order is None:
            A = (sp.identity(self.N, format="csc") / self.tau[l] + self.v[l] * self._direction(i)[0]).tocsc()
            lu = spla.splu(A)
            self._lu[key] = lu
            return lu
        Kp = self._ordered.get(i)
        if Kp is None:
            Kp = self._direction(i)[0].tocsr()[order][:, order].tocsc()
            if sp.triu(Kp, 1).nnz != 0:
                raise AssertionError("upwind order does not make K_i lower triangular")
            self._ordered[i] = Kp
        return _OrderedSystem(order, Kp, 1.0 / self.tau[l], self.v[l])

    def sweep(self, Tdev, eb_prev, store_e=False, tasks=None, e_prev=None, e_in=None, eb_dirs=None):
        """One transport pass over every (band, direction) task of Eq. (4).

        Returns the moments of the new distribution, its values at the wall
        cells (for the next iteration's wall coupling), the incoming wall
        values that were used, and optionally the full distribution.  With
        ``e_prev`` (N, B, D), the previous distribution, the interior face
        values are second order (:meth:`second_order_source`).

        A pass may be split over several callers by task: ``tasks`` lists the
        (direction, band) pairs to solve (the moments are then those tasks'
        terms), ``e_in`` supplies the incoming wall values instead of
        computing them from ``eb_prev`` (any object indexed as
        ``e_in[half_faces, band, direction]``), and ``eb_dirs`` lists the
        directions whose wall-cell values are returned (the last axis of
        ``eb``)."""
        if e_in is None:
            e_in = self.incoming(eb_prev)
        S = self.source()
        NL = np.zeros(self.N)
        E = np.zeros(self.N)
        q = np.zeros((self.N, self.dim))
        col = {i: k for k, i in enumerate(eb_dirs)} if eb_dirs is not None else None
        eb_new = np.empty((self.bcells.size, self.B, self.D if col is None else len(col)))
        e_all = np.zeros((self.N, self.B, self.D)) if store_e else None
        todo = tasks if tasks is not None else [(i, l) for i in range(self.D) for l in range(self.B)]
        for (i, l) in todo:
            bi, coef = self._direction(i)[1]
            rhs = self.C[l] * Tdev / (self.W * self.tau[l]) + S[:, l]
            rhs += self.v[l] * np.bincount(self.bcell_of_hf[bi], weights=coef * e_in[bi, l, i],
                                           minlength=self.N)
            if e_prev is not None:
                rhs += self.v[l] * self.second_order_source(e_prev[:, l, i], i)
            e = self._factor(i, l).solve(rhs)
            NL += self.w[i] * e / self.tau[l]
            E += self.w[i] * e
            q += (self.w[i] * self.v[l] * e)[:, None] * self.s[i][None, :]
            eb_new[:, l, i if col is None else col[i]] = e[self.bcells]
            if store_e:
                e_all[:, l, i] = e
        return dict(NL=NL, E=E, q=q, eb=eb_new, e_in=e_in, e=e_all)

    def kappa_bulk(self):
        """kappa = sum_l C_l v_l^2 tau_l * (1/dim) sum_i w_i |s_i|^2 / W (in-domain s)."""
        ang = np.sum(self.w * np.sum(self.s ** 2, axis=1)) / (self.dim * self.W)
        return float(np.sum(self.C * self.v ** 2 * self.tau) * ang)

    def numerical_diffusivity(self):
        """Coefficient k1 of ``kappa_f = kappa_bulk + k1 h_f``:
        ``k1 = <|s|> sum_l C_l v_l / 4``."""
        mean_abs = np.sum(self.w[:, None] * np.abs(self.s)) / (self.dim * self.W)
        return float(0.25 * mean_abs * np.sum(self.C * self.v))

    def laplacian(self):
        """Integrated TPFA operator ``(L d)_c = sum_f g_f (d_c - d_nb)`` of the
        synthetic correction (Eq. (10)).

        ``g_f = kappa_f |An_f| / d_f`` with ``d_f = |(x_nb - x_c) . n_f|``; on
        thermalizing walls ``d = 0`` at the face (``d_f = |(x_f - x_c) . n_f|``,
        cell width ``2 d_f``); other walls carry no diffusive flux.

        ``kappa_f = kappa_bulk + (h_f / 4) <|s|> sum_l C_l v_l`` with ``h_f`` the
        cell width across the face and ``<|s|> = sum_i w_i sum_k |s_ik| /
        (dim W)``: the bulk conductivity of Eq. (8) plus half the numerical
        diffusivity of the first-order upwind flux (C v h <|s.n|> / 2).  Without
        the second term the correction over-shoots on cells thicker than the
        mean free path, where the discrete transport is more diffusive than
        kappa_bulk, and the iteration diverges; the term only changes the rate,
        never the fixed point."""
        if self._lap is not None:
            return self._lap
        g = self.g
        kap = self.kappa_bulk()
        k1 = self.numerical_diffusivity()
        area = np.linalg.norm(g.hf_An, axis=1)
        n = g.hf_An / area[:, None]
        rows, cols, vals = [], [], []
        diag = np.zeros(self.N)
        m = g.hf_nb >= 0
        dist = np.abs(np.sum((g.xc[g.hf_nb[m]] - g.xc[g.hf_cell[m]]) * n[m], axis=1))
        gf = (kap + k1 * dist) * area[m] / dist
        np.add.at(diag, g.hf_cell[m], gf)
        rows.append(g.hf_cell[m]); cols.append(g.hf_nb[m]); vals.append(-gf)
        th = self.bhf[self.btype == THERMALIZING]
        dist = np.abs(np.sum((g.hf_xf[th] - g.xc[g.hf_cell[th]]) * n[th], axis=1))
        np.add.at(diag, g.hf_cell[th], (kap + k1 * 2.0 * dist) * area[th] / dist)
        L = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.N, self.N)) + sp.diags(diag)
        # a symmetric fill-reducing ordering (the operator is symmetric)
        self._lap = spla.splu(L.tocsc(), permc_spec="MMD_AT_PLUS_A")
        self._lap_matrix = L.tocsr()
        return self._lap

    def fourier_guess(self):
        """Initial temperature deviation from the diffusion limit (the
        Fourier solution the paper starts from, Sec. IV): ``L T' = Qdot V +
        sum over thermalizing faces g_f T'_w``, the same TPFA operator as the
        synthetic correction (:meth:`laplacian`) with the thermalizing wall
        temperatures as Dirichlet data; other walls carry no flux.  Only the
        starting point changes, never the fixed point."""
        g = self.g
        lap = self.laplacian()
        kap = self.kappa_bulk()
        k1 = self.numerical_diffusivity()
        area = np.linalg.norm(g.hf_An, axis=1)
        n = g.hf_An / area[:, None]
        sel = self.btype == THERMALIZING
        th = self.bhf[sel]
        dist = np.abs(np.sum((g.hf_xf[th] - g.xc[g.hf_cell[th]]) * n[th], axis=1))
        gf = (kap + k1 * 2.0 * dist) * area[th] / dist
        rhs = self.Qdot * g.V + np.bincount(g.hf_cell[th], weights=gf * self.bTw[sel], minlength=self.N)
        return lap.solve(rhs)

    def wall_flux(self, eb, e_in):
        """Net outward heat flow through each boundary tag,
        sum_l sum_i w_i v_l (s_i . An_f) e~_f over the tag's faces."""
        g = self.g
        a = g.hf_An[self.bhf] @ self.s.T                          # (nb, D)
        e_cell = eb[self.bidx]                                    # (nb, B, D)
        et = np.where((a > 0)[:, None, :], e_cell, e_in)
        flow = np.einsum("hld,hd,l->h", et, a * self.w[None, :], self.v)
        tags = g.hf_tag[self.bhf]
        return {int(t): float(flow[tags == t].sum()) for t in np.unique(tags)}

    def face_divergence(self, e_all, e_in):
        """Per-cell upwind face-flux divergence sum_f F_f of the full distribution."""
        g = self.g
        div = np.zeros(self.N)
        wv = self.w[None, :] * self.v[:, None]                    # (B, D)
        for h in range(g.hf_cell.size):
            c = g.hf_cell[h]
            a = self.s @ g.hf_An[h]                               # (D,)
            nb = g.hf_nb[h]
            if nb >= 0:
                up = np.where(a[None, :] > 0, e_all[c], e_all[nb])
            else:
                k = np.searchsorted(self.bhf, h)
                up = np.where(a[None, :] > 0, e_all[c], e_in[k])
            div[c] += np.sum(wv * a[None, :] * up)
        return div

    # ---------------------------------------------------------- iteration loop
    def solve(self, scheme=None, tol=None, max_iter=None, n_iter=None, T_init=None, init="tref",
              store_e=False, verbose=False, order=1, sweep=None, callback=None):
        """Run the outer iteration.

        ``n_iter`` runs exactly that many sweeps (no convergence test);
        otherwise iterate until ``r = |T'^{n+1} - T'^n|_inf / |T'^{n+1}|_inf < tol``.
        ``init="fourier"`` starts from :meth:`fourier_guess` (walls at
        equilibrium with it) instead of T_init / T_ref.  ``order=2`` uses
        second-order upwind face values, each sweep reconstructing from the
        distribution of the sweep before it (none before the first sweep).
        ``sweep`` replaces :meth:`sweep` (same arguments and result), e.g. by
        one that splits the pass over processes by task.  ``callback``, if
        given, is called after every iteration with its number, the new
        temperature, the kinetic temperature and the sweep's heat flux.
        Returned temperatures are absolute (K)."""
        sweep = sweep or self.sweep
        if order not in (1, 2):
            raise ValueError(order)
        scheme = scheme or self.p.scheme
        tol = self.p.tol if tol is None else tol
        max_iter = self.p.max_iter if max_iter is None else max_iter
        if init == "fourier":
            T = self.fourier_guess()
        elif init == "tref":
            T = np.zeros(self.N) if T_init is None else np.asarray(T_init, dtype=np.float64) - self.T_ref
        else:
            raise ValueError(init)
        eb = self.equilibrium_walls(T)
        hist = []
        it = 0
        t0 = time.perf_counter()
        limit = n_iter if n_iter is not None else max_iter
        out = None
        TL = T
        e_prev = None
        while it < limit:
            out = sweep(T, eb, store_e=store_e or order == 2, e_prev=e_prev)
            if order == 2:
                e_prev = out["e"]
            TL = out["NL"] / self.beta
            if scheme == "sequential":
                Tn = TL
            elif scheme in ("synthetic", "synthetic_literal"):
                rhs = self.g.V * self.beta * (TL - T)
                delta = self.laplacian().solve(rhs)
                Tn = (TL if scheme == "synthetic" else T) + delta
            else:
                raise ValueError(scheme)
            r = np.max(np.abs(Tn - T)) / max(np.max(np.abs(Tn)), 1e-300)
            hist.append(float(r))
            # the lagged wall distributions take the equilibrium part of the
            # synthetic correction, so the next sweep's reflections start from
            # the corrected state (zero for the sequential scheme)
            eb = out["eb"] + ((Tn - TL)[self.bcells][:, None] * self.C[None, :] / self.W)[:, :, None]
            T = Tn
            it += 1
            if callback is not None:
                callback(it, T + self.T_ref, TL + self.T_ref, out["q"])
            if verbose:
                print(it, r)
            if n_iter is None and r < tol:
                break
        secs = time.perf_counter() - t0
        flux = self.wall_flux(out["eb"], out["e_in"])
        therm_tags = {int(t) for t in np.unique(self.g.hf_tag[self.bhf][self.btype == THERMALIZING])}
        q_total = float(np.sum(self.Qdot * self.g.V))
        out_therm = sum(v for k, v in flux.items() if k in therm_tags)
        scale = max(abs(q_total), sum(abs(v) for v in flux.values()), 1e-300)
        return dict(
            T=T + self.T_ref, T_kinetic=TL + self.T_ref, T_energy=out["E"] / self.Ctot + self.T_ref,
            q=out["q"], iterations=it, residuals=hist, wall_flux=flux, Q_total=q_total,
            energy_imbalance=abs(out_therm - q_total) / scale, seconds=secs,
            e=out["e"], e_in=out["e_in"], eb=out["eb"], converged=bool(hist and hist[-1] < tol))
