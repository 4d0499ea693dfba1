"""The oracle's one-task entry points (used for sampled parity on meshes too
large for a full oracle iteration) against its full transport pass."""
import numpy as np

from oracle import OracleSolver
from cases import CASES, tets_cyclic


def test_incoming_band_and_solve_task_match_full_pass():
    for name in ("fin2d_mixed", "fin3d_tets"):
        p = CASES[name]()
        o = OracleSolver(p)
        rng = np.random.default_rng(5)
        T = rng.uniform(-1.0, 1.0, o.N)
        eb = rng.uniform(0.0, 1.0, (o.bcells.size, o.B, o.D)) * (o.C / o.W)[None, :, None]
        e_in = o.incoming(eb)
        tasks = [(0, 0), (o.D // 2, o.B - 1), (o.D - 1, o.B // 2)]
        full = o.sweep(T, eb, store_e=True, tasks=tasks)
        for (i, l) in tasks:
            eib = o.incoming_band(eb[:, l, :], l)
            assert np.allclose(eib, e_in[:, l, :], rtol=1e-14, atol=0.0)
            e = o.solve_task(T, eib, i, l)
            ref = full["e"][:, l, i]
            assert np.abs(e - ref).max() <= 1e-13 * np.abs(ref).max()


def _upwind_edges(o, i):
    """(upstream, downstream) cell pairs of direction i: across every
    interior face, from the cell the flow leaves to the cell it enters."""
    g = o.g
    a = g.hf_An @ o.s[i]
    m = (a < 0) & (g.hf_nb >= 0)
    return g.hf_nb[m], g.hf_cell[m]


def test_upwind_order_is_topological():
    """The order the oracle factorises in places every cell after each
    upstream neighbour, on every cell type."""
    for name in ("square_mixed", "fin2d_mixed", "fin3d_tets", "cube_hex"):
        o = OracleSolver(CASES[name]())
        for i in range(o.D):
            order = o.upwind_order(i)
            assert order is not None and np.array_equal(np.sort(order), np.arange(o.N))
            pos = np.empty(o.N, dtype=np.int64)
            pos[order] = np.arange(o.N)
            up, dn = _upwind_edges(o, i)
            assert np.all(pos[up] < pos[dn]), (name, i)


def test_ordered_factorisation_solves_the_task_system():
    """The task system of Eq. (13) solved in the upwind order agrees with a
    sparse LU in SuperLU's own ordering and leaves a rounding-level
    residual."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    for name in ("fin2d_mixed", "fin3d_tets", "cube_hex"):
        o = OracleSolver(CASES[name]())
        rng = np.random.default_rng(2)
        for (i, l) in [(0, 0), (o.D // 2, o.B - 1)]:
            A = (sp.identity(o.N, format="csc") / o.tau[l] + o.v[l] * o._direction(i)[0]).tocsc()
            b = rng.standard_normal(o.N)
            e = o._factor(i, l).solve(b)
            ref = spla.splu(A).solve(b)
            assert np.abs(e - ref).max() <= 1e-13 * np.abs(ref).max()
            assert np.abs(A @ e - b).max() <= 1e-13 * np.abs(b).max()


def test_cyclic_mesh_has_upwind_cycles_and_is_solved_exactly():
    """The twisted annulus of the cycle-breaking test: the mesh is untangled
    (the two sides of every interior face see opposite face vectors), a
    cycle exists in the upwind graph of many directions (found by networkx,
    an independent graph search, with every face on it crossed at a visible
    angle), the oracle finds a topological order exactly for the others, and
    its sparse LU solves the task system of a cyclic direction to rounding."""
    import networkx as nx
    import scipy.sparse as sp
    p = tets_cyclic()
    o = OracleSolver(p)
    g = o.g
    twin = {(c, nb): h for h, (c, nb) in enumerate(zip(g.hf_cell.tolist(), g.hf_nb.tolist())) if nb >= 0}
    area = np.linalg.norm(g.hf_An, axis=1)
    for (c, nb), h in twin.items():
        assert np.linalg.norm(g.hf_An[h] + g.hf_An[twin[(nb, c)]]) <= 1e-12 * area[h]
    cyclic = []
    for i in range(o.D):
        up, dn = _upwind_edges(o, i)
        G = nx.DiGraph()
        G.add_edges_from(zip(up.tolist(), dn.tolist()))
        try:
            cyc = nx.find_cycle(G)
        except nx.NetworkXNoCycle:
            cyc = []
        if cyc:
            cyclic.append(i)
            assert len(cyc) >= 3
            a = g.hf_An @ o.s[i]
            for (u, d) in cyc:       # every face on the cycle carries a visible flux
                h = twin[(d, u)]
                assert a[h] < -1e-3 * area[h]
            assert o.upwind_order(i) is None
        else:
            assert o.upwind_order(i) is not None
    assert len(cyclic) >= o.D // 4, cyclic
    i, l = cyclic[0], 1
    A = (sp.identity(o.N, format="csc") / o.tau[l] + o.v[l] * o._direction(i)[0]).tocsc()
    b = np.random.default_rng(4).standard_normal(o.N)
    e = o._factor(i, l).solve(b)
    assert np.abs(A @ e - b).max() <= 1e-12 * np.abs(b).max()
