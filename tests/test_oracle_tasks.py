"""The oracle's one-task entry points (used for sampled parity on meshes too
large for a full oracle iteration) against its full transport pass."""
import numpy as np

from oracle import OracleSolver
from cases import CASES


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
