"""Upwind-graph cycles on the GPU: the twisted annulus of tetrahedra
(cases.tets_cyclic, 288 cells, 32 directions of which 16 have cycles in
their upwind graph).  The planner breaks each cycle by lagging the faces it
cannot order (they take the previous iteration's value), so single
iterations differ from the oracle's exact per-task LU solves; the converged
fields do not: both are the fixed point of Eq. (4) with the walls of Sec. II.
Tolerances as for the other converged FP64 fields (T 1e-9, q 1e-8) and the
FP32 sweep (T 1e-6)."""
import numpy as np
import pytest

from oracle import OracleSolver
from cases import tets_cyclic, rel_T, rel_q

pytestmark = pytest.mark.gpu
_ref = {}


def _oracle(scheme):
    if scheme not in _ref:
        _ref[scheme] = OracleSolver(tets_cyclic()).solve(scheme=scheme, tol=1e-14, max_iter=50000)
    return _ref[scheme]


@pytest.fixture(scope="module")
def nbte_mod(gpu_lib):
    from paper_2607_03226_b300 import nbte
    return nbte


@pytest.mark.parametrize("scheme", ["sequential", "synthetic"])
def test_cyclic_mesh_converged_fp64(nbte_mod, scheme):
    p = tets_cyclic()
    s = nbte_mod.Solver(p)
    st = s.plan_stats(precision="fp64", band_group=1, cta_threads=64)
    assert st["lagged_faces"] > 0
    info = s.solve(scheme=scheme, precision="fp64", tol=1e-13, max_iter=50000, band_group=1, cta_threads=64)
    assert info["status"] == 0 and info["lagged_faces"] == st["lagged_faces"]
    r = _oracle(scheme)
    assert r["converged"]
    eT = rel_T(s.temperature(0), r["T"], p.T_ref)
    eq = rel_q(s.heat_flux(), r["q"])
    print(f"{scheme}: {info['lagged_faces']} lagged faces, {info['iterations']} iterations, T {eT:.2e}, q {eq:.2e}")
    assert eT < 1e-9 and eq < 1e-8
    assert info["energy_imbalance"] < 1e-9
    for tag in (1, 2, 3, 4):
        assert s.wall_heat(tag) == pytest.approx(r["wall_flux"][tag], rel=1e-7, abs=1e-9 * abs(r["Q_total"]))
    s.close()


def test_cyclic_mesh_converged_fp32_every_layout(nbte_mod):
    """The FP32 sweep in several launch layouts (band groups, chunk lengths)
    reaches the same field within 1e-6."""
    p = tets_cyclic()
    r = _oracle("sequential")
    s = nbte_mod.Solver(p)
    for G, cta in ((1, 64), (2, 96), (2, 160)):
        info = s.solve(scheme="sequential", precision="fp32", tol=1e-9, max_iter=50000, band_group=G, cta_threads=cta)
        assert info["status"] == 0 and info["lagged_faces"] > 0
        e = rel_T(s.temperature(0), r["T"], p.T_ref)
        print(f"fp32 band group {G}, {cta} threads: T {e:.2e}")
        assert e < 1e-6
    s.close()
