"""Full-size parity on the two 3D workloads (the 64^3 hex cube: 262,144
cells, 40 bands, 128 directions; the FinFET: 1.14M tets, 40 bands, 200
directions), in the autotuned launch configuration a user gets.

The oracle's values are stored (tests/golden/make_golden.py), on 4096 seeded
sample cells:
* the distribution e'_{l i} of a few (direction, band) tasks in the first
  sequential iteration from T_ref (device values from nbte_get_distribution;
  relative to max|e'| of the task: FP64 1e-11, rounding order only; FP32
  sweep 1e-6);
* the FinFET's temperature after sequential iterations 1, 2 and 3 from T_ref
  and the heat flux of the third sweep: from the second iteration on every
  diffuse, specular and partially specular wall feeds back the previous
  sweep (FP64 1e-11 of the largest deviation, q 1e-10; FP32 1e-6);
* the cube converged with the synthetic scheme (the CG correction at full
  size): T 1e-9 and q 1e-8 in FP64, T 1e-6 with the FP32 sweep.
"""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_solvers = {}


@pytest.fixture(scope="module")
def nbte_mod(gpu_lib):
    from paper_2607_03226_b300 import nbte
    yield nbte
    for s in _solvers.values():
        s.close()
    _solvers.clear()


def _solver(nbte, name):
    if name not in _solvers:
        for other in list(_solvers):   # one large solver on the device at a time
            _solvers.pop(other).close()
        _solvers[name] = nbte.Solver(getattr(W.problems, name)())
    return _solvers[name]


@pytest.mark.parametrize("name", ["cube3d", "finfet3d"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-6)])
def test_full_size_first_iteration_tasks(nbte_mod, name, precision, tol):
    path = os.path.join(GOLDEN, f"{name}_tasks.json")
    if not os.path.exists(path):
        pytest.skip(f"{name}_tasks.json not generated")
    g = json.load(open(path))
    s = _solver(nbte_mod, name)
    info = s.solve(scheme="sequential", precision=precision, n_iter=1, skip_outputs=True)
    assert info["iterations"] == 1
    idx = np.array(g["cells"])
    for t in g["tasks"]:
        e = s.distribution(t["direction"], t["band"])[idx]
        err = np.abs(e - np.array(t["e"])).max() / t["max_abs"]
        print(f"{name} {precision} task ({t['direction']}, {t['band']}): rel err {err:.2e}")
        assert err < tol


def _stream_problems():
    """The smallest request of each mesh kind in the benchmark's 24-request
    stream (same seed): a 2D triangle fin, a 3D hex box and a 3D tet fin with
    random wall mixes and a heat box."""
    reqs = W.stream.requests(24, 1.0)
    out = []
    for kind in ("tri2d", "hex3d", "tet3d"):
        r = min((r for r in reqs if r.kind == kind), key=lambda r: r.n_cells_target)
        out.append(W.stream.build(r))
    return out


@pytest.mark.parametrize("k", range(3))
def test_stream_requests_first_iteration_tasks(nbte_mod, k):
    """Stream requests at their full size: the first sequential iteration's
    distribution of three (direction, band) tasks against the oracle's
    sparse solve of the same tasks (walls at equilibrium with T_ref), every
    cell, relative to max|e'| of the task.  FP64 1e-11 (rounding order).
    FP32 4e-6: the 1e-6 target is for the temperature, an average over all
    tasks; one task's distribution carries the FP32 rounding of its own level
    chain, up to about a thousand dependent updates of relative error 2^-24
    each (a random walk of ~2e-6 at that length), with a factor 2 margin."""
    from oracle import OracleSolver
    p = _stream_problems()[k]
    o = OracleSolver(p)
    T0 = np.zeros(o.N)
    eb0 = np.zeros((o.bcells.size, o.D))
    tasks = [(0, 0), (p.n_dirs // 2, p.n_bands // 2), (p.n_dirs - 1, p.n_bands - 1)]
    ref = {(i, l): o.solve_task(T0, o.incoming_band(eb0, l), i, l) for (i, l) in tasks}
    s = nbte_mod.Solver(p)
    for precision, tol in (("fp64", 1e-11), ("fp32", 4e-6)):
        s.solve(scheme="sequential", precision=precision, n_iter=1, skip_outputs=True)
        for (i, l), e in ref.items():
            err = np.abs(s.distribution(i, l) - e).max() / np.abs(e).max()
            print(f"{p.name} ({p.n_cells} cells) {precision} task ({i}, {l}): rel err {err:.2e}")
            assert err < tol
    s.close()


def _golden(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    return json.load(open(path))


@pytest.mark.parametrize("precision,tol_T,tol_q", [("fp64", 1e-11, 1e-10), ("fp32", 1e-6, 1e-5)])
def test_finfet3d_full_size_three_iterations(nbte_mod, precision, tol_T, tol_q):
    g = _golden("finfet3d_steps.json")
    s = _solver(nbte_mod, "finfet3d")
    idx = np.array(g["cells"])
    for n in (1, 2, 3):
        info = s.solve(scheme="sequential", precision=precision, n_iter=n, use_graph=True, skip_outputs=n < 3)
        assert info["iterations"] == n
        err = np.abs(s.temperature(0)[idx] - np.array(g[f"T_iter{n}"])).max() / g[f"T_iter{n}_max_dev"]
        print(f"finfet3d {precision} iteration {n}: T rel err {err:.2e}")
        assert err < tol_T
    eq = np.abs(s.heat_flux()[idx] - np.array(g["q_iter3"])).max() / g["q_iter3_max"]
    print(f"finfet3d {precision} iteration 3: q rel err {eq:.2e}")
    assert eq < tol_q


def test_cube3d_full_size_converged(nbte_mod):
    g = _golden("cube3d_converged.json")
    assert g["tol"] <= 1e-12
    s = _solver(nbte_mod, "cube3d")
    idx = np.array(g["cells"])
    Tg, qg = np.array(g["T"]), np.array(g["q"])
    dev = max(g["T_max"] - 300.0, 300.0 - g["T_min"])
    info = s.solve(scheme="synthetic", precision="fp64", tol=1e-13, max_iter=5000, init="fourier")
    assert info["status"] == 0
    eT = np.abs(s.temperature(0)[idx] - Tg).max() / dev
    eq = np.abs(s.heat_flux()[idx] - qg).max() / g["q_max"]
    print(f"cube3d fp64 synthetic: {info['iterations']} iterations, T {eT:.2e}, q {eq:.2e}")
    assert eT < 1e-9 and eq < 1e-8
    assert info["energy_imbalance"] < 1e-9
    info = s.solve(scheme="synthetic", precision="fp32", tol=1e-9, max_iter=5000)
    assert info["status"] == 0
    eT = np.abs(s.temperature(0)[idx] - Tg).max() / dev
    print(f"cube3d fp32 synthetic: {info['iterations']} iterations (floor {info['residual']:.1e}), T {eT:.2e}")
    assert eT < 1e-6


@pytest.mark.parametrize("k,kind", [(0, "tri2d"), (1, "hex3d"), (2, "tet3d")])
def test_stream_requests_converged(nbte_mod, k, kind):
    """The smallest 2D-triangle, 3D-hex and 3D-tet requests of the serving
    stream (random wall mixes with partially specular and specular walls,
    heat boxes) converged with the synthetic scheme, against the oracle's
    field converged to 1e-12: FP64 T 1e-9, q 1e-8; the FP32 sweep T 1e-6."""
    g = _golden("stream_converged.json")
    assert g["tol"] <= 1e-12
    r = g["requests"][kind]
    p = _stream_problems()[k]
    assert p.n_cells == r["n_cells"] and r["converged"]
    idx = np.array(r["cells"])
    Tg, qg = np.array(r["T"]), np.array(r["q"])
    dev = max(r["T_max"] - p.T_ref, p.T_ref - r["T_min"])
    s = nbte_mod.Solver(p)
    info = s.solve(scheme="synthetic", precision="fp64", tol=1e-13, max_iter=20000, init="fourier")
    assert info["status"] == 0
    eT = np.abs(s.temperature(0)[idx] - Tg).max() / dev
    eq = np.abs(s.heat_flux()[idx] - qg).max() / r["q_max"]
    print(f"{kind} ({p.n_cells} cells) fp64: {info['iterations']} iterations, T {eT:.2e}, q {eq:.2e}")
    assert eT < 1e-9 and eq < 1e-8
    info = s.solve(scheme="synthetic", precision="fp32", tol=1e-9, max_iter=20000, init="fourier")
    assert info["status"] == 0
    eT = np.abs(s.temperature(0)[idx] - Tg).max() / dev
    print(f"{kind} fp32: {info['iterations']} iterations (floor {info['residual']:.1e}), T {eT:.2e}")
    assert eT < 1e-6
    s.close()
