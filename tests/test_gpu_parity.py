"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (written here, from the stated targets): FP64 path, converged
fields: temperature 1e-9 and heat flux 1e-8 relative (|.|_inf over the
oracle's deviation / flux magnitude); single iterations from the same state
agree to rounding (1e-11).  FP32-sweep path: temperature 1e-6.
"""
import json
import os

import numpy as np
import pytest

from oracle import OracleSolver
import workloads as W
from cases import CASES, rel_T, rel_q

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def nbte_mod(gpu_lib):
    from paper_2607_03226_b300 import nbte
    return nbte


_oracle_cache = {}


def oracle_run(name, **kw):
    key = (name, tuple(sorted(kw.items())))
    if key not in _oracle_cache:
        p = CASES[name]()
        _oracle_cache[key] = OracleSolver(p).solve(**kw)
    return _oracle_cache[key]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("n_iter", [1, 3])
def test_single_iterations_fp64(nbte_mod, name, n_iter):
    """Same start state, same number of sequential iterations: every moment
    agrees with the oracle to rounding (no cycle-breaking lag on these meshes)."""
    p = CASES[name]()
    s = nbte_mod.Solver(p)
    info = s.solve(scheme="sequential", precision="fp64", n_iter=n_iter)
    assert info["iterations"] == n_iter and info["lagged_faces"] == 0
    r = oracle_run(name, scheme="sequential", n_iter=n_iter)
    assert rel_T(s.temperature(0), r["T"], p.T_ref) < 1e-11
    assert rel_T(s.temperature(2), r["T_kinetic"], p.T_ref) < 1e-11
    assert rel_T(s.temperature(1), r["T_energy"], p.T_ref) < 1e-11
    assert rel_q(s.heat_flux(), r["q"]) < 1e-10
    s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_single_iterations_synthetic_fp64(nbte_mod, name):
    """Two synthetic (diffusion-corrected) iterations, CG converged tightly:
    the correction, the corrected wall values and the update agree."""
    p = CASES[name]()
    s = nbte_mod.Solver(p)
    s.solve(scheme="synthetic", precision="fp64", n_iter=2, cg_tol=1e-14, cg_max_iter=20000)
    r = oracle_run(name, scheme="synthetic", n_iter=2)
    assert rel_T(s.temperature(0), r["T"], p.T_ref) < 1e-9
    assert rel_T(s.temperature(2), r["T_kinetic"], p.T_ref) < 1e-9
    s.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("scheme", ["sequential", "synthetic"])
def test_converged_fp64(nbte_mod, name, scheme):
    """Converged FP64 fields: T within 1e-9 and q within 1e-8 of the oracle;
    the energy balance closes."""
    p = CASES[name]()
    s = nbte_mod.Solver(p)
    info = s.solve(scheme=scheme, precision="fp64", tol=1e-13, max_iter=20000)
    assert info["status"] == 0
    r = oracle_run(name, scheme="synthetic", tol=1e-14, max_iter=20000)
    assert rel_T(s.temperature(0), r["T"], p.T_ref) < 1e-9
    assert rel_q(s.heat_flux(), r["q"]) < 1e-8
    assert info["energy_imbalance"] < 1e-8
    for tag, f in r["wall_flux"].items():
        assert abs(s.wall_heat(tag) - f) <= 1e-8 * max(abs(v) for v in r["wall_flux"].values())
    s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_converged_fp32_sweep(nbte_mod, name):
    """FP32 sweep with FP64 moments, update and residual: temperature within
    1e-6 of the FP64 oracle (heat-flux error recorded, bounded at 1e-4)."""
    p = CASES[name]()
    s = nbte_mod.Solver(p)
    # FP32 distributions put a rounding floor under the relative increment;
    # the solve stops there (NBTE_OK) when tol is below it
    info = s.solve(scheme="synthetic", precision="fp32", tol=1e-9, max_iter=20000)
    assert info["status"] == 0
    assert info["residual"] < 1e-6
    r = oracle_run(name, scheme="synthetic", tol=1e-14, max_iter=20000)
    eT = rel_T(s.temperature(0), r["T"], p.T_ref)
    eq = rel_q(s.heat_flux(), r["q"])
    print(f"{name}: FP32 iterations {info['iterations']} residual {info['residual']:.2e} T err {eT:.2e} q err {eq:.2e}")
    assert eT < 1e-6
    assert eq < 1e-4
    s.close()


def test_square_full_size_golden(nbte_mod):
    """The 40x40 in-plane square (FP64 sequential to 1e-10, and FP32) against
    the stored oracle solution."""
    g = json.load(open(os.path.join(GOLDEN, "square_inplane_converged.json")))
    p = W.problems.square_inplane()
    s = nbte_mod.Solver(p)
    info = s.solve(scheme="sequential", precision="fp64", tol=1e-12)
    assert info["status"] == 0
    assert rel_T(s.temperature(0), np.array(g["T"]), p.T_ref) < 1e-9
    assert rel_q(s.heat_flux(), np.array(g["q"])) < 1e-8
    info = s.solve(scheme="sequential", precision="fp32", tol=1e-10)
    assert rel_T(s.temperature(0), np.array(g["T"]), p.T_ref) < 1e-6
    s.close()


@pytest.mark.parametrize("variant", [dict(band_group=1), dict(band_group=2, cta_threads=96),
                                     dict(use_graph=True), dict(band_group=4, cta_threads=544, use_graph=True),
                                     dict(ring="global"), dict(band_group=4, cta_threads=160, ring="global")])
def test_launch_variants_identical(nbte_mod, variant):
    """Band grouping, CTA size (chunk length of the copy pipeline), the value
    ring's placement (shared or global memory) and graph replay change only
    the launch shape: FP64 results are identical to the default to rounding."""
    p = CASES["fin2d_mixed"]()
    p.C, p.v, p.tau = (np.tile(x, 2)[:4] for x in (p.C, p.v, p.tau))
    s = nbte_mod.Solver(p)
    s.solve(scheme="sequential", precision="fp64", n_iter=4)
    T0, q0 = s.temperature(0), s.heat_flux()
    s.solve(scheme="sequential", precision="fp64", n_iter=4, **variant)
    assert np.abs(s.temperature(0) - T0).max() <= 1e-12 * np.abs(T0 - 300).max()
    assert np.abs(s.heat_flux() - q0).max() <= 1e-11 * np.abs(q0).max()
    s.close()


@pytest.mark.parametrize("name", ["fin2d_mixed", "fin3d_tets", "cube_hex"])
def test_tilted_plan_same_iterates(nbte_mod, monkeypatch, name):
    """Tilted fronts (release levels along the long axis) only reorder the
    triangular solve of Eq. (13): three FP64 iterations with every direction
    tilted match the untilted plan to rounding and the oracle at 1e-11, and
    the FP32 sweep at 1e-6."""
    p = CASES[name]()
    ref = OracleSolver(p).solve(scheme="sequential", n_iter=3)
    out = {}
    for tilt in ("0", "force"):
        monkeypatch.setenv("NBTE_PLAN_TILT", tilt)
        s = nbte_mod.Solver(p)
        s.solve(scheme="sequential", precision="fp64", n_iter=3)
        out[tilt] = s.temperature(0)
        assert rel_T(out[tilt], ref["T"], p.T_ref) < 1e-11
        s.solve(scheme="sequential", precision="fp32", n_iter=3)
        assert rel_T(s.temperature(0), ref["T"], p.T_ref) < 1e-5
        s.close()
    assert rel_T(out["force"], out["0"], p.T_ref) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_collision_moment_forms(nbte_mod, precision):
    """The 140k-tet FinFET (the 1.14M-tet workload's geometry at 4 nm cells,
    40 bands, 200 directions) is large enough for the default layout to sum
    the collision moment of Eq. (5) with FP64 atomic adds; deterministic=1
    keeps fixed-order partials.  The fixed-order form repeats bit for bit;
    the two forms agree to FP64 rounding (FP64 sweep) or to the FP32 sweep's
    rounding (a temperature rounded to the neighbouring FP32 value)."""
    import workloads as W
    p = W.problems.finfet3d(h=4e-9)
    s = nbte_mod.Solver(p)
    kw = dict(scheme="sequential", precision=precision, n_iter=2, band_group=8 if precision == "fp32" else 4,
              cta_threads=544 if precision == "fp32" else 320)
    s.solve(deterministic=True, **kw)
    T_det = s.temperature(0)
    s.solve(deterministic=True, **kw)
    assert np.array_equal(s.temperature(0), T_det)
    s.solve(**kw)
    T_acc = s.temperature(0)
    e = rel_T(T_acc, T_det, p.T_ref)
    print(f"{precision}: atomic sums vs fixed order {e:.2e}")
    assert e <= (1e-13 if precision == "fp64" else 1e-6)
    s.close()


def test_warm_start_continues(nbte_mod):
    """Two solves of n iterations with warm=True equal one solve of 2n."""
    p = CASES["cube_hex"]()
    s = nbte_mod.Solver(p)
    s.solve(scheme="sequential", precision="fp64", n_iter=6)
    Ta = s.temperature(0)
    s.solve(scheme="sequential", precision="fp64", n_iter=3)
    s.solve(scheme="sequential", precision="fp64", n_iter=3, warm=True)
    assert np.abs(s.temperature(0) - Ta).max() <= 1e-12 * np.abs(Ta - 300).max()
    s.close()


def test_results_into_pinned_buffers(nbte_mod):
    """Results read into page-locked caller arrays (copied there by DMA)
    equal the same results read into ordinary arrays, for every temperature
    kind and the heat flux; a heat source set from a pinned array gives the
    same solve as from an ordinary one (bitwise, with the fixed-order
    collision moment)."""
    import torch
    p = CASES["fin2d_mixed"]()
    s = nbte_mod.Solver(p)
    Qp = torch.empty(p.n_cells, dtype=torch.float64, pin_memory=True).numpy()
    Qp[:] = p.Q
    nbte_mod.nbte_set_heat_source(s.solver, Qp)
    s.solve(scheme="sequential", precision="fp64", n_iter=3, deterministic=True)
    for kind in (0, 1, 2):
        out = torch.full((p.n_cells,), np.nan, dtype=torch.float64, pin_memory=True).numpy()
        r = s.temperature(kind, out=out)
        assert r is out
        assert np.array_equal(out, s.temperature(kind))
    qp = torch.full((p.n_cells, p.mesh.dim), np.nan, dtype=torch.float64, pin_memory=True).numpy()
    assert np.array_equal(s.heat_flux(out=qp), s.heat_flux())
    T_pinned_src = s.temperature(0)
    nbte_mod.nbte_set_heat_source(s.solver, np.array(p.Q))
    s.solve(scheme="sequential", precision="fp64", n_iter=3, deterministic=True)
    assert np.array_equal(s.temperature(0), T_pinned_src)
    s.close()


def test_uniform_temperature_invariant_fp32(nbte_mod):
    """All thermalizing walls at one temperature and no source: the converged
    field is that temperature everywhere, on a mixed-wall tet mesh, in FP32."""
    p = W.problems.finfet3d(h=15e-9, B=4, n_pol=2, n_az=8, q_fin=0.0)
    for b in p.boundaries:
        if b.type == 0:
            b.T_wall = 303.0
    p.Q = None
    s = nbte_mod.Solver(p)
    info = s.solve(scheme="synthetic", precision="fp32", tol=1e-9, max_iter=5000)
    assert info["status"] == 0
    assert np.abs(s.temperature(0) - 303.0).max() < 3e-6 * 3.0
    s.close()


def _fin2d_golden(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    return json.load(open(path))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-6)])
def test_finfet2d_full_size_steps(nbte_mod, precision, tol):
    """The full-size 2D fin (50,474 triangles, 20 bands, 64 directions), in
    the launch configuration the benchmark times (autotuned layout, graph
    replay): T after sequential iterations 1 and 2 from T_ref on 4096 stored
    oracle sample cells."""
    g = _fin2d_golden("finfet2d_steps.json")
    p = W.problems.finfet2d()
    idx = np.array(g["cells"])
    s = nbte_mod.Solver(p)
    for n in (1, 2):
        info = s.solve(scheme="sequential", precision=precision, n_iter=n, use_graph=True)
        assert info["iterations"] == n
        T = s.temperature(0)[idx]
        err = np.abs(T - np.array(g[f"T_iter{n}"])).max() / g[f"T_iter{n}_max_dev"]
        print(f"{precision} iteration {n}: rel err {err:.2e}")
        assert err < tol
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-6)])
def test_finfet2d_full_size_every_layout(nbte_mod, precision, tol):
    """Sweep layouts the autotuner may pick (band group x chunk length: the
    powers of two and the multiples of 32 it refines around the best)
    on the full-size 2D fin: T after one and two sequential iterations on the
    stored oracle sample cells.  Layouts that do not fit shared memory are
    refused with NBTE_ERR_ARG and skipped."""
    g = _fin2d_golden("finfet2d_steps.json")
    p = W.problems.finfet2d()
    idx = np.array(g["cells"])
    s = nbte_mod.Solver(p)
    groups = (1, 2, 4) if precision == "fp64" else (1, 2, 4, 8)
    bad, ran = [], 0
    for G in groups:
        for cap in (64, 128, 160, 192, 256, 512):
            for n in (1, 2):
                try:
                    s.solve(scheme="sequential", precision=precision, n_iter=n, band_group=G,
                            cta_threads=cap + 32)
                except nbte_mod.NbteError as e:
                    assert e.code == nbte_mod.NBTE_ERR_ARG
                    break
                ran += 1
                err = np.abs(s.temperature(0)[idx] - np.array(g[f"T_iter{n}"])).max() / g[f"T_iter{n}_max_dev"]
                if not err < tol:
                    bad.append((G, cap, n, float(err)))
    s.close()
    print(f"{precision}: {ran} layout runs, failing: {bad}")
    assert ran >= 8 and not bad


def test_finfet2d_full_size_converged(nbte_mod):
    """The full-size 2D fin converged, FP64 and FP32 sweep, against the
    oracle's field converged to 1e-13 (728 sequential iterations): T and q
    on the stored sample cells, relative to the oracle's largest deviation
    and heat flux over all cells.  FP64: T 1e-9, q 1e-8; FP32 sweep: T 1e-6
    (the stated targets)."""
    g = _fin2d_golden("finfet2d_converged.json")
    assert g["tol"] <= 1e-13
    p = W.problems.finfet2d()
    idx = np.array(g["cells"])
    Tg, qg = np.array(g["T"]), np.array(g["q"])
    dev = g["T_max"] - p.T_ref
    s = nbte_mod.Solver(p)
    for scheme in ("synthetic", "sequential"):
        info = s.solve(scheme=scheme, precision="fp64", tol=1e-13, max_iter=20000)
        assert info["status"] == 0
        eT = np.abs(s.temperature(0)[idx] - Tg).max() / dev
        eq = np.abs(s.heat_flux()[idx] - qg).max() / g["q_max"]
        print(f"fp64 {scheme}: {info['iterations']} iterations, T {eT:.2e}, q {eq:.2e}")
        assert eT < 1e-9 and eq < 1e-8
    info = s.solve(scheme="synthetic", precision="fp32", tol=1e-9, max_iter=20000)
    assert info["status"] == 0
    eT = np.abs(s.temperature(0)[idx] - Tg).max() / dev
    eq = np.abs(s.heat_flux()[idx] - qg).max() / g["q_max"]
    print(f"fp32 synthetic: {info['iterations']} iterations (floor {info['residual']:.1e}), T {eT:.2e}, q {eq:.2e}")
    assert eT < 1e-6
    s.close()


@pytest.mark.parametrize("name", ["fin2d_mixed", "fin3d_tets", "cube_hex"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-6)])
def test_distribution_every_task(nbte_mod, name, precision, tol):
    """e'_{band,direction} of the last sweep (nbte_get_distribution) for every
    task after three sequential iterations, against the oracle's last sweep
    (relative to max|e'| over the task)."""
    p = CASES[name]()
    s = nbte_mod.Solver(p)
    s.solve(scheme="sequential", precision=precision, n_iter=3)
    r = oracle_run(name, scheme="sequential", n_iter=3, store_e=True)
    worst = 0.0
    for i in range(p.n_dirs):
        for l in range(p.n_bands):
            ref = r["e"][:, l, i]
            scale = max(np.abs(ref).max(), 1e-300)
            worst = max(worst, np.abs(s.distribution(i, l) - ref).max() / scale)
    print(f"{name} {precision}: worst task error {worst:.2e}")
    assert worst < tol
    s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_fourier_initial_guess(nbte_mod, name):
    """Iterations from the diffusion-limit initial guess (init="fourier")
    against the oracle's, which solves the guess exactly; the device solves it
    by CG to a 1e-12 relative residual, so the bound is 1e-8.  The converged
    field does not depend on the starting point (1e-9)."""
    p = CASES[name]()
    s = nbte_mod.Solver(p)
    for n in (1, 2):
        s.solve(scheme="sequential", precision="fp64", n_iter=n, init="fourier")
        r = oracle_run(name, scheme="sequential", n_iter=n, init="fourier")
        err = rel_T(s.temperature(0), r["T"], p.T_ref)
        print(f"{name}: {n} iteration(s) from the Fourier guess, T error {err:.2e}")
        assert err < 1e-8
    a = s.solve(scheme="synthetic", precision="fp64", tol=1e-13, max_iter=20000, init="fourier")
    Ta = s.temperature(0)
    b = s.solve(scheme="synthetic", precision="fp64", tol=1e-13, max_iter=20000)
    assert a["status"] == 0 and b["status"] == 0
    assert rel_T(Ta, s.temperature(0), p.T_ref) < 1e-9
    s.close()
