"""Write the stored oracle results the GPU parity tests compare against.

Calls only ``oracle/`` and the seeded generators in ``workloads/``.  Each
output file records the command, the problem parameters and the oracle's
iteration count; values are absolute temperatures (K) and heat fluxes (W/m^2).

Usage:  python tests/golden/make_golden.py [square|finfet2d_steps|finfet2d_converged|
                                            finfet2d_order2_steps ...]

* ``square``              - the 40x40 in-plane square, sequential to 1e-12
                            (all 1600 cells).
* ``finfet2d_steps``      - the ~50k-triangle fin, 20 bands, 64 directions:
                            the lattice temperature after sequential iterations
                            1 and 2 from T_ref, on 4096 seeded sample cells.
* ``finfet2d_converged``  - the same problem converged (sequential, 1e-10),
                            T_L and q on the sample cells.
* ``finfet2d_order2_steps`` - the same fin with second-order upwind face
                            values: T_L after sequential iterations 2 and 3
                            from T_ref (the first iteration has no
                            reconstruction yet), on the sample cells.
* ``cube3d_tasks`` / ``finfet3d_tasks`` - the 64^3 cube and the 1.14M-tet
                            FinFET at full size: the distribution e'_{l i} of
                            a few (direction, band) tasks in the first
                            sequential iteration from T_ref (walls at
                            equilibrium with T_ref), on 4096 sample cells.
                            Each task is one sparse solve of Eq. (4).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import OracleSolver  # noqa: E402

SAMPLE_SEED = 7
N_SAMPLE = 4096


def _write(name, payload):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        json.dump(payload, f, indent=None, separators=(",", ":"))
    print("wrote", path)


def square():
    p = W.problems.square_inplane()
    t = time.time()
    r = OracleSolver(p).solve(scheme="sequential", tol=1e-12)
    _write("square_inplane_converged.json", dict(
        problem="square_inplane()", scheme="sequential", tol=1e-12, iterations=r["iterations"],
        seconds=time.time() - t, T=r["T"].tolist(), q=r["q"].tolist(),
        T_energy=r["T_energy"].tolist()))


def _sample(n_cells):
    rng = np.random.default_rng(SAMPLE_SEED)
    return np.sort(rng.choice(n_cells, size=min(N_SAMPLE, n_cells), replace=False))


def finfet2d_steps():
    p = W.problems.finfet2d()
    o = OracleSolver(p)
    idx = _sample(p.n_cells)
    out = dict(problem="finfet2d()", scheme="sequential", sample_seed=SAMPLE_SEED, cells=idx.tolist())
    for n in (1, 2):
        t = time.time()
        r = o.solve(scheme="sequential", n_iter=n)
        out[f"T_iter{n}"] = r["T"][idx].tolist()
        out[f"T_iter{n}_max_dev"] = float(np.abs(r["T"] - p.T_ref).max())
        out[f"seconds_iter{n}"] = time.time() - t
        print("iter", n, "done", time.time() - t)
    _write("finfet2d_steps.json", out)


def finfet2d_converged():
    p = W.problems.finfet2d()
    o = OracleSolver(p)
    idx = _sample(p.n_cells)
    t = time.time()
    r = o.solve(scheme="sequential", tol=1e-10, verbose=True)
    _write("finfet2d_converged.json", dict(
        problem="finfet2d()", scheme="sequential", tol=1e-10, iterations=r["iterations"],
        converged=r["converged"], seconds=time.time() - t, sample_seed=SAMPLE_SEED,
        cells=idx.tolist(), T=r["T"][idx].tolist(), q=r["q"][idx].tolist(),
        T_max=float(r["T"].max()), energy_imbalance=r["energy_imbalance"]))


def finfet2d_order2_steps():
    p = W.problems.finfet2d()
    o = OracleSolver(p)
    idx = _sample(p.n_cells)
    out = dict(problem="finfet2d()", scheme="sequential", order=2, sample_seed=SAMPLE_SEED,
               cells=idx.tolist())
    for n in (2, 3):
        t = time.time()
        r = o.solve(scheme="sequential", n_iter=n, order=2)
        out[f"T_iter{n}"] = r["T"][idx].tolist()
        out[f"T_iter{n}_max_dev"] = float(np.abs(r["T"] - p.T_ref).max())
        out[f"seconds_iter{n}"] = time.time() - t
        print("iter", n, "done", time.time() - t, flush=True)
    _write("finfet2d_order2_steps.json", out)


def _tasks(name, p, tasks):
    o = OracleSolver(p)
    idx = _sample(p.n_cells)
    T0 = np.zeros(o.N)
    eb0 = np.zeros((o.bcells.size, o.D))    # wall cells at equilibrium with T_ref
    out = dict(problem=f"{name}()", scheme="sequential", iteration=1, sample_seed=SAMPLE_SEED,
               cells=idx.tolist(), tasks=[])
    for (i, l) in tasks:
        t = time.time()
        e = o.solve_task(T0, o.incoming_band(eb0, l), i, l)
        out["tasks"].append(dict(direction=int(i), band=int(l), e=e[idx].tolist(),
                                 max_abs=float(np.abs(e).max()), seconds=time.time() - t))
        print(name, "task", i, l, "done", time.time() - t, flush=True)
    _write(f"{name}_tasks.json", out)


def cube3d_tasks():
    p = W.problems.cube3d()
    s = np.asarray(p.s)
    along = np.argsort(-s[:, 0])            # most nearly +x first (the hot wall is x = 0)
    _tasks("cube3d", p, [(int(along[0]), 0), (int(along[5]), p.n_bands - 1), (int(along[20]), 21)])


def finfet3d_tasks():
    p = W.problems.finfet3d()
    _tasks("finfet3d", p, [(0, 0), (p.n_dirs // 2, 21), (p.n_dirs - 1, p.n_bands - 1)])


if __name__ == "__main__":
    for name in (sys.argv[1:] or ["square"]):
        globals()[name]()
