"""Write the stored oracle results the GPU parity tests compare against.

Calls only ``oracle/`` and the seeded generators in ``workloads/``.  Each
output file records the command, the problem parameters and the oracle's
iteration count; values are absolute temperatures (K) and heat fluxes (W/m^2).

Usage:  python tests/golden/make_golden.py [square|finfet2d_steps|finfet2d_converged|
                                            finfet2d_order2_steps|cube3d_tasks|finfet3d_tasks|
                                            cube3d_converged|stream_converged|finfet3d_steps ...]

* ``square``              - the 40x40 in-plane square, sequential to 1e-12
                            (all 1600 cells).
* ``finfet2d_steps``      - the ~50k-triangle fin, 20 bands, 64 directions:
                            the lattice temperature after sequential iterations
                            1 and 2 from T_ref, on 4096 seeded sample cells.
* ``finfet2d_converged``  - the same problem converged (sequential, 1e-13),
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
* ``cube3d_converged``    - the 64^3 cube converged with the synthetic scheme
                            (1e-12, from the diffusion guess): T_L and q on
                            the sample cells.
* ``stream_converged``    - the smallest 2D-triangle, 3D-hex and 3D-tet
                            requests of the serving stream, each converged
                            (synthetic, 1e-12): T_L and q on sample cells.
* ``finfet3d_steps``      - the 1.14M-tet FinFET: T_L after sequential
                            iterations 1, 2 and 3 from T_ref and q of the
                            third sweep, on the sample cells.

The 3D ones and the stream requests split every pass over worker processes by direction (one per
available core, or GOLDEN_WORKERS; ``PoolSweep``).
"""
from __future__ import annotations

import json
import multiprocessing as mp
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


# ---------------------------------------------------------------- task pool
# An oracle pass at the 3D workloads' sizes is thousands of sparse solves.
# The pool below splits each pass by direction over worker processes (each
# builds its own OracleSolver of the same problem) and adds up their moments;
# every solve and every moment term is the oracle's own.  Only the order in
# which the per-task terms are summed differs from a serial pass (rounding).
_O = None


_KEEP = True


def _problem(name, kwargs):
    """A workload by name: a family of workloads.problems, or
    "stream:<kind>" for the smallest request of that mesh kind in the
    benchmark's seeded 24-request stream."""
    if name.startswith("stream:"):
        kind = name.split(":", 1)[1]
        reqs = W.stream.requests(24, 1.0)
        return W.stream.build(min((r for r in reqs if r.kind == kind), key=lambda r: r.n_cells_target))
    return getattr(W.problems, name)(**kwargs)


def _pool_init(name, kwargs, keep):
    global _O, _KEEP
    _O = OracleSolver(_problem(name, kwargs))
    _KEEP = keep


class _Cols:
    """Incoming wall values of some directions, indexed like the full
    (half-face, band, direction) array."""

    def __init__(self, a, dirs):
        self.a = a
        self.col = {i: k for k, i in enumerate(dirs)}

    def __getitem__(self, key):
        h, l, i = key
        return self.a[h, l, self.col[i]]


def _pool_sweep(Tdev, e_in_sub, dirs):
    """The worker's directions one at a time (all bands of each); without
    _KEEP each direction's cached operators are dropped after its bands."""
    e_in = _Cols(e_in_sub, dirs)
    NL, E, q = np.zeros(_O.N), np.zeros(_O.N), np.zeros((_O.N, _O.dim))
    eb = np.empty((_O.bcells.size, _O.B, len(dirs)))
    for k, i in enumerate(dirs):
        r = _O.sweep(Tdev, None, tasks=[(i, l) for l in range(_O.B)], e_in=e_in, eb_dirs=[i])
        NL += r["NL"]
        E += r["E"]
        q += r["q"]
        eb[:, :, k] = r["eb"][:, :, 0]
        if not _KEEP:
            _O.forget_direction(i)
    return NL, E, q, eb


class PoolSweep:
    """Drop-in for ``OracleSolver.sweep`` (first-order passes) that solves
    the (direction, band) tasks on ``workers`` processes."""

    def __init__(self, o, name, kwargs=None, workers=None, keep=True):
        self.o = o
        workers = workers or int(os.environ.get("GOLDEN_WORKERS", "0")) or max(1, len(os.sched_getaffinity(0)))
        self.dirs = [list(range(k, o.D, workers)) for k in range(workers)]
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_pool_init,
                                                 initargs=(name, kwargs or {}, keep))

    def __call__(self, Tdev, eb_prev, store_e=False, e_prev=None):
        if store_e or e_prev is not None:
            raise ValueError("the pool runs first-order passes without the full distribution")
        o = self.o
        e_in = o.incoming(eb_prev)
        jobs = [(Tdev, np.ascontiguousarray(e_in[:, :, d]), d) for d in self.dirs]
        NL, E, q = np.zeros(o.N), np.zeros(o.N), np.zeros((o.N, o.dim))
        eb = np.empty((o.bcells.size, o.B, o.D))
        for d, (nl, en, qq, ebk) in zip(self.dirs, self.pool.starmap(_pool_sweep, jobs)):
            NL += nl
            E += en
            q += qq
            eb[:, :, d] = ebk
        return dict(NL=NL, E=E, q=q, eb=eb, e_in=e_in, e=None)

    def close(self):
        self.pool.close()
        self.pool.join()


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
    pool = PoolSweep(o, "finfet2d")
    idx = _sample(p.n_cells)
    t = time.time()
    r = o.solve(scheme="sequential", tol=1e-13, max_iter=20000, sweep=pool, verbose=True)
    pool.close()
    _write("finfet2d_converged.json", dict(
        problem="finfet2d()", scheme="sequential", tol=1e-13, iterations=r["iterations"],
        converged=r["converged"], seconds=time.time() - t, sample_seed=SAMPLE_SEED,
        command="python tests/golden/make_golden.py finfet2d_converged",
        cells=idx.tolist(), T=r["T"][idx].tolist(), q=r["q"][idx].tolist(),
        T_max=float(r["T"].max()), q_max=float(np.abs(r["q"]).max()),
        energy_imbalance=r["energy_imbalance"]))


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


def cube3d_converged():
    """The 64^3 cube, synthetic scheme to 1e-12 from the diffusion (Fourier)
    initial guess (the oracle's correction is an exact sparse LU solve of
    Eq. (10)); the fixed point does not depend on the start."""
    p = W.problems.cube3d()
    o = OracleSolver(p)
    pool = PoolSweep(o, "cube3d")
    idx = _sample(p.n_cells)
    t = time.time()
    r = o.solve(scheme="synthetic", tol=1e-12, max_iter=5000, init="fourier", sweep=pool, verbose=True)
    pool.close()
    _write("cube3d_converged.json", dict(
        problem="cube3d()", scheme="synthetic", init="fourier", tol=1e-12, iterations=r["iterations"],
        converged=r["converged"], seconds=time.time() - t, sample_seed=SAMPLE_SEED,
        command="python tests/golden/make_golden.py cube3d_converged",
        cells=idx.tolist(), T=r["T"][idx].tolist(), q=r["q"][idx].tolist(),
        T_max=float(r["T"].max()), T_min=float(r["T"].min()), q_max=float(np.abs(r["q"]).max()),
        energy_imbalance=r["energy_imbalance"], residuals=r["residuals"]))


def stream_converged():
    """The smallest request of each mesh kind in the benchmark's seeded
    24-request stream (a 2D triangle fin, a 3D hex box, a 3D tet fin, with
    their random wall mixes and heat boxes), each converged with the
    synthetic scheme to 1e-12 from the diffusion guess: T_L and q on up to
    4096 sample cells of each."""
    out = dict(command="python tests/golden/make_golden.py stream_converged", scheme="synthetic",
               init="fourier", tol=1e-12, sample_seed=SAMPLE_SEED, requests={})
    for kind in ("tri2d", "hex3d", "tet3d"):
        name = "stream:" + kind
        p = _problem(name, {})
        o = OracleSolver(p)
        pool = PoolSweep(o, name)
        idx = _sample(p.n_cells)
        t = time.time()
        r = o.solve(scheme="synthetic", tol=1e-12, max_iter=5000, init="fourier", sweep=pool, verbose=True)
        pool.close()
        out["requests"][kind] = dict(
            n_cells=p.n_cells, bands=p.n_bands, directions=p.n_dirs, iterations=r["iterations"],
            converged=r["converged"], seconds=time.time() - t, cells=idx.tolist(), T=r["T"][idx].tolist(),
            q=r["q"][idx].tolist(), T_max=float(r["T"].max()), T_min=float(r["T"].min()),
            q_max=float(np.abs(r["q"]).max()), energy_imbalance=r["energy_imbalance"])
        print(kind, r["iterations"], time.time() - t, flush=True)
    _write("stream_converged.json", out)


def finfet3d_steps():
    """The 1.14M-tet FinFET, sequential iterations 1, 2 and 3 from T_ref:
    T_L after each and the heat flux of the third sweep, on the sample
    cells.  From the second iteration on, the diffuse, specular and
    partially specular walls feed in the previous sweep's values."""
    p = W.problems.finfet3d()
    o = OracleSolver(p)
    pool = PoolSweep(o, "finfet3d", keep=False)   # per-direction operators are rebuilt each pass (memory)
    idx = _sample(p.n_cells)
    out = dict(problem="finfet3d()", scheme="sequential", sample_seed=SAMPLE_SEED,
               command="python tests/golden/make_golden.py finfet3d_steps", cells=idx.tolist())
    t = time.time()

    def keep(it, T, TL, q):
        out[f"T_iter{it}"] = T[idx].tolist()
        out[f"T_iter{it}_max_dev"] = float(np.abs(T - p.T_ref).max())
        out[f"seconds_iter{it}"] = time.time() - t
        if it == 3:
            out["q_iter3"] = q[idx].tolist()
            out["q_iter3_max"] = float(np.abs(q).max())
        print("iteration", it, time.time() - t, flush=True)

    o.solve(scheme="sequential", n_iter=3, sweep=pool, callback=keep)
    pool.close()
    _write("finfet3d_steps.json", out)


if __name__ == "__main__":
    for name in (sys.argv[1:] or ["square"]):
        globals()[name]()
