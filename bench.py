"""Throughput benchmark: band-direction cell updates per second on the
1.14M-tet 3D FinFET workload (fin 7 x 50 x 100 nm on a 300 x 100 x 50 nm
substrate, 40 bands, 200 directions, 5e17 W/m^3 in the fin), in the scheme
that workload is specified with (synthetic: the sweep plus the diffusion
correction), FP32 sweeps with FP64 moments, update and correction; the same
line carries the FP64 path's step (the paper's precision).

A step is one outer iteration of the hot path: wall coupling, the
level-scheduled sweep over every (direction, band) with the fused collision
moment, the moment reduction and the temperature update (plus the CG
correction for the synthetic scheme), on inputs resident in device memory.
The line also reports the time to a converged field, the end-to-end rate
through the C ABI with host buffers, the sweep's roofline and the FP64
oracle timed on this host's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload finfet3d|finfet2d|cube3d] [--precision fp32|fp64]
                    [--scheme synthetic|sequential]
    python bench.py --workload stream [--requests R] [--load L]     (serving)
    python bench.py --converge --workload cube3d|finfet3d           (time to converged field)

Prints one JSON line.  Under torchrun (N > 1) every rank solves its own
replica (no data exchange); rank 0 prints the aggregate over all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "band-dir cell updates/s"
UNIT = "updates/s"
# name -> (description, scheme the workload is specified with)
WORKLOADS = {
    "finfet3d": ("finfet3d: 1.14M-tet FinFET (fin 7 x 50 x 100 nm on a 300 x 100 x 50 nm substrate), "
                 "40 bands, 200 directions, 5e17 W/m^3 in the fin, mixed walls (p = 0.5 fin sides)", "synthetic"),
    "finfet2d": ("finfet2d: ~50k-triangle fin-on-substrate, 20 bands, 64 directions, Gaussian hot spot",
                 "sequential"),
    "cube3d": ("cube3d: 500 nm cube, 64^3 hexes, 40 bands (Kn 0.01-1), 128 directions, 310/300 K walls",
               "synthetic"),
}
# nominal FP64 (non-tensor) arithmetic rate of one B300 (FLOP/s): the FP64
# sweep's roof; there is no measured figure for it
FP64_NOMINAL_FLOPS = 1.25e12


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest value of x over all ranks (the job's time is its slowest
    rank's); x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_step, steps, world_size, t_max_ms):
    """Whole-job throughput: every rank processed units_per_step per step
    (replicas, weak scaling), over the slowest rank's time."""
    return units_per_step * steps * world_size / (t_max_ms * 1e-3)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        busy = [s for s in sm if mx and s > 0.3 * max(mx)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def sweep_algorithmic_bytes(updates, prec_bytes):
    """Algorithmic bytes of one sweep launch by the scope table's count for a
    resident-distribution sweep: every band-direction cell update writes its
    value once and reads it once (8 B in FP32, 16 B in FP64).  This is the
    roofline's byte count."""
    return 2 * prec_bytes * updates


def sweep_design_bytes(st, n_cells, n_dirs, prec_bytes, Bp, order=1):
    """Bytes this design's sweep launch must move to or from HBM at minimum
    (reported beside the roofline; no distribution is stored):
    * each direction's position records once (cell, ring slot, export index,
      diagonal G, and K inflow references and coefficients; the 16-byte
      padding of the packed record is not counted) -- the band groups of a
      direction read the same records, which L2 serves after the first;
    * the per-cell FP64 collision-moment sum once (the sweep's atomic adds
      resolve in L2);
    * the (T', Qdot) pair of every cell once;
    * the wall/lag import values read and the export values written
      (boundary cells only), all bands.
    Upwind values live in the value ring (shared memory, or an L2-resident
    global region) and are not counted.  Second order adds, per (direction,
    cell, band), the reconstruction source read and the outgoing value kept
    for the next iteration's gradients."""
    K = st["K"]
    rec = 3 * 4 + prec_bytes + K * (4 + prec_bytes)
    b = (n_dirs * n_cells * rec + n_cells * 8 + n_cells * 2 * prec_bytes
         + (st["exports"] + st["imports"]) * Bp * prec_bytes)
    if order == 2:
        b += 2 * n_dirs * n_cells * Bp * prec_bytes
    return b


def sweep_flops_per_update(n_faces):
    """FP operations of one band-direction cell update: an inflow face's
    term is one FMA (about n_faces / 2 inflow faces per cell), plus the
    equilibrium product, the source FMA, the division (FP64: a product with
    the precomputed denominator), the update and the collision-moment FMA."""
    return 2 * (n_faces / 2) + 7


def _sweep_traffic(workload, precision, G, threads, updates):
    """DRAM bytes per sweep launch from the committed ncu summary of this
    workload's sweep, if that capture was taken with the current sweep
    sources and this launch layout (else None).  A capture on a smaller case
    of the same workload (the summary's updates_per_launch) is scaled to a
    full launch by the updates it processes."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"sweep_kernel_{workload}_{precision}.md")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and not line.startswith(("|", "#", " ", "*", "`")):
            k, _, v = line.partition(":")
            fields[k.strip()] = v.strip()
    h = hashlib.sha256()
    for f in ("sweep.cu", "vecio.cuh", "layout.h", "sweep_args.h"):
        with open(os.path.join(ROOT, "paper_2607_03226_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if fields.get("sweep_source_digest") != h.hexdigest()[:16]:
        return None
    if fields.get("layout") != f"band_group={G} cta_threads={threads}":
        return None
    try:
        t = int(fields["traffic_bytes_per_launch"])
        n = int(fields.get("updates_per_launch", updates))
    except (KeyError, ValueError):
        return None
    return int(round(t * updates / n))


def _event_time(stream, fn):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def _step_record(solver, stream, kw, steps, upd, n_faces, prec):
    """ms per step (graph replay, CUDA events), the sweep's own duration
    (events around each launch) and its roofline."""
    solver.solve(n_iter=3, warm=True, **kw)
    ms, info = _event_time(stream, lambda: solver.solve(n_iter=steps, warm=True, **kw))
    prof = solver.solve(n_iter=steps, warm=True, profile=True, **{k: v for k, v in kw.items() if k != "use_graph"})
    sweep_ms = prof["sweep_seconds"] * 1e3 / max(1, prof["sweep_launches"])
    rec = {"ms_per_step": ms / steps, "updates_per_s": upd / (ms / steps * 1e-3), "sweep_ms": sweep_ms,
           "cg_iterations_per_step": info["cg_iterations"] / max(1, steps)}
    return rec, info


def _fp64_roofline(sweep_ms, upd, n_faces):
    flops = sweep_flops_per_update(n_faces) * upd
    achieved = flops / (sweep_ms * 1e-3) / 1e12
    peak = FP64_NOMINAL_FLOPS / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": "nominal FP64 rate (no measured FP64 figure)", "traffic": None,
            "kernel": "sweep_kernel", "sweep_ms": sweep_ms, "flops_per_update": sweep_flops_per_update(n_faces)}


def run_gpu(args):
    import numpy as np
    import torch
    import workloads as W
    from paper_2607_03226_b300 import nbte

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    desc, scheme0 = WORKLOADS[args.workload]
    scheme = args.scheme or scheme0
    p = getattr(W.problems, args.workload)()
    n_faces = {3: 3, 4: 4, 10: 4, 12: 6}[int(p.mesh.cell_type)]
    stream = torch.cuda.Stream()
    solver = nbte.Solver(p, stream=stream.cuda_stream)
    kw = dict(scheme=scheme, precision=args.precision, cg_tol=args.cg_tol, cg_max_iter=args.cg_max_iter,
              band_group=args.band_group, cta_threads=args.cta_threads, use_graph=True,
              skip_outputs=True, order=args.order)
    t_setup = time.perf_counter()
    stats = solver.plan_stats(**kw)          # plan, upload and (band_group = cta_threads = 0) the autotuner
    upd = p.updates_per_iteration
    # warm-up (graph capture) then the timed steps
    solver.solve(n_iter=max(args.warmup, 3), **kw)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        # the NVTX range lets a profiler select exactly the timed launches
        torch.cuda.nvtx.range_push("timed_steps")
        e0.record(stream)
        info = solver.solve(n_iter=args.steps, warm=True, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    clocks = clk.summary()
    t_max = max_over_ranks(ms, dist, "cuda")
    value = aggregate_rate(upd, args.steps, ws, t_max)

    # the sweep kernel's own duration: events around each launch, same stream
    prof = solver.solve(n_iter=args.steps, warm=True, profile=True,
                        **{k: v for k, v in kw.items() if k != "use_graph"})
    sweep_ms = prof["sweep_seconds"] * 1e3 / max(1, prof["sweep_launches"])
    prec_b = 4 if args.precision == "fp32" else 8
    G = stats["band_group"]
    n_items = stats["items"]
    Bp = n_items // p.n_dirs * G
    bytes_launch = sweep_algorithmic_bytes(upd, prec_b)
    design_bytes = sweep_design_bytes(stats, p.n_cells, p.n_dirs, prec_b, Bp, args.order)
    peak, peak_kind = _peaks()
    achieved = bytes_launch / (sweep_ms * 1e-3) / 1e9
    if args.precision == "fp32":
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": peak_kind,
                    "traffic": (_sweep_traffic(args.workload, args.precision, G, stats["cta_threads"], upd)
                                if args.order == 1 else None),
                    "kernel": "sweep_kernel", "sweep_ms": sweep_ms, "algorithmic_bytes_per_launch": bytes_launch,
                    "bytes_per_update": 2 * prec_b, "design_bytes_per_launch": design_bytes,
                    "design_frac": design_bytes / (sweep_ms * 1e-3) / 1e9 / peak}
    else:
        roofline = _fp64_roofline(sweep_ms, upd, n_faces)

    # end to end through the public API with pinned host buffers: per step the
    # heat source goes host->device, one iteration runs, the temperature comes
    # back; the second loop also computes and returns the heat flux (the
    # output sweep of Eq. (7))
    Qh = torch.empty(p.n_cells, dtype=torch.float64, pin_memory=True).numpy()
    Qh[:] = p.Q if p.Q is not None else 0.0
    Th = torch.empty(p.n_cells, dtype=torch.float64, pin_memory=True).numpy()
    qh = torch.empty((p.n_cells, p.mesh.dim), dtype=torch.float64, pin_memory=True).numpy()
    e2e_steps = max(3, min(args.steps, 10))
    e2e = {}
    for label, outputs in (("T", False), ("T+q", True)):
        kw_e = dict(kw, skip_outputs=not outputs)
        nbte.nbte_set_heat_source(solver.solver, Qh)      # untimed warm-up of this loop (graph re-capture)
        solver.solve(n_iter=1, warm=True, **kw_e)
        solver.temperature(0, out=Th)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            nbte.nbte_set_heat_source(solver.solver, Qh)
            solver.solve(n_iter=1, warm=True, **kw_e)
            solver.temperature(0, out=Th)
            if outputs:
                solver.heat_flux(out=qh)
        e2e[label] = (time.perf_counter() - t0, int(Th.nbytes + (qh.nbytes if outputs else 0)))
    e2e_line = {"value": upd * e2e_steps / e2e["T"][0], "unit": UNIT, "h2d_bytes_per_step": int(Qh.nbytes),
                "d2h_bytes_per_step": e2e["T"][1],
                "per_step": "heat source up, one iteration, temperature down (one call each)",
                "with_heat_flux": {"value": upd * e2e_steps / e2e["T+q"][0], "unit": UNIT,
                                   "h2d_bytes_per_step": int(Qh.nbytes), "d2h_bytes_per_step": e2e["T+q"][1],
                                   "per_step": "as above plus the output sweep of Eq. (7) and the heat flux down"}}

    # the other scheme's step, and the time to a converged field from T_ref
    other = "synthetic" if scheme == "sequential" else "sequential"
    other_rec, _ = _step_record(solver, stream, dict(kw, scheme=other), max(3, args.steps // 2), upd, n_faces,
                                args.precision)
    ttc = None
    if not args.no_converge:
        tol_c = args.converge_tol or (1e-6 if args.precision == "fp32" else 1e-8)
        kw_c = dict(kw, tol=tol_c, max_iter=args.max_iter)
        ms_c, ic = _event_time(stream, lambda: solver.solve(**kw_c))
        ttc = {"scheme": scheme, "seconds": ms_c * 1e-3, "iterations": ic["iterations"],
               "residual": ic["residual"], "status": ic["status"], "tol": tol_c, "start": "T_ref"}

    # the FP64 path (all sweeps, moments and corrections in FP64)
    fp64 = None
    if args.precision == "fp32" and not args.no_fp64:
        kw64 = dict(kw, precision="fp64", band_group=args.fp64_band_group, cta_threads=args.fp64_cta_threads)
        t64 = time.perf_counter()
        st64 = solver.plan_stats(**kw64)
        solver.solve(n_iter=3, **kw64)
        t64 = time.perf_counter() - t64
        rec64, _ = _step_record(solver, stream, kw64, max(3, args.fp64_steps), upd, n_faces, "fp64")
        fp64 = dict(rec64, roofline=_fp64_roofline(rec64["sweep_ms"], upd, n_faces), band_group=st64["band_group"],
                    cta_threads=st64["cta_threads"], setup_s=t64,
                    dtype="f64", scheme=scheme)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 sweep / f64 moments+update+CG" if args.precision == "fp32" else "f64",
        "data": "synthetic (seeded mesh, spectrum and heat source)",
        "config": {"workload": desc, "n_cells": p.n_cells, "bands": p.n_bands, "directions": p.n_dirs,
                   "updates_per_step": upd, "scheme": scheme, "precision": args.precision, "cg_tol": args.cg_tol,
                   "upwind_order": args.order,
                   "band_group": G, "cta_threads": stats["cta_threads"], "items": n_items,
                   "levels_max": stats["max_levels"], "ring_slots_max": stats["max_slots"],
                   "ring": "global" if stats["ring"] == 2 else "shared", "lagged_faces": stats["lagged_faces"],
                   "parallelism": f"replicas x{ws}", "setup_s": t_setup,
                   "l2": "inputs larger than L2: per-step device footprint %.0f MB > 126 MB" % (
                       stats["device_bytes"] / 1e6)},
        "e2e": e2e_line,
        "gpu_launches": int(info["kernel_launches"]),
        "cg_iterations_per_step": info["cg_iterations"] / max(1, args.steps),
        "sweep_ms": sweep_ms,
        other + "_step": other_rec,
        "time_to_converged": ttc,
        "fp64": fp64,
        "roofline": roofline,
        "clocks": clocks,
    }
    solver.close()
    if rank == 0 and ws == 1 and not args.no_serve:
        out["serving"] = serving_summary()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, max_seconds=args.cpu_seconds)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


# ---------------------------------------------------------------- CPU baseline
# The FP64 oracle on this host's cores: worker processes (spawned, so that no
# CUDA state is inherited), each with its own OracleSolver of the workload,
# each solving a sample of (direction, band) tasks of the first transport
# pass from T_ref (every wall then feeds in the equilibrium at T_ref).
_BASE = None


class _FirstPassIncoming:
    """Incoming wall values of the first pass from T_ref, indexed like the
    oracle's (half-face, band, direction) array, one band at a time."""

    def __init__(self, o):
        import numpy as np
        self.o = o
        self.eb0 = np.zeros((o.bcells.size, o.D))
        self.band = {}

    def __getitem__(self, key):
        h, l, i = key
        if l not in self.band:
            self.band = {l: self.o.incoming_band(self.eb0, l)}
        return self.band[l][h, i]


def _base_init(workload):
    global _BASE
    import numpy as np
    import workloads as W
    from oracle import OracleSolver
    o = OracleSolver(getattr(W.problems, workload)())
    _BASE = (o, np.zeros(o.N), _FirstPassIncoming(o))


def _base_run(tasks):
    """Solve `tasks` (one transport pass over them, moments included);
    returns the seconds it took."""
    o, T0, e_in = _BASE
    dirs = sorted({i for i, _ in tasks})
    t0 = time.perf_counter()
    o.sweep(T0, None, tasks=tasks, e_in=e_in, eb_dirs=dirs)
    return time.perf_counter() - t0


class OraclePool:
    """``workers`` processes, each owning a set of directions of the
    workload; ``run(k)`` has every worker solve k tasks of its directions
    (bands in turn) at once and returns the wall time."""

    def __init__(self, workload, workers=None):
        import multiprocessing as mp
        import workloads as W
        p = getattr(W.problems, workload)()
        self.n_cells, self.n_bands, self.n_dirs = p.n_cells, p.n_bands, p.n_dirs
        avail = len(os.sched_getaffinity(0))
        self.workers = max(1, min(workers or avail, 32, p.n_dirs))
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_base_init, initargs=(workload,))
        self.next = [0] * self.workers

    def _tasks(self, w, k):
        out = []
        for _ in range(k):
            j = self.next[w]
            self.next[w] += 1
            i = (w + self.workers * (j // self.n_bands)) % self.n_dirs
            out.append((i, j % self.n_bands))
        return out

    def run(self, k):
        jobs = [self._tasks(w, k) for w in range(self.workers)]
        t0 = time.perf_counter()
        self.pool.map(_base_run, jobs, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(workload, max_seconds=20.0, steps=1, warmup=1, pool=None):
    """The FP64 oracle on this host's cores on a bounded sample of the same
    workload: each worker solves the same number of (direction, band) tasks
    of one transport pass (the per-direction set-up of each worker's first
    direction runs in an untimed warm-up), scaled to updates/s."""
    own = pool is None
    pool = pool or OraclePool(workload)
    t_one = pool.run(1)                                   # warm-up: builds every worker's first direction
    k = int(max(1, min(pool.n_bands, max_seconds / (max(steps, 1) * max(t_one, 1e-3)))))
    for _ in range(warmup):
        pool.run(k)
    dt = 0.0
    for _ in range(steps):
        dt += pool.run(k)
    dt /= steps
    n_tasks = k * pool.workers
    if own:
        pool.close()
    return {"value": n_tasks * pool.n_cells / dt, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
            "sample": f"{n_tasks} of {pool.n_dirs * pool.n_bands} (direction, band) tasks of one transport pass "
                      f"from T_ref ({pool.n_cells} cells each; moments included), {k} per worker process; "
                      f"sparse LU of Eq. (13) in a fill-free upwind order (SciPy), one process per core",
            "seconds_per_step": dt}


def serving_summary(n_requests=8, n_range=(20000, 80000), tol=1e-8):
    """Batched and served forms against one solve at a time, on a small
    seeded request stream (2D tri / 3D hex / 3D tet geometries, mixed band
    counts, direction sets, heat loads and walls), every request submitted
    at once: one at a time (nbte_solve_steady per request, planning
    included), one nbte_solve_batch call, and the continuous-batching server.
    Same options and tolerance in every arm (synthetic scheme, FP32 sweep,
    fixed layout); the largest relative temperature difference between each
    arm's results and the one-at-a-time ones is reported beside the rates."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2607_03226_b300 import nbte

    reqs = W.stream.requests(n_requests, rate=1.0, n_range=n_range)
    probs = [W.stream.build(r) for r in reqs]
    opts = dict(scheme="synthetic", precision="fp32", tol=tol, max_iter=20000, band_group=2, cta_threads=160,
                use_graph=True, skip_outputs=True)
    upd = [p.updates_per_iteration for p in probs]

    def rel(T, Tref, p):
        return float(np.abs(T - Tref).max() / max(np.abs(Tref - p.T_ref).max(), 1e-300))

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    alone, work1 = [], 0
    for p, u in zip(probs, upd):
        s = nbte.Solver(p)
        info = s.solve(**opts)
        alone.append(s.temperature(0))
        work1 += u * info["iterations"]
        s.close()
    t_one = time.perf_counter() - t0

    solvers = [nbte.Solver(p) for p in probs]
    t0 = time.perf_counter()
    infos = nbte.solve_batch(solvers, **opts)
    t_batch = time.perf_counter() - t0
    work2 = sum(u * i["iterations"] for u, i in zip(upd, infos))
    d_batch = max(rel(s.temperature(0), T, p) for s, T, p in zip(solvers, alone, probs))
    for s in solvers:
        s.close()

    solvers = [nbte.Solver(p) for p in probs]
    srv = nbte.Server(max_active=32, n_planners=4, **opts)
    t0 = time.perf_counter()
    ids = [srv.submit(s) for s in solvers]
    srv.drain(timeout_s=600)
    t_srv = time.perf_counter() - t0
    polls = [srv.poll(i) for i in ids]
    work3 = sum(u * pl[0]["iterations"] for u, pl in zip(upd, polls))
    failed = sum(pl[0]["status"] != 0 for pl in polls)
    lat = np.array([pl[1] for pl in polls])
    d_srv = max(rel(s.temperature(0), T, p) for s, T, p in zip(solvers, alone, probs))
    srv.close()
    for s in solvers:
        s.close()
    return {"requests": len(probs), "cells": list(n_range), "tol": tol,
            "one_at_a_time": {"updates_per_s": work1 / t_one, "makespan_s": t_one},
            "batched": {"updates_per_s": work2 / t_batch, "makespan_s": t_batch, "max_rel_T_vs_alone": d_batch},
            "served": {"updates_per_s": work3 / t_srv, "makespan_s": t_srv, "max_rel_T_vs_alone": d_srv,
                       "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                       "failed": int(failed)},
            "speedup_batched": (work2 / t_batch) / (work1 / t_one),
            "speedup_served": (work3 / t_srv) / (work1 / t_one),
            "layout": "band_group=2 cta_threads=160, synthetic scheme, FP32 sweep, every request at once"}


def run_stream(args):
    """Serving: a seeded stream of steady solves (2D tri / 3D hex / 3D tet
    geometries, mixed sizes, band counts, direction sets, heat loads and
    walls) with Poisson arrivals.  One-at-a-time arm: each request solved
    alone with nbte_solve_steady (planning included), its FIFO queueing
    replayed from the measured service times.  Served arm: the same requests
    submitted in real time to the continuous-batching server.  Both report
    throughput and p50/p99 time-to-converged (arrival to converged field)."""
    import threading
    import numpy as np
    import torch
    import workloads as W
    from paper_2607_03226_b300 import nbte

    ws, rank = _dist()
    if rank != 0:
        return
    torch.cuda.set_device(0)
    reqs = W.stream.requests(args.requests, rate=1.0, n_range=(args.min_cells, args.max_cells))
    probs = [W.stream.build(r) for r in reqs]
    opts = dict(scheme="synthetic", precision=args.precision, tol=args.stream_tol, max_iter=20000,
                band_group=2, cta_threads=160, use_graph=True, skip_outputs=False)
    upd = [p.updates_per_iteration for p in probs]
    # ---- one at a time
    service, iters = [], []
    for p in probs:
        s = nbte.Solver(p)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = s.solve(**opts)
        service.append(time.perf_counter() - t0)
        iters.append(info["iterations"])
        s.close()
    mu = len(service) / sum(service)                     # one-at-a-time service rate (requests/s)
    rate = args.load * mu
    rng = np.random.default_rng(2607032265)
    arrival = np.cumsum(rng.exponential(1.0 / rate, size=len(probs)))
    arrival -= arrival[0]
    finish, free = [], 0.0
    for a, sv in zip(arrival, service):
        free = max(free, a) + sv
        finish.append(free)
    lat1 = np.array(finish) - arrival
    work = sum(u * it for u, it in zip(upd, iters))
    one = {"throughput_req_s": len(probs) / finish[-1], "updates_per_s": work / finish[-1],
           "p50_s": float(np.percentile(lat1, 50)), "p99_s": float(np.percentile(lat1, 99)),
           "mean_service_s": float(np.mean(service))}
    # ---- served
    solvers = [nbte.Solver(p) for p in probs]
    srv = nbte.Server(max_active=args.max_active, n_planners=args.planners, **opts)
    ids = [None] * len(probs)
    t_start = time.perf_counter()

    def feeder():
        for k, a in enumerate(arrival):
            dt = t_start + a - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ids[k] = srv.submit(solvers[k])

    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    srv.drain(timeout_s=3600)
    makespan = time.perf_counter() - t_start
    lat2, iters2, errs = [], [], 0
    for k in range(len(probs)):
        info, total, queued = srv.poll(ids[k])
        lat2.append(total)
        iters2.append(info["iterations"])
        errs += info["status"] != 0
    work2 = sum(u * it for u, it in zip(upd, iters2))
    st = srv.stats()
    srv.close()
    for s in solvers:
        s.close()
    lat2 = np.array(lat2)
    served = {"throughput_req_s": len(probs) / makespan, "updates_per_s": work2 / makespan,
              "p50_s": float(np.percentile(lat2, 50)), "p99_s": float(np.percentile(lat2, 99)),
              "batched_iterations": st["iterations"], "failed": int(errs)}
    # ---- capacity: every request submitted at once (throughput is then the
    # server's, not the arrival rate's); one at a time it is the summed service
    solvers = [nbte.Solver(p) for p in probs]
    srv = nbte.Server(max_active=args.max_active, n_planners=args.planners, **opts)
    t0 = time.perf_counter()
    ids = [srv.submit(s) for s in solvers]
    srv.drain(timeout_s=3600)
    burst = time.perf_counter() - t0
    iters3 = [srv.poll(i)[0]["iterations"] for i in ids]
    srv.close()
    for s in solvers:
        s.close()
    work3 = sum(u * it for u, it in zip(upd, iters3))
    capacity = {"served_updates_per_s": work3 / burst, "served_req_s": len(probs) / burst,
                "one_at_a_time_updates_per_s": work / sum(service), "one_at_a_time_req_s": mu,
                "served_makespan_s": burst, "one_at_a_time_makespan_s": sum(service)}
    out = {"metric": "serve time-to-converged p50 (p99 beside)", "value": served["p50_s"], "unit": "s",
           "n_gpus": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 sweep / f64 moments+update+CG" if args.precision == "fp32" else "f64",
           "data": "synthetic (seeded request stream)",
           "config": {"workload": "stream: Poisson arrivals of 2D tri / 3D hex / 3D tet steady solves",
                      "requests": len(probs), "cells": [args.min_cells, args.max_cells],
                      "load": args.load, "arrival_rate_req_s": rate, "tol": args.stream_tol,
                      "max_active": args.max_active, "layout": "band_group=2 cta_threads=160"},
           "served": served, "one_at_a_time": one, "capacity": capacity,
           "speedup_capacity": capacity["served_updates_per_s"] / capacity["one_at_a_time_updates_per_s"]}
    print(json.dumps(out))


def run_converge(args):
    """The 3D workloads' measurement: time and iterations to a converged
    field, synthetic against sequential, from T_ref and from the diffusion
    (Fourier) guess, plus the per-step rate of each scheme.  FP64 sweeps
    reach the 1e-8 tolerance these workloads are specified with; FP32 sweeps
    stop at their rounding floor (about 5e-8), so they are run to 1e-6."""
    import torch
    import workloads as W
    from paper_2607_03226_b300 import nbte

    ws, rank = _dist()
    if rank != 0:
        return
    torch.cuda.set_device(0)
    p = getattr(W.problems, args.workload)()
    solver = nbte.Solver(p)
    tol = 1e-8 if args.precision == "fp64" else 1e-6
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    runs = {}
    for sch in ("synthetic", "sequential"):
        for init in ("tref", "fourier"):
            kw = dict(scheme=sch, precision=args.precision, tol=tol, max_iter=args.max_iter, cg_tol=args.cg_tol,
                      use_graph=True, skip_outputs=True, init=init)
            solver.solve(n_iter=2, **{k: v for k, v in kw.items() if k not in ("tol", "max_iter")})  # plan, tune, graph
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = solver.solve(**kw)
            torch.cuda.synchronize()
            runs[f"{sch}_{init}"] = {"seconds": time.perf_counter() - t0, "iterations": info["iterations"],
                                     "residual": info["residual"], "status": info["status"],
                                     "cg_iterations": info["cg_iterations"]}
            print(json.dumps({sch + "_" + init: runs[f"{sch}_{init}"]}), file=sys.stderr, flush=True)
    steps = {}
    for sch in ("synthetic", "sequential"):
        kw = dict(scheme=sch, precision=args.precision, cg_tol=args.cg_tol, use_graph=True, skip_outputs=True)
        solver.solve(n_iter=3, warm=True, **kw)
        torch.cuda.synchronize()
        e0.record(stream)
        solver.solve(n_iter=args.steps, warm=True, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        steps[sch] = {"ms_per_step": ms, "updates_per_s": p.updates_per_iteration / (ms * 1e-3)}
    st = solver.plan_stats(precision=args.precision, scheme="synthetic")
    solver.close()
    best = min(runs, key=lambda k: runs[k]["seconds"] if runs[k]["status"] == 0 else 1e30)
    out = {"metric": "time to converged field", "value": runs[best]["seconds"], "unit": "s", "n_gpus": 1,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 sweep / f64 moments+update+CG" if args.precision == "fp32" else "f64",
           "data": "synthetic (seeded mesh and spectrum)",
           "config": {"workload": args.workload, "n_cells": p.n_cells, "bands": p.n_bands, "directions": p.n_dirs,
                      "tol": tol, "precision": args.precision, "cg_tol": args.cg_tol, "best": best,
                      "band_group": st["band_group"], "cta_threads": st["cta_threads"],
                      "ring": "global" if st["ring"] == 2 else "shared"},
           "runs": runs, "steps": steps,
           "synthetic_vs_sequential_iterations": runs["sequential_tref"]["iterations"] /
           max(1, runs["synthetic_tref"]["iterations"])}
    print(json.dumps(out))


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on this host's cores,
    timed on a bounded sample of the same workload each step (one transport
    pass over an equal number of (direction, band) tasks per worker process),
    so that the whole --steps/--warmup run ends within a few minutes."""
    ws, rank = _dist()
    if rank != 0:
        return
    desc, scheme0 = WORKLOADS[args.workload]
    pool = OraclePool(args.workload)
    t_one = pool.run(1)                                   # untimed: every worker's first direction
    per_step = max(1.0, 150.0 / max(1, args.steps + args.warmup))
    k = int(max(1, min(pool.n_bands, per_step / max(t_one, 1e-3))))
    for _ in range(args.warmup):
        pool.run(k)
    dts = [pool.run(k) for _ in range(args.steps)]
    pool.close()
    dt = sum(dts) / len(dts)
    n_tasks = k * pool.workers
    value = n_tasks * pool.n_cells / dt
    sample = (f"{n_tasks} of {pool.n_dirs * pool.n_bands} (direction, band) tasks of one transport pass from T_ref "
              f"per step ({pool.n_cells} cells each), {k} per worker process; sparse LU of Eq. (13) in a fill-free "
              f"upwind order (SciPy), one process per core")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded mesh, spectrum and heat source)",
           "config": {"workload": desc, "scheme": f"{scheme0} (oracle transport pass)", "n_cells": pool.n_cells,
                      "bands": pool.n_bands, "directions": pool.n_dirs},
           "impl": "reference",
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.workers, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="nbte", choices=["nbte", "reference"])
    ap.add_argument("--workload", default="finfet3d", choices=["finfet3d", "finfet2d", "cube3d", "stream"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--scheme", default=None, choices=["synthetic", "sequential"],
                    help="default: the scheme the workload is specified with")
    ap.add_argument("--band-group", type=int, default=0)
    ap.add_argument("--cta-threads", type=int, default=0)
    ap.add_argument("--cg-tol", type=float, default=1e-2)
    ap.add_argument("--order", type=int, default=1, choices=[1, 2],
                    help="upwind order of the face values (2: deferred least-squares reconstruction)")
    ap.add_argument("--cg-max-iter", type=int, default=5000)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 path's step")
    ap.add_argument("--fp64-band-group", type=int, default=0)
    ap.add_argument("--fp64-cta-threads", type=int, default=0)
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--no-converge", action="store_true", help="skip the time to a converged field")
    ap.add_argument("--converge-tol", type=float, default=0.0)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the batched / served / one-at-a-time comparison on a small request stream")
    ap.add_argument("--converge", action="store_true",
                    help="time and iterations to a converged field, both schemes and starts (3D workloads)")
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--min-cells", type=int, default=20000)
    ap.add_argument("--max-cells", type=int, default=500000)
    ap.add_argument("--load", type=float, default=0.9)
    ap.add_argument("--stream-tol", type=float, default=1e-8)
    ap.add_argument("--max-active", type=int, default=32)
    ap.add_argument("--planners", type=int, default=4)
    args = ap.parse_args()
    if args.impl == "reference":
        if args.workload == "stream":
            args.workload = "finfet3d"
        run_reference(args)
    elif args.workload == "stream":
        run_stream(args)
    elif args.converge:
        run_converge(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
