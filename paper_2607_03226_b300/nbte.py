"""Python binding of libnanobte (ctypes; argument marshalling only).

Every function mirrors one ``nbte_*`` call of ``include/nbte.h`` and converts
NumPy arrays to the C layout; every computation runs in the library's CUDA
kernels.  There is no fallback: if the library is not built, :func:`load`
raises.  :class:`Solver` bundles the calls for one problem.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnanobte.so")

NBTE_OK = 0
NBTE_ERR_ARG = -1
NBTE_ERR_MESH = -2
NBTE_ERR_OOM = -3
NBTE_ERR_CUDA = -4
NBTE_ERR_NOT_CONVERGED = -5
NBTE_ERR_DIVERGED = -6
NBTE_ERR_DEVICE_TIMEOUT = -7
NBTE_ERR_STATE = -8
ERR_NAMES = {0: "OK", -1: "ARG", -2: "MESH", -3: "OOM", -4: "CUDA", -5: "NOT_CONVERGED", -6: "DIVERGED",
             -7: "DEVICE_TIMEOUT", -8: "STATE"}

NBTE_TRI, NBTE_QUAD, NBTE_TET, NBTE_HEX = 3, 4, 10, 12
NBTE_THERMALIZING, NBTE_DIFFUSE, NBTE_SPECULAR, NBTE_PARTIAL = 0, 1, 2, 3
SCHEMES = {"sequential": 0, "synthetic": 1, "synthetic_literal": 2}

# every symbol include/nbte.h declares
EXPORTS = [
    "nbte_mesh_create", "nbte_mesh_destroy", "nbte_mesh_info", "nbte_solver_create", "nbte_solver_destroy",
    "nbte_solver_set_stream", "nbte_set_bands", "nbte_set_quadrature", "nbte_set_boundaries",
    "nbte_set_heat_source", "nbte_default_opts", "nbte_solve_steady", "nbte_get_temperature",
    "nbte_get_heat_flux", "nbte_get_wall_heat", "nbte_plan_stats", "nbte_last_error", "nbte_version",
    "nbte_laplacian_solve_noalloc", "nbte_get_distribution", "nbte_solve_batch", "nbte_server_create",
    "nbte_server_submit", "nbte_server_poll", "nbte_server_drain", "nbte_server_stats", "nbte_server_destroy",
    "nbte_test_timeouts",
]


class nbte_boundary(C.Structure):
    _fields_ = [("tag", C.c_int32), ("type", C.c_int32), ("T_wall", C.c_double), ("specularity", C.c_double)]


class nbte_solve_opts(C.Structure):
    _fields_ = [("scheme", C.c_int32), ("precision", C.c_int32), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("n_iter", C.c_int32), ("T_init", C.POINTER(C.c_double)),
                ("warm", C.c_int32), ("band_group", C.c_int32), ("threads_per_cell", C.c_int32),
                ("cg_tol", C.c_double), ("cg_max_iter", C.c_int32), ("use_graph", C.c_int32),
                ("skip_outputs", C.c_int32), ("profile", C.c_int32), ("cta_threads", C.c_int32),
                ("ring", C.c_int32), ("init", C.c_int32), ("order", C.c_int32), ("deterministic", C.c_int32)]


class nbte_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("residual", C.c_double), ("energy_imbalance", C.c_double),
                ("lagged_faces", C.c_int64), ("seconds", C.c_double), ("cg_iterations", C.c_int64),
                ("sweep_seconds", C.c_double), ("sweep_launches", C.c_int64), ("kernel_launches", C.c_int64),
                ("status", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class NbteError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nbte error {code} ({ERR_NAMES.get(code, '?')}): {msg}")
        self.code = code


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_I32 = C.POINTER(C.c_int32)


def load(path: str | None = None):
    """Load the built library (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -m paper_2607_03226_b300.build`")
    lib = C.CDLL(path)
    sig = {
        "nbte_mesh_create": ([C.c_int, C.c_int64, _D, C.c_int, C.c_int64, _I64, C.c_int64, _I64, _I32,
                              C.POINTER(_P)], C.c_int),
        "nbte_mesh_destroy": ([_P], C.c_int),
        "nbte_mesh_info": ([_P, _I64, _D], C.c_int),
        "nbte_solver_create": ([_P, C.c_double, C.POINTER(_P)], C.c_int),
        "nbte_solver_destroy": ([_P], C.c_int),
        "nbte_solver_set_stream": ([_P, _P], C.c_int),
        "nbte_set_bands": ([_P, C.c_int, _D, _D, _D], C.c_int),
        "nbte_set_quadrature": ([_P, C.c_int, _D, _D], C.c_int),
        "nbte_set_boundaries": ([_P, C.c_int, C.POINTER(nbte_boundary)], C.c_int),
        "nbte_set_heat_source": ([_P, _D], C.c_int),
        "nbte_default_opts": ([C.POINTER(nbte_solve_opts)], C.c_int),
        "nbte_solve_steady": ([_P, C.POINTER(nbte_solve_opts), C.POINTER(nbte_solve_info)], C.c_int),
        "nbte_get_temperature": ([_P, C.c_int, _D], C.c_int),
        "nbte_get_heat_flux": ([_P, _D], C.c_int),
        "nbte_get_wall_heat": ([_P, C.c_int32, _D], C.c_int),
        "nbte_get_distribution": ([_P, C.c_int32, C.c_int32, _D], C.c_int),
        "nbte_solve_batch": ([C.POINTER(_P), C.c_int32, C.POINTER(nbte_solve_opts), C.POINTER(nbte_solve_info)],
                             C.c_int),
        "nbte_server_create": ([C.POINTER(nbte_solve_opts), C.c_size_t, C.c_int32, C.c_int32, C.POINTER(_P)], C.c_int),
        "nbte_server_submit": ([_P, _P, _I64], C.c_int),
        "nbte_server_poll": ([_P, C.c_int64, _I32, C.POINTER(nbte_solve_info), _D], C.c_int),
        "nbte_server_drain": ([_P, C.c_double], C.c_int),
        "nbte_server_stats": ([_P, _I64], C.c_int),
        "nbte_server_destroy": ([_P], C.c_int),
        "nbte_plan_stats": ([_P, C.POINTER(nbte_solve_opts), _I64], C.c_int),
        "nbte_last_error": ([], C.c_char_p),
        "nbte_version": ([], C.c_char_p),
        "nbte_laplacian_solve_noalloc": ([C.c_int, _P, _P, _P, _P, _P, C.c_double, C.c_int, _I32, _D, _P],
                                         C.c_int),
        "nbte_test_timeouts": ([C.c_int32], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc, allow=()):
    if rc != NBTE_OK and rc not in allow:
        raise NbteError(rc, load().nbte_last_error().decode())
    return rc


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_I64)


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_I32)


# ------------------------------------------------------------------ thin calls
def nbte_mesh_create(dim, nodes, cell_type, cells, bfaces, btags):
    lib = load()
    nodes, pn = _d(nodes)
    cells, pc = _i64(cells)
    bfaces, pb = _i64(bfaces)
    btags, pt = _i32(btags)
    out = _P()
    _check(lib.nbte_mesh_create(int(dim), nodes.shape[0], pn, int(cell_type), cells.shape[0], pc,
                                bfaces.shape[0], pb, pt, C.byref(out)))
    return out


def nbte_mesh_destroy(mesh):
    return _check(load().nbte_mesh_destroy(mesh))


def nbte_mesh_info(mesh):
    n = C.c_int64()
    v = C.c_double()
    _check(load().nbte_mesh_info(mesh, C.byref(n), C.byref(v)))
    return n.value, v.value


def nbte_solver_create(mesh, T_ref):
    out = _P()
    _check(load().nbte_solver_create(mesh, float(T_ref), C.byref(out)))
    return out


def nbte_solver_destroy(solver):
    return _check(load().nbte_solver_destroy(solver))


def nbte_solver_set_stream(solver, stream_ptr):
    return _check(load().nbte_solver_set_stream(solver, _P(stream_ptr) if stream_ptr else None))


def nbte_set_bands(solver, C_, v, tau):
    C_, pc = _d(C_)
    v, pv = _d(v)
    tau, pt = _d(tau)
    return _check(load().nbte_set_bands(solver, C_.size, pc, pv, pt))


def nbte_set_quadrature(solver, s, w):
    s, ps = _d(np.asarray(s, dtype=np.float64).reshape(-1, 3))
    w, pw = _d(w)
    return _check(load().nbte_set_quadrature(solver, w.size, ps, pw))


def nbte_set_boundaries(solver, bcs):
    arr = (nbte_boundary * len(bcs))()
    for k, b in enumerate(bcs):
        arr[k].tag, arr[k].type = int(b.tag), int(b.type)
        arr[k].T_wall, arr[k].specularity = float(b.T_wall), float(b.specularity)
    return _check(load().nbte_set_boundaries(solver, len(bcs), arr))


def nbte_set_heat_source(solver, Qdot):
    if Qdot is None:
        return _check(load().nbte_set_heat_source(solver, None))
    Qdot, pq = _d(Qdot)
    return _check(load().nbte_set_heat_source(solver, pq))


def nbte_default_opts():
    o = nbte_solve_opts()
    _check(load().nbte_default_opts(C.byref(o)))
    return o


def make_opts(scheme="sequential", precision="fp64", tol=1e-10, max_iter=10000, n_iter=0, T_init=None,
              warm=False, band_group=0, threads_per_cell=0, cg_tol=0.0, cg_max_iter=0, use_graph=False,
              skip_outputs=False, profile=False, cta_threads=0, ring=0, init="tref", order=1,
              deterministic=False):
    o = nbte_default_opts()
    o.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    o.precision = {"fp64": 0, "fp32": 1}[precision] if isinstance(precision, str) else int(precision)
    o.tol, o.max_iter, o.n_iter = float(tol), int(max_iter), int(n_iter)
    o.warm, o.band_group, o.threads_per_cell = int(bool(warm)), int(band_group), int(threads_per_cell)
    o.cg_tol, o.cg_max_iter, o.use_graph = float(cg_tol), int(cg_max_iter), int(bool(use_graph))
    o.skip_outputs, o.profile, o.cta_threads = int(bool(skip_outputs)), int(bool(profile)), int(cta_threads)
    o.ring = {"auto": 0, "shared": 1, "global": 2}[ring] if isinstance(ring, str) else int(ring)
    o.init = {"tref": 0, "fourier": 1}[init] if isinstance(init, str) else int(init)
    o.order = int(order)
    o.deterministic = int(bool(deterministic))
    keep = None
    if T_init is not None:
        keep, o.T_init = _d(T_init)
    o._keep = keep  # keeps T_init alive for the call
    return o


def nbte_solve_steady(solver, opts):
    info = nbte_solve_info()
    rc = _check(load().nbte_solve_steady(solver, C.byref(opts), C.byref(info)),
                allow=(NBTE_ERR_NOT_CONVERGED,))
    return rc, info


def nbte_solve_batch(solvers, opts):
    """Solve several solvers together; returns (rc, [info per solver])."""
    n = len(solvers)
    arr = (_P * n)(*solvers)
    infos = (nbte_solve_info * n)()
    rc = _check(load().nbte_solve_batch(arr, n, C.byref(opts), infos), allow=(NBTE_ERR_NOT_CONVERGED,))
    return rc, list(infos)


def solve_batch(solvers, **kw):
    """Solve several :class:`Solver` objects together (one options set);
    returns the per-solver info dicts."""
    rc, infos = nbte_solve_batch([s.solver for s in solvers], make_opts(**kw))
    return [i.as_dict() for i in infos]


class Server:
    """Continuous-batching request queue (nbte_server_*): submit set-up
    :class:`Solver` objects, poll or drain, read results from the solvers."""

    def __init__(self, budget_bytes=0, max_active=64, n_planners=2, **opts):
        self._opts = make_opts(**opts)
        h = _P()
        _check(load().nbte_server_create(C.byref(self._opts), int(budget_bytes), int(max_active), int(n_planners),
                                         C.byref(h)))
        self.server = h

    def submit(self, solver):
        rid = C.c_int64()
        _check(load().nbte_server_submit(self.server, solver.solver, C.byref(rid)))
        return rid.value

    def poll(self, request):
        """None while queued or running, else (info dict, seconds submit-to-done,
        seconds submit-to-admission)."""
        state = C.c_int32()
        info = nbte_solve_info()
        sec = (C.c_double * 2)()
        rc = load().nbte_server_poll(self.server, int(request), C.byref(state), C.byref(info), sec)
        if state.value != 3:
            _check(rc)
            return None
        d = info.as_dict()
        d["status"] = rc
        return d, sec[0], sec[1]

    def drain(self, timeout_s=0.0):
        _check(load().nbte_server_drain(self.server, float(timeout_s)))

    def stats(self):
        st = np.zeros(4, dtype=np.int64)
        _check(load().nbte_server_stats(self.server, st.ctypes.data_as(_I64)))
        return dict(zip(["iterations", "submitted", "done", "bytes_in_use"], (int(x) for x in st)))

    def close(self):
        if getattr(self, "server", None):
            load().nbte_server_destroy(self.server)
            self.server = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _out(out, shape):
    """The caller's result array (C-contiguous float64 of this shape), or a
    new one.  A page-locked array (e.g. a pinned torch tensor's .numpy())
    is filled by DMA directly."""
    if out is None:
        return np.empty(shape, dtype=np.float64)
    if out.dtype != np.float64 or out.shape != shape or not out.flags.c_contiguous or not out.flags.writeable:
        raise ValueError(f"out must be a writeable C-contiguous float64 array of shape {shape}")
    return out


def nbte_get_temperature(solver, kind, n_cells, out=None):
    out = _out(out, (n_cells,))
    _check(load().nbte_get_temperature(solver, int(kind), out.ctypes.data_as(_D)))
    return out


def nbte_get_heat_flux(solver, n_cells, dim, out=None):
    out = _out(out, (n_cells, dim))
    _check(load().nbte_get_heat_flux(solver, out.ctypes.data_as(_D)))
    return out


def nbte_get_distribution(solver, direction, band, n_cells):
    out = np.empty(n_cells, dtype=np.float64)
    _check(load().nbte_get_distribution(solver, int(direction), int(band), out.ctypes.data_as(_D)))
    return out


def nbte_get_wall_heat(solver, tag):
    v = C.c_double()
    _check(load().nbte_get_wall_heat(solver, int(tag), C.byref(v)))
    return v.value


def nbte_plan_stats(solver, opts=None):
    st = np.zeros(12, dtype=np.int64)
    _check(load().nbte_plan_stats(solver, C.byref(opts) if opts is not None else None, st.ctypes.data_as(_I64)))
    keys = ["total_levels", "max_levels", "max_slots", "lagged_faces", "items", "band_group",
            "ring", "device_bytes", "K", "exports", "imports", "cta_threads"]
    return dict(zip(keys, (int(x) for x in st)))


def nbte_laplacian_solve_noalloc(n, row_ptr_dev, col_dev, val_dev, rhs_dev, x_dev, tol, max_iter, stream=0):
    """Allocation-free CG solve on caller-owned device buffers (raw device
    addresses as ints).  Returns (status, iterations, residual)."""
    it = C.c_int32()
    res = C.c_double()
    rc = _check(load().nbte_laplacian_solve_noalloc(
        int(n), _P(row_ptr_dev), _P(col_dev), _P(val_dev), _P(rhs_dev), _P(x_dev), float(tol), int(max_iter),
        C.byref(it), C.byref(res), _P(stream) if stream else None), allow=(NBTE_ERR_NOT_CONVERGED,))
    return rc, it.value, res.value


def nbte_test_timeouts(on):
    """Make every bounded device wait of later launches run out (on), or
    restore normal operation."""
    _check(load().nbte_test_timeouts(int(bool(on))))


def nbte_last_error():
    return load().nbte_last_error().decode()


def nbte_version():
    return load().nbte_version().decode()


# ------------------------------------------------------------------ helper
class Solver:
    """One mesh + solver pair set up from a problem description (any object
    with ``mesh, C, v, tau, s, w, boundaries, Q, T_ref``)."""

    def __init__(self, problem, stream=None):
        m = problem.mesh
        self.dim = int(m.dim)
        self.n_cells = int(m.cells.shape[0])
        self.mesh = nbte_mesh_create(m.dim, m.nodes, m.cell_type, m.cells, m.bfaces, m.btags)
        self.solver = nbte_solver_create(self.mesh, problem.T_ref)
        if stream is not None:
            nbte_solver_set_stream(self.solver, stream)
        nbte_set_bands(self.solver, problem.C, problem.v, problem.tau)
        nbte_set_quadrature(self.solver, problem.s, problem.w)
        nbte_set_boundaries(self.solver, problem.boundaries)
        nbte_set_heat_source(self.solver, problem.Q)
        self.tags = sorted({int(b.tag) for b in problem.boundaries})

    def solve(self, **kw):
        opts = make_opts(**kw)
        rc, info = nbte_solve_steady(self.solver, opts)
        d = info.as_dict()
        d["status"] = rc
        return d

    def temperature(self, kind=0, out=None):
        return nbte_get_temperature(self.solver, kind, self.n_cells, out)

    def heat_flux(self, out=None):
        return nbte_get_heat_flux(self.solver, self.n_cells, self.dim, out)

    def wall_heat(self, tag):
        return nbte_get_wall_heat(self.solver, tag)

    def distribution(self, direction, band):
        return nbte_get_distribution(self.solver, direction, band, self.n_cells)

    def plan_stats(self, **kw):
        return nbte_plan_stats(self.solver, make_opts(**kw))

    def close(self):
        if getattr(self, "solver", None):
            nbte_solver_destroy(self.solver)
            self.solver = None
        if getattr(self, "mesh", None):
            nbte_mesh_destroy(self.mesh)
            self.mesh = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
