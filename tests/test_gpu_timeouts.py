"""Failure detection without a GPU fault: every device-side wait of the
library is bounded, and nbte_test_timeouts makes the waits run out -- the
sweep's producer issues no copy (a barrier phase nothing completes, so each
consumer's wait runs out on its bound of about a second) and the CG barriers
give up after one poll.  Each kernel then sets its error word and returns
(a sweep consumer whose wait ran out stops computing and keeps the barrier
sequence); the call reports NBTE_ERR_DEVICE_TIMEOUT, and the same solver,
back in normal operation, solves to the oracle's result on the next call.
Nothing here hangs or faults: a wait that runs out only ends its kernel
early."""
import numpy as np
import pytest

from oracle import OracleSolver
from cases import fin2d_mixed, rel_T

pytestmark = pytest.mark.gpu


@pytest.fixture
def nbte_mod(gpu_lib):
    from paper_2607_03226_b300 import nbte
    nbte.nbte_test_timeouts(0)
    yield nbte
    nbte.nbte_test_timeouts(0)


def _timed_out(nbte, call, tries=3):
    """Run call() with every wait made to run out until it reports a
    timeout (a CG barrier whose blocks all arrived at once passes its single
    poll, so a launch may occasionally get through); returns the status code
    seen."""
    code = None
    for _ in range(tries):
        nbte.nbte_test_timeouts(1)
        try:
            call()
            code = nbte.NBTE_OK
        except nbte.NbteError as e:
            code = e.code
        finally:
            nbte.nbte_test_timeouts(0)
        if code == nbte.NBTE_ERR_DEVICE_TIMEOUT:
            break
    return code


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_sweep_wait_gives_up_then_next_solve_is_exact(nbte_mod, precision, tol):
    nbte = nbte_mod
    p = fin2d_mixed()
    s = nbte.Solver(p)
    kw = dict(scheme="sequential", precision=precision, band_group=1, cta_threads=64)
    s.solve(n_iter=1, **kw)    # plan and layout with the default limit
    code = _timed_out(nbte, lambda: s.solve(n_iter=1, **kw))
    assert code == nbte.NBTE_ERR_DEVICE_TIMEOUT
    assert "gave up" in nbte.nbte_last_error()
    # warm is asked for, but after a timeout the solver starts over from T_ref
    s.solve(n_iter=3, warm=True, **kw)
    ref = OracleSolver(p).solve(scheme="sequential", n_iter=3)
    assert rel_T(s.temperature(0), ref["T"], p.T_ref) < tol
    s.close()


def test_cg_barrier_gives_up_then_next_solve_is_exact(nbte_mod):
    """The diffusion initial guess runs the synthetic correction's CG (a
    cooperative grid of many blocks) before any sweep: with one poll per
    barrier wait the early blocks give up."""
    nbte = nbte_mod
    p = fin2d_mixed()
    s = nbte.Solver(p)
    kw = dict(scheme="synthetic", precision="fp64", init="fourier", cg_tol=1e-12, cg_max_iter=20000)
    s.solve(n_iter=1, **kw)
    code = _timed_out(nbte, lambda: s.solve(n_iter=2, **kw))
    assert code == nbte.NBTE_ERR_DEVICE_TIMEOUT
    info = s.solve(tol=1e-13, max_iter=20000, **kw)
    assert info["status"] == 0
    ref = OracleSolver(p).solve(scheme="synthetic", tol=1e-14, max_iter=20000)
    assert rel_T(s.temperature(0), ref["T"], p.T_ref) < 1e-9
    s.close()


def test_batched_sweep_wait_gives_up(nbte_mod):
    """The fused multi-solver sweep: a timeout is reported for the batch and
    both solvers solve correctly afterwards."""
    nbte = nbte_mod
    p = fin2d_mixed()
    a, b = nbte.Solver(p), nbte.Solver(p)
    kw = dict(scheme="sequential", precision="fp64", band_group=1, cta_threads=64)
    nbte.solve_batch([a, b], n_iter=1, **kw)

    def batch():
        infos = nbte.solve_batch([a, b], n_iter=1, **kw)
        codes = {i["status"] for i in infos}
        if nbte.NBTE_ERR_DEVICE_TIMEOUT in codes:
            raise nbte.NbteError(nbte.NBTE_ERR_DEVICE_TIMEOUT, "batch")

    assert _timed_out(nbte, batch) == nbte.NBTE_ERR_DEVICE_TIMEOUT
    infos = nbte.solve_batch([a, b], n_iter=3, **kw)
    assert all(i["status"] == 0 for i in infos)
    ref = OracleSolver(p).solve(scheme="sequential", n_iter=3)
    for s in (a, b):
        assert rel_T(s.temperature(0), ref["T"], p.T_ref) < 1e-11
        s.close()
