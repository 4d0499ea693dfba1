"""Serving (nbte_server_*): solves of different meshes, band counts and heat
loads submitted over time to a continuous-batching server.  Requests that
arrive while others are iterating join the batch; each result must equal
the same solve alone: FP64 temperature within 1e-9 (the CG's block share,
and with it its rounding, depends on the mix)."""
import time

import numpy as np
import pytest

from cases import rel_T
from test_gpu_batch import _problems

pytestmark = pytest.mark.gpu

OPTS = dict(scheme="synthetic", precision="fp64", tol=1e-12, max_iter=20000, use_graph=True)


@pytest.fixture(scope="module")
def nbte_mod(gpu_lib):
    from paper_2607_03226_b300 import nbte
    return nbte


@pytest.fixture(scope="module")
def alone(nbte_mod):
    out = []
    for p in _problems():
        s = nbte_mod.Solver(p)
        info = s.solve(**OPTS)
        assert info["status"] == 0
        out.append(s.temperature(0))
        s.close()
    return out


@pytest.mark.parametrize("budget", [0, 1])
def test_served_results_equal_alone(nbte_mod, alone, budget):
    """budget 0: all requests fit and are iterated together; budget 1 byte:
    admission by memory lets one request run at a time."""
    probs = _problems()
    srv = nbte_mod.Server(budget_bytes=budget, max_active=8, n_planners=2, **OPTS)
    ss = [nbte_mod.Solver(p) for p in probs]
    ids = [srv.submit(s) for s in ss[:3]]
    t0 = time.time()
    while srv.stats()["iterations"] == 0 and time.time() - t0 < 120:   # the first wave is iterating
        time.sleep(0.005)
    ids += [srv.submit(s) for s in ss[3:]]
    srv.drain(timeout_s=600)
    st = srv.stats()
    assert st["done"] == len(probs) and st["bytes_in_use"] == 0
    admits = []
    for p, s, rid, T in zip(probs, ss, ids, alone):
        info, total, queued = srv.poll(rid)
        assert info["status"] == 0
        err = rel_T(s.temperature(0), T, p.T_ref)
        print(f"{p.name}: {info['iterations']} iterations, {total:.3f} s in the server "
              f"({queued:.3f} s before admission), T difference to the solve alone {err:.2e}")
        assert err < 1e-9
        admits.append(queued)
    srv.close()
    for s in ss:
        s.close()


def test_served_second_order_equals_alone(nbte_mod):
    """Second-order solves through the server (its options carry order=2)
    converge to the same fields as alone."""
    probs = _problems()[:3]
    opts = dict(OPTS, order=2)
    ref = []
    for p in probs:
        s = nbte_mod.Solver(p)
        assert s.solve(**opts)["status"] == 0
        ref.append(s.temperature(0))
        s.close()
    srv = nbte_mod.Server(max_active=8, n_planners=2, **opts)
    ss = [nbte_mod.Solver(p) for p in probs]
    ids = [srv.submit(s) for s in ss]
    srv.drain(timeout_s=600)
    for p, s, rid, T in zip(probs, ss, ids, ref):
        info, _, _ = srv.poll(rid)
        assert info["status"] == 0
        err = rel_T(s.temperature(0), T, p.T_ref)
        print(f"{p.name}: served second order, {info['iterations']} iterations, difference {err:.2e}")
        assert err < 1e-9
    srv.close()
    for s in ss:
        s.close()
