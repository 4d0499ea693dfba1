"""The host's stopping rule for the outer iteration
(paper_2607_03226_b300/csrc/iteration_monitor.h), compiled with the host C++
compiler and fed increment sequences of known behaviour: a converging linear
iteration, a diverging one (spectral radius above one), an FP32-like rounding
floor, a non-finite value, a fixed iteration count and a transient that grows
briefly before converging.  No GPU needed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2607_03226_b300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "iteration_monitor.h"
using nbte::IterationMonitor;
int main() {
  int n; double tol; int limit, fixed, fp32;
  while (std::scanf("%d %lf %d %d %d", &n, &tol, &limit, &fixed, &fp32) == 5) {
    IterationMonitor m; m.tol = tol; m.limit = limit; m.fixed = fixed; m.fp32 = fp32;
    int stop_it = -1, verdict = 0;
    for (int k = 0; k < n; ++k) {
      double d, t; std::scanf("%lf %lf", &d, &t);
      if (stop_it >= 0) continue;
      const int v = m.step(d, t);
      if (v != IterationMonitor::CONTINUE) { stop_it = m.it; verdict = v; }
    }
    std::printf("%d %d %.17g\n", verdict, stop_it, m.r);
  }
  return 0;
}
"""

CONVERGED, FLOOR, LIMIT, DIVERGED = 1, 2, 3, 4


@pytest.fixture(scope="module")
def monitor(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("monitor")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(dmax, tmax, tol=1e-10, limit=10000, fixed=False, fp32=False):
        lines = [f"{len(dmax)} {tol!r} {limit} {int(fixed)} {int(fp32)}"]
        lines += [f"{float(a)!r} {float(b)!r}" for a, b in zip(dmax, tmax)]
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout.split()
        return int(out[0]), int(out[1]), float(out[2])
    return run


def _linear(rho, n, T_inf=1.0, T0=0.0):
    """max|dT| and max|T| of T_n = T_inf + (T0 - T_inf) rho^n (a scalar
    linear fixed-point iteration)."""
    T = T_inf + (T0 - T_inf) * rho ** np.arange(n + 1)
    return np.abs(np.diff(T)), np.abs(T[1:])


def test_converging_iteration_stops_at_tolerance(monitor):
    d, t = _linear(0.9, 400)
    v, it, r = monitor(d, t, tol=1e-8)
    r_all = d / t
    assert v == CONVERGED
    assert it == int(np.argmax(r_all < 1e-8)) + 1 and r < 1e-8


def test_diverging_iteration_is_detected(monitor):
    """rho = 1.05: the relative increment levels off near 0.048 (never below
    any tolerance), the absolute increment grows geometrically."""
    d, t = _linear(1.05, 2000, T_inf=1.0, T0=0.999)
    v, it, r = monitor(d, t, tol=1e-8, limit=5000)
    assert v == DIVERGED
    # detected once the increment has grown 1e4 above its first value
    assert it == int(np.argmax(d > 1e4 * d[0])) + 1


def test_slow_divergence_is_detected_not_mistaken_for_convergence(monitor):
    d, t = _linear(1.002, 12000, T_inf=1.0, T0=0.9999)
    v, it, r = monitor(d, t, tol=1e-12, limit=20000)
    assert v == DIVERGED


def test_fp32_floor(monitor):
    """The relative increment falls to a noise level around 3e-8 and stays
    there: an FP32 sweep stops there (FLOOR) instead of running to max_iter;
    an FP64 solve with the same sequence is not converged (LIMIT)."""
    rng = np.random.default_rng(1)
    d1, t1 = _linear(0.9, 150)
    noise = 3e-8 * (1.0 + rng.random(600))
    d = np.concatenate([d1, noise])
    t = np.concatenate([t1, np.ones(600)])
    v, it, r = monitor(d, t, tol=1e-9, limit=700, fp32=True)
    assert v == FLOOR and 200 <= it - 150 <= 400 and r < 1e-5
    v, it, r = monitor(d, t, tol=1e-9, limit=700, fp32=False)
    assert v == LIMIT and it == 700


def test_non_finite_values(monitor):
    d, t = _linear(0.9, 20)
    d[5] = np.nan
    v, it, r = monitor(d, t)
    assert v == DIVERGED and it == 6
    d, t = _linear(0.9, 20)
    t[3] = np.inf
    assert monitor(d, t)[:2] == (DIVERGED, 4)


def test_fixed_count_ignores_tolerance(monitor):
    d, t = _linear(0.5, 60)
    v, it, r = monitor(d, t, tol=1e-3, limit=50, fixed=True)
    assert v == LIMIT and it == 50


def test_transient_growth_then_convergence_is_not_divergence(monitor):
    """A non-normal iteration may grow for a while (here 100x over 8
    iterations) before it converges; that is below the growth threshold."""
    d1 = 1e-3 * 1.8 ** np.arange(8)
    d2 = d1[-1] * 0.8 ** np.arange(1, 200)
    d = np.concatenate([d1, d2])
    t = np.ones_like(d)
    v, it, r = monitor(d, t, tol=1e-10)
    assert v == CONVERGED


def test_uniform_field_converges_at_once(monitor):
    """All increments and the field deviation exactly zero (e.g. every wall
    at T_ref, no heat): r = 0, converged in the first iteration."""
    v, it, r = monitor(np.zeros(5), np.zeros(5), tol=1e-12)
    assert (v, it, r) == (CONVERGED, 1, 0.0)
