// The host's stopping rule for the outer iteration (Eq. (6) / Eq. (12)):
// after every iteration it reads two FP64 words from the device, the largest
// absolute increment max|T'^{n+1} - T'^n| and max|T'^{n+1}|, and decides
// whether to go on.  Plain C++ with no CUDA dependency, so that the rule can
// be exercised on the host alone.
#pragma once

#include <cmath>

namespace nbte {

struct IterationMonitor {
  enum Verdict { CONTINUE = 0, CONVERGED = 1, FLOOR = 2, LIMIT = 3, DIVERGED = 4 };

  // configuration
  double tol = 1e-10;       // on the relative increment r = max|dT'| / max|T'|
  int limit = 10000;        // iteration cap (or the exact count when fixed)
  bool fixed = false;       // run exactly `limit` iterations, no convergence test
  bool fp32 = false;        // FP32 sweep: stop at the rounding floor of r
  // divergence: after at least kDivMinIter iterations, the absolute increment
  // has grown kDivGrowth times above its smallest value so far while still
  // being a visible fraction (kDivRelative) of the field -- a linear
  // iteration whose spectral radius exceeds one does exactly that (the
  // relative increment itself levels off at (rho - 1) / rho), while a
  // converging one, or rounding noise at the FP32 floor, never grows by
  // orders of magnitude
  static constexpr int kDivMinIter = 10;
  static constexpr double kDivGrowth = 1e4;
  static constexpr double kDivRelative = 1e-4;
  // FP32 floor: r below kFloorMax and not improved by 10% for kFloorIter
  // iterations
  static constexpr double kFloorMax = 1e-5;
  static constexpr int kFloorIter = 200;

  // state
  int it = 0;
  double r = INFINITY;
  double best_r = INFINITY;
  int it_best = 0;
  double dmin = INFINITY;
  Verdict last = CONTINUE;

  // Record iteration `it + 1` with its increment and field maxima; returns
  // what to do next.
  Verdict step(double dmax, double tmax) {
    ++it;
    if (!std::isfinite(dmax) || !std::isfinite(tmax)) {
      r = INFINITY;
      return last = DIVERGED;
    }
    r = dmax / (tmax > 1e-300 ? tmax : 1e-300);
    if (tmax == 0.0 && dmax == 0.0) r = 0.0;
    if (it >= kDivMinIter && dmax > kDivGrowth * dmin && dmax > kDivRelative * tmax) return last = DIVERGED;
    if (dmax < dmin) dmin = dmax;
    if (!fixed && r < tol) return last = CONVERGED;
    if (fp32 && !fixed) {
      if (r < 0.9 * best_r) {
        best_r = r;
        it_best = it;
      }
      if (best_r < kFloorMax && it - it_best >= kFloorIter) return last = FLOOR;
    }
    if (it >= limit) return last = LIMIT;
    return last = CONTINUE;
  }
};

}  // namespace nbte
