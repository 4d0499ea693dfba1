// Coarse space of the synthetic-correction solver: geometric aggregation of
// cells and the dense inverse of the Galerkin coarse operator.
#include <algorithm>
#include <cmath>
#include <thread>

#include "nbte_internal.h"

namespace nbte {

int build_aggregates(const Mesh& m, int target, std::vector<int32_t>& agg) {
  const int dim = m.dim;
  const int64_t N = m.n_cells;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t c = 0; c < N; ++c)
    for (int d = 0; d < dim; ++d) {
      lo[d] = std::min(lo[d], m.xc[c * dim + d]);
      hi[d] = std::max(hi[d], m.xc[c * dim + d]);
    }
  // boxes of equal edge h over the bounding box, sized from the occupied
  // volume so that about `target` boxes hold cells
  const double vol = m.volume > 0 ? m.volume : 1.0;
  double h = std::pow(vol / std::max(1, target), 1.0 / dim);
  int nb[3] = {1, 1, 1};
  for (int d = 0; d < dim; ++d) nb[d] = std::max(1, (int)std::ceil((hi[d] - lo[d]) / h));
  std::vector<int64_t> box(N);
  for (int64_t c = 0; c < N; ++c) {
    int64_t id = 0;
    for (int d = dim - 1; d >= 0; --d) {
      int k = (int)((m.xc[c * dim + d] - lo[d]) / h);
      k = std::min(std::max(k, 0), nb[d] - 1);
      id = id * nb[d] + k;
    }
    box[c] = id;
  }
  std::vector<int64_t> ids(box);
  std::sort(ids.begin(), ids.end());
  ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
  agg.resize(N);
  for (int64_t c = 0; c < N; ++c) agg[c] = (int32_t)(std::lower_bound(ids.begin(), ids.end(), box[c]) - ids.begin());
  return (int)ids.size();
}

// In-place inverse of a dense symmetric positive-definite matrix (row-major
// n x n) through its Cholesky factor: A = L L^T, A^{-1} = L^{-T} L^{-1}.
bool dense_spd_inverse(std::vector<double>& A, int n) {
  auto at = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  // Cholesky (lower triangle)
  for (int j = 0; j < n; ++j) {
    double d = at(j, j);
    for (int k = 0; k < j; ++k) d -= at(j, k) * at(j, k);
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    at(j, j) = d;
    const int nt = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
    auto rows = [&](int t) {
      for (int i = j + 1 + t; i < n; i += nt) {
        double s = at(i, j);
        const double* ri = &A[(size_t)i * n];
        const double* rj = &A[(size_t)j * n];
        for (int k = 0; k < j; ++k) s -= ri[k] * rj[k];
        at(i, j) = s / d;
      }
    };
    if (n - j > 256 && nt > 1) {
      std::vector<std::thread> th;
      for (int t = 1; t < nt; ++t) th.emplace_back(rows, t);
      rows(0);
      for (auto& x : th) x.join();
    } else {
      for (int i = j + 1; i < n; ++i) {
        double s = at(i, j);
        for (int k = 0; k < j; ++k) s -= at(i, k) * at(j, k);
        at(i, j) = s / d;
      }
    }
  }
  // Linv = L^{-1} (lower triangular), stored separately
  std::vector<double> Li((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    Li[(size_t)i * n + i] = 1.0 / at(i, i);
    for (int j = 0; j < i; ++j) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s += at(i, k) * Li[(size_t)k * n + j];
      Li[(size_t)i * n + j] = -s / at(i, i);
    }
  }
  // A^{-1} = Li^T Li
  const int nt = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
  auto work = [&](int t) {
    for (int i = t; i < n; i += nt)
      for (int j = 0; j <= i; ++j) {
        double s = 0.0;
        for (int k = i; k < n; ++k) s += Li[(size_t)k * n + i] * Li[(size_t)k * n + j];
        A[(size_t)i * n + j] = s;
        A[(size_t)j * n + i] = s;
      }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& x : th) x.join();
  return true;
}

}  // namespace nbte
