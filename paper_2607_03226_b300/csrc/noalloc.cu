// nbte_laplacian_solve_noalloc: a conjugate-gradient solve of a caller's
// sparse symmetric positive-definite system that allocates no memory.
//
// Who needs it: code that may not call cudaMalloc -- for example a caller
// running inside another framework's memory pool or under a fixed device
// memory budget, or a real-time loop where an allocation could block or
// fail.  Such a caller hands over its own input and output buffers; this
// call's working vectors live in a fixed-size array in the library's device
// image instead of in memory it would otherwise allocate.  With lazy module
// loading (the CUDA default) the driver allocates that array when the first
// call on a device loads this file's device code; n = 0 does only that
// set-up, so that a caller can do it before its memory budget applies.
//
// It is a one-level (Jacobi-preconditioned) variant of the persistent CG
// kernel the synthetic correction uses; the arithmetic of a CG solve is
// unchanged, only the preconditioner is simpler, because the caller passes a
// bare matrix with no coarse space.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "nbte.h"
#include "nbte_internal.h"

namespace {

constexpr int kNoAllocMaxRows = 1 << 18;   // 262,144 rows
constexpr int kNoAllocMaxGrid = 256;
constexpr int kNoAllocThreads = 512;
constexpr int kMaxDevices = 64;
constexpr unsigned long long kNoAllocSpinLimit = 1ull << 25;

// Scratch of every call on a device: r, z, p, Ap and the inverse diagonal
// (kNoAllocMaxRows doubles each), 3 x kNoAllocMaxGrid reduction partials, and
// 8 control words (barrier counter, barrier error, iteration count, residual,
// converged flag, bad-diagonal flag).  About 10 MB, held by every GPU on which
// the library's device code is loaded until the process exits.
constexpr size_t kScratchDoubles = 5 * (size_t)kNoAllocMaxRows + 3 * kNoAllocMaxGrid + 8;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

struct Scratch {
  double* r;
  double* z;
  double* p;
  double* Ap;
  double* dinv;
  double* partial;
  unsigned* bar;
  int* err;
  int* iters;
  double* res;
  int* converged;
  int* bad_diag;
};

__host__ __device__ inline Scratch carve(double* base) {
  Scratch s;
  s.r = base;
  s.z = base + kNoAllocMaxRows;
  s.p = base + 2 * (size_t)kNoAllocMaxRows;
  s.Ap = base + 3 * (size_t)kNoAllocMaxRows;
  s.dinv = base + 4 * (size_t)kNoAllocMaxRows;
  s.partial = base + 5 * (size_t)kNoAllocMaxRows;
  double* ctl = s.partial + 3 * kNoAllocMaxGrid;
  s.bar = reinterpret_cast<unsigned*>(ctl);          // ctl[0]
  s.err = reinterpret_cast<int*>(ctl + 1);            // ctl[1]
  s.iters = reinterpret_cast<int*>(ctl + 2);          // ctl[2]
  s.res = ctl + 3;                                    // ctl[3]
  s.converged = reinterpret_cast<int*>(ctl + 4);      // ctl[4]
  s.bad_diag = reinterpret_cast<int*>(ctl + 5);       // ctl[5]
  return s;
}
constexpr int kCtlWords = 6;

// bounded grid barrier for a cooperative launch (see the synthetic CG
// kernel); the give-up decision is the same for every thread of a block
__device__ bool noalloc_grid_sync(unsigned* bar, int* err, unsigned nblocks, unsigned long long spin_limit) {
  __shared__ int s_abort;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned old = atomicAdd(bar, 1u);
    const unsigned target = (old / nblocks + 1) * nblocks;
    volatile unsigned* vc = bar;
    int abort = 0;
    unsigned long long spins = 0;
    while ((int)(*vc - target) < 0) {
      if (++spins > spin_limit) {
        atomicExch(err, 1);
        abort = 1;
        break;
      }
      if (spins > 2048) __nanosleep(32);
    }
    __threadfence();
    if (*(volatile int*)err != 0) abort = 1;
    s_abort = abort;
  }
  __syncthreads();
  return s_abort != 0;
}

__device__ double noalloc_block_sum(double x) {
  __shared__ double sh[32];
  __shared__ double tot;
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    double y = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    if (l == 0) tot = y;
  }
  __syncthreads();
  return tot;
}

__device__ double noalloc_grid_total(const double* partial, int slot) {
  __shared__ double tot;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) s += __ldcg(partial + slot * gridDim.x + b);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) tot = s;
  }
  __syncthreads();
  const double r = tot;
  __syncthreads();
  return r;
}

// Jacobi-preconditioned CG from x = 0; the scratch pointer is the device
// address of g_noalloc_scratch looked up on the host.  The inverse diagonal
// is gathered once; a row without a positive diagonal entry sets the
// bad-diagonal flag and every block leaves after the first barrier.
__global__ void __launch_bounds__(kNoAllocThreads)
noalloc_cg_kernel(int n, const int32_t* rp, const int32_t* col, const double* val, const double* b, double* x,
                  double tol, int max_it, double* scratch, unsigned long long spin_limit) {
  const Scratch S = carve(scratch);
  const unsigned nb = gridDim.x;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  double rz_l = 0.0, bb_l = 0.0;
  for (int c = t0; c < n; c += stride) {
    double d = 0.0;
    for (int k = rp[c]; k < rp[c + 1]; ++k)
      if (col[k] == c) d = val[k];
    if (!(d > 0.0)) {
      atomicExch(S.bad_diag, 1);
      d = 1.0;
    }
    const double di = 1.0 / d;
    const double r = b[c];
    const double z = r * di;
    S.dinv[c] = di;
    x[c] = 0.0;
    S.r[c] = r;
    S.z[c] = z;
    S.p[c] = z;
    rz_l += r * z;
    bb_l += r * r;
  }
  double s = noalloc_block_sum(rz_l);
  if (threadIdx.x == 0) S.partial[0 * nb + blockIdx.x] = s;
  s = noalloc_block_sum(bb_l);
  if (threadIdx.x == 0) S.partial[1 * nb + blockIdx.x] = s;
  if (noalloc_grid_sync(S.bar, S.err, nb, spin_limit)) return;
  if (*(volatile int*)S.bad_diag != 0) return;   // the same answer in every block, after the barrier
  double rz = noalloc_grid_total(S.partial, 0);
  const double bb = noalloc_grid_total(S.partial, 1);
  const double stop = tol * tol * bb;
  int it = 0;
  double rr = bb;
  bool conv = !(rr > stop);
  while (!conv && it < max_it) {
    double pap_l = 0.0;
    for (int c = t0; c < n; c += stride) {
      double y = 0.0;
      for (int k = rp[c]; k < rp[c + 1]; ++k) y += val[k] * __ldcg(S.p + col[k]);
      S.Ap[c] = y;
      pap_l += S.p[c] * y;
    }
    s = noalloc_block_sum(pap_l);
    if (threadIdx.x == 0) S.partial[2 * nb + blockIdx.x] = s;
    if (noalloc_grid_sync(S.bar, S.err, nb, spin_limit)) return;
    const double alpha = rz / noalloc_grid_total(S.partial, 2);
    double rzn_l = 0.0, rr_l = 0.0;
    for (int c = t0; c < n; c += stride) {
      x[c] += alpha * S.p[c];
      const double r = S.r[c] - alpha * S.Ap[c];
      const double z = r * S.dinv[c];
      S.r[c] = r;
      S.z[c] = z;
      rzn_l += r * z;
      rr_l += r * r;
    }
    s = noalloc_block_sum(rzn_l);
    if (threadIdx.x == 0) S.partial[0 * nb + blockIdx.x] = s;
    s = noalloc_block_sum(rr_l);
    if (threadIdx.x == 0) S.partial[1 * nb + blockIdx.x] = s;
    if (noalloc_grid_sync(S.bar, S.err, nb, spin_limit)) return;
    const double rzn = noalloc_grid_total(S.partial, 0);
    rr = noalloc_grid_total(S.partial, 1);
    ++it;
    conv = !(rr > stop);
    if (conv) break;
    const double beta = rzn / rz;
    rz = rzn;
    for (int c = t0; c < n; c += stride) S.p[c] = S.z[c] + beta * S.p[c];
    if (noalloc_grid_sync(S.bar, S.err, nb, spin_limit)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *S.iters = it;
    *S.res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    *S.converged = conv ? 1 : 0;   // the stopping test the host reports
  }
}

// Per device: the device address of the scratch array and the cooperative
// grid size, found once with that device current.
struct DeviceSetup {
  double* base = nullptr;
  int grid = 0;
};
std::mutex g_mu;
DeviceSetup g_setup[kMaxDevices];

int setup_device(int dev, DeviceSetup* out) {
  using nbte::set_error;
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceSetup& d = g_setup[dev];
  if (!d.base) {
    // Loading the kernel's module is what makes the driver allocate the
    // scratch array on this device (with lazy module loading, the CUDA
    // default, that happens here and not when the library is loaded).
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, noalloc_cg_kernel);
    double* base = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&base), g_noalloc_scratch);
    int nsm = 1, per_sm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_cg_kernel, kNoAllocThreads, 0);
    if (e != cudaSuccess) {
      set_error(std::string("allocation-free solve set-up: ") + cudaGetErrorString(e));
      return NBTE_ERR_CUDA;
    }
    d.grid = std::max(1, std::min(kNoAllocMaxGrid, nsm * std::max(1, per_sm)));
    d.base = base;
  }
  *out = d;
  return NBTE_OK;
}

}  // namespace

extern "C" int nbte_laplacian_solve_noalloc(int n, const int32_t* row_ptr, const int32_t* col, const double* val,
                                            const double* rhs, double* x, double tol, int max_iter,
                                            int32_t* iterations, double* residual, void* cuda_stream) {
  using nbte::set_error;
  if (n < 0) { set_error("n must not be negative"); return NBTE_ERR_ARG; }
  if (n > kNoAllocMaxRows) {
    set_error("n = " + std::to_string(n) + " exceeds the fixed scratch of " + std::to_string(kNoAllocMaxRows) +
              " rows of nbte_laplacian_solve_noalloc");
    return NBTE_ERR_ARG;
  }
  if (n > 0 && (!row_ptr || !col || !val || !rhs || !x)) { set_error("null device pointer"); return NBTE_ERR_ARG; }
  if (n > 0 && (!(tol > 0.0) || max_iter <= 0)) {
    set_error("tol must be positive and max_iter > 0");
    return NBTE_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error(std::string("no usable CUDA device: ") + cudaGetErrorString(e));
    return NBTE_ERR_CUDA;
  }
  DeviceSetup d;
  const int rc = setup_device(dev, &d);
  if (rc) return rc;
  if (n == 0) return NBTE_OK;   // the per-device set-up only
  double* base = d.base;
  const Scratch S = carve(base);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int grid = std::max(1, std::min(d.grid, (n + kNoAllocThreads - 1) / kNoAllocThreads));
  unsigned long long spin_limit = nbte::wait_limit_or(kNoAllocSpinLimit);
  // control words start at zero for every call (barrier counter, flags)
  e = cudaMemsetAsync(S.bar, 0, kCtlWords * sizeof(double), st);
  if (e != cudaSuccess) { set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)); return NBTE_ERR_CUDA; }
  void* args[] = {&n, &row_ptr, &col, &val, &rhs, &x, &tol, &max_iter, &base, &spin_limit};
  e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(noalloc_cg_kernel), dim3(grid), dim3(kNoAllocThreads), args,
                                  0, st);
  if (e != cudaSuccess) {
    set_error(std::string("cooperative launch failed: ") + cudaGetErrorString(e));
    return NBTE_ERR_CUDA;
  }
  double ctl[kCtlWords] = {0, 0, 0, 0, 0, 0};
  e = cudaMemcpyAsync(ctl, S.bar, sizeof(ctl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { set_error(std::string("CUDA error: ") + cudaGetErrorString(e)); return NBTE_ERR_CUDA; }
  int err_word = 0, it = 0, conv = 0, bad = 0;
  memcpy(&err_word, &ctl[1], sizeof(int));
  memcpy(&it, &ctl[2], sizeof(int));
  memcpy(&conv, &ctl[4], sizeof(int));
  memcpy(&bad, &ctl[5], sizeof(int));
  if (err_word != 0) {
    set_error("a bounded grid barrier of the CG gave up");
    return NBTE_ERR_DEVICE_TIMEOUT;
  }
  if (bad != 0) {
    set_error("a row of the matrix has no positive diagonal entry");
    return NBTE_ERR_ARG;
  }
  if (iterations) *iterations = it;
  if (residual) *residual = ctl[3];
  if (!conv) {
    set_error("CG reached max_iter before tol");
    return NBTE_ERR_NOT_CONVERGED;
  }
  return NBTE_OK;
}
