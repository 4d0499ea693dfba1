// Device kernels of libnanobte (sm_103a), except the sweep (sweep.cu):
//
//  walls         - thermalizing / diffuse / specular / partial wall values and
//                  lagged cycle faces for the next sweep.
//  update        - moment reduction over work items, lattice temperature
//                  (Eq. (5)), sequential update (Eq. (6)) or synthetic
//                  right-hand side and update (Eqs. (8)-(10), (12)), FP64
//                  residual.
//  cg            - persistent Jacobi-preconditioned CG for the synthetic
//                  correction on the TPFA cell Laplacian, with a bounded-spin
//                  grid barrier.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cstdint>

#include "kernels.h"

namespace nbte {

// ============================================================================ walls
template <typename R>
__global__ void init_exports_kernel(R* exp, const int32_t* exp_cell, const double* Tdev, const double* CoW, int Bp,
                                    int G, int Gpad, int64_t n_exp) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_exp * Bp) return;
  const int64_t x = t / Bp;
  const int b = (int)(t - x * Bp);
  exp[io_index(x, b, n_exp, G, Gpad)] = (R)(CoW[b] * Tdev[exp_cell[x]]);
}

template <typename R>
void launch_init_exports(R* exp, const int32_t* exp_cell, const double* Tdev, const double* CoW, int Bp, int G,
                         int Gpad, int64_t n_exp, cudaStream_t st) {
  const int64_t n = n_exp * Bp;
  if (n == 0) return;
  init_exports_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(exp, exp_cell, Tdev, CoW, Bp, G, Gpad, n_exp);
}

// exported value of entry x, band b, with the synthetic correction's
// equilibrium part added (zero for the sequential scheme)
template <typename R>
__device__ __forceinline__ double exported(const WallArgs<R>& a, int64_t x, int b) {
  return (double)a.exp[io_index(x, b, a.n_exp, a.G, a.Gpad)] + a.CoW[b] * a.Delta[a.exp_cell[x]];
}

// diffuse re-emission: one value per (diffuse face, band)
template <typename R>
__global__ void diffuse_kernel(const WallArgs<R> a) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.n_dbf * a.Bp) return;
  const int64_t f = t / a.Bp;
  const int b = (int)(t - f * a.Bp);
  double s = 0.0;
  for (int64_t k = a.dif_ptr[f]; k < a.dif_ptr[f + 1]; ++k) s += a.dif_wt[k] * exported(a, a.dif_src[k], b);
  a.dsum[t] = s;
}

template <typename R>
__global__ void imports_kernel(const WallArgs<R> a) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.n_imp * a.Bp) return;
  const int64_t x = t / a.Bp;
  const int b = (int)(t - x * a.Bp);
  double v;
  switch (a.imp_kind[x]) {
    case 0:  // thermalizing: equilibrium at the wall temperature
      v = a.CoW[b] * a.imp_par[x];
      break;
    case 1:  // diffuse
      v = a.dsum[(int64_t)a.imp_dbf[x] * a.Bp + b];
      break;
    case 2:  // specular
      v = exported(a, a.imp_src[x], b);
      break;
    case 3: {  // partially specular
      const double p = a.imp_par[x];
      v = p * exported(a, a.imp_src[x], b) + (1.0 - p) * a.dsum[(int64_t)a.imp_dbf[x] * a.Bp + b];
      break;
    }
    default:  // lagged cycle face
      v = exported(a, a.imp_src[x], b);
      break;
  }
  a.imp[io_index(x, b, a.n_imp, a.G, a.Gpad)] = (R)v;
}

template <typename R>
void launch_walls(const WallArgs<R>& a, cudaStream_t st) {
  if (a.n_dbf > 0) {
    const int64_t n = a.n_dbf * a.Bp;
    diffuse_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
  }
  if (a.n_imp > 0) {
    const int64_t n = a.n_imp * a.Bp;
    imports_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
  }
}

// ============================================================================ update
__device__ __forceinline__ void block_max2(double& x, double& y, unsigned long long* res) {
  __shared__ double sx[32], sy[32];
  for (int o = 16; o > 0; o >>= 1) {
    x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    y = fmax(y, __shfl_xor_sync(0xffffffffu, y, o));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sx[w] = x; sy[w] = y; }
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    x = l < nw ? sx[l] : 0.0;
    y = l < nw ? sy[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
      y = fmax(y, __shfl_xor_sync(0xffffffffu, y, o));
    }
    if (l == 0) {
      // non-negative doubles order like their bit patterns; NaN sorts above +inf
      atomicMax(res, (unsigned long long)__double_as_longlong(x));
      atomicMax(res + 1, (unsigned long long)__double_as_longlong(y));
    }
  }
}

template <typename R>
__global__ void update_kernel(const UpdateArgs<R> a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double dmax = 0.0, tmax = 0.0;
  if (c < a.N) {
    const double Told = a.T[c];
    double TL = 0.0;
    if (a.mode == 0 || a.mode == 3) {
      double s = 0.0;
      for (int it = 0; it < a.n_items; ++it) s += a.part[(int64_t)it * a.N + c];
      // Eq. (5) as a deviation from T_ref: the equilibrium part of every
      // distribution sums to beta T'_used, T'_used being the (possibly
      // reduced-precision) temperature the sweep emitted from
      TL = (double)a.srcTQ_next[2 * c] + s * a.inv_beta;
      a.Tkin[c] = TL;
    } else {
      TL = a.Tkin[c];
    }
    if (a.mode == 3) {
      a.rhs[c] = a.V[c] * a.beta * (TL - Told);  // right-hand side of Eq. (10), DSA form
    } else {
      double Tn;
      if (a.mode == 0) Tn = TL;                   // Eq. (6)
      else Tn = (a.mode == 1 ? TL : Told) + a.delta[c];
      a.Delta[c] = Tn - TL;
      dmax = fabs(Tn - Told);
      tmax = fabs(Tn);
      if (!isfinite(dmax) || !isfinite(tmax)) dmax = tmax = CUDART_INF;
      a.T[c] = Tn;
      a.srcTQ_next[2 * c] = (R)Tn;
      a.srcTQ_next[2 * c + 1] = (R)a.Q[c];
    }
  }
  if (a.mode != 3) block_max2(dmax, tmax, a.res);
}

template <typename R>
void launch_update(const UpdateArgs<R>& a, cudaStream_t st) {
  update_kernel<R><<<(a.N + 255) / 256, 256, 0, st>>>(a);
}

template <typename R>
__global__ void fill_srcTQ_kernel(R* srcTQ, const double* T, const double* Q, int N) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  srcTQ[2 * c] = (R)T[c];
  srcTQ[2 * c + 1] = (R)Q[c];
}

template <typename R>
void launch_fill_srcTQ(R* srcTQ, const double* T, const double* Q, int N, cudaStream_t st) {
  fill_srcTQ_kernel<R><<<(N + 255) / 256, 256, 0, st>>>(srcTQ, T, Q, N);
}

// ============================================================================ CG
namespace {
constexpr unsigned long long kSpinLimit = 1ull << 25;   // ~seconds with nanosleep

// Grid barrier for a cooperative launch (all blocks co-resident).  bar[0] is
// a counter that only grows: a block arriving as number k waits until the
// counter reaches the next multiple of the block count.  The host zeroes it
// before each launch.  The wait spins tightly first, then backs off, and is
// bounded: on timeout the error word is set and every block leaves.
__device__ bool grid_sync(unsigned* bar, int32_t* err, unsigned nblocks) {
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
      if (++spins > kSpinLimit) {
        atomicExch(err, (int32_t)DEV_BARRIER_TIMEOUT);
        abort = 1;
        break;
      }
      if (spins > 2048) __nanosleep(32);
    }
    __threadfence();
    if (*(volatile int32_t*)err != 0) abort = 1;
    s_abort = abort;
  }
  __syncthreads();
  return s_abort != 0;
}

// block-wide sum, result valid in every thread
__device__ double block_sum(double x) {
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

// sum of the per-block partials written before the last grid barrier: every
// block reads them with the same lane split and the same shuffle tree, so all
// blocks get the same (deterministic) value
__device__ double grid_total(const double* partial, int slot) {
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

__device__ __forceinline__ double warp_sum(double s) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}
}  // namespace

// Persistent two-level PCG (one launch per synthetic correction).  Three grid
// barriers per iteration: after p.Ap, after the aggregate restriction, after
// r.z.  A p is updated as A z + beta A p_old so that the SpMV only needs z,
// which is complete at the r.z barrier.
__global__ void __launch_bounds__(kCGThreads) cg_kernel(const CGArgs a) {
  const unsigned nb = gridDim.x;
  const int c0 = a.blk_cell[blockIdx.x], c1 = a.blk_cell[blockIdx.x + 1];
  const int a0 = a.blk_agg[blockIdx.x], a1 = a.blk_agg[blockIdx.x + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;

  // aggregate restriction of r for the block's own aggregates
  auto restrict_r = [&]() {
    for (int g = a0 + warp; g < a1; g += nwarp) {
      double s = 0.0;
      for (int c = a.agg_cell[g] + lane; c < a.agg_cell[g + 1]; c += 32) s += a.r[c];
      s = warp_sum(s);
      if (lane == 0) a.rc[g] = s;
    }
  };
  // coarse correction rows for the block's own aggregates: the restricted
  // residual is staged in shared memory, the (symmetric, FP32-stored) coarse
  // inverse is read four entries per load, sums are FP64
  __shared__ double rc_s[kMaxCoarse];
  auto coarse_rows = [&]() {
    const int nc4 = a.Nc4;
    for (int k = threadIdx.x; k < 4 * nc4; k += blockDim.x) rc_s[k] = k < a.Nc ? __ldcg(a.rc + k) : 0.0;
    __syncthreads();
    for (int g = a0 + warp; g < a1; g += nwarp) {
      const float4* row = reinterpret_cast<const float4*>(a.Ainv + (int64_t)g * nc4 * 4);
      double s = 0.0;
#pragma unroll 4
      for (int k = lane; k < nc4; k += 32) {
        const float4 v = __ldg(row + k);
        const double* r = rc_s + 4 * k;
        s += (double)v.x * r[0] + (double)v.y * r[1] + (double)v.z * r[2] + (double)v.w * r[3];
      }
      s = warp_sum(s);
      if (lane == 0) a.yc[g] = s;
    }
  };
  auto spmv = [&](const double* v, int c) {
    double y = 0.0;
    for (int k = a.rp[c]; k < a.rp[c + 1]; ++k) y += a.val[k] * __ldcg(v + a.col[k]);
    return y;
  };

  // ---- initial guess: the previous correction scaled by its Galerkin
  // factor theta = (x_prev . b) / (x_prev . A x_prev) (zero on first use);
  // successive synthetic corrections share their slowly decaying shape
  double xb_l = 0.0, xax_l = 0.0, bb_l = 0.0;
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const double b = a.b[a.perm[c]];
    const double xp = a.x[c];
    const double q = spmv(a.x, c);
    a.r[c] = b;
    a.Ap[c] = q;   // A x_prev, scaled below
    xb_l += xp * b;
    xax_l += xp * q;
    bb_l += b * b;
  }
  double s = block_sum(xb_l);
  if (threadIdx.x == 0) a.partial[0 * nb + blockIdx.x] = s;
  s = block_sum(xax_l);
  if (threadIdx.x == 0) a.partial[1 * nb + blockIdx.x] = s;
  s = block_sum(bb_l);
  if (threadIdx.x == 0) a.partial[3 * nb + blockIdx.x] = s;
  if (grid_sync(a.bar, a.err, nb)) return;
  const double xb = grid_total(a.partial, 0);
  const double xax = grid_total(a.partial, 1);
  const double bb = grid_total(a.partial, 3);
  const double theta = (xax > 0.0 && isfinite(xb / xax)) ? xb / xax : 0.0;
  double rr0_l = 0.0;
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const double r = a.r[c] - theta * a.Ap[c];
    a.r[c] = r;
    a.x[c] = theta * a.x[c];
    rr0_l += r * r;
  }
  __syncthreads();
  restrict_r();
  s = block_sum(rr0_l);
  if (threadIdx.x == 0) a.partial[4 * nb + blockIdx.x] = s;   // own slot: 0-3 may still be read
  if (grid_sync(a.bar, a.err, nb)) return;
  const double rr0 = grid_total(a.partial, 4);
  int it = 0;
  double rr = rr0;
  if (bb > 0.0 && rr0 > a.tol * a.tol * bb) {
    coarse_rows();
    __syncthreads();
    double rz_l = 0.0;
    for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
      const double z = a.dinv[c] * a.r[c] + a.yc[a.agg[c]];
      a.z[c] = z;
      a.p[c] = z;
      rz_l += a.r[c] * z;
    }
    s = block_sum(rz_l);
    if (threadIdx.x == 0) a.partial[2 * nb + blockIdx.x] = s;
    if (grid_sync(a.bar, a.err, nb)) return;
    double rz = grid_total(a.partial, 2);
    double beta = 0.0;
    for (it = 0; it < a.max_it;) {
      // p = z + beta p ; Ap = A z + beta Ap
      double pap_l = 0.0;
      for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        const double az = spmv(a.z, c);
        const double p = it == 0 ? a.z[c] : a.z[c] + beta * a.p[c];
        const double ap = it == 0 ? az : az + beta * a.Ap[c];
        a.p[c] = p;
        a.Ap[c] = ap;
        pap_l += p * ap;
      }
      s = block_sum(pap_l);
      if (threadIdx.x == 0) a.partial[0 * nb + blockIdx.x] = s;
      if (grid_sync(a.bar, a.err, nb)) return;
      const double alpha = rz / grid_total(a.partial, 0);
      double rr_l = 0.0;
      for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        a.x[c] += alpha * a.p[c];
        const double r = a.r[c] - alpha * a.Ap[c];
        a.r[c] = r;
        rr_l += r * r;
      }
      __syncthreads();
      restrict_r();
      s = block_sum(rr_l);
      if (threadIdx.x == 0) a.partial[1 * nb + blockIdx.x] = s;
      if (grid_sync(a.bar, a.err, nb)) return;
      rr = grid_total(a.partial, 1);
      ++it;
      if (!(rr > a.tol * a.tol * bb)) break;
      coarse_rows();
      __syncthreads();
      double rz_n = 0.0;
      for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        const double z = a.dinv[c] * a.r[c] + a.yc[a.agg[c]];
        a.z[c] = z;
        rz_n += a.r[c] * z;
      }
      s = block_sum(rz_n);
      if (threadIdx.x == 0) a.partial[2 * nb + blockIdx.x] = s;
      if (grid_sync(a.bar, a.err, nb)) return;
      const double rzn = grid_total(a.partial, 2);
      beta = rzn / rz;
      rz = rzn;
    }
  }
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) a.x_out[a.perm[c]] = a.x[c];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.it_out += it;
    *a.res_out = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
}

cudaError_t launch_cg(const CGArgs& a, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kCGThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cg_kernel, a);
}

// ============================================================================ wall heat
template <typename R>
__global__ void wall_heat_kernel(const WallHeatArgs<R> a) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= a.n_wf) return;
  double h = 0.0;
  for (int64_t k = a.wf_ptr[f]; k < a.wf_ptr[f + 1]; ++k) {
    const int64_t v = a.wf_val[k];
    double s = 0.0;
    for (int b = 0; b < a.Bp; ++b) {
      const R val = v >= 0 ? a.exp[io_index(v, b, a.n_exp, a.G, a.Gpad)]
                           : a.imp[io_index(-1 - v, b, a.n_imp, a.G, a.Gpad)];
      s += a.band_v[b] * (double)val;
    }
    h += a.wf_coef[k] * s;
  }
  a.heat[f] = h;
}

template <typename R>
void launch_wall_heat(const WallHeatArgs<R>& a, cudaStream_t st) {
  if (a.n_wf == 0) return;
  wall_heat_kernel<R><<<(unsigned)((a.n_wf + 127) / 128), 128, 0, st>>>(a);
}

// ---------------------------------------------------------------- instantiations
#define NBTE_INST(R)                                                                                      \
  template void launch_init_exports<R>(R*, const int32_t*, const double*, const double*, int, int, int,   \
                                       int64_t, cudaStream_t);                                            \
  template void launch_walls<R>(const WallArgs<R>&, cudaStream_t);                                        \
  template void launch_update<R>(const UpdateArgs<R>&, cudaStream_t);                                     \
  template void launch_wall_heat<R>(const WallHeatArgs<R>&, cudaStream_t);                                \
  template void launch_fill_srcTQ<R>(R*, const double*, const double*, int, cudaStream_t);
NBTE_INST(float)
NBTE_INST(double)
#undef NBTE_INST

}  // namespace nbte
