// Device kernels of libnanobte (sm_103a).
//
//  sweep_kernel  - the per-(direction, band group) transport solve of Eq. (4)
//                  as a level-scheduled sweep over the direction's upwind
//                  graph (the triangular solve of the cached factorisation of
//                  Eq. (13)), bands innermost in registers, upwind values in a
//                  shared-memory ring, fused with the collision moment of
//                  Eq. (5) (and, on request, the energy/flux moments of
//                  Eq. (7)).
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

namespace {

template <typename R>
struct Vec2;
template <>
struct Vec2<float> { using T = float2; };
template <>
struct Vec2<double> { using T = double2; };

// BPT consecutive values of one cell's band group
template <typename R, int BPT>
__device__ __forceinline__ void load_bands(const R* p, R (&v)[BPT]) {
  if constexpr (sizeof(R) == 4 && BPT % 4 == 0) {
#pragma unroll
    for (int b = 0; b < BPT; b += 4) {
      const float4 t = *reinterpret_cast<const float4*>(p + b);
      v[b] = t.x; v[b + 1] = t.y; v[b + 2] = t.z; v[b + 3] = t.w;
    }
  } else if constexpr (BPT % 2 == 0) {
#pragma unroll
    for (int b = 0; b < BPT; b += 2) {
      const typename Vec2<R>::T t = *reinterpret_cast<const typename Vec2<R>::T*>(p + b);
      v[b] = t.x; v[b + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int b = 0; b < BPT; ++b) v[b] = p[b];
  }
}

template <typename R, int BPT>
__device__ __forceinline__ void store_bands(R* p, const R (&v)[BPT]) {
  if constexpr (sizeof(R) == 4 && BPT % 4 == 0) {
#pragma unroll
    for (int b = 0; b < BPT; b += 4) *reinterpret_cast<float4*>(p + b) = make_float4(v[b], v[b + 1], v[b + 2], v[b + 3]);
  } else if constexpr (BPT % 2 == 0) {
#pragma unroll
    for (int b = 0; b < BPT; b += 2) {
      typename Vec2<R>::T t;
      t.x = v[b]; t.y = v[b + 1];
      *reinterpret_cast<typename Vec2<R>::T*>(p + b) = t;
    }
  } else {
#pragma unroll
    for (int b = 0; b < BPT; ++b) p[b] = v[b];
  }
}

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <int LANES, typename R>
__device__ __forceinline__ R lane_sum(R x) {
  if constexpr (LANES > 1) {
    const unsigned lid = threadIdx.x & 31u;
    const unsigned mask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << (lid & ~(unsigned)(LANES - 1)));
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
  }
  return x;
}

}  // namespace

// ============================================================================ sweep
// One CTA owns one work item (direction i, band group g) and walks the levels
// of direction i in order; a __syncthreads() between levels makes level l's
// values visible to level l+1.  Thread t serves lane (t % LANES) of cells
// (t / LANES), (t / LANES) + blockDim/LANES, ... of each level; lane j holds
// bands [g*G + j*BPT, g*G + (j+1)*BPT) in registers.  Per cell and band the
// upwind balance of Eq. (4) is solved for the deviation from the cell's own
// equilibrium e0 = C T'/W (Eq. (11)):
//   e = e0 + (Qdot C/(C_tot W) + v sum_in c_k (e_up,k - e0)) / (1/tau + v G),
//   c_k = |s.An_k|/V,  G = sum_in c_k  (= sum_out (s.An)/V for a closed cell),
// which equals e = (e0/tau + S + v sum_in c_k e_up)/(1/tau + v G).  Written
// this way a uniform equilibrium is reproduced exactly in any precision and
// rounding errors scale with the local differences e_up - e0.
template <typename R, int K, int BPT, int LANES>
__global__ void __launch_bounds__(512) sweep_kernel(const SweepArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* ring = reinterpret_cast<R*>(smem_raw);
  const int item = blockIdx.x;
  const int i = a.item_dir[item];
  const int g = a.item_grp[item];
  const int G = BPT * LANES;
  const int lane = LANES > 1 ? (int)(threadIdx.x & (LANES - 1)) : 0;
  const int band0 = g * G + lane * BPT;
  const int N = a.N;

  for (int t = threadIdx.x; t < G; t += blockDim.x) ring[t] = R(0);   // zero slot

  const double wi = a.dir_w[i];
  R vb[BPT], itau[BPT], cw[BPT], aQ[BPT], wt[BPT];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    vb[b] = a.band_v[band0 + b];
    itau[b] = a.band_inv_tau[band0 + b];
    cw[b] = a.band_cw[band0 + b];
    aQ[b] = a.band_aQ[band0 + b];
    wt[b] = (R)(wi * (double)itau[b]);
  }
  __syncthreads();

  const int64_t dbase = (int64_t)i * N;
  const int32_t* lp = a.level_ptr + a.lvl_off[i];
  const int L = (int)(a.lvl_off[i + 1] - a.lvl_off[i]) - 1;
  const R* imp_i = a.imp + a.imp_off[i] * a.Bp + band0;
  R* exp_i = a.exp + a.exp_off[i] * a.Bp + band0;
  const int per_pass = blockDim.x / LANES;
  const int cidx = threadIdx.x / LANES;
  double* part = a.part + (int64_t)item * N;
  const typename Vec2<R>::T* tq = reinterpret_cast<const typename Vec2<R>::T*>(a.srcTQ);

  for (int l = 0; l < L; ++l) {
    const int p1 = lp[l + 1];
    for (int p = lp[l] + cidx; p < p1; p += per_pass) {
      const int64_t q = dbase + p;
      const int cell = a.pos_cell[q];
      const int slot = a.pos_slot[q];
      const int ex = a.pos_exp[q];
      const R Gc = a.pos_G[q];
      const typename Vec2<R>::T src = tq[cell];
      R e0[BPT], up[BPT];
#pragma unroll
      for (int b = 0; b < BPT; ++b) {
        e0[b] = cw[b] * src.x;
        up[b] = R(0);
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int64_t qk = ((int64_t)i * K + k) * N + p;
        const int ref = a.pos_ref[qk];
        const R cf = a.pos_coef[qk];
        const R* sp = ref >= 0 ? ring + ref * G + lane * BPT : imp_i + (int64_t)(-1 - ref) * a.Bp;
        R e_up[BPT];
        load_bands<R, BPT>(sp, e_up);
#pragma unroll
        for (int b = 0; b < BPT; ++b) up[b] += cf * (e_up[b] - e0[b]);
      }
      R e[BPT];
      R nl = R(0);
#pragma unroll
      for (int b = 0; b < BPT; ++b) {
        e[b] = e0[b] + (aQ[b] * src.y + vb[b] * up[b]) * recip(itau[b] + vb[b] * Gc);
        nl += wt[b] * e[b];
      }
      if (slot >= 0) store_bands<R, BPT>(ring + slot * G + lane * BPT, e);
      if (ex >= 0) store_bands<R, BPT>(exp_i + (int64_t)ex * a.Bp, e);
      nl = lane_sum<LANES>(nl);
      if (lane == 0) part[cell] = (double)nl;
      if (a.full) {
        R es = R(0), evs = R(0);
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
          es += e[b];
          evs += vb[b] * e[b];
        }
        es = lane_sum<LANES>(es);
        evs = lane_sum<LANES>(evs);
        if (lane == 0) {
          atomicAdd(a.accE + cell, wi * (double)es);
          for (int d = 0; d < a.dim; ++d) atomicAdd(a.accQ + (int64_t)cell * a.dim + d, wi * a.dir_s[i * 3 + d] * (double)evs);
        }
      }
    }
    __syncthreads();
  }
}

template <typename R, int K, int BPT>
static cudaError_t launch_sweep_l(const SweepArgs<R>& a, int lanes, int n_items, int threads, size_t smem,
                                  cudaStream_t st) {
  switch (lanes) {
#define NBTE_L(Lv)                                                                                    \
  case Lv: {                                                                                          \
    auto kern = sweep_kernel<R, K, BPT, Lv>;                                                          \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                                   \
    kern<<<n_items, threads, smem, st>>>(a);                                                          \
    return cudaGetLastError();                                                                        \
  }
    NBTE_L(1) NBTE_L(2) NBTE_L(4) NBTE_L(8)
#undef NBTE_L
    default: return cudaErrorInvalidConfiguration;
  }
}

template <typename R, int K>
static cudaError_t launch_sweep_b(const SweepArgs<R>& a, int bpt, int lanes, int n_items, int threads, size_t smem,
                                  cudaStream_t st) {
  switch (bpt) {
    case 1: return launch_sweep_l<R, K, 1>(a, lanes, n_items, threads, smem, st);
    case 2: return launch_sweep_l<R, K, 2>(a, lanes, n_items, threads, smem, st);
    case 4: return launch_sweep_l<R, K, 4>(a, lanes, n_items, threads, smem, st);
    case 8:
      if constexpr (sizeof(R) == 4) return launch_sweep_l<R, K, 8>(a, lanes, n_items, threads, smem, st);
      return cudaErrorInvalidConfiguration;
    default: return cudaErrorInvalidConfiguration;
  }
}

// Launches the variant for (K inflow entries, BPT bands per thread, lanes);
// an unsupported combination returns cudaErrorInvalidConfiguration without
// launching anything.
template <typename R>
cudaError_t launch_sweep(const SweepArgs<R>& a, int K, int bpt, int lanes, int n_items, int threads, size_t smem,
                         cudaStream_t st) {
  switch (K) {
    case 1: return launch_sweep_b<R, 1>(a, bpt, lanes, n_items, threads, smem, st);
    case 2: return launch_sweep_b<R, 2>(a, bpt, lanes, n_items, threads, smem, st);
    case 3: return launch_sweep_b<R, 3>(a, bpt, lanes, n_items, threads, smem, st);
    case 4: return launch_sweep_b<R, 4>(a, bpt, lanes, n_items, threads, smem, st);
    case 5: return launch_sweep_b<R, 5>(a, bpt, lanes, n_items, threads, smem, st);
    default: return cudaErrorInvalidConfiguration;
  }
}

// ============================================================================ walls
template <typename R>
__global__ void init_exports_kernel(R* exp, const int32_t* exp_cell, const double* Tdev, const double* CoW, int Bp,
                                    int64_t n_exp) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_exp * Bp) return;
  const int64_t x = t / Bp;
  const int b = (int)(t - x * Bp);
  exp[t] = (R)(CoW[b] * Tdev[exp_cell[x]]);
}

template <typename R>
void launch_init_exports(R* exp, const int32_t* exp_cell, const double* Tdev, const double* CoW, int Bp, int64_t n_exp,
                         cudaStream_t st) {
  const int64_t n = n_exp * Bp;
  if (n == 0) return;
  init_exports_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(exp, exp_cell, Tdev, CoW, Bp, n_exp);
}

// exported value of entry x, band b, with the synthetic correction's
// equilibrium part added (zero for the sequential scheme)
template <typename R>
__device__ __forceinline__ double exported(const WallArgs<R>& a, int64_t x, int b) {
  return (double)a.exp[x * a.Bp + b] + a.CoW[b] * a.Delta[a.exp_cell[x]];
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
  a.imp[t] = (R)v;
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
      TL = s * a.inv_beta;                        // Eq. (5), as a deviation from T_ref
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
constexpr int kCGThreads = 256;
constexpr unsigned long long kSpinLimit = 1ull << 25;   // ~seconds with nanosleep

// Grid barrier for a cooperative launch (all blocks co-resident).  Every wait
// is bounded: on timeout the error word is set and every block leaves.
__device__ bool grid_sync(unsigned* bar, int32_t* err, unsigned nblocks) {
  __shared__ int s_abort;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned g0 = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    int abort = 0;
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long spins = 0;
      while (*vgen == g0) {
        if (++spins > kSpinLimit) {
          atomicExch(err, (int32_t)DEV_BARRIER_TIMEOUT);
          abort = 1;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
    if (*(volatile int32_t*)err != 0) abort = 1;
    s_abort = abort;
  }
  __syncthreads();
  return s_abort != 0;
}

__device__ double block_sum(double x) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = x;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
  return r;  // valid in thread 0
}

// sum of the per-block partials, same order in every block (deterministic)
__device__ double grid_total(const double* partial, int slot) {
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) s += ((volatile const double*)partial)[slot * gridDim.x + b];
    tot = s;
  }
  __syncthreads();
  const double r = tot;
  __syncthreads();
  return r;
}
}  // namespace

__global__ void __launch_bounds__(kCGThreads) cg_kernel(const CGArgs a) {
  const int n = a.N;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nb = gridDim.x;
  double rz_l = 0.0, bb_l = 0.0;
  for (int c = t0; c < n; c += stride) {
    const double r = a.b[c];
    const double z = a.dinv[c] * r;
    a.x[c] = 0.0;
    a.r[c] = r;
    a.z[c] = z;
    a.p[c] = z;
    rz_l += r * z;
    bb_l += r * r;
  }
  double s = block_sum(rz_l);
  if (threadIdx.x == 0) a.partial[1 * nb + blockIdx.x] = s;
  s = block_sum(bb_l);
  if (threadIdx.x == 0) a.partial[2 * nb + blockIdx.x] = s;
  if (grid_sync(a.bar, a.err, nb)) return;
  double rz = grid_total(a.partial, 1);
  const double bb = grid_total(a.partial, 2);
  int it = 0;
  double rr = bb;
  if (bb > 0.0) {
    for (it = 0; it < a.max_it;) {
      double pap_l = 0.0;
      for (int c = t0; c < n; c += stride) {
        double y = 0.0;
        for (int k = a.rp[c]; k < a.rp[c + 1]; ++k) y += a.val[k] * __ldcg(a.p + a.col[k]);
        a.Ap[c] = y;
        pap_l += a.p[c] * y;
      }
      s = block_sum(pap_l);
      if (threadIdx.x == 0) a.partial[0 * nb + blockIdx.x] = s;
      if (grid_sync(a.bar, a.err, nb)) return;
      const double alpha = rz / grid_total(a.partial, 0);
      double rzn_l = 0.0, rr_l = 0.0;
      for (int c = t0; c < n; c += stride) {
        a.x[c] += alpha * a.p[c];
        const double r = a.r[c] - alpha * a.Ap[c];
        const double z = a.dinv[c] * r;
        a.r[c] = r;
        a.z[c] = z;
        rzn_l += r * z;
        rr_l += r * r;
      }
      s = block_sum(rzn_l);
      if (threadIdx.x == 0) a.partial[1 * nb + blockIdx.x] = s;
      s = block_sum(rr_l);
      if (threadIdx.x == 0) a.partial[2 * nb + blockIdx.x] = s;
      if (grid_sync(a.bar, a.err, nb)) return;
      const double rzn = grid_total(a.partial, 1);
      rr = grid_total(a.partial, 2);
      ++it;
      if (!(rr > a.tol * a.tol * bb)) break;
      const double beta = rzn / rz;
      rz = rzn;
      for (int c = t0; c < n; c += stride) a.p[c] = a.z[c] + beta * a.p[c];
      if (grid_sync(a.bar, a.err, nb)) return;
    }
  } else {
    for (int c = t0; c < n; c += stride) a.x[c] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.it_out += it;
    *a.res_out = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
}

int cg_max_grid(int device) {
  int nsm = 0, per_sm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_kernel, kCGThreads, 0);
  return nsm * (per_sm < 1 ? 1 : per_sm);
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
    const R* src = v >= 0 ? a.exp + v * a.Bp : a.imp + (-1 - v) * a.Bp;
    double s = 0.0;
    for (int b = 0; b < a.Bp; ++b) s += a.band_v[b] * (double)src[b];
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
  template cudaError_t launch_sweep<R>(const SweepArgs<R>&, int, int, int, int, int, size_t, cudaStream_t); \
  template void launch_init_exports<R>(R*, const int32_t*, const double*, const double*, int, int64_t,    \
                                       cudaStream_t);                                                     \
  template void launch_walls<R>(const WallArgs<R>&, cudaStream_t);                                        \
  template void launch_update<R>(const UpdateArgs<R>&, cudaStream_t);                                     \
  template void launch_wall_heat<R>(const WallHeatArgs<R>&, cudaStream_t);                                \
  template void launch_fill_srcTQ<R>(R*, const double*, const double*, int, cudaStream_t);
NBTE_INST(float)
NBTE_INST(double)
#undef NBTE_INST

}  // namespace nbte
