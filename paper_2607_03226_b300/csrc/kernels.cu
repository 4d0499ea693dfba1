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
//
// The collision moment of Eq. (5) is accumulated as sum_l w_i (e - e0)/tau_l;
// the equilibrium part sums to beta T' exactly and is added back in FP64 by
// the update kernel, so reduced-precision partials carry only the deviation.
//
// Latency: everything a cell needs except its upwind ring values (its record,
// its (T', Qdot) pair and any wall/lag import values) is loaded one level
// ahead, so a level's critical path is: barrier, shared-memory reads,
// arithmetic, shared-memory store.
namespace {
template <typename R, int K>
struct Rec {
  int cell, slot, ex;
  R G;
  int ref[K];
  R cf[K];
};
template <typename R, int K, int BPT>
struct Pre {
  R t, q;
  R imp[K][BPT];
};
}  // namespace

template <typename R, int K, int BPT, int LANES>
__global__ void __launch_bounds__(512) sweep_kernel(const SweepArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* ring = reinterpret_cast<R*>(smem_raw);
  int* lps = reinterpret_cast<int*>(smem_raw + a.lp_smem_off);
  const int item = blockIdx.x;
  const int i = a.item_dir[item];
  const int g = a.item_grp[item];
  const int G = BPT * LANES;
  const int lane = LANES > 1 ? (int)(threadIdx.x & (LANES - 1)) : 0;
  const int band0 = g * G + lane * BPT;
  const int N = a.N;
  const int L = (int)(a.lvl_off[i + 1] - a.lvl_off[i]) - 1;
  {
    const int32_t* lp = a.level_ptr + a.lvl_off[i];
    for (int t = threadIdx.x; t <= L; t += blockDim.x) lps[t] = lp[t];
  }
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
  const R* imp_i = a.imp + a.imp_off[i] * a.Bp + band0;
  R* exp_i = a.exp + a.exp_off[i] * a.Bp + band0;
  const int per_pass = blockDim.x / LANES;
  const int cidx = threadIdx.x / LANES;
  double* part = a.part + (int64_t)item * N;
  const typename Vec2<R>::T* tq = reinterpret_cast<const typename Vec2<R>::T*>(a.srcTQ);

  auto load_rec = [&](int p, Rec<R, K>& r) {
    const int64_t q = dbase + p;
    r.cell = a.pos_cell[q];
    r.slot = a.pos_slot[q];
    r.ex = a.pos_exp[q];
    r.G = a.pos_G[q];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t qk = ((int64_t)i * K + k) * N + p;
      r.ref[k] = a.pos_ref[qk];
      r.cf[k] = a.pos_coef[qk];
    }
  };
  auto load_pre = [&](const Rec<R, K>& r, Pre<R, K, BPT>& d) {
    const typename Vec2<R>::T s = tq[r.cell];
    d.t = s.x;
    d.q = s.y;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (r.ref[k] < 0) load_bands<R, BPT>(imp_i + (int64_t)(-1 - r.ref[k]) * a.Bp, d.imp[k]);
  };
  auto compute = [&](const Rec<R, K>& r, const Pre<R, K, BPT>& d) {
    R e0[BPT], up[BPT];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
      e0[b] = cw[b] * d.t;
      up[b] = R(0);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      R e_up[BPT];
      if (r.ref[k] >= 0) {
        load_bands<R, BPT>(ring + r.ref[k] * G + lane * BPT, e_up);
      } else {
#pragma unroll
        for (int b = 0; b < BPT; ++b) e_up[b] = d.imp[k][b];
      }
#pragma unroll
      for (int b = 0; b < BPT; ++b) up[b] += r.cf[k] * (e_up[b] - e0[b]);
    }
    R e[BPT];
    R nl = R(0);
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
      const R phi = (aQ[b] * d.q + vb[b] * up[b]) * recip(itau[b] + vb[b] * r.G);
      e[b] = e0[b] + phi;
      nl += wt[b] * phi;
    }
    if (r.slot >= 0) store_bands<R, BPT>(ring + r.slot * G + lane * BPT, e);
    if (r.ex >= 0) store_bands<R, BPT>(exp_i + (int64_t)r.ex * a.Bp, e);
    nl = lane_sum<LANES>(nl);
    if (lane == 0) part[r.cell] = (double)nl;
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
        atomicAdd(a.accE + r.cell, wi * (double)es);
        for (int d = 0; d < a.dim; ++d)
          atomicAdd(a.accQ + (int64_t)r.cell * a.dim + d, wi * a.dir_s[i * 3 + d] * (double)evs);
      }
    }
  };

  // pipeline: r0/d0 = this level's first-pass cell, r1 = next level's record
  Rec<R, K> r0, r1;
  Pre<R, K, BPT> d0;
  bool v0 = L > 0 && lps[0] + cidx < lps[1];
  bool v1 = L > 1 && lps[1] + cidx < lps[2];
  if (v0) {
    load_rec(lps[0] + cidx, r0);
    load_pre(r0, d0);
  }
  if (v1) load_rec(lps[1] + cidx, r1);
  for (int l = 0; l < L; ++l) {
    Pre<R, K, BPT> d1;
    if (v1) load_pre(r1, d1);                       // level l+1, issued now
    Rec<R, K> r2;
    const bool v2 = l + 2 < L && lps[l + 2] + cidx < lps[l + 3];
    if (v2) load_rec(lps[l + 2] + cidx, r2);        // level l+2, issued now
    if (v0) compute(r0, d0);
    for (int p = lps[l] + cidx + per_pass; p < lps[l + 1]; p += per_pass) {   // wide levels
      Rec<R, K> rw;
      Pre<R, K, BPT> dw;
      load_rec(p, rw);
      load_pre(rw, dw);
      compute(rw, dw);
    }
    __syncthreads();
    r0 = r1;
    d0 = d1;
    v0 = v1;
    r1 = r2;
    v1 = v2;
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
