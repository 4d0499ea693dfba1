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

// diffuse re-emission: one value per (diffuse face, band).  One block per
// face; thread (band, slice) sums every kDifSlices-th outgoing direction of
// the face, and the slice sums are combined in a fixed order (so results do
// not depend on scheduling).  FP64 sums, as the wall balance needs.
constexpr int kDifSlices = 8;

constexpr int kDifBands = 64;   // bands per block (blockIdx.y covers the rest)

template <typename R>
__global__ void diffuse_kernel(const WallArgs<R> a) {
  __shared__ double dif_red[kDifSlices][kDifBands];
  const int64_t f = blockIdx.x;
  const int b = blockIdx.y * kDifBands + threadIdx.x;
  const int j = threadIdx.y;
  const int64_t k0 = a.dif_ptr[f], k1 = a.dif_ptr[f + 1];
  double s = 0.0;
  if (b < a.Bp)
    for (int64_t k = k0 + j; k < k1; k += kDifSlices) s += a.dif_wt[k] * exported(a, a.dif_src[k], b);
  dif_red[j][threadIdx.x] = s;
  __syncthreads();
  if (j == 0 && b < a.Bp) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kDifSlices; ++q) t += dif_red[q][threadIdx.x];
    a.dsum[f * a.Bp + b] = t;
  }
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
    const int bx = a.Bp < kDifBands ? a.Bp : kDifBands;
    diffuse_kernel<R><<<dim3((unsigned)a.n_dbf, (unsigned)((a.Bp + kDifBands - 1) / kDifBands)),
                        dim3(bx, kDifSlices), 0, st>>>(a);
  }
  if (a.n_imp > 0) {
    const int64_t n = a.n_imp * a.Bp;
    imports_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
  }
}

// ============================================================================ update
// One block per 32 cell slots (V cells each: V = 2 for FP32 partials with an
// even cell count, read as float2, else 1).  The collision moment comes in one
// of two forms:
//  * per-cell FP64 sums of the sweep's atomic adds (part null): read, then
//    cleared for the next sweep;
//  * per-(work item, cell) partials (deterministic): summed by 8 item slices
//    per cell and combined in shared memory in a fixed order; one warp then
//    applies the update.  FP32 partials are summed with compensation (Kahan)
//    in FP32, which keeps the sum to FP32 rounding of the total while
//    spending no FP64 instruction per partial; FP64 partials are summed in
//    FP64.  Every cell's summation order is the same for V = 1 and V = 2.
constexpr int kUpdCells = 32, kUpdSlices = 8;

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

template <int V>
__device__ __forceinline__ void load_part(const float* p, int64_t k, float (&x)[V]) {
  if constexpr (V == 2) {
    const float2 v = __ldcs(reinterpret_cast<const float2*>(p) + k);
    x[0] = v.x;
    x[1] = v.y;
  } else {
    x[0] = __ldcs(p + k);
  }
}

template <typename R, int V>
__global__ void __launch_bounds__(kUpdCells * kUpdSlices) update_kernel(const UpdateArgs<R> a) {
  static_assert(V == 1 || (V == 2 && sizeof(R) == 4), "two cells per thread with FP32 partials only");
  const int c0 = (blockIdx.x * kUpdCells + threadIdx.x) * V;
  const bool reduce = a.mode == 0 || a.mode == 3;
  double s[V];
#pragma unroll
  for (int v = 0; v < V; ++v) s[v] = 0.0;
  if (reduce && a.part == nullptr) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int c = c0 + v;
      if (c < a.N) {
        s[v] = a.acc[c];
        a.acc[c] = 0.0;
      }
    }
  } else if (reduce) {
    if constexpr (sizeof(R) == 4) {
      __shared__ float red_s[kUpdSlices][V][kUpdCells], red_c[kUpdSlices][V][kUpdCells];
      float ks[V], kc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) ks[v] = kc[v] = 0.0f;
      if (c0 < a.N) {
        // in units of V floats: the row of item it starts at it * (N / V)
        const float* p = a.part + c0;
        const int64_t NV = a.N / V;
        int it = threadIdx.y;
        for (; it + 3 * kUpdSlices < a.n_items; it += 4 * kUpdSlices) {
          float x0[V], x1[V], x2[V], x3[V];
          load_part<V>(p, it * NV, x0);
          load_part<V>(p, (it + kUpdSlices) * NV, x1);
          load_part<V>(p, (it + 2 * kUpdSlices) * NV, x2);
          load_part<V>(p, (it + 3 * kUpdSlices) * NV, x3);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            kahan_add(ks[v], kc[v], x0[v]);
            kahan_add(ks[v], kc[v], x1[v]);
            kahan_add(ks[v], kc[v], x2[v]);
            kahan_add(ks[v], kc[v], x3[v]);
          }
        }
        for (; it < a.n_items; it += kUpdSlices) {
          float x[V];
          load_part<V>(p, it * NV, x);
#pragma unroll
          for (int v = 0; v < V; ++v) kahan_add(ks[v], kc[v], x[v]);
        }
      }
#pragma unroll
      for (int v = 0; v < V; ++v) {
        red_s[threadIdx.y][v][threadIdx.x] = ks[v];
        red_c[threadIdx.y][v][threadIdx.x] = kc[v];
      }
      __syncthreads();
      if (threadIdx.y != 0) return;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        float ts = 0.0f, tc = 0.0f;
#pragma unroll
        for (int y = 0; y < kUpdSlices; ++y) {
          kahan_add(ts, tc, red_s[y][v][threadIdx.x]);
          kahan_add(ts, tc, -red_c[y][v][threadIdx.x]);
        }
        s[v] = (double)ts - (double)tc;
      }
    } else {
      __shared__ double red[kUpdSlices][kUpdCells];
      double t = 0.0;
      if (c0 < a.N) {
        const R* p = a.part + c0;
        const int64_t N = a.N;
        double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
        int it = threadIdx.y;
        for (; it + 3 * kUpdSlices < a.n_items; it += 4 * kUpdSlices) {
          acc0 += __ldcs(p + it * N);
          acc1 += __ldcs(p + (it + kUpdSlices) * N);
          acc2 += __ldcs(p + (it + 2 * kUpdSlices) * N);
          acc3 += __ldcs(p + (it + 3 * kUpdSlices) * N);
        }
        for (; it < a.n_items; it += kUpdSlices) acc0 += __ldcs(p + it * N);
        t = (acc0 + acc1) + (acc2 + acc3);
      }
      red[threadIdx.y][threadIdx.x] = t;
      __syncthreads();
      if (threadIdx.y != 0) return;
      t = 0.0;
#pragma unroll
      for (int y = 0; y < kUpdSlices; ++y) t += red[y][threadIdx.x];
      s[0] = t;
    }
  } else if (threadIdx.y != 0) {
    return;
  }
  // one warp per block from here on
  double dmax = 0.0, tmax = 0.0;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int c = c0 + v;
    if (c >= a.N) break;
    const double Told = a.T[c];
    double TL = 0.0;
    if (reduce) {
      // Eq. (5) as a deviation from T_ref: the equilibrium part of every
      // distribution sums to beta T'_used, T'_used being the (possibly
      // reduced-precision) temperature the sweep emitted from
      TL = (double)a.srcTQ_next[2 * c] + s[v] * a.inv_beta;
      a.Tkin[c] = TL;
      // the first update of an iteration keeps the iterate the sweep started
      // from (the final moments replay that sweep)
      a.Tprev[c] = Told;
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
      double d = fabs(Tn - Told), t = fabs(Tn);
      if (!isfinite(d) || !isfinite(t)) d = t = CUDART_INF;
      dmax = fmax(dmax, d);
      tmax = fmax(tmax, t);
      a.T[c] = Tn;
      a.srcTQ_next[2 * c] = (R)Tn;
      a.srcTQ_next[2 * c + 1] = (R)a.Q[c];
    }
  }
  if (a.mode != 3) {
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      tmax = fmax(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
    }
    if (threadIdx.x == 0) {
      // non-negative doubles order like their bit patterns; NaN sorts above +inf
      atomicMax(a.res, (unsigned long long)__double_as_longlong(dmax));
      atomicMax(a.res + 1, (unsigned long long)__double_as_longlong(tmax));
    }
  }
}

template <typename R>
void launch_update(const UpdateArgs<R>& a, cudaStream_t st) {
  const bool reduce = a.mode == 0 || a.mode == 3;
  const dim3 block(kUpdCells, reduce && a.part ? kUpdSlices : 1);
  if (sizeof(R) == 4 && a.N % 2 == 0) {
    const int slots = a.N / 2;
    update_kernel<R, (sizeof(R) == 4 ? 2 : 1)><<<(slots + kUpdCells - 1) / kUpdCells, block, 0, st>>>(a);
  } else {
    update_kernel<R, 1><<<(a.N + kUpdCells - 1) / kUpdCells, block, 0, st>>>(a);
  }
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

// Between the caller's cell order and the library's: perm[c] is the caller
// index of internal cell c.
__global__ void from_caller_kernel(double* dst, const double* src, const int32_t* perm, int N) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < N) dst[c] = __ldg(src + __ldg(perm + c));
}
__global__ void to_caller_kernel(double* dst, const double* src, const int32_t* perm, int N, int dim,
                                 double scale, double offset) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * dim) return;
  const int c = (int)(t / dim), d = (int)(t - (int64_t)c * dim);
  dst[(int64_t)__ldg(perm + c) * dim + d] = src[t] * scale + offset;
}
cudaError_t launch_from_caller(double* dst, const double* src, const int32_t* perm, int N, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  from_caller_kernel<<<(N + 255) / 256, 256, 0, st>>>(dst, src, perm, N);
  return cudaGetLastError();
}
cudaError_t launch_to_caller(double* dst, const double* src, const int32_t* perm, int N, int dim, double scale,
                             double offset, cudaStream_t st) {
  const int64_t n = (int64_t)N * dim;
  if (n <= 0) return cudaSuccess;
  to_caller_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dst, src, perm, N, dim, scale, offset);
  return cudaGetLastError();
}

// ============================================================================ CG
// FP64 arithmetic is scarce on this part (a warp-wide FP64 instruction holds
// its scheduler's FP64 pipe for tens of cycles), so the kernel below spends
// FP64 instructions only where the correction's accuracy needs them: the
// vectors, the matrix product and the inner products.  Scalars are formed by
// one thread, block sums go through shared memory to one warp per value, and
// with a loose tolerance the coarse preconditioner runs in FP32.
namespace {

__device__ __forceinline__ double warp_sum(double s) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}
__device__ __forceinline__ float warp_sumf(float s) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Grid barrier fused with a reduction of NV (<= 3) values.  Thread values go
// to red_s[j][tid]; warp j sums column j and writes the block's sum into its
// slot (buffer gen & 1); thread 0 arrives on a 64-bit counter that only grows
// (a block arriving as number k waits for the next multiple of the block
// count); after the barrier warp j loads every block's sum j at once and adds
// them in one fixed order, so all blocks get the same totals.  The wait is
// bounded: on timeout, or when another block reported one, the error word is
// set and the function returns true.  Thread 0 replaces inv[0..n_inv) by
// their reciprocals while it waits (work off the critical path).
template <int NV>
__device__ bool grid_reduce(const double* v, double* tot, double* red_s, CGSlot* slots, unsigned long long* bar,
                            unsigned gen, int32_t* err, int blk, unsigned nb, unsigned long long spin_limit,
                            double* inv = nullptr, int n_inv = 0) {
  static_assert(NV >= 0 && NV <= 3, "a slot carries up to three sums");
  __shared__ double s_tot[3];
  __shared__ int s_abort;
  const int tid = threadIdx.x, T = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int buf = gen & 1;
#pragma unroll
  for (int j = 0; j < NV; ++j) red_s[j * T + tid] = v[j];
  __syncthreads();
  if (warp < NV) {
    double y = 0.0;
    for (int i = lane; i < T; i += 32) y += red_s[warp * T + i];
    y = warp_sum(y);
    if (lane == 0) slots[blk].v[buf][warp] = y;
  }
  __syncthreads();   // orders every thread's global writes (and the slot sums) before the fence below
  if (tid == 0) {
    int abort = 0;
    __threadfence();
    const unsigned long long old = atomicAdd(bar, 1ull);
    const unsigned long long target = (old / nb + 1) * nb;
    for (int k = 0; k < n_inv; ++k) inv[k] = 1.0 / inv[k];
    volatile unsigned long long* vb = bar;
    unsigned long long spins = 0;
    while (*vb < target) {
      if (++spins > spin_limit) {
        atomicExch(err, (int32_t)DEV_BARRIER_TIMEOUT);
        abort = 1;
        break;
      }
      if (spins > 4096) __nanosleep(64);
    }
    __threadfence();
    if (*(volatile int32_t*)err != 0) abort = 1;
    s_abort = abort;
  }
  __syncthreads();
  if (warp < NV) {
    // every block's sum at once (grid <= 256), added in one fixed order
    double t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) t[k] = (unsigned)(k * 32 + lane) < nb ? __ldcg(&slots[k * 32 + lane].v[buf][warp]) : 0.0;
    double y = t[0];
#pragma unroll
    for (int k = 1; k < 8; ++k)
      if ((unsigned)(k * 32) < nb) y += t[k];
    y = warp_sum(y);
    if (lane == 0) s_tot[warp] = y;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) tot[j] = s_tot[j];
  return s_abort != 0;
}

template <bool C32>
struct CoarseT { using T = double; };
template <>
struct CoarseT<true> { using T = float; };
}  // namespace

// Persistent two-level PCG (one launch per synthetic correction), in the
// Chronopoulos-Gear arrangement: with u = M^{-1} r and w = A u, the two inner
// products (r,u) and (w,u) come from one reduction, and s = A p follows the
// recurrence s = w + beta s.  Two grid barriers per iteration:
//   X  after w = A u, carrying (r,u), (w,u), (r,r);
//   Z  after u = M^{-1} r, so the next product A u sees every row of u.
// The coarse part of M needs every aggregate's sum of r.  Each block keeps all
// of them in shared memory and advances them with the same linear recurrence
// as r itself (P^T r <- P^T r - alpha (P^T w + beta P^T s)), starting each
// step from the exact sums the owning blocks computed one step earlier, so no
// third barrier is needed and rounding does not accumulate.
//
// A block's own rows of x, r, p, s, w, u, D^{-1} (and, when they fit, its
// ELL matrix rows) live in shared memory; only u is mirrored to global memory
// for the neighbours' products.  Row l of the block is cell c0 + l.  C32: the
// coarse sums, the coarse inverse product and the correction it yields are
// FP32 (a preconditioner only has to be fixed and SPD to rounding; the
// iteration's vectors and inner products stay FP64).
template <bool C32>
__device__ __forceinline__ void cg_body(const CGArgs& a, const int blk, const unsigned nb, unsigned char* cg_smem) {
  using CT = typename CoarseT<C32>::T;
  const int c0 = a.blk_cell[blk], nr = a.blk_cell[blk + 1] - c0;
  const int a0 = a.blk_agg[blk], na = a.blk_agg[blk + 1] - a0;
  const int tid = threadIdx.x, T = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = T >> 5;
  const int Nc = a.Nc, nc4 = a.Nc4, W = a.W;
  __shared__ double s_scal[4];
  CgSmem L = cg_smem_layout(nc4, a.max_rows, a.max_na, W, T, a.smem_vec, a.smem_ell, (int)sizeof(CT));
  double* red_s = reinterpret_cast<double*>(cg_smem + L.red);
  CT* rc_s = reinterpret_cast<CT*>(cg_smem + L.rc);   // aggregate sums of r, every aggregate
  CT* sc_s = reinterpret_cast<CT*>(cg_smem + L.sc);   // aggregate sums of s
  CT* yc_s = reinterpret_cast<CT*>(cg_smem + L.yc);   // coarse correction, own aggregates
  CT* fr_s = reinterpret_cast<CT*>(cg_smem + L.fr);   // own rows of the vector being restricted
  int32_t* ab_s = reinterpret_cast<int32_t*>(cg_smem + L.ab);   // own aggregates' first rows
  for (int g = tid; g <= na; g += T) ab_s[g] = a.agg_cell[a0 + g] - c0;
  double *x, *r, *p, *s, *w, *u, *dv;
  const int32_t* ag;   // aggregate of each own row, relative to a0
  if (a.smem_vec) {
    x = reinterpret_cast<double*>(cg_smem + L.vec);
    r = x + a.max_rows;
    p = r + a.max_rows;
    s = p + a.max_rows;
    w = s + a.max_rows;
    u = w + a.max_rows;
    dv = u + a.max_rows;
    int32_t* ag_s = reinterpret_cast<int32_t*>(dv + a.max_rows);
    for (int l = tid; l < nr; l += T) {
      x[l] = a.x[c0 + l];
      dv[l] = a.dinv[c0 + l];
      ag_s[l] = a.agg_rel[c0 + l];
    }
    ag = ag_s;
  } else {
    x = a.x_work + c0;
    r = a.r + c0;
    p = a.p + c0;
    s = a.s + c0;
    w = a.w + c0;
    u = a.u + c0;
    dv = const_cast<double*>(a.dinv) + c0;
    ag = a.agg_rel + c0;
    for (int l = tid; l < nr; l += T) x[l] = a.x[c0 + l];
  }
  // ELL off-diagonals [k][row] and the diagonal
  const double* ev;
  const int32_t* ec;
  const double* dg;
  int es;
  if (a.smem_ell) {
    double* v_s = reinterpret_cast<double*>(cg_smem + L.ell);
    double* d_s = v_s + (size_t)W * a.max_rows;
    int32_t* c_s = reinterpret_cast<int32_t*>(d_s + a.max_rows);
    for (int l = tid; l < nr; l += T) {
      d_s[l] = a.diag[c0 + l];
      for (int k = 0; k < W; ++k) {
        v_s[k * a.max_rows + l] = a.ell_val[(int64_t)k * a.N + c0 + l];
        c_s[k * a.max_rows + l] = a.ell_col[(int64_t)k * a.N + c0 + l];
      }
    }
    ev = v_s;
    ec = c_s;
    dg = d_s;
    es = a.max_rows;
  } else {
    ev = a.ell_val + c0;
    ec = a.ell_col + c0;
    dg = a.diag + c0;
    es = a.N;
  }
  for (int k = Nc + tid; k < 4 * nc4; k += T) rc_s[k] = CT(0);   // row padding of the coarse inverse
  const CT* Ainv = reinterpret_cast<const CT*>(C32 ? static_cast<const void*>(a.Ainv32) : static_cast<const void*>(a.Ainv64));
  CT* rcx = static_cast<CT*>(a.rcx);
  CT* scx = static_cast<CT*>(a.scx);
  CT* rw = static_cast<CT*>(a.rw);
  unsigned gen = 0;
  __syncthreads();

  // (A v)_row for row l; v is a global vector in aggregate order.  The
  // neighbour loads are issued together, the products form one FMA chain.
  auto spmv = [&](const double* vg, int l) {
    double t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < W) t[k] = __ldcg(vg + ec[k * es + l]);
    double y = dg[l] * __ldcg(vg + c0 + l);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < W) y = fma(ev[k * es + l], t[k], y);
    return y;
  };
  // aggregate sums of fr_s (own rows) over the own aggregates, one warp per
  // aggregate, written to out[global aggregate]
  auto restrict_own = [&](CT* out) {
    for (int g = warp; g < na; g += nwarp) {
      CT t = CT(0);
      for (int l = ab_s[g] + lane; l < ab_s[g + 1]; l += 32) t += fr_s[l];
      if constexpr (C32) t = warp_sumf(t);
      else t = warp_sum(t);
      if (lane == 0) out[a0 + g] = t;
    }
  };
  // u = D^{-1} r + P Ac^{-1} rc on own rows: the coarse rows of the own
  // aggregates (the symmetric inverse read four entries per load), then the
  // fine rows; u is mirrored to global memory
  auto precondition = [&]() {
    for (int g = warp; g < na; g += nwarp) {
      const CT* row = Ainv + (int64_t)(a0 + g) * nc4 * 4;
      CT t = CT(0);
#pragma unroll 8
      for (int k = lane; k < nc4; k += 32) {
        const CT* rr = rc_s + 4 * k;
        if constexpr (C32) {
          const float4 f = __ldg(reinterpret_cast<const float4*>(row) + k);
          t = fmaf(f.x, rr[0], t);
          t = fmaf(f.y, rr[1], t);
          t = fmaf(f.z, rr[2], t);
          t = fmaf(f.w, rr[3], t);
        } else {
          const double2 f0 = __ldg(reinterpret_cast<const double2*>(row) + 2 * k);
          const double2 f1 = __ldg(reinterpret_cast<const double2*>(row) + 2 * k + 1);
          t = fma(f0.x, rr[0], t);
          t = fma(f0.y, rr[1], t);
          t = fma(f1.x, rr[2], t);
          t = fma(f1.y, rr[3], t);
        }
      }
      if constexpr (C32) t = warp_sumf(t);
      else t = warp_sum(t);
      if (lane == 0) yc_s[g] = t;
    }
    __syncthreads();
    for (int l = tid; l < nr; l += T) {
      const double v = fma(dv[l], r[l], (double)yc_s[ag[l]]);
      u[l] = v;
      if (a.smem_vec) a.u[c0 + l] = v;
    }
  };

  // ---- initial guess: the previous correction scaled by its Galerkin
  // factor theta = (x_prev . b) / (x_prev . A x_prev) (zero on first use);
  // successive synthetic corrections share their slowly decaying shape
  double v3[3] = {0.0, 0.0, 0.0}, t3[3];
  for (int l = tid; l < nr; l += T) {
    const double b = a.b[a.perm[c0 + l]];
    const double qx = spmv(a.x, l);
    r[l] = b;
    s[l] = qx;   // A x_prev, scaled below
    v3[0] = fma(x[l], b, v3[0]);
    v3[1] = fma(x[l], qx, v3[1]);
    v3[2] = fma(b, b, v3[2]);
  }
  if (grid_reduce<3>(v3, t3, red_s, a.slots, a.bar, gen++, a.err, blk, nb, a.spin_limit)) return;
  if (tid == 0) {
    const double th = t3[1] > 0.0 ? t3[0] / t3[1] : 0.0;
    s_scal[0] = isfinite(th) ? th : 0.0;
  }
  __syncthreads();
  const double bb = t3[2];
  const double theta = s_scal[0];
  double v1[1] = {0.0}, t1[1];
  for (int l = tid; l < nr; l += T) {
    const double rv = fma(-theta, s[l], r[l]);
    r[l] = rv;
    fr_s[l] = (CT)rv;
    x[l] = theta * x[l];
    v1[0] = fma(rv, rv, v1[0]);
  }
  __syncthreads();
  restrict_own(rcx);
  if (grid_reduce<1>(v1, t1, red_s, a.slots, a.bar, gen++, a.err, blk, nb, a.spin_limit)) return;
  double rho = t1[0];
  const double stop = a.tol * a.tol * bb;
  int it = 0;
  if (bb > 0.0 && rho > stop) {
    for (int k = tid; k < Nc; k += T) rc_s[k] = __ldcg(rcx + k);
    __syncthreads();
    precondition();
    if (grid_reduce<0>(nullptr, nullptr, red_s, a.slots, a.bar, gen++, a.err, blk, nb, a.spin_limit)) return;
    // s_scal[2], s_scal[3]: 1/gamma and 1/alpha of the previous step (thread 0)
    while (true) {
      // -- w = A u, (r,u), (w,u), (r,r), aggregate sums of w
      if (it > 0) {
        for (int k = tid; k < Nc; k += T) {
          rc_s[k] = __ldcg(rcx + k);
          sc_s[k] = __ldcg(scx + k);
        }
      }
      v3[0] = v3[1] = v3[2] = 0.0;
      for (int l = tid; l < nr; l += T) {
        const double wv = spmv(a.u, l);
        w[l] = wv;
        fr_s[l] = (CT)wv;
        const double rv = r[l], uv = u[l];
        v3[0] = fma(rv, uv, v3[0]);
        v3[1] = fma(wv, uv, v3[1]);
        v3[2] = fma(rv, rv, v3[2]);
      }
      __syncthreads();
      restrict_own(rw);
      if (grid_reduce<3>(v3, t3, red_s, a.slots, a.bar, gen++, a.err, blk, nb, a.spin_limit)) return;
      const double gamma = t3[0], delta = t3[1];
      rho = t3[2];
      if (!(rho > stop) || it >= a.max_it) break;
      if (tid == 0) {
        const double beta = it == 0 ? 0.0 : gamma * s_scal[2];
        s_scal[0] = beta;
        s_scal[1] = gamma / (it == 0 ? delta : delta - beta * gamma * s_scal[3]);
      }
      __syncthreads();
      const double beta = s_scal[0], alpha = s_scal[1];
      // -- p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s
      for (int l = tid; l < nr; l += T) {
        const double pv = it == 0 ? u[l] : fma(beta, p[l], u[l]);
        const double sv = it == 0 ? w[l] : fma(beta, s[l], w[l]);
        p[l] = pv;
        s[l] = sv;
        x[l] = fma(alpha, pv, x[l]);
        r[l] = fma(-alpha, sv, r[l]);
      }
      // the same recurrence on the aggregate sums, in every block
      const CT cb = (CT)beta, ca = (CT)alpha;
      for (int k = tid; k < Nc; k += T) {
        const CT rwk = __ldcg(rw + k);
        const CT sc = it == 0 ? rwk : rwk + cb * sc_s[k];
        sc_s[k] = sc;
        rc_s[k] -= ca * sc;
      }
      __syncthreads();
      // exact aggregate sums of r and s for the next step
      for (int l = tid; l < nr; l += T) fr_s[l] = (CT)r[l];
      __syncthreads();
      restrict_own(rcx);
      __syncthreads();
      for (int l = tid; l < nr; l += T) fr_s[l] = (CT)s[l];
      __syncthreads();
      restrict_own(scx);
      precondition();
      if (tid == 0) {
        s_scal[2] = gamma;   // inverted by thread 0 inside the barrier below
        s_scal[3] = alpha;
      }
      ++it;
      if (grid_reduce<0>(nullptr, nullptr, red_s, a.slots, a.bar, gen++, a.err, blk, nb, a.spin_limit, s_scal + 2, 2)) return;
    }
  }
  // every read of the previous correction happened before the first barrier
  for (int l = tid; l < nr; l += T) {
    a.x_out[a.perm[c0 + l]] = x[l];
    a.x[c0 + l] = x[l];
  }
  if (blk == 0 && tid == 0) {
    *a.it_out += it;
    *a.res_out = bb > 0.0 ? sqrt(rho / bb) : 0.0;
  }
}

template <bool C32>
__global__ void __launch_bounds__(kCGThreads) cg_kernel(const CGArgs a) {
  extern __shared__ __align__(16) unsigned char cg_smem[];
  cg_body<C32>(a, blockIdx.x, gridDim.x, cg_smem);
}

// The corrections of several solvers in one cooperative launch: block b works
// for solver s as its block b - blk_start[s]; each solver has its own rows,
// barrier counter and slots, so the solvers never wait on one another.
template <bool C32>
__global__ void __launch_bounds__(kCGThreads) cg_batch_kernel(const CGArgs* args, const int32_t* blk_start, int n) {
  extern __shared__ __align__(16) unsigned char cg_smem[];
  __shared__ CGArgs sa;
  __shared__ int s_blk, s_nb;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (blk_start[mid] <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    sa = args[lo];
    s_blk = (int)blockIdx.x - blk_start[lo];
    s_nb = blk_start[lo + 1] - blk_start[lo];
  }
  __syncthreads();
  cg_body<C32>(sa, s_blk, (unsigned)s_nb, cg_smem);
}

cudaError_t launch_cg_batch(const CGArgs* args, const int32_t* blk_start, int n, bool coarse32, int grid,
                            int threads, size_t smem, cudaStream_t st) {
  if (n < 1) return cudaSuccess;
  if (grid < 1 || threads < 128 || threads > kCGThreads || threads % 32 != 0) return cudaErrorInvalidConfiguration;
  auto kern = coarse32 ? cg_batch_kernel<true> : cg_batch_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args, blk_start, n);
}

cudaError_t launch_cg(const CGArgs& a, bool coarse32, int grid, int threads, size_t smem, cudaStream_t st) {
  if (grid < 1 || grid > 256 || threads < 128 || threads > kCGThreads || threads % 32 != 0)
    return cudaErrorInvalidConfiguration;
  if (a.Nc > kMaxCoarse || a.W > 8) return cudaErrorInvalidValue;
  auto kern = coarse32 ? cg_kernel<true> : cg_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
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

// ============================================================================ balance
// One block; every sum is a per-thread strided sum followed by a fixed tree
// over the block, so the result does not depend on scheduling.
constexpr int kBalThreads = 512;

__device__ double block_sum_fixed(double x, double* sh) {
  sh[threadIdx.x] = x;
  __syncthreads();
  for (int o = kBalThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double t = sh[0];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kBalThreads)
wall_balance_kernel(const double* heat, const int32_t* tag_of, const int32_t* therm, int n_tags, int64_t n_wf,
                    const double* Q, const double* V, int64_t N, double* out) {
  __shared__ double sh[kBalThreads];
  double habs = 0.0;
  for (int64_t f = threadIdx.x; f < n_wf; f += kBalThreads) habs += fabs(heat[f]);
  const double absall = block_sum_fixed(habs, sh);
  double therm_sum = 0.0;
  for (int t = 0; t < n_tags; ++t) {
    double h = 0.0;
    for (int64_t f = threadIdx.x; f < n_wf; f += kBalThreads)
      if (tag_of[f] == t) h += heat[f];
    const double tot = block_sum_fixed(h, sh);
    if (therm[t]) therm_sum += tot;
    if (threadIdx.x == 0) out[3 + t] = tot;
  }
  double q = 0.0, qa = 0.0;
  for (int64_t c = threadIdx.x; c < N; c += kBalThreads) {
    const double x = Q[c] * V[c];
    q += x;
    qa += fabs(x);
  }
  const double qtot = block_sum_fixed(q, sh);
  const double qabs = block_sum_fixed(qa, sh);
  if (threadIdx.x == 0) {
    out[0] = fabs(therm_sum - qtot) / fmax(fmax(qabs, absall), 1e-300);
    out[1] = therm_sum;
    out[2] = qtot;
  }
}

cudaError_t launch_wall_balance(const double* heat, const int32_t* tag_of, const int32_t* therm, int n_tags,
                                int64_t n_wf, const double* Q, const double* V, int64_t N, double* out,
                                cudaStream_t st) {
  wall_balance_kernel<<<1, kBalThreads, 0, st>>>(heat, tag_of, therm, n_tags, n_wf, Q, V, N, out);
  return cudaGetLastError();
}

__global__ void fourier_rhs_kernel(double* rhs, const double* Q, const double* V, const double* bc, int64_t N) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c < N) rhs[c] = fma(Q[c], V[c], bc[c]);
}

cudaError_t launch_fourier_rhs(double* rhs, const double* Q, const double* V, const double* bc, int64_t N,
                               cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  fourier_rhs_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(rhs, Q, V, bc, N);
  return cudaGetLastError();
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
