// Data preparation around the transport sweep (sm_103a): packing the
// position records into chunk blocks, the per-iteration gather of (T', Qdot)
// into those blocks, the FP64 denominators, and the second-order upwind
// sources the sweep adds to its upwind sums.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "layout.h"
#include "vecio.cuh"

namespace nbte {

// One block per chunk: its positions' records (multiples of 16 bytes, copied
// as 16-byte words) to the chunk's block, and each position's pair index
__global__ void pack_blocks_kernel(unsigned char* blk, int2* tq_dst, const unsigned char* rec_pos,
                                   const Chunk* chunks, const int64_t* chunk_doff, const int32_t* chunk_dir,
                                   const int64_t* sub_ptr, const int32_t* sub_end, int64_t N, int rec_size,
                                   int pair_bytes) {
  const int64_t c = blockIdx.x;
  const Chunk ch = chunks[c];
  const int64_t doff = chunk_doff[c];
  const int64_t q0 = (int64_t)chunk_dir[c] * N + ch.pos;
  const int n_lev = chunk_levels(ch.nimp_end);
  int32_t* hdr = reinterpret_cast<int32_t*>(blk + doff);
  for (int t = threadIdx.x; t <= n_lev; t += blockDim.x) hdr[t] = t == 0 ? n_lev : sub_end[sub_ptr[c] + t - 1];
  const int64_t roff = doff + chunk_header_bytes(n_lev);
  const int w16 = rec_size / 16;
  const uint4* src = reinterpret_cast<const uint4*>(rec_pos + (size_t)q0 * rec_size);
  uint4* dst = reinterpret_cast<uint4*>(blk + roff);
  for (int t = threadIdx.x; t < ch.len * w16; t += blockDim.x) dst[t] = src[t];
  const uint32_t tq0 = (uint32_t)((roff + (int64_t)ch.len * rec_size) / pair_bytes);
  // the cell is the record's first word
  for (int j = threadIdx.x; j < ch.len; j += blockDim.x)
    tq_dst[q0 + j] = make_int2(*reinterpret_cast<const int32_t*>(rec_pos + (size_t)(q0 + j) * rec_size),
                               (int32_t)(tq0 + (uint32_t)j));
}

cudaError_t launch_pack_blocks(unsigned char* blk, int2* tq_dst, const unsigned char* rec_pos,
                               const Chunk* chunks, const int64_t* chunk_doff, const int32_t* chunk_dir,
                               const int64_t* sub_ptr, const int32_t* sub_end, int64_t n_chunks, int64_t N,
                               int rec_size, int pair_bytes, cudaStream_t st) {
  if (n_chunks == 0) return cudaSuccess;
  if (rec_size % 16 != 0 || n_chunks > 0x7fffffff) return cudaErrorInvalidValue;
  pack_blocks_kernel<<<(unsigned)n_chunks, 128, 0, st>>>(blk, tq_dst, rec_pos, chunks, chunk_doff, chunk_dir,
                                                         sub_ptr, sub_end, N, rec_size, pair_bytes);
  return cudaGetLastError();
}

// FP64 denominators of every (work item, position); one thread per pair
__global__ void fill_dinv_kernel(double* dinv, const double* pos_G, const double* band_v, const double* band_inv_tau,
                                 int D, int ng, int G, int64_t N) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)D * ng * N) return;
  const int64_t item = t / N, pos = t - item * N;
  const int i = (int)(item / ng), g = (int)(item - (int64_t)i * ng);
  const double Gc = pos_G[(size_t)i * N + pos];
  for (int b = 0; b < G; ++b) dinv[t * G + b] = 1.0 / (band_inv_tau[g * G + b] + band_v[g * G + b] * Gc);
}

cudaError_t launch_fill_dinv(double* dinv, const double* pos_G, const double* band_v, const double* band_inv_tau,
                             int D, int n_groups, int G, int64_t N, cudaStream_t st) {
  const int64_t n = (int64_t)D * n_groups * N;
  if (n == 0) return cudaSuccess;
  fill_dinv_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dinv, pos_G, band_v, band_inv_tau, D, n_groups, G,
                                                                N);
  return cudaGetLastError();
}

// (T', Qdot) of every position's cell, in each direction's level order, so
// the sweep's producer can bulk-copy them with the position records
template <typename R>
__global__ void gather_tq_kernel(R* data, const int2* tq_dst, const R* srcTQ, int64_t n,
                                 unsigned long long* res_zero) {
  using R2 = typename Vec2<R>::T;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (res_zero && q < 2) res_zero[q] = 0ull;
  if (q >= n) return;
  const int2 cd = __ldcs(tq_dst + q);   // (cell, pair index)
  reinterpret_cast<R2*>(data)[(uint32_t)cd.y] = __ldg(reinterpret_cast<const R2*>(srcTQ) + cd.x);
}

// Second-order upwind sources in one pass (triangles, quadrilaterals,
// tetrahedra).  One thread per (direction, position): it
// resolves the cell's faces once -- upwind cell, its neighbours and the
// reconstruction weights toward the face -- and keeps them in registers
// while it walks the band groups along each needed row of the direction's
// distribution (N*Bp values, L2-resident while the direction's blocks run).
// Consecutive threads take consecutive positions, so each band group's
// results are stored as one contiguous run of the [item][position][G]
// layout the sweep copies.  Wall faces get d = 0 and read the cell itself;
// a wall neighbour of the upwind cell reads the upwind cell (zero difference,
// zero weight): no branches between the loads.
template <typename R, int G, int NF>
__global__ void __launch_bounds__(256, 1) src2_kernel(const Src2Args<R> a) {
  static_assert(NF <= 4, "hexahedra take the two-pass form");
  const int i = a.dir0 + blockIdx.y;   // direction (a 2D grid: no division by N)
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.N) return;
  const int c = __ldg(a.pos_cell + (int64_t)i * a.N + p);
  const R sx = (R)a.dir_s[i * 3], sy = (R)a.dir_s[i * 3 + 1], sz = (R)a.dir_s[i * 3 + 2];
  R d[NF], w[NF][NF];
  int u[NF], h[NF], nbu[NF][NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const int nk = __ldg(a.nb + (int64_t)c * NF + k);
    const int tw = __ldg(a.twin + (int64_t)c * NF + k);
    const R* An = a.AnV + ((int64_t)c * NF + k) * 3;
    R dk = sx * __ldg(An) + sy * __ldg(An + 1) + sz * __ldg(An + 2);
    if (nk < 0) dk = R(0);
    const bool in = dk < R(0);
    d[k] = dk;
    u[k] = in ? nk : c;
    h[k] = in ? tw : k;
#pragma unroll
    for (int m2 = 0; m2 < NF; ++m2) {
      const int nm = __ldg(a.nb + (int64_t)u[k] * NF + m2);
      nbu[k][m2] = nm >= 0 ? nm : u[k];
      w[k][m2] = __ldg(a.rc_a + ((int64_t)u[k] * NF + h[k]) * NF + m2);
    }
  }
  const R* e = a.e + (size_t)i * a.N * a.Bp;
  R* out = a.src2 + ((size_t)i * a.n_groups * a.N + p) * G;
  for (int g = 0; g < a.n_groups; ++g) {
    const R* eg = e + g * G;
    R acc[G];
#pragma unroll
    for (int b = 0; b < G; ++b) acc[b] = R(0);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      R eu[G], inc[G];
      load_vals<R, G>(eg + (size_t)u[k] * a.Bp, eu);
#pragma unroll
      for (int b = 0; b < G; ++b) inc[b] = R(0);
#pragma unroll
      for (int m2 = 0; m2 < NF; ++m2) {
        R en[G];
        load_vals<R, G>(eg + (size_t)nbu[k][m2] * a.Bp, en);
#pragma unroll
        for (int b = 0; b < G; ++b) inc[b] += w[k][m2] * (en[b] - eu[b]);
      }
#pragma unroll
      for (int b = 0; b < G; ++b) acc[b] -= d[k] * inc[b];
    }
    store_vals<R, G>(out + (size_t)g * a.N * G, acc);
  }
}

// Second-order upwind sources in two passes (hexahedra), over a batch of
// directions.
//  1. grad_kernel: one thread per (direction, cell) takes the least-squares
//     gradient of every band, grad_d = sum_m gw[c, m, d] (e[nb m] - e[c]),
//     from the cell's row of the previous sweep's distribution and its
//     neighbours' rows (NF + 1 gathered rows per cell), stored as
//     grad[dir][cell][group][d][G].
//  2. face_src_kernel: one thread per (direction, position) sums over the
//     cell's interior faces f: -(s . An_f / V) (grad_u . rf[u, f_u]), u the
//     face's upwind cell (the cell itself on outflow faces) and f_u the
//     face's local index in u: NF gathered gradient blocks per position.
// The single pass gathers NF (NF + 1) rows per position (the upwind cell
// and its neighbours, for every face): 42 for hexahedra against 7 + 6 here.
// For NF <= 4 the gradient buffer's traffic outweighs the saving (measured
// on triangles and tetrahedra), so those meshes keep the single pass.  Wall faces get d = 0; a wall
// neighbour reads the cell itself (zero difference, zero weight).  Results
// go to the [item][position][G] layout the sweep copies, one contiguous run
// per band group.
template <typename R, int G, int NF, int DIM>
__global__ void __launch_bounds__(256) grad_kernel(const Src2Args<R> a) {
  const int i = a.dir0 + blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.N) return;
  int nb[NF];
  R w[NF][DIM];
#pragma unroll
  for (int m = 0; m < NF; ++m) {
    const int nm = __ldg(a.nb + (int64_t)c * NF + m);
    nb[m] = nm >= 0 ? nm : c;
#pragma unroll
    for (int d = 0; d < DIM; ++d) w[m][d] = __ldg(a.gw + ((int64_t)c * NF + m) * 3 + d);
  }
  const R* e = a.e + (size_t)i * a.N * a.Bp;
  R* gr = a.grad + ((size_t)blockIdx.y * a.N + c) * a.Bp * DIM;
  for (int g = 0; g < a.n_groups; ++g) {
    const R* eg = e + g * G;
    R ec[G], acc[DIM][G];
    load_vals<R, G>(eg + (size_t)c * a.Bp, ec);
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int b = 0; b < G; ++b) acc[d][b] = R(0);
#pragma unroll
    for (int m = 0; m < NF; ++m) {
      R en[G];
      load_vals<R, G>(eg + (size_t)nb[m] * a.Bp, en);
#pragma unroll
      for (int b = 0; b < G; ++b) {
        const R diff = en[b] - ec[b];
#pragma unroll
        for (int d = 0; d < DIM; ++d) acc[d][b] += w[m][d] * diff;
      }
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) store_vals<R, G>(gr + (size_t)(g * DIM + d) * G, acc[d]);
  }
}

template <typename R, int G, int NF, int DIM>
__global__ void __launch_bounds__(256) face_src_kernel(const Src2Args<R> a) {
  const int bi = blockIdx.y;   // direction within the batch (a 2D grid: no division by N)
  const int i = a.dir0 + bi;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.N) return;
  const int c = __ldg(a.pos_cell + (int64_t)i * a.N + p);
  const R sx = (R)a.dir_s[i * 3], sy = (R)a.dir_s[i * 3 + 1], sz = (R)a.dir_s[i * 3 + 2];
  R dk[NF], rf[NF][DIM];
  int u[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const int nk = __ldg(a.nb + (int64_t)c * NF + k);
    const int tw = __ldg(a.twin + (int64_t)c * NF + k);
    const R* An = a.AnV + ((int64_t)c * NF + k) * 3;
    R d = sx * __ldg(An) + sy * __ldg(An + 1) + sz * __ldg(An + 2);
    if (nk < 0) d = R(0);
    const bool in = d < R(0);
    dk[k] = d;
    u[k] = in ? nk : c;
    const int h = in ? tw : k;
#pragma unroll
    for (int q = 0; q < DIM; ++q) rf[k][q] = __ldg(a.rf + ((int64_t)u[k] * NF + h) * 3 + q);
  }
  const R* grad = a.grad + (size_t)bi * a.N * a.Bp * DIM;
  R* out = a.src2 + ((size_t)i * a.n_groups * a.N + p) * G;
  for (int g = 0; g < a.n_groups; ++g) {
    R acc[G];
#pragma unroll
    for (int b = 0; b < G; ++b) acc[b] = R(0);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const R* gu = grad + ((size_t)u[k] * a.Bp + g * G) * DIM;
      R face[G];
#pragma unroll
      for (int b = 0; b < G; ++b) face[b] = R(0);
#pragma unroll
      for (int q = 0; q < DIM; ++q) {
        R gq[G];
        load_vals<R, G>(gu + q * G, gq);
#pragma unroll
        for (int b = 0; b < G; ++b) face[b] += rf[k][q] * gq[b];
      }
#pragma unroll
      for (int b = 0; b < G; ++b) acc[b] -= dk[k] * face[b];
    }
    store_vals<R, G>(out + (size_t)g * a.N * G, acc);
  }
}

template <typename R, int G, int NF, int DIM>
static cudaError_t launch_src2_fd(const Src2Args<R>& a, cudaStream_t st) {
  const dim3 grid((unsigned)((a.N + 255) / 256), (unsigned)a.n_dirs);
  grad_kernel<R, G, NF, DIM><<<grid, 256, 0, st>>>(a);
  face_src_kernel<R, G, NF, DIM><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename R, int G>
static cudaError_t launch_src2_g(const Src2Args<R>& a, cudaStream_t st) {
  if (a.nfc == 6 && a.dim == 3) return launch_src2_fd<R, G, 6, 3>(a, st);
  const dim3 grid((unsigned)((a.N + 255) / 256), (unsigned)a.n_dirs);
  switch (a.nfc) {
    case 3: src2_kernel<R, G, 3><<<grid, 256, 0, st>>>(a); break;
    case 4: src2_kernel<R, G, 4><<<grid, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_src2(const Src2Args<R>& a, cudaStream_t st) {
  if ((int64_t)a.n_dirs * a.N == 0) return cudaSuccess;
  if (a.Bp != a.n_groups * a.G || a.n_dirs > 65535 || a.dir0 < 0 || a.dir0 + a.n_dirs > a.D)
    return cudaErrorInvalidValue;
  switch (a.G) {
    case 1: return launch_src2_g<R, 1>(a, st);
    case 2: return launch_src2_g<R, 2>(a, st);
    case 4: return launch_src2_g<R, 4>(a, st);
    case 8:
      if constexpr (sizeof(R) == 4) return launch_src2_g<R, 8>(a, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_gather_tq(unsigned char* data, const int2* tq_dst, const R* srcTQ, int64_t n,
                             unsigned long long* res_zero, cudaStream_t st) {
  if (n == 0 && !res_zero) return cudaSuccess;
  const int64_t blocks = n > 0 ? (n + 255) / 256 : 1;
  gather_tq_kernel<R><<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<R*>(data), tq_dst, srcTQ, n, res_zero);
  return cudaGetLastError();
}

template cudaError_t launch_src2<float>(const Src2Args<float>&, cudaStream_t);
template cudaError_t launch_src2<double>(const Src2Args<double>&, cudaStream_t);
template cudaError_t launch_gather_tq<float>(unsigned char*, const int2*, const float*, int64_t, unsigned long long*,
                                              cudaStream_t);
template cudaError_t launch_gather_tq<double>(unsigned char*, const int2*, const double*, int64_t, unsigned long long*,
                                               cudaStream_t);

}  // namespace nbte
