// Launch interface of the device kernels (internal; no torch types).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "layout.h"
#include "sweep_args.h"

namespace nbte {

template <typename R>
cudaError_t launch_sweep(const SweepArgs<R>& a, int K, int G, int n_items, int threads, size_t smem,
                         cudaStream_t st);
// work items of several solvers sharing (R, K, G, ring placement, upwind order) in one
// launch; args[s] and item_start[s] (prefix sums, n_solvers+1 entries) are
// device arrays
template <typename R>
cudaError_t launch_sweep_batch(const SweepArgs<R>* args, const int32_t* item_start, int n_solvers, int K, int G,
                               bool global_ring, bool order2, int n_items, int threads, size_t smem,
                               cudaStream_t st);
// dinv[(item*N + pos)*G + b] = 1 / (band_inv_tau[g*G+b] + band_v[g*G+b] G_pos),
// item = i*n_groups + g, G_pos = pos_G[i*N + pos]
cudaError_t launch_fill_dinv(double* dinv, const double* pos_G, const double* band_v, const double* band_inv_tau,
                             int D, int n_groups, int G, int64_t N, cudaStream_t st);
// Rearrange position-ordered records into chunk blocks (header with the
// chunk's level ends, records, then room for the chunk's (T', Qdot) pairs)
// and set tq_dst (per position: its cell and the index of its (T', Qdot)
// pair in the blocks, in pairs): one block per chunk.
cudaError_t launch_pack_blocks(unsigned char* blk, int2* tq_dst, const unsigned char* rec_pos,
                               const Chunk* chunks, const int64_t* chunk_doff, const int32_t* chunk_dir,
                               const int64_t* sub_ptr, const int32_t* sub_end, int64_t n_chunks, int64_t N,
                               int rec_size, int pair_bytes, cudaStream_t st);
// (T', Qdot) of every position's cell into its chunk's block:
// ((R2*)data)[tq_dst[q].y] = ((R2*)srcTQ)[tq_dst[q].x], q = i*N + position.
// res_zero, if not null, gets its two words cleared (the residual maxima the
// iteration's update collects).
template <typename R>
cudaError_t launch_gather_tq(unsigned char* data, const int2* tq_dst, const R* srcTQ, int64_t n,
                             unsigned long long* res_zero, cudaStream_t st);

// Second-order upwind source of every work item and position of the
// directions [dir0, dir0 + n_dirs), from the previous sweep's distribution
// e[(i*N + cell)*Bp + band] (direction i, all bands of a cell contiguous):
//   src2 = -sum over the cell's interior faces f of (s_i . An_f / V) *
//          grad_u . rf[u, f_u],
//   grad_u = sum_m gw[u, m] (e[nb(u, m)] - e[u]),
// u the face's upwind cell (the cell itself on outflow faces) and f_u the
// face's local index in u.  Hexahedra take two launches: the gradients of
// the batch into grad[(j*N + cell)*Bp*dim + (group*dim + d)*G + b]
// (j = i - dir0), then the face sums.  Other cells take one, with the
// weights toward each face precombined (rc_a).  Written at
// src2[(item*N + pos)*G + b], item = i*n_groups + g, the layout the sweep's
// chunks copy.
template <typename R>
struct Src2Args {
  int N, nfc, dim, G, n_items, n_groups, Bp, D;
  int dir0, n_dirs;              // the batch of directions
  const R* e;
  R* src2;
  R* grad;                       // [n_dirs*N*Bp*dim] gradients of the batch
  const int32_t* pos_cell;       // [D*N] cell of each position
  const int32_t* nb;             // [N*nfc] neighbour or -1
  const int32_t* twin;           // [N*nfc] the face's local index in the neighbour
  const R* AnV;                  // [N*nfc*3] outward face vector / cell volume
  const R* rc_a;                 // [N*nfc*nfc] weights toward each face (one pass: nfc <= 4)
  const R* gw;                   // [N*nfc*3] gradient weights, zero without a gradient (two
                                 // passes: hexahedra)
  const R* rf;                   // [N*nfc*3] face centroid minus cell centroid (two passes)
  const double* dir_s;           // [D*3]
};
template <typename R>
cudaError_t launch_src2(const Src2Args<R>& a, cudaStream_t st);

template <typename R>
void launch_init_exports(R* exp, const int32_t* exp_cell, const double* Tdev, const double* CoW, int Bp, int G,
                         int Gpad, int64_t n_exp, cudaStream_t st);

template <typename R>
struct WallArgs {
  int Bp, G, Gpad;
  int64_t n_exp, n_imp, n_dbf;
  const R* exp;
  R* imp;
  const int32_t* exp_cell;
  const double* Delta;           // [N] synthetic correction carried by lagged values
  const double* CoW;             // [Bp] C / W
  const int32_t* imp_kind;
  const int32_t* imp_dbf;
  const int64_t* imp_src;
  const double* imp_par;
  const int64_t* dif_ptr;
  const int64_t* dif_src;
  const double* dif_wt;
  double* dsum;                  // [n_dbf*Bp]
};
template <typename R>
void launch_walls(const WallArgs<R>& a, cudaStream_t st);

// collision-moment reduction + temperature update
template <typename R>
struct UpdateArgs {
  int N, n_items;
  int mode;                      // 0 sequential, 1 synthetic (DSA), 2 synthetic (literal), 3 rhs only
  double inv_beta, beta;
  const R* part;                 // [n_items*N] collision-moment partials of e - e0, or null:
  double* acc;                   // [N] their FP64 sums from the sweep's atomic adds (read, then cleared)
  const double* Q;
  const double* V;
  double* T;                     // T' iterate (in/out)
  double* Tprev;                 // T' the sweep started from (written by modes 0 and 3)
  double* Tkin;                  // kinetic T'_L of this sweep
  double* Delta;                 // T'^{n+1} - T'_L
  double* rhs;                   // synthetic right-hand side
  const double* delta;           // synthetic correction
  R* srcTQ_next;                 // [2*N]
  unsigned long long* res;       // [2] max |dT|, max |T'| (as ordered bits)
};
template <typename R>
void launch_update(const UpdateArgs<R>& a, cudaStream_t st);

// Two-level preconditioned CG on the synthetic-correction Laplacian.  Rows
// are in aggregate order (cells of one aggregate contiguous); block k owns
// aggregates [blk_agg[k], blk_agg[k+1]) and their cells
// [blk_cell[k], blk_cell[k+1]).  M^{-1} r = D^{-1} r + P Ac^{-1} P^T r with P
// the piecewise-constant aggregate prolongation and Ac^{-1} dense.

// One block's published partial sums, one 64-byte line per block,
// double-buffered by barrier parity: a block can only write the sums of
// barrier k+2 after every block has arrived at barrier k+1, i.e. has finished
// reading the sums of barrier k.
struct alignas(64) CGSlot {
  double v[2][3];
  double pad[2];
};

struct CGArgs {
  int N, Nc, W;                  // rows, aggregates, ELL width (off-diagonals per row, <= 8)
  const int32_t* ell_col;        // [W][N] off-diagonal columns (padding: own row)
  const double* ell_val;         // [W][N] off-diagonal values (padding: 0)
  const double* diag;            // [N]
  const double* dinv;            // [N]
  const int32_t* perm;           // aggregate-order row -> internal cell
  const int32_t* agg_rel;        // aggregate of each row minus its block's first aggregate
  const int32_t* agg_cell;       // [Nc+1] first row of each aggregate
  const int32_t* blk_cell;       // [grid+1]
  const int32_t* blk_agg;        // [grid+1]
  const float* Ainv32;           // [Nc * Nc4*4] coarse inverse, rows padded with zeros to Nc4*4
  const double* Ainv64;          // the same in FP64
  int Nc4;                       // ceil(Nc / 4)
  int max_rows, max_na;          // largest block's rows / aggregates
  int smem_vec, smem_ell;        // own-row vectors / ELL rows held in shared memory
  const double* b;               // right-hand side, internal order
  double* x_out;                 // solution, internal order
  double* x;                     // [N] previous correction in, new correction out (aggregate order)
  double* u;                     // [N] M^{-1} r (read by the neighbours' products)
  double* x_work;                // [N] work vectors when not in shared memory
  double* r;
  double* p;
  double* s;
  double* w;
  void* rw;                      // [Nc] aggregate sums of w (coarse precision)
  void* rcx;                     // [Nc] aggregate sums of r
  void* scx;                     // [Nc] aggregate sums of s
  CGSlot* slots;                 // [grid]
  unsigned long long* bar;       // barrier counter (only grows)
  int32_t* err;
  unsigned long long spin_limit; // polls of the barrier word before giving up (kCgSpinPolls; one
                                 // poll under nbte_test_timeouts)
  double tol;
  int max_it;
  int32_t* it_out;
  double* res_out;
};
// default polls of the CG grid barrier before it gives up (seconds)
constexpr unsigned long long kCgSpinPolls = 1ull << 24;
// persistent cooperative PCG; coarse32 selects the FP32 coarse preconditioner
cudaError_t launch_cg(const CGArgs& a, bool coarse32, int grid, int threads, size_t smem, cudaStream_t st);
// several solvers' corrections in one cooperative launch; args[s] and
// blk_start[s] (prefix sums of blocks, n+1 entries) are device arrays
cudaError_t launch_cg_batch(const CGArgs* args, const int32_t* blk_start, int n, bool coarse32, int grid,
                            int threads, size_t smem, cudaStream_t st);

// dynamic shared memory of the CG kernel (byte offsets, 16-byte aligned)
struct CgSmem {
  size_t red, rc, sc, yc, fr, ab, vec, ell, total;
};
NBTE_HD constexpr size_t cg_align16(size_t x) { return (x + 15) / 16 * 16; }
NBTE_HD inline CgSmem cg_smem_layout(int nc4, int max_rows, int max_na, int W, int threads, int vec, int ell,
                                     int coarse_bytes) {
  CgSmem L{};
  size_t o = 0;
  L.red = o;
  o = cg_align16(o + (size_t)3 * threads * 8);
  L.rc = o;
  o = cg_align16(o + (size_t)4 * nc4 * coarse_bytes);
  L.sc = o;
  o = cg_align16(o + (size_t)4 * nc4 * coarse_bytes);
  L.yc = o;
  o = cg_align16(o + (size_t)max_na * coarse_bytes);
  L.fr = o;
  o = cg_align16(o + (size_t)max_rows * coarse_bytes);
  L.ab = o;
  o = cg_align16(o + (size_t)(max_na + 1) * 4);
  L.vec = o;
  if (vec) o = cg_align16(o + (size_t)7 * max_rows * 8 + (size_t)max_rows * 4);
  L.ell = o;
  if (ell) o = cg_align16(o + (size_t)W * max_rows * 8 + (size_t)max_rows * 8 + (size_t)W * max_rows * 4);
  L.total = o;
  return L;
}
constexpr int kCGThreads = 512;
constexpr int kMaxCoarse = 2048;   // aggregates of the coarse space (staged in shared memory)

template <typename R>
struct WallHeatArgs {
  int Bp, G, Gpad;
  int64_t n_exp, n_imp;
  int64_t n_wf;
  const int64_t* wf_ptr;
  const int64_t* wf_val;
  const double* wf_coef;
  const R* exp;
  const R* imp;
  const double* band_v;          // [Bp] FP64
  double* heat;                  // [n_wf]
};
template <typename R>
void launch_wall_heat(const WallHeatArgs<R>& a, cudaStream_t st);

// Wall heat per boundary tag and the energy balance of the last sweep, FP64,
// in one block with a fixed summation order:
//   out[0]            |sum_thermalizing tags heat - integral Qdot| /
//                     max(integral |Qdot|, sum |heat|)
//   out[1], out[2]    sum over thermalizing tags of the heat, integral Qdot
//   out[3 + t]        heat through tag index t (t < n_tags)
// heat[f] is the net outward flow through wall face f (launch_wall_heat),
// tag_of[f] its tag index, therm[t] = 1 for thermalizing tags.
cudaError_t launch_wall_balance(const double* heat, const int32_t* tag_of, const int32_t* therm, int n_tags,
                                int64_t n_wf, const double* Q, const double* V, int64_t N, double* out,
                                cudaStream_t st);
// rhs[c] = Q[c] V[c] + bc[c]: the right-hand side of the diffusion initial
// guess (bc holds the thermalizing walls' Dirichlet terms)
cudaError_t launch_fourier_rhs(double* rhs, const double* Q, const double* V, const double* bc, int64_t N,
                               cudaStream_t st);

template <typename R>
void launch_fill_srcTQ(R* srcTQ, const double* T, const double* Q, int N, cudaStream_t st);
// dst[c] = src[perm[c]] (caller order -> internal order)
cudaError_t launch_from_caller(double* dst, const double* src, const int32_t* perm, int N, cudaStream_t st);
// dst[perm[c]*dim + d] = src[c*dim + d] * scale + offset (internal -> caller order)
cudaError_t launch_to_caller(double* dst, const double* src, const int32_t* perm, int N, int dim, double scale,
                             double offset, cudaStream_t st);

}  // namespace nbte
