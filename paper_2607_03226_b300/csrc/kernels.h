// Launch interface of the device kernels (internal; no torch types).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace nbte {

// device error word values (written by bounded waits, read by the host)
enum DevError : int32_t { DEV_OK = 0, DEV_BARRIER_TIMEOUT = 1, DEV_QUEUE_TIMEOUT = 2 };

template <typename R>
struct SweepArgs {
  int N, Bp, G, n_groups, dim;
  int full;                      // also accumulate E and q (atomics)
  int lp_smem_off;               // byte offset of the level pointers after the ring
  const int32_t* item_dir;       // [n_items]
  const int32_t* item_grp;       // [n_items]
  const int64_t* lvl_off;        // [D+1]
  const int32_t* level_ptr;
  const int32_t* pos_cell;       // [D*N]
  const int32_t* pos_slot;
  const int32_t* pos_exp;
  const R* pos_G;
  const int32_t* pos_ref;        // [D*K*N]
  const R* pos_coef;
  const int64_t* exp_off;        // [D+1]
  const int64_t* imp_off;
  const R* imp;                  // [n_imp*Bp]
  R* exp;                        // [n_exp*Bp]
  const R* srcTQ;                // [2*N] (T', Qdot) per cell
  const R* band_v;               // [Bp]
  const R* band_inv_tau;
  const R* band_cw;              // C / W
  const R* band_aQ;              // C / (C_tot W)
  const double* dir_w;           // [D]
  const double* dir_s;           // [D*3]
  double* part;                  // [n_items*N] collision-moment partials
  double* accE;                  // [N]   (full)
  double* accQ;                  // [N*dim] (full)
};

template <typename R>
cudaError_t launch_sweep(const SweepArgs<R>& a, int K, int bpt, int lanes, int n_items, int threads,
                  size_t smem, cudaStream_t st);

template <typename R>
void launch_init_exports(R* exp, const int32_t* exp_cell, const double* Tdev, const double* CoW, int Bp,
                         int64_t n_exp, cudaStream_t st);

template <typename R>
struct WallArgs {
  int Bp;
  int64_t n_imp, n_dbf;
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
  const double* part;
  const double* Q;
  const double* V;
  double* T;                     // T' iterate (in/out)
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
struct CGArgs {
  int N, Nc;
  const int32_t* rp;
  const int32_t* col;
  const double* val;
  const double* dinv;
  const int32_t* perm;           // aggregate-order row -> internal cell
  const int32_t* agg;            // aggregate of each row
  const int32_t* agg_cell;       // [Nc+1] first row of each aggregate
  const int32_t* blk_cell;       // [grid+1]
  const int32_t* blk_agg;        // [grid+1]
  const float* Ainv;             // [Nc * Nc4*4], rows padded with zeros to Nc4*4
  int Nc4;                       // ceil(Nc / 4)
  const double* b;               // right-hand side, internal order
  double* x_out;                 // solution, internal order
  double* x;                     // work vectors in aggregate order
  double* r;
  double* z;
  double* p;
  double* Ap;
  double* rc;                    // [Nc]
  double* yc;                    // [Nc]
  double* partial;               // [5*grid]
  unsigned* bar;                 // [2] count, generation
  int32_t* err;
  double tol;
  int max_it;
  int32_t* it_out;
  double* res_out;
};
// persistent cooperative PCG; returns cudaError of the launch
cudaError_t launch_cg(const CGArgs& a, int grid, cudaStream_t st);
constexpr int kCGThreads = 1024;
constexpr int kMaxCoarse = 2048;   // aggregates of the coarse space (rc staged in shared memory)

template <typename R>
struct WallHeatArgs {
  int Bp;
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

template <typename R>
void launch_fill_srcTQ(R* srcTQ, const double* T, const double* Q, int N, cudaStream_t st);

}  // namespace nbte
