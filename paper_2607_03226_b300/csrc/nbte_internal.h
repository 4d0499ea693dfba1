// Internal structures of libnanobte (host side).  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "nbte.h"

namespace nbte {

void set_error(const std::string& msg);

// Builds with NBTE_CHECKS defined add device-side consistency checks to the
// sweep (index bounds, upstream level before the reading level, ring-slot
// reuse only after the slot's last reader); a failed check is reported as
// NBTE_ERR_STATE.  Normal builds carry none of them.
#ifdef NBTE_CHECKS
constexpr bool kChecks = true;
#else
constexpr bool kChecks = false;
#endif

// nbte_test_timeouts (a diagnostic for testing the timeout paths): whether
// every bounded device wait of the launches made now must run out, and the
// poll limit a run-time-bounded wait then uses (one poll; else `dflt`).
bool test_timeouts();
unsigned long long wait_limit_or(unsigned long long dflt);

struct Status {
  int code = NBTE_OK;
  std::string msg;
  static Status ok() { return {}; }
  static Status err(int c, std::string m) { return {c, std::move(m)}; }
  bool good() const { return code == NBTE_OK; }
};

// Finite-volume mesh in the library's internal cell order (space-filling
// curve).  Half-face h = c * nfc + k is local face k of internal cell c.
struct Mesh {
  int dim = 0, cell_type = 0;
  int nvc = 0;   // nodes per cell
  int nfc = 0;   // faces per cell
  int nvf = 0;   // nodes per face
  int64_t n_nodes = 0, n_cells = 0, n_bfaces = 0;
  std::vector<int64_t> perm;    // internal -> caller cell index
  std::vector<int64_t> iperm;   // caller -> internal
  std::vector<double> V;        // [N]
  std::vector<double> xc;       // [N*dim]
  std::vector<int64_t> nb;      // [N*nfc] neighbour (internal) or -1
  std::vector<int64_t> twin;    // [N*nfc] matching half-face of the neighbour or -1
  std::vector<double> An;       // [N*nfc*dim] outward area vectors
  std::vector<double> xf;       // [N*nfc*dim] face centroids
  std::vector<int32_t> tag;     // [N*nfc] boundary tag (valid when nb < 0)
  std::vector<int32_t> tags_present;
  double volume = 0.0;
};

Status build_mesh(int dim, int64_t n_nodes, const double* xyz, int cell_type, int64_t n_cells,
                  const int64_t* cell_nodes, int64_t n_bfaces, const int64_t* bface_nodes,
                  const int32_t* bface_tag, Mesh& m);

// ------------------------------------------------------------------ plan --
// Import entry kinds (values a sweep reads from outside its direction's DAG).
enum ImportKind : int32_t { IMP_THERM = 0, IMP_DIFFUSE = 1, IMP_SPECULAR = 2, IMP_PARTIAL = 3, IMP_LAG = 4 };

struct Plan {
  int D = 0, N = 0, K = 0;                 // directions, cells, inflow entries per cell
  std::vector<int64_t> lvl_off;            // [D+1] offsets into level_ptr
  std::vector<int32_t> level_ptr;          // per direction: n_levels+1 positions
  std::vector<int32_t> n_slots;            // [D] ring slots used (excluding the zero slot)
  std::vector<int32_t> max_width;          // [D] widest level (cells)
  // position records, direction-major, N per direction
  std::vector<int32_t> pos_cell, pos_slot, pos_exp;   // [D*N]
  std::vector<int32_t> pos_last;                      // [D*N] last level that reads the position's value
                                                      // (-1: none); filled in NBTE_CHECKS builds only
  std::vector<double> pos_G;                          // [D*N]
  std::vector<int32_t> pos_ref;                       // [D*K*N]
  std::vector<double> pos_coef;                       // [D*K*N]
  // exports (values the sweep writes) and imports (values it reads)
  std::vector<int64_t> exp_off, imp_off;    // [D+1]
  std::vector<int32_t> exp_cell;            // [n_exp]
  std::vector<int32_t> imp_kind;            // [n_imp]
  std::vector<int32_t> imp_dbf;             // [n_imp] diffuse-face index (diffuse/partial)
  std::vector<int64_t> imp_src;             // [n_imp] export index (specular/partial/lag)
  std::vector<double> imp_par;              // [n_imp] T_wall' (therm) or p (partial)
  // diffuse re-emission: per diffuse/partial boundary half-face, CSR over the
  // outgoing directions: export index and weight w_j (s_j.n) / sum_in w |s.n|
  std::vector<int64_t> dif_ptr;             // [n_dbf+1]
  std::vector<int64_t> dif_src;
  std::vector<double> dif_wt;
  // energy balance: per boundary half-face in the wall-flux table
  std::vector<int32_t> wf_tag;              // [n_wf] tag of the face
  std::vector<int32_t> wf_cell;             // [n_wf]
  std::vector<int64_t> wf_ptr;              // [n_wf+1] CSR over directions
  std::vector<int64_t> wf_val;              // export index (>=0) or -(1+import index)
  std::vector<double> wf_coef;              // w_i (s_i . An) (signed)
  int64_t lagged_faces = 0;
  int64_t total_levels = 0;
  int max_levels = 0, max_slots = 0, max_width_all = 0;
};

struct BC {
  int32_t tag;
  int32_t type;
  double T_wall;
  double p;
};

Status build_plan(const Mesh& m, int D, const double* s, const double* w, const std::vector<BC>& bcs,
                  double T_ref, Plan& plan, int n_threads);

// TPFA Laplacian of the synthetic correction (CSR, internal cell order).
struct Laplacian {
  std::vector<int32_t> row_ptr, col;
  std::vector<double> val, diag;
  // per cell, over its thermalizing faces: sum g_f and sum g_f T_wall (the
  // Dirichlet data of a diffusion solve with the wall temperatures)
  std::vector<double> bc_g, bc_gT;
};
void build_laplacian(const Mesh& m, const std::vector<BC>& bcs, double kappa_bulk, double k1,
                     Laplacian& L);

// Second-order upwind reconstruction tables (internal cell order): per
// half-face h = c*nfc + k the neighbour (or -1), the face's local index in the
// neighbour, An/V (3 components, z = 0 in 2D), and per (h, m) the weight
// a[h*nfc + m] = (P_c r_m) . (x_f - x_c) of the least-squares gradient
// (P_c the pseudo-inverse of sum_m r_m r_m^T, r_m = x_nb(m) - x_c), so that
// e_f - e_c = sum_m a (e_nb(m) - e_c); zero for wall faces m and for cells
// with fewer than dim + 1 face neighbours.
struct Reconstruction {
  std::vector<int32_t> nb, twin;
  std::vector<double> AnV, a;
  // the same operator in two factors: gradient weights gw[(c*nf + m)*3 + d]
  // (grad_d = sum_m gw (e[nb m] - e[c]); zero without a gradient) and face
  // offsets rf[(c*nf + k)*3 + d] (face centroid minus cell centroid), so
  // that a[(c*nf + k)*nf + m] = sum_d gw[(c*nf + m)*3 + d] rf[(c*nf + k)*3 + d]
  std::vector<double> gw, rf;
  int64_t cells_with_gradient = 0;
};
void build_reconstruction(const Mesh& m, Reconstruction& rc);

// geometric aggregates (boxes of the cell-centroid bounding box); returns the
// number of non-empty aggregates, agg[c] in [0, n)
int build_aggregates(const Mesh& m, int target, std::vector<int32_t>& agg);
// dense SPD inverse in place (row-major); false if not positive definite
bool dense_spd_inverse(std::vector<double>& A, int n);

}  // namespace nbte
