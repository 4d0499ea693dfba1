// extern "C" entry points of libnanobte (see include/nbte.h) and the solve
// iteration loop.  One outer iteration (Sec. II, Eq. (6) / Eq. (12)) is
//   walls -> sweep -> moment reduction + update [-> CG correction -> update]
// on the solver's stream; the host reads two residual words per iteration
// and stops at tol.  With use_graph the iteration is captured once as a CUDA
// graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <cstdlib>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "iteration_monitor.h"
#include "kernels.h"
#include "nbte_internal.h"

using namespace nbte;

namespace nbte {
static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
// nbte_test_timeouts: every bounded device wait of later launches runs out
static std::atomic<int> g_test_timeouts{0};
bool test_timeouts() { return g_test_timeouts.load(std::memory_order_relaxed) != 0; }
unsigned long long wait_limit_or(unsigned long long dflt) { return test_timeouts() ? 1ull : dflt; }
}  // namespace nbte

#define NBTE_CK(call)                                                                               \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      set_error(std::string("CUDA error in ") + #call + ": " + cudaGetErrorString(e_));             \
      return e_ == cudaErrorMemoryAllocation ? NBTE_ERR_OOM : NBTE_ERR_CUDA;                        \
    }                                                                                               \
  } while (0)

namespace {

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

// RAII device allocation
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t alloc(size_t n) {
    if (n == 0) n = 16;
    if (p && n == bytes) return cudaSuccess;
    release();
    cudaError_t e = cudaMalloc(&p, n);
    if (e == cudaSuccess) bytes = n;
    else p = nullptr;
    return e;
  }
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
};

// A plain cudaMemcpy from pageable memory may return before its DMA lands,
// and it runs on the legacy stream, which the solvers' non-blocking streams
// do not wait for: wait for it here, so that every later launch sees the data.
template <typename T>
cudaError_t upload(DBuf& b, const std::vector<T>& v) {
  cudaError_t e = b.alloc(v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
  return e;
}

// Zero device memory in the order of `st` and wait for it (device error
// words and set-up buffers that the next launches on `st` read).
inline cudaError_t zero_now(void* p, size_t n, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(p, 0, n, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

template <typename T>
std::vector<float> to_float(const std::vector<T>& v) {
  std::vector<float> f(v.size());
  for (size_t i = 0; i < v.size(); ++i) f[i] = (float)v[i];
  return f;
}

}  // namespace

struct nbte_mesh {
  Mesh m;
};

// sweep launch shape picked by timing candidates (band group, chunk length)
struct Tuned {
  bool valid = false;
  int G = 0, cap = 0;
  int64_t key = -1;
  double ms = 0.0;
};

struct nbte_solver {
  const nbte_mesh* mesh = nullptr;
  int device = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  double T_ref = 300.0;
  // inputs (caller order for Q converted to internal)
  int B = 0;
  std::vector<double> C, v, tau;
  int D = 0;
  std::vector<double> s, w;
  std::vector<BC> bcs;
  bool bcs_set = false;
  // heat source: caller order in pinned host memory (what the caller set),
  // internal order on the device (Qd)
  double* h_qc = nullptr;   // pinned, or ordinary memory where pinning is unavailable
  bool h_qc_pinned = false;
  int64_t q_dev_version = -1;
  int64_t version_plan = 0, version_bands = 0, version_q = 0;

  // ---- plan (depends on quadrature and walls)
  int64_t plan_built = -1;
  int K = 0, D_plan = 0;
  int64_t n_exp = 0, n_imp = 0, n_dbf = 0, n_wf = 0, lagged = 0, total_levels = 0;
  int max_levels = 0, max_slots = 0, max_width = 0;
  std::vector<int32_t> wf_tag_h;
  Plan plan;                                  // host copy: records are packed per precision from it
  DBuf exp_off, imp_off, exp_cell, imp_kind, imp_dbf, imp_src, imp_par, dif_ptr, dif_src, dif_wt;
  DBuf wf_ptr, wf_val, wf_coef, dir_w, dir_s;
  // ---- band layout (depends on bands, precision and tuning)
  std::string layout_key, rec_key, chunk_key;
  int prec = 0, G = 1, Gpad = 4, n_groups = 1, Bp = 1, n_items = 0, threads = 160, n_stages = 4;
  int stage_bytes = 0, off_ring = 0, off_stage = 0, off_imp = 0, off_den = 0, off_src2 = 0;
  size_t smem = 0;
  int order = 1;                              // upwind order of the current layout
  bool partials = false;                      // collision moment as (item, cell) partials, else atomic sums
  std::vector<int32_t> item_of;               // [D*n_groups] CTA index of (direction i, band group g) at i*n_groups+g
  // second-order upwind: previous distribution [n_items*N*G], per-position
  // sources [n_items*N*G], gradients of one batch of directions
  // [o2_db*N*Bp*dim], reconstruction tables (mesh only; kept per precision)
  DBuf o2_e, o2_src, o2_grad, rc_nb, rc_twin, rc_AnV, rc_a, rc_gw, rc_rf;
  int o2_db = 0;                              // directions per gradient batch
  int rc_prec = -1;
  int64_t rc_cells = 0;
  // most wall/lag imports in one chunk, per chunk length (sizes the stages' import region)
  int64_t cimp_plan = -1;
  std::map<int, int> cimp_max, csub_max;
  double W = 0, beta = 0, Ctot = 0;
  DBuf rec_pos, rec, pos_cell, chunks, chunk_off, chunk_doff, chunk_dir, chunk_sub_ptr, chunk_sub_end, tq_dst, gring,
      e_scratch, dinv;
  std::string blk_key;
  std::vector<Chunk> h_chunks;                // host copy of the chunks of the current chunk length
  std::vector<int64_t> h_chunk_off;           // [D+1] first chunk of each direction
  std::vector<int64_t> h_sub_ptr;             // [chunks+1] CSR of the chunks' level ends
  std::vector<int32_t> h_sub_end;
  int64_t gring_stride = 0;
  DBuf item_dir, item_grp, band_v, band_itau, band_aT, band_aQ, band_CoW, band_v64;
  DBuf expt, impt, srcTQ, srcTQ_fin, part, acc, T, Tprev, Tkin, Delta, rhs, delta, Qd, Vd, dsum, accE, accQ, res, heat;
  DBuf perm_d, io_d;   // caller index of each internal cell; caller-order staging on the device
  DBuf cg_r, cg_u, cg_w, cg_p, cg_s, cg_xw, cg_slots, cg_bar, cg_err, cg_it, cg_res;
  DBuf cg_Ainv64;
  DBuf cg_x, cg_rw, cg_rcx, cg_scx, cg_perm, cg_agg_rel, cg_agg_cell, cg_blk_cell, cg_blk_agg, cg_Ainv;
  int cg_grid = 0, cg_threads = kCGThreads, cg_Nc = 0, cg_Nc4 = 0, cg_W = 0;
  int cg_max_rows = 0, cg_max_na = 0, cg_smem_vec = 0, cg_smem_ell = 0;
  int64_t cg_part_key = -1;
  std::vector<int32_t> h_agg_cell, h_agg_p;   // aggregate row ranges / aggregate of each row (aggregate order)
  std::vector<double> h_fourier_bc;           // [N] Dirichlet rhs of the diffusion initial guess
  // ---- laplacian (synthetic)
  int64_t lap_built = -1;
  DBuf L_ecol, L_eval, L_diag, L_dinv;
  // ---- autotuned sweep layout per precision
  Tuned tuned[2];
  // ---- state
  bool have_state = false;
  bool have_results = false;   // T (kind 0, 2) of the last solve
  bool have_outputs = false;   // E, q, wall heat of the last sweep
  unsigned long long* h_res = nullptr;   // pinned: [2] residual words
  int32_t* h_misc = nullptr;             // pinned: [2] device error, cg iterations
  mutable double* h_stage = nullptr;     // pinned staging of result fields read back to the host
  mutable size_t h_stage_n = 0;
  cudaGraphExec_t graph = nullptr;
  std::string graph_key;
  double last_energy_imbalance = 0;
  // wall heat per tag of the last output sweep, computed on the device:
  // tag_list[t] is the tag of index t, wall_heat_by_tag[t] its heat
  std::vector<int32_t> tag_list;
  std::vector<double> wall_heat_by_tag;
  DBuf wf_tagidx, tag_therm, balance, fbc;
  DBuf pos_last, chk_level, chk_last;         // NBTE_CHECKS builds only

  ~nbte_solver() {
    if (graph) cudaGraphExecDestroy(graph);
    if (h_qc && h_qc_pinned) cudaFreeHost(h_qc);
    if (h_qc && !h_qc_pinned) std::free(h_qc);
    if (h_res) cudaFreeHost(h_res);
    if (h_misc) cudaFreeHost(h_misc);
    if (h_stage) cudaFreeHost(h_stage);
    if (own_stream) cudaStreamDestroy(own_stream);
  }
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

size_t device_bytes(const nbte_solver* S) {
  const DBuf* all[] = {&S->rec_pos, &S->rec, &S->pos_cell, &S->gring, &S->e_scratch, &S->dinv, &S->chunks,
                       &S->chunk_off, &S->chunk_doff, &S->chunk_dir, &S->chunk_sub_ptr, &S->chunk_sub_end,
                       &S->tq_dst, &S->exp_off, &S->imp_off,
                       &S->exp_cell, &S->imp_kind, &S->imp_dbf, &S->imp_src, &S->imp_par, &S->dif_ptr,
                       &S->dif_src, &S->dif_wt, &S->wf_ptr, &S->wf_val, &S->wf_coef, &S->dir_w, &S->dir_s,
                       &S->item_dir, &S->item_grp, &S->band_v, &S->band_itau, &S->band_aT, &S->band_aQ,
                       &S->band_CoW, &S->band_v64, &S->expt, &S->impt, &S->srcTQ, &S->srcTQ_fin, &S->part, &S->acc,
                       &S->T, &S->Tprev, &S->Tkin, &S->Delta, &S->rhs, &S->delta, &S->Qd, &S->Vd, &S->dsum,
                       &S->perm_d, &S->io_d,
                       &S->accE, &S->accQ, &S->res, &S->heat, &S->cg_r, &S->cg_u, &S->cg_p, &S->cg_s,
                       &S->cg_w, &S->cg_slots, &S->cg_err, &S->cg_it, &S->cg_res, &S->cg_x, &S->cg_rw,
                       &S->cg_rcx, &S->cg_scx, &S->cg_xw, &S->cg_bar, &S->cg_Ainv64,
                       &S->cg_perm, &S->cg_agg_rel, &S->cg_agg_cell, &S->cg_blk_cell, &S->cg_blk_agg,
                       &S->cg_Ainv, &S->L_ecol, &S->L_eval,
                       &S->L_diag, &S->L_dinv, &S->o2_e, &S->o2_src, &S->o2_grad, &S->rc_nb, &S->rc_twin,
                       &S->rc_AnV, &S->rc_a, &S->rc_gw, &S->rc_rf, &S->wf_tagidx, &S->tag_therm, &S->balance,
                       &S->fbc, &S->pos_last, &S->chk_level, &S->chk_last};
  size_t t = 0;
  for (auto* b : all) t += b->bytes;
  return t;
}

void drop_graph(nbte_solver* S) {
  if (S->graph) cudaGraphExecDestroy(S->graph);
  S->graph = nullptr;
  S->graph_key.clear();
}

// status of a non-zero sweep error word (a bounded wait gave up, or, in
// NBTE_CHECKS builds, a consistency check failed)
int sweep_error(uint64_t word) {
  if (word == (uint64_t)DEV_CHECK_FAILED)
    return fail(NBTE_ERR_STATE, "a device-side consistency check of the sweep failed (index bounds or level order)");
  return fail(NBTE_ERR_DEVICE_TIMEOUT, "a bounded wait of the sweep's copy pipeline gave up");
}

// ------------------------------------------------------------------ plan
int ensure_plan(nbte_solver* S) {
  if (S->plan_built == S->version_plan) return NBTE_OK;
  if (S->D <= 0) return fail(NBTE_ERR_STATE, "nbte_set_quadrature must be called before solving");
  if (!S->bcs_set) return fail(NBTE_ERR_STATE, "nbte_set_boundaries must be called before solving");
  const Mesh& m = S->mesh->m;
  Plan P;
  const int nt = (int)std::max(1u, std::thread::hardware_concurrency());
  Status st = build_plan(m, S->D, S->s.data(), S->w.data(), S->bcs, S->T_ref, P, nt);
  if (!st.good()) return fail(st.code, st.msg);
  // compact the inflow entries to the largest count actually used
  const int64_t N = P.N;
  int K = 1;
  for (int i = 0; i < P.D; ++i)
    for (int k = P.K - 1; k >= K; --k) {
      bool any = false;
      const size_t off = ((size_t)i * P.K + k) * N;
      for (int64_t p = 0; p < N && !any; ++p) any = P.pos_coef[off + p] != 0.0 || P.pos_ref[off + p] != 0;
      if (any) { K = k + 1; break; }
    }
  if (K < P.K) {
    std::vector<int32_t> ref((size_t)P.D * K * N);
    std::vector<double> coef((size_t)P.D * K * N);
    for (int i = 0; i < P.D; ++i)
      for (int k = 0; k < K; ++k) {
        std::copy_n(P.pos_ref.begin() + ((size_t)i * P.K + k) * N, N, ref.begin() + ((size_t)i * K + k) * N);
        std::copy_n(P.pos_coef.begin() + ((size_t)i * P.K + k) * N, N, coef.begin() + ((size_t)i * K + k) * N);
      }
    P.pos_ref.swap(ref);
    P.pos_coef.swap(coef);
    P.K = K;
  }
  DeviceGuard g(S->device);
  drop_graph(S);
  S->rec.release();
  S->rec_key.clear();
  S->chunk_key.clear();
  S->blk_key.clear();
  NBTE_CK(upload(S->exp_off, P.exp_off));
  NBTE_CK(upload(S->imp_off, P.imp_off));
  NBTE_CK(upload(S->exp_cell, P.exp_cell));
  NBTE_CK(upload(S->imp_kind, P.imp_kind));
  NBTE_CK(upload(S->imp_dbf, P.imp_dbf));
  NBTE_CK(upload(S->imp_src, P.imp_src));
  NBTE_CK(upload(S->imp_par, P.imp_par));
  NBTE_CK(upload(S->dif_ptr, P.dif_ptr));
  NBTE_CK(upload(S->dif_src, P.dif_src));
  NBTE_CK(upload(S->dif_wt, P.dif_wt));
  NBTE_CK(upload(S->wf_ptr, P.wf_ptr));
  NBTE_CK(upload(S->wf_val, P.wf_val));
  NBTE_CK(upload(S->wf_coef, P.wf_coef));
  NBTE_CK(upload(S->dir_w, S->w));
  NBTE_CK(upload(S->dir_s, S->s));
  S->K = K;
  S->D_plan = P.D;
  S->n_exp = P.exp_off.back();
  S->n_imp = P.imp_off.back();
  S->n_dbf = (int64_t)P.dif_ptr.size() - 1;
  S->n_wf = (int64_t)P.wf_tag.size();
  S->wf_tag_h = P.wf_tag;
  {
    // wall faces by tag index, and which tags are thermalizing (the energy
    // balance and the per-tag wall heat are summed on the device)
    std::vector<int32_t> tags(P.wf_tag.begin(), P.wf_tag.end());
    std::sort(tags.begin(), tags.end());
    tags.erase(std::unique(tags.begin(), tags.end()), tags.end());
    std::vector<int32_t> idx(P.wf_tag.size()), th(tags.size(), 0);
    for (size_t f = 0; f < P.wf_tag.size(); ++f)
      idx[f] = (int32_t)(std::lower_bound(tags.begin(), tags.end(), P.wf_tag[f]) - tags.begin());
    for (const BC& b : S->bcs) {
      auto it = std::lower_bound(tags.begin(), tags.end(), b.tag);
      if (it != tags.end() && *it == b.tag && b.type == NBTE_THERMALIZING) th[it - tags.begin()] = 1;
    }
    NBTE_CK(upload(S->wf_tagidx, idx));
    NBTE_CK(upload(S->tag_therm, th));
    NBTE_CK(S->balance.alloc((3 + tags.size()) * 8));
    S->tag_list = tags;
  }
  S->lagged = P.lagged_faces;
  S->total_levels = P.total_levels;
  S->max_levels = P.max_levels;
  S->max_slots = P.max_slots;
  S->max_width = P.max_width_all;
  S->plan = std::move(P);
  S->plan_built = S->version_plan;
  S->layout_key.clear();
  S->have_state = false;
  return NBTE_OK;
}

// Packed position records of precision R (see layout.h), direction-major,
// uploaded once per plan and precision; ensure_blocks rearranges them per
// chunk length.
template <typename R>
int ensure_records(nbte_solver* S) {
  const std::string key = std::to_string(sizeof(R)) + "/" + std::to_string(S->plan_built);
  if (key == S->rec_key && S->rec_pos.p) return NBTE_OK;
  const Plan& P = S->plan;
  const int K = P.K;
  const RecLayout L = rec_layout((int)sizeof(R), K);
  const size_t n = (size_t)P.D * P.N;
  std::vector<unsigned char> buf(n * L.size, 0);
  for (int i = 0; i < P.D; ++i)
    for (int64_t p = 0; p < P.N; ++p) {
      const size_t q = (size_t)i * P.N + p;
      unsigned char* r = buf.data() + q * L.size;
      std::memcpy(r, &P.pos_cell[q], 4);
      std::memcpy(r + 4, &P.pos_slot[q], 4);
      std::memcpy(r + 8, &P.pos_exp[q], 4);
      const R G = (R)P.pos_G[q];
      std::memcpy(r + L.off_G, &G, sizeof(R));
      for (int k = 0; k < K; ++k) {
        const size_t qk = ((size_t)i * K + k) * P.N + p;
        const R c = (R)P.pos_coef[qk];
        std::memcpy(r + L.off_ref + 4 * k, &P.pos_ref[qk], 4);
        std::memcpy(r + L.off_coef + sizeof(R) * k, &c, sizeof(R));
      }
    }
  NBTE_CK(upload(S->rec_pos, buf));
  NBTE_CK(upload(S->pos_cell, P.pos_cell));
  if (kChecks) NBTE_CK(upload(S->pos_last, P.pos_last));
  S->rec_key = key;
  S->blk_key.clear();
  return NBTE_OK;
}

// The sweep's chunk blocks for the current chunks: each chunk's header (its
// level count and level ends), its records, then room for its (T', Qdot)
// pairs, so that one bulk copy brings all three.
// chunk_doff holds each block's byte offset; tq_dst, per position
// (direction-major), its cell and the index of its pair in units of pairs.
// Packed on the device from the position-ordered records.
template <typename R>
int ensure_blocks(nbte_solver* S, int cap) {
  const std::string key = S->rec_key + "/" + S->chunk_key;
  if (key == S->blk_key && S->rec.p) return NBTE_OK;
  const Plan& P = S->plan;
  const RecLayout L = rec_layout((int)sizeof(R), P.K);
  const int pair = 2 * (int)sizeof(R);
  const size_t nch = S->h_chunks.size();
  std::vector<int64_t> doff(nch);
  std::vector<int32_t> cdir(nch);
  size_t total = 0;
  for (int i = 0; i < P.D; ++i)
    for (int64_t c = S->h_chunk_off[i]; c < S->h_chunk_off[i + 1]; ++c) {
      doff[c] = (int64_t)total;
      cdir[c] = i;
      const Chunk& ch = S->h_chunks[c];
      total += chunk_header_bytes(chunk_levels(ch.nimp_end)) + (size_t)ch.len * L.size +
               chunk_tq_bytes(ch.len, (int)sizeof(R));
    }
  if (total / pair > 0xffffffffull) return fail(NBTE_ERR_OOM, "position records exceed the 32-bit pair index");
  NBTE_CK(upload(S->chunk_doff, doff));
  NBTE_CK(upload(S->chunk_dir, cdir));
  NBTE_CK(upload(S->chunk_sub_ptr, S->h_sub_ptr));
  NBTE_CK(upload(S->chunk_sub_end, S->h_sub_end));
  NBTE_CK(S->rec.alloc(total));
  NBTE_CK(S->tq_dst.alloc((size_t)P.D * P.N * 8));
  NBTE_CK(cudaMemsetAsync(S->rec.p, 0, S->rec.bytes, S->stream));
  NBTE_CK(launch_pack_blocks(S->rec.as<unsigned char>(), S->tq_dst.as<int2>(), S->rec_pos.as<unsigned char>(),
                             S->chunks.as<Chunk>(), S->chunk_doff.as<int64_t>(), S->chunk_dir.as<int32_t>(),
                             S->chunk_sub_ptr.as<int64_t>(), S->chunk_sub_end.as<int32_t>(), (int64_t)nch, P.N,
                             L.size, pair, S->stream));
  NBTE_CK(cudaStreamSynchronize(S->stream));
  S->blk_key = key;
  return NBTE_OK;
}

// Chunks of one sweep: consecutive whole levels of a direction are packed
// into one chunk while they total at most cap positions (the consumers
// separate them with a named barrier, the copy and stage hand-off are
// shared); a level wider than cap is split into chunks of its own.
// sub_end lists, per chunk, where each of its levels ends (relative to the
// chunk's first position).  Imports are numbered in position order, so each
// chunk's imports are one contiguous slice.
struct ChunkList {
  std::vector<Chunk> ch;
  std::vector<int64_t> off;        // [D+1] first chunk of each direction
  std::vector<int64_t> sub_ptr;    // [chunks+1]
  std::vector<int32_t> sub_end;
  int max_imp = 0, max_sub = 0;
};

int build_chunks(const Plan& P, int cap, ChunkList& out) {
  out = ChunkList{};
  out.off.assign(P.D + 1, 0);
  out.sub_ptr.push_back(0);
  for (int i = 0; i < P.D; ++i) {
    int32_t imp = 0;
    const int32_t* lp = P.level_ptr.data() + P.lvl_off[i];
    const int L = (int)(P.lvl_off[i + 1] - P.lvl_off[i]) - 1;
    auto n_imports = [&](int32_t p0, int32_t p1) {
      int32_t n = 0;
      for (int k = 0; k < P.K; ++k) {
        const int32_t* ref = P.pos_ref.data() + ((size_t)i * P.K + k) * P.N;
        for (int32_t p = p0; p < p1; ++p) n += ref[p] < 0;
      }
      return n;
    };
    auto emit = [&](int32_t p0, int32_t p1, bool level_end, const std::vector<int32_t>& ends) {
      const int32_t nimp = n_imports(p0, p1);
      Chunk c;
      c.pos = p0;
      c.len = p1 - p0;
      c.imp = imp;
      c.nimp_end = chunk_flags(nimp, (int)ends.size(), level_end);
      out.ch.push_back(c);
      for (int32_t e : ends) out.sub_end.push_back(e);
      out.sub_ptr.push_back((int64_t)out.sub_end.size());
      out.max_imp = std::max(out.max_imp, (int)nimp);
      out.max_sub = std::max(out.max_sub, (int)ends.size());
      imp += nimp;
    };
    int32_t b0 = -1;                 // first position of the chunk being filled
    std::vector<int32_t> ends;       // its level ends, relative to b0
    for (int l = 0; l < L; ++l) {
      const int32_t w = lp[l + 1] - lp[l];
      if (w > cap) {
        if (b0 >= 0) emit(b0, lp[l], true, ends);
        b0 = -1;
        ends.clear();
        for (int32_t p0 = lp[l]; p0 < lp[l + 1]; p0 += cap) {
          const int32_t p1 = std::min(lp[l + 1], p0 + cap);
          emit(p0, p1, p1 == lp[l + 1], {p1 - p0});
        }
        continue;
      }
      if (b0 >= 0 && lp[l + 1] - b0 > cap) {
        emit(b0, lp[l], true, ends);
        b0 = -1;
        ends.clear();
      }
      if (b0 < 0) b0 = lp[l];
      ends.push_back(lp[l + 1] - b0);
    }
    if (b0 >= 0) emit(b0, lp[L], true, ends);
    if (imp != P.imp_off[i + 1] - P.imp_off[i]) return fail(NBTE_ERR_MESH, "internal: import numbering");
    out.off[i + 1] = (int64_t)out.ch.size();
  }
  if (out.max_imp > kChunkMaxImports || out.max_sub > kChunkMaxLevels)
    return fail(NBTE_ERR_MESH, "internal: chunk descriptor field overflow");
  return NBTE_OK;
}

// the most imports and levels any chunk of length <= cap holds (they size a
// copy stage's import region and block header)
int chunk_extents(nbte_solver* S, int cap, int* max_imp, int* max_sub) {
  if (S->cimp_plan != S->plan_built) {
    S->cimp_max.clear();
    S->csub_max.clear();
    S->cimp_plan = S->plan_built;
  }
  auto it = S->cimp_max.find(cap);
  if (it == S->cimp_max.end()) {
    ChunkList cl;
    int rc = build_chunks(S->plan, cap, cl);
    if (rc) return rc;
    S->cimp_max[cap] = cl.max_imp;
    S->csub_max[cap] = cl.max_sub;
  }
  *max_imp = S->cimp_max[cap];
  *max_sub = S->csub_max[cap];
  return NBTE_OK;
}

int ensure_chunks(nbte_solver* S, int cap) {
  const std::string key = std::to_string(cap) + "/" + std::to_string(S->plan_built);
  if (key == S->chunk_key && S->chunks.p) return NBTE_OK;
  ChunkList cl;
  int rc = build_chunks(S->plan, cap, cl);
  if (rc) return rc;
  NBTE_CK(upload(S->chunks, cl.ch));
  NBTE_CK(upload(S->chunk_off, cl.off));
  S->h_chunks = std::move(cl.ch);
  S->h_chunk_off = std::move(cl.off);
  S->h_sub_ptr = std::move(cl.sub_ptr);
  S->h_sub_end = std::move(cl.sub_end);
  S->chunk_key = key;
  return NBTE_OK;
}

int64_t tune_key(const nbte_solver* S) { return S->plan_built * 1000003 + S->version_bands; }

// ------------------------------------------------------------------ layout
// Chooses and allocates the sweep layout for options o.  With `estimate`
// non-null nothing is allocated: *estimate receives the device bytes the
// layout would hold (records, tables, distributions' in-flight buffers,
// per-cell fields), for admission by memory budget.
// bytes of second-order gradients held at once (hexahedra compute them in
// direction batches of this size): 2 GiB, or NBTE_O2_GRAD_BYTES when set
// (smaller batches exercise the batching on small meshes)
static size_t o2_grad_budget() {
  size_t budget = (size_t)2 << 30;
  if (const char* v = std::getenv("NBTE_O2_GRAD_BYTES")) {
    const long long x = std::atoll(v);
    if (x > 0) budget = (size_t)x;
  }
  return budget;
}

// largest per-(work item, cell) partial table of the collision moment kept in
// the fixed-order form without being asked for (see ensure_layout)
constexpr size_t kPartialsMaxBytes = (size_t)256 << 20;

int ensure_layout(nbte_solver* S, const nbte_solve_opts& o, size_t* estimate = nullptr) {
  if (S->B <= 0) return fail(NBTE_ERR_STATE, "nbte_set_bands must be called before solving");
  const int prec = o.precision;
  const int sz = prec ? 4 : 8;
  const int K = S->K;
  const RecLayout RL = rec_layout(sz, K);
  // the autotuner's choice stands in for "planner's choice" (0, 0)
  int want_G = o.band_group, want_threads = o.cta_threads;
  const Tuned& tu = S->tuned[prec];
  if (want_G == 0 && want_threads == 0 && o.ring == 0 && tu.valid && tu.key == tune_key(S)) {
    want_G = tu.G;
    want_threads = tu.cap + 32;
  }
  // consumer threads of a sweep CTA = positions per chunk
  int cap = 128;
  if (want_threads != 0) {
    if (want_threads < 64 || want_threads > 544 || want_threads % 32 != 0)
      return fail(NBTE_ERR_ARG, "cta_threads must be a multiple of 32 in [64, 544]");
    cap = want_threads - 32;
  }
  if (o.threads_per_cell > 1) return fail(NBTE_ERR_ARG, "threads_per_cell must be 0 or 1");
  // shared memory of one CTA: barriers and chunk headers, the value ring, and
  // the copy stages (records, (T', Qdot) pairs, imports, and with FP64 the
  // precomputed denominators 1/(1/tau + v G) of the chunk's positions)
  const bool order2 = o.order == 2;
  int off_src2 = 0;
  // import rows of a chunk: sized by the fullest chunk, not by cap * K; the
  // block header by the chunk with the most levels
  int cimp = 0, csub = 0;
  {
    const int rc0 = chunk_extents(S, cap, &cimp, &csub);
    if (rc0) return rc0;
  }
  // a stage: the chunk block (header, records, (T', Qdot) pairs), the
  // chunk's import rows, FP64 denominators, second-order sources
  auto stage_of = [&](int Gv, int& off_imp, int& off_den) {
    const int gpad = padded_group(Gv, sz);
    const int rec = (int)chunk_header_bytes(csub) + cap * RL.size;
    const int tq = ((cap + 2) * 2 * sz + 15) / 16 * 16;
    const int imp = cimp * gpad * sz;
    const int den = prec ? 0 : ((cap + 2) * Gv * 8 + 15) / 16 * 16;
    // second order: the chunk's reconstruction sources (superset of at most cap + 3 positions)
    const int src2 = order2 ? ((cap + 4) * Gv * sz + 15) / 16 * 16 : 0;
    off_imp = rec + tq;
    off_den = rec + tq + imp;
    off_src2 = rec + tq + imp + den;
    return rec + tq + imp + den + src2;
  };
  // the value ring: in shared memory when it fits beside two copy stages,
  // else one global-memory region per CTA
  auto ring_of = [&](int Gv) { return (int)(((size_t)(S->max_slots + 1) * Gv * sz + 15) / 16 * 16); };
  const int head = 32 * 8;   // up to 8 stages: full + empty barriers and chunk headers
  auto smem_ring = [&](int Gv) {
    int a, b;
    return (int64_t)head + ring_of(Gv) + 2 * (int64_t)stage_of(Gv, a, b) <= kSweepSmemMax;
  };
  auto ring_smem_bytes = [&](int Gv) { return smem_ring(Gv) ? ring_of(Gv) : 0; };
  const int maxG = prec ? 8 : 4;
  int G = want_G;
  if (G > 0) {
    if (!(G == 1 || G == 2 || G == 4 || G == 8) || G > maxG)
      return fail(NBTE_ERR_ARG, prec ? "band_group must be 1, 2, 4 or 8" : "band_group must be 1, 2 or 4 in FP64");
  } else {
    G = 0;
    double best = 1e300;
    for (int c : {8, 4, 2, 1}) {
      if (c > maxG) continue;
      const int ng = (S->B + c - 1) / c;
      const double waste = (double)(ng * c - S->B) / S->B;
      // prefer wide groups with a shared-memory ring, unless they pad more than 12.5%
      const double score = (waste <= 0.125 ? -c : 1000.0 * waste - c) + (smem_ring(c) ? 0.0 : 100.0);
      if (score < best) { best = score; G = c; }
    }
  }
  if (o.ring == 1 && !smem_ring(G))
    return fail(NBTE_ERR_ARG, "the value ring does not fit in shared memory (" + std::to_string(S->max_slots) +
                                  " live cells in one direction)");
  const bool gr = o.ring == 2 || !smem_ring(G);
  {
    int a, b;
    if ((int64_t)head + 2 * (int64_t)stage_of(G, a, b) > kSweepSmemMax)
      return fail(NBTE_ERR_ARG, "cta_threads too large for shared memory with this band group");
  }
  // stages: 2..8.  The sweep of one item is a long dependent chain of
  // levels, so co-resident CTAs are what hides its latency: aim for every
  // work item resident at once, else for as many CTAs per SM as still get
  // three stages each, then give each CTA as many stages as that allows
  int off_imp = 0, off_den = 0;
  const int stage = stage_of(G, off_imp, off_den);
  const int off_src2_sel = off_src2;
  const int ng = (S->B + G - 1) / G;
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, S->device);
  const int64_t ringB = ring_smem_bytes(G);
  auto total = [&](int ns) { return (int64_t)head + ringB + (int64_t)ns * stage; };
  auto budget = [&](int t) { return (int64_t)(228 * 1024) / t - 1024; };
  int per_sm = std::max(1, (S->D * ng + nsm - 1) / nsm);
  while (per_sm > 1 && total(3) > budget(per_sm)) --per_sm;
  // a global-memory value ring is served by L1, which shares the SM's 256 KB
  // with shared memory: past about 96 KB of copy stages per CTA the ring's
  // loads fall through to L2 (1.14M-tet FinFET, band group 8: 57 ms per sweep
  // at 96 KB, 70 ms at 225 KB)
  const int64_t smem_cap = gr ? std::min<int64_t>(kSweepSmemMax, 96 * 1024) : kSweepSmemMax;
  int ns = 8;
  while (ns > 2 && total(ns) > std::min<int64_t>(budget(per_sm), smem_cap)) --ns;
  const int Bp = ng * G;
  const int threads = cap + 32;
  if (estimate) {
    const size_t N = (size_t)S->mesh->m.n_cells, D = (size_t)S->D, Gp = (size_t)padded_group(G, sz);
    size_t b = D * N * (2 * RL.size + 12 + 2 * sz);                     // records (by position and in chunk
                                                                         // blocks), cells, (cell, pair) index,
                                                                         // (T', Qdot)
    b += N * 8;                                                          // collision moment (FP64)
    if (o.deterministic != 0 || (size_t)D * ng * N * sz <= kPartialsMaxBytes)
      b += D * ng * N * sz;                                              // its fixed-order partials
    b += (size_t)ng * (S->n_exp + S->n_imp) * Gp * sz;                   // export / import rows
    if (gr) b += (size_t)D * ng * (((size_t)(S->max_slots + 1) * G + 3) / 4 * 4) * sz;   // global rings
    b += N * (4 * sz + 12 * 8 + 8 * (size_t)S->mesh->m.dim);            // per-cell fields
    if (!prec) b += (size_t)D * Bp * N * 8;                              // FP64 denominators
    if (order2) {                                                        // previous distribution, sources,
      const size_t nf = (size_t)S->mesh->m.nfc;                         // gradients of one batch, tables
      const size_t grad_dir = N * Bp * (size_t)S->mesh->m.dim * sz;
      b += 2 * D * Bp * N * sz + N * nf * (8 + 3 * sz);
      if (nf == 6) b += std::max<size_t>(1, std::min<size_t>(D, o2_grad_budget() / grad_dir)) * grad_dir + N * nf * 6 * sz;
      else b += N * nf * nf * sz;
    }
    b += D * N / 8 + (size_t)S->n_dbf * Bp * 8 + (size_t)S->n_wf * 16;  // chunks, diffuse sums, wall heat
    *estimate = b;
    return NBTE_OK;
  }
  // the collision moment: fixed-order partials per (work item, cell) when
  // they are small (they stay mostly in L2 and are written about as fast as
  // atomic adds resolve) or when asked for, else FP64 atomic sums per cell
  // (the partials' scattered 4-byte writes went to HBM sector by sector on
  // the 1.14M-tet FinFET: 38 ms per sweep against 32 ms with atomic sums; on
  // the 2D fin the atomic adds cost 0.43 against 0.33 ms)
  const bool partials = o.deterministic != 0 || (size_t)S->D * ng * S->mesh->m.n_cells * sz <= kPartialsMaxBytes;
  const std::string key = std::to_string(prec) + "/" + std::to_string(G) + "/" + std::to_string(cap) + "/" +
                          std::to_string(S->version_bands) + "/" + std::to_string(S->plan_built) + "/" +
                          std::to_string(ns) + (gr ? "/global" : "/shared") + (order2 ? "/o2" : "/o1") +
                          (partials ? "/part" : "/acc");
  if (key == S->layout_key) return NBTE_OK;
  DeviceGuard dg(S->device);
  drop_graph(S);
  int rc = prec ? ensure_records<float>(S) : ensure_records<double>(S);
  if (rc) return rc;
  rc = ensure_chunks(S, cap);
  if (rc) return rc;
  rc = prec ? ensure_blocks<float>(S, cap) : ensure_blocks<double>(S, cap);
  if (rc) return rc;
  S->prec = prec; S->G = G; S->Gpad = padded_group(G, sz); S->n_groups = ng; S->Bp = Bp;
  S->n_items = S->D * ng;
  S->threads = threads;
  S->n_stages = ns;
  S->stage_bytes = stage;
  S->off_imp = off_imp;
  S->off_den = off_den;
  S->off_src2 = off_src2_sel;
  S->order = order2 ? 2 : 1;
  S->off_ring = head;
  S->off_stage = head + (int)ringB;
  S->gring_stride = gr ? ((int64_t)(S->max_slots + 1) * G + 3) / 4 * 4 : 0;
  S->smem = (size_t)S->off_stage + (size_t)ns * stage;
  const int64_t N = S->mesh->m.n_cells;
  // band constants, padded bands are inert (C = 0, v = 0, 1/tau = 1)
  S->W = 0;
  for (double x : S->w) S->W += x;
  S->beta = 0;
  S->Ctot = 0;
  for (int l = 0; l < S->B; ++l) { S->beta += S->C[l] / S->tau[l]; S->Ctot += S->C[l]; }
  std::vector<double> bv(Bp, 0.0), bit(Bp, 1.0), baT(Bp, 0.0), baQ(Bp, 0.0), bCoW(Bp, 0.0);
  for (int l = 0; l < S->B; ++l) {
    bv[l] = S->v[l];
    bit[l] = 1.0 / S->tau[l];
    baT[l] = S->C[l] / S->W;   // e0 = (C/W) T' of Eq. (11)
    baQ[l] = S->C[l] / (S->Ctot * S->W);
    bCoW[l] = S->C[l] / S->W;
  }
  if (prec) {
    NBTE_CK(upload(S->band_v, to_float(bv)));
    NBTE_CK(upload(S->band_itau, to_float(bit)));
    NBTE_CK(upload(S->band_aT, to_float(baT)));
    NBTE_CK(upload(S->band_aQ, to_float(baQ)));
  } else {
    NBTE_CK(upload(S->band_v, bv));
    NBTE_CK(upload(S->band_itau, bit));
    NBTE_CK(upload(S->band_aT, baT));
    NBTE_CK(upload(S->band_aQ, baQ));
  }
  NBTE_CK(upload(S->band_CoW, bCoW));
  NBTE_CK(upload(S->band_v64, bv));
  // CTA order of the work items: direction by direction, a direction's band
  // groups side by side (they read the same records, which L2 then serves
  // after the first).  Longest directions first measured no better on the
  // 1.14M-tet FinFET (31.36 against 31.25 ms, same box).
  std::vector<int32_t> idir(S->n_items), igrp(S->n_items), dorder(S->D);
  for (int i = 0; i < S->D; ++i) dorder[i] = i;
  S->item_of.assign(S->n_items, 0);
  for (int k = 0; k < S->D; ++k)
    for (int g = 0; g < ng; ++g) {
      const int it = k * ng + g, i = dorder[k];
      idir[it] = i;
      igrp[it] = g;
      S->item_of[i * ng + g] = it;
    }
  NBTE_CK(upload(S->item_dir, idir));
  NBTE_CK(upload(S->item_grp, igrp));
  NBTE_CK(S->expt.alloc((size_t)ng * S->n_exp * S->Gpad * sz));
  NBTE_CK(S->impt.alloc((size_t)ng * S->n_imp * S->Gpad * sz));
  NBTE_CK(S->srcTQ.alloc((size_t)2 * N * sz));
  NBTE_CK(S->srcTQ_fin.alloc((size_t)2 * N * sz));
  NBTE_CK(S->acc.alloc((size_t)N * 8));
  NBTE_CK(cudaMemsetAsync(S->acc.p, 0, (size_t)N * 8, S->stream));
  S->partials = partials;
  if (partials) NBTE_CK(S->part.alloc((size_t)S->n_items * N * sz));
  else S->part.release();
  if (gr) {
    NBTE_CK(S->gring.alloc((size_t)S->n_items * S->gring_stride * sz));
  } else {
    S->gring.release();
  }
  if (kChecks) {
    NBTE_CK(S->chk_level.alloc((size_t)S->n_items * (S->max_slots + 1) * 4));
    NBTE_CK(S->chk_last.alloc((size_t)S->n_items * (S->max_slots + 1) * 4));
  }
  if (!prec) {
    // FP64: the denominators 1/(1/tau + v G) of every (work item, position),
    // iteration-independent, so the sweep reads them instead of dividing
    // (+16 doubles: a chunk's 16-byte aligned copy may run one position past the last)
    NBTE_CK(S->dinv.alloc(((size_t)S->n_items * N * G + 16) * 8));
    NBTE_CK(cudaMemsetAsync(S->dinv.p, 0, S->dinv.bytes, S->stream));
    DBuf posG;
    NBTE_CK(upload(posG, S->plan.pos_G));
    NBTE_CK(launch_fill_dinv(S->dinv.as<double>(), posG.as<double>(), S->band_v.as<double>(),
                             S->band_itau.as<double>(), S->D, ng, G, N, S->stream));
    NBTE_CK(cudaStreamSynchronize(S->stream));
  } else {
    S->dinv.release();
  }
  if (order2) {
    // second-order upwind: the previous sweep's distribution (zero = no
    // reconstruction yet) and the per-position sources (+16 positions: a
    // chunk's 16-byte aligned copy may run past the last position)
    NBTE_CK(S->o2_e.alloc((size_t)S->n_items * N * G * sz));
    NBTE_CK(S->o2_src.alloc(((size_t)S->n_items * N + 16) * G * sz));
    NBTE_CK(cudaMemsetAsync(S->o2_e.p, 0, S->o2_e.bytes, S->stream));
    NBTE_CK(cudaMemsetAsync(S->o2_src.p, 0, S->o2_src.bytes, S->stream));
    // hexahedra: the gradients of as many directions as fit in the gradient
    // budget at once (two passes); other cells: one pass over all directions
    const bool two_pass = S->mesh->m.nfc == 6;
    const size_t grad_dir = (size_t)N * S->Bp * S->mesh->m.dim * sz;
    S->o2_db = two_pass ? (int)std::max<size_t>(1, std::min<size_t>((size_t)S->D, o2_grad_budget() / grad_dir))
                        : S->D;
    if (two_pass) NBTE_CK(S->o2_grad.alloc((size_t)S->o2_db * grad_dir));
    else S->o2_grad.release();
    if (S->rc_prec != prec || !S->rc_AnV.p) {
      Reconstruction rcn;
      build_reconstruction(S->mesh->m, rcn);
      NBTE_CK(upload(S->rc_nb, rcn.nb));
      NBTE_CK(upload(S->rc_twin, rcn.twin));
      if (prec) {
        NBTE_CK(upload(S->rc_AnV, to_float(rcn.AnV)));
        if (two_pass) {
          NBTE_CK(upload(S->rc_gw, to_float(rcn.gw)));
          NBTE_CK(upload(S->rc_rf, to_float(rcn.rf)));
        } else {
          NBTE_CK(upload(S->rc_a, to_float(rcn.a)));
        }
      } else {
        NBTE_CK(upload(S->rc_AnV, rcn.AnV));
        if (two_pass) {
          NBTE_CK(upload(S->rc_gw, rcn.gw));
          NBTE_CK(upload(S->rc_rf, rcn.rf));
        } else {
          NBTE_CK(upload(S->rc_a, rcn.a));
        }
      }
      S->rc_prec = prec;
      S->rc_cells = rcn.cells_with_gradient;
    }
  } else {
    S->o2_e.release();
    S->o2_src.release();
    S->o2_grad.release();
    S->o2_db = 0;
  }
  NBTE_CK(S->T.alloc(N * 8));
  NBTE_CK(S->Tprev.alloc(N * 8));
  NBTE_CK(S->Tkin.alloc(N * 8));
  NBTE_CK(S->Delta.alloc(N * 8));
  NBTE_CK(S->rhs.alloc(N * 8));
  NBTE_CK(S->delta.alloc(N * 8));
  NBTE_CK(S->Qd.alloc(N * 8));
  NBTE_CK(S->Vd.alloc(N * 8));
  NBTE_CK(S->dsum.alloc((size_t)S->n_dbf * Bp * 8));
  NBTE_CK(S->accE.alloc(N * 8));
  NBTE_CK(S->accQ.alloc((size_t)N * S->mesh->m.dim * 8));
  NBTE_CK(S->res.alloc(32));   // [0,1] residual words, [2] sweep error word (sticky)
  NBTE_CK(cudaMemsetAsync(S->res.p, 0, 32, S->stream));
  NBTE_CK(S->heat.alloc((size_t)S->n_wf * 8));
  NBTE_CK(cudaMemcpyAsync(S->Vd.p, S->mesh->m.V.data(), N * 8, cudaMemcpyHostToDevice, S->stream));
  NBTE_CK(cudaStreamSynchronize(S->stream));
  S->q_dev_version = -2;   // Qd was reallocated: upload the heat source again
  S->layout_key = key;
  S->have_state = false;
  return NBTE_OK;
}

// the caller's cell index of every internal cell, on the device
int ensure_perm(nbte_solver* S) {
  const int64_t N = S->mesh->m.n_cells;
  if (S->perm_d.p && S->perm_d.bytes == (size_t)N * 4) return NBTE_OK;
  std::vector<int32_t> p(N);
  for (int64_t c = 0; c < N; ++c) p[c] = (int32_t)S->mesh->m.perm[c];
  NBTE_CK(upload(S->perm_d, p));
  return NBTE_OK;
}

// device heat source (internal order) for the caller's last setting: the
// pinned caller-order copy goes up once and is reordered on the device
int ensure_q(nbte_solver* S) {
  const int64_t N = S->mesh->m.n_cells;
  if (S->q_dev_version == S->version_q && S->Qd.p) return NBTE_OK;
  if (!S->h_qc) {
    NBTE_CK(cudaMemsetAsync(S->Qd.p, 0, N * 8, S->stream));
  } else {
    int rc = ensure_perm(S);
    if (rc) return rc;
    NBTE_CK(S->io_d.alloc(std::max<size_t>(S->io_d.bytes, (size_t)N * 8 * S->mesh->m.dim)));
    NBTE_CK(cudaMemcpyAsync(S->io_d.p, S->h_qc, N * 8, cudaMemcpyHostToDevice, S->stream));
    NBTE_CK(launch_from_caller(S->Qd.as<double>(), S->io_d.as<double>(), S->perm_d.as<int32_t>(), (int)N,
                               S->stream));
  }
  S->q_dev_version = S->version_q;
  return NBTE_OK;
}

int ensure_laplacian(nbte_solver* S) {
  const int64_t want = S->version_bands * 1000003 + S->version_plan;
  if (S->lap_built == want && S->L_diag.p) return NBTE_OK;
  const Mesh& m = S->mesh->m;
  // kappa_bulk = sum C v^2 tau * (1/dim) sum_i w_i |s_i|^2 / W  (in-domain s)
  double ang = 0, mean_abs = 0, W = 0;
  for (int i = 0; i < S->D; ++i) {
    double s2 = 0, sa = 0;
    for (int d = 0; d < m.dim; ++d) { s2 += S->s[i * 3 + d] * S->s[i * 3 + d]; sa += std::fabs(S->s[i * 3 + d]); }
    ang += S->w[i] * s2;
    mean_abs += S->w[i] * sa;
    W += S->w[i];
  }
  ang /= (m.dim * W);
  mean_abs /= (m.dim * W);
  double kb = 0, cv = 0;
  for (int l = 0; l < S->B; ++l) { kb += S->C[l] * S->v[l] * S->v[l] * S->tau[l]; cv += S->C[l] * S->v[l]; }
  kb *= ang;
  const double k1 = 0.25 * mean_abs * cv;
  Laplacian L;
  build_laplacian(m, S->bcs, kb, k1, L);
  // Dirichlet data of the diffusion initial guess: sum over thermalizing
  // faces of g_f (T_wall - T_ref), per internal cell
  S->h_fourier_bc.resize(m.n_cells);
  for (int64_t c = 0; c < m.n_cells; ++c) S->h_fourier_bc[c] = L.bc_gT[c] - S->T_ref * L.bc_g[c];
  {
    DeviceGuard g0(S->device);
    NBTE_CK(upload(S->fbc, S->h_fourier_bc));
  }
  const int64_t N = m.n_cells;
  // ---- coarse space: geometric aggregates, rows reordered so each
  // aggregate's cells are contiguous, blocks owning whole aggregates
  std::vector<int32_t> agg;
  int target = N <= 4096 ? (int)std::max<int64_t>(1, N / 16)
                          : (int)std::min<int64_t>(N > 400000 ? 1536 : 1024, N / 32);
  int Nc = build_aggregates(m, target, agg);
  while (Nc > kMaxCoarse) {   // partly filled boxes can push the count over the target
    target = target * 3 / 4;
    Nc = build_aggregates(m, target, agg);
  }
  std::vector<int32_t> perm(N), iperm(N);
  for (int64_t c = 0; c < N; ++c) perm[c] = (int32_t)c;
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t x, int32_t y) { return agg[x] < agg[y]; });
  for (int64_t c = 0; c < N; ++c) iperm[perm[c]] = (int32_t)c;
  std::vector<int32_t> agg_p(N), agg_cell(Nc + 1, 0);
  for (int64_t c = 0; c < N; ++c) {
    agg_p[c] = agg[perm[c]];
    agg_cell[agg_p[c] + 1]++;
  }
  for (int k = 0; k < Nc; ++k) agg_cell[k + 1] += agg_cell[k];
  // ELL off-diagonals [k][row] (padding: own row, value 0) and the diagonal,
  // rows in aggregate order; Galerkin coarse operator Ac = P^T A P
  const int Wl = m.nfc;
  std::vector<int32_t> ecol((size_t)Wl * N);
  std::vector<double> eval((size_t)Wl * N, 0.0), diag(N), dinv(N);
  std::vector<double> Ac((size_t)Nc * Nc, 0.0);
  for (int64_t r = 0; r < N; ++r) {
    const int32_t c = perm[r];
    int k = 0;
    for (int32_t j = L.row_ptr[c]; j < L.row_ptr[c + 1]; ++j) {
      Ac[(size_t)agg[c] * Nc + agg[L.col[j]]] += L.val[j];
      if (L.col[j] == c) continue;
      ecol[(size_t)k * N + r] = iperm[L.col[j]];
      eval[(size_t)k * N + r] = L.val[j];
      ++k;
    }
    for (; k < Wl; ++k) ecol[(size_t)k * N + r] = (int32_t)r;
    diag[r] = L.diag[c];
    dinv[r] = 1.0 / L.diag[c];
  }
  if (!dense_spd_inverse(Ac, Nc))
    return fail(NBTE_ERR_ARG, "synthetic correction: coarse operator is not positive definite");
  const int Nc4 = (Nc + 3) / 4;
  DeviceGuard g(S->device);
  NBTE_CK(upload(S->L_ecol, ecol));
  NBTE_CK(upload(S->L_eval, eval));
  NBTE_CK(upload(S->L_diag, diag));
  NBTE_CK(upload(S->L_dinv, dinv));
  NBTE_CK(upload(S->cg_perm, perm));
  NBTE_CK(upload(S->cg_agg_cell, agg_cell));
  std::vector<float> Af((size_t)Nc * Nc4 * 4, 0.0f);
  for (int r = 0; r < Nc; ++r)
    for (int c = 0; c < Nc; ++c) Af[(size_t)r * Nc4 * 4 + c] = (float)Ac[(size_t)r * Nc + c];
  NBTE_CK(upload(S->cg_Ainv, Af));
  std::vector<double> Ad((size_t)Nc * Nc4 * 4, 0.0);
  for (int r = 0; r < Nc; ++r)
    for (int c = 0; c < Nc; ++c) Ad[(size_t)r * Nc4 * 4 + c] = Ac[(size_t)r * Nc + c];
  NBTE_CK(upload(S->cg_Ainv64, Ad));
  S->cg_Nc4 = Nc4;
  S->cg_W = Wl;
  S->cg_Nc = Nc;
  S->h_agg_cell = agg_cell;
  S->h_agg_p = agg_p;
  NBTE_CK(S->cg_x.alloc(N * 8));
  NBTE_CK(S->cg_u.alloc(N * 8));
  NBTE_CK(S->cg_rw.alloc((size_t)Nc * 8));
  NBTE_CK(S->cg_rcx.alloc((size_t)Nc * 8));
  NBTE_CK(S->cg_scx.alloc((size_t)Nc * 8));
  NBTE_CK(zero_now(S->cg_x.p, N * 8, S->stream));   // no previous correction yet
  NBTE_CK(S->cg_bar.alloc(16));
  NBTE_CK(S->cg_err.alloc(16));
  NBTE_CK(S->cg_it.alloc(16));
  NBTE_CK(S->cg_res.alloc(16));
  NBTE_CK(zero_now(S->cg_err.p, 16, S->stream));
  S->cg_part_key = -1;
  S->lap_built = want;
  drop_graph(S);
  return NBTE_OK;
}

// Blocks of the CG launch and what each owns: `grid` blocks, each a run of
// whole aggregates with about N/grid rows, and at least `threads_min`
// threads per block (a batched launch shares one block size).  Chooses which
// per-block arrays fit in shared memory for that block size.
int cg_partition(nbte_solver* S, int grid, int threads_min) {
  const int N = (int)S->mesh->m.n_cells;
  const int Nc = S->cg_Nc;
  grid = std::max(1, std::min(std::min(grid, 256), Nc));
  std::vector<int32_t> blk_cell(grid + 1, 0), blk_agg(grid + 1, 0);
  const std::vector<int32_t>& agg_cell = S->h_agg_cell;
  {
    int b = 0;
    for (int k = 0; k < Nc && b < grid; ++k) {
      // close block b once it reaches its share of cells, keeping one
      // aggregate for each block still to come
      const int64_t share = (int64_t)(b + 1) * N / grid;
      if (agg_cell[k + 1] >= share || Nc - (k + 1) <= grid - (b + 1)) {
        blk_agg[b + 1] = k + 1;
        ++b;
      }
    }
    blk_agg[grid] = Nc;
    for (int k = 0; k <= grid; ++k) blk_cell[k] = agg_cell[blk_agg[k]];
  }
  std::vector<int32_t> agg_rel(N);
  int max_rows = 1, max_na = 1;
  for (int k = 0; k < grid; ++k) {
    max_rows = std::max(max_rows, blk_cell[k + 1] - blk_cell[k]);
    max_na = std::max(max_na, blk_agg[k + 1] - blk_agg[k]);
    for (int32_t r = blk_cell[k]; r < blk_cell[k + 1]; ++r) agg_rel[r] = S->h_agg_p[r] - blk_agg[k];
  }
  // threads per block: enough for one pass over the largest block's rows
  const int threads = std::min(kCGThreads, std::max(std::max(128, threads_min), (max_rows + 31) / 32 * 32));
  const int64_t key = ((int64_t)grid << 20) + threads;
  if (key == S->cg_part_key) return NBTE_OK;
  // shared memory: own-row vectors first, then the ELL rows, as far as they
  // fit (sized for the FP64 coarse variant, the larger one)
  const size_t budget = (size_t)kSweepSmemMax - 2048;
  auto need = [&](int v, int e) {
    return cg_smem_layout(S->cg_Nc4, max_rows, max_na, S->cg_W, threads, v, e, 8).total;
  };
  const int vec = need(1, 0) <= budget;
  const int ell = vec && need(1, 1) <= budget;
  if (need(0, 0) > budget) return fail(NBTE_ERR_ARG, "synthetic correction: too many aggregates per block");
  DeviceGuard g(S->device);
  NBTE_CK(upload(S->cg_agg_rel, agg_rel));
  NBTE_CK(upload(S->cg_blk_cell, blk_cell));
  NBTE_CK(upload(S->cg_blk_agg, blk_agg));
  const size_t work = vec ? 16 : (size_t)N * 8;   // global work vectors only when not in shared memory
  NBTE_CK(S->cg_xw.alloc(work));
  NBTE_CK(S->cg_r.alloc(work));
  NBTE_CK(S->cg_p.alloc(work));
  NBTE_CK(S->cg_s.alloc(work));
  NBTE_CK(S->cg_w.alloc(work));
  NBTE_CK(S->cg_slots.alloc((size_t)grid * sizeof(CGSlot)));
  NBTE_CK(zero_now(S->cg_slots.p, S->cg_slots.bytes, S->stream));
  NBTE_CK(zero_now(S->cg_bar.p, 16, S->stream));   // arrivals must start at a multiple of the block count
  S->cg_max_rows = max_rows;
  S->cg_max_na = max_na;
  S->cg_smem_vec = vec;
  S->cg_smem_ell = ell;
  S->cg_grid = grid;
  S->cg_threads = threads;
  S->cg_part_key = key;
  drop_graph(S);
  return NBTE_OK;
}

// the partition a solver uses on its own: one block per SM
int cg_default_partition(nbte_solver* S) {
  int nsm = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, S->device);
  return cg_partition(S, nsm, 0);
}

size_t cg_smem_for(const nbte_solver* S, bool c32) {
  return cg_smem_layout(S->cg_Nc4, S->cg_max_rows, S->cg_max_na, S->cg_W, S->cg_threads, S->cg_smem_vec,
                        S->cg_smem_ell, c32 ? 4 : 8)
      .total;
}

// ------------------------------------------------------------------ iteration body
template <typename R>
SweepArgs<R> sweep_args(nbte_solver* S, int full) {
  SweepArgs<R> a{};
  a.N = (int)S->mesh->m.n_cells;
  a.dim = S->mesh->m.dim;
  a.full = full;
  a.Gpad = S->Gpad;
  a.n_stages = S->n_stages;
  a.stage_bytes = S->stage_bytes;
  a.off_ring = S->off_ring;
  a.off_stage = S->off_stage;
  a.off_imp = S->off_imp;
  a.off_den = S->off_den;
  a.off_src2 = S->off_src2;
  a.dinv = S->dinv.p ? S->dinv.as<R>() : nullptr;
  a.src2 = S->order == 2 ? S->o2_src.as<R>() : nullptr;
  a.e_out = S->order == 2 ? S->o2_e.as<R>() : nullptr;
  // second order keeps the distribution as [direction][cell][band]
  a.e_out_dstride = (int64_t)a.N * S->Bp;
  a.e_out_gstride = S->G;
  a.e_out_cstride = S->Bp;
  a.n_exp = S->n_exp;
  a.n_imp = S->n_imp;
  a.item_dir = S->item_dir.as<int32_t>();
  a.item_grp = S->item_grp.as<int32_t>();
  a.n_groups = S->n_groups;
  a.chunk_off = S->chunk_off.as<int64_t>();
  a.chunks = S->chunks.as<Chunk>();
  a.rec = S->rec.as<unsigned char>();
  a.chunk_doff = S->chunk_doff.as<int64_t>();
  a.exp_off = S->exp_off.as<int64_t>();
  a.imp_off = S->imp_off.as<int64_t>();
  a.imp = S->impt.as<R>();
  a.exp = S->expt.as<R>();
  a.err = reinterpret_cast<int32_t*>(S->res.as<unsigned long long>() + 2);
  a.band_v = S->band_v.as<R>();
  a.band_inv_tau = S->band_itau.as<R>();
  a.band_cw = S->band_aT.as<R>();
  a.band_aQ = S->band_aQ.as<R>();
  a.dir_w = S->dir_w.as<double>();
  a.dir_s = S->dir_s.as<double>();
  a.part = S->partials ? S->part.as<R>() : nullptr;
  a.acc = S->acc.as<double>();
  a.gring = S->gring.p ? S->gring.as<R>() : nullptr;
  a.gring_stride = S->gring_stride;
  a.accE = S->accE.as<double>();
  a.accQ = S->accQ.as<double>();
  a.hold_copies = test_timeouts() ? 1 : 0;
  a.ring_slots = S->max_slots + 1;
  if (kChecks) {
    a.chk_level = S->chk_level.as<int32_t>();
    a.chk_last = S->chk_last.as<int32_t>();
    a.pos_last = S->pos_last.as<int32_t>();
  }
  return a;
}

template <typename R>
WallArgs<R> wall_args(nbte_solver* S) {
  WallArgs<R> a{};
  a.Bp = S->Bp;
  a.G = S->G;
  a.Gpad = S->Gpad;
  a.n_exp = S->n_exp;
  a.n_imp = S->n_imp;
  a.n_dbf = S->n_dbf;
  a.exp = S->expt.as<R>();
  a.imp = S->impt.as<R>();
  a.exp_cell = S->exp_cell.as<int32_t>();
  a.Delta = S->Delta.as<double>();
  a.CoW = S->band_CoW.as<double>();
  a.imp_kind = S->imp_kind.as<int32_t>();
  a.imp_dbf = S->imp_dbf.as<int32_t>();
  a.imp_src = S->imp_src.as<int64_t>();
  a.imp_par = S->imp_par.as<double>();
  a.dif_ptr = S->dif_ptr.as<int64_t>();
  a.dif_src = S->dif_src.as<int64_t>();
  a.dif_wt = S->dif_wt.as<double>();
  a.dsum = S->dsum.as<double>();
  return a;
}

template <typename R>
UpdateArgs<R> update_args(nbte_solver* S, int mode) {
  UpdateArgs<R> a{};
  a.N = (int)S->mesh->m.n_cells;
  a.n_items = S->n_items;
  a.mode = mode;
  a.beta = S->beta;
  a.inv_beta = 1.0 / S->beta;
  a.part = S->partials ? S->part.as<R>() : nullptr;
  a.acc = S->acc.as<double>();
  a.Q = S->Qd.as<double>();
  a.V = S->Vd.as<double>();
  a.T = S->T.as<double>();
  a.Tprev = S->Tprev.as<double>();
  a.Tkin = S->Tkin.as<double>();
  a.Delta = S->Delta.as<double>();
  a.rhs = S->rhs.as<double>();
  a.delta = S->delta.as<double>();
  a.srcTQ_next = S->srcTQ.as<R>();
  a.res = S->res.as<unsigned long long>();
  return a;
}

CGArgs cg_args(nbte_solver* S, double tol, int max_it) {
  CGArgs a{};
  a.N = (int)S->mesh->m.n_cells;
  a.Nc = S->cg_Nc;
  a.W = S->cg_W;
  a.ell_col = S->L_ecol.as<int32_t>();
  a.ell_val = S->L_eval.as<double>();
  a.diag = S->L_diag.as<double>();
  a.dinv = S->L_dinv.as<double>();
  a.perm = S->cg_perm.as<int32_t>();
  a.agg_rel = S->cg_agg_rel.as<int32_t>();
  a.agg_cell = S->cg_agg_cell.as<int32_t>();
  a.blk_cell = S->cg_blk_cell.as<int32_t>();
  a.blk_agg = S->cg_blk_agg.as<int32_t>();
  a.Ainv32 = S->cg_Ainv.as<float>();
  a.Ainv64 = S->cg_Ainv64.as<double>();
  a.Nc4 = S->cg_Nc4;
  a.max_rows = S->cg_max_rows;
  a.max_na = S->cg_max_na;
  a.smem_vec = S->cg_smem_vec;
  a.smem_ell = S->cg_smem_ell;
  a.b = S->rhs.as<double>();
  a.x_out = S->delta.as<double>();
  a.x = S->cg_x.as<double>();
  a.u = S->cg_u.as<double>();
  a.x_work = S->cg_xw.as<double>();
  a.r = S->cg_r.as<double>();
  a.p = S->cg_p.as<double>();
  a.s = S->cg_s.as<double>();
  a.w = S->cg_w.as<double>();
  a.rw = S->cg_rw.p;
  a.rcx = S->cg_rcx.p;
  a.scx = S->cg_scx.p;
  a.slots = S->cg_slots.as<CGSlot>();
  a.bar = S->cg_bar.as<unsigned long long>();
  a.err = S->cg_err.as<int32_t>();
  a.spin_limit = wait_limit_or(kCgSpinPolls);
  a.tol = tol;
  a.max_it = max_it;
  a.it_out = S->cg_it.as<int32_t>();
  a.res_out = S->cg_res.as<double>();
  return a;
}

// One outer iteration, stream-ordered (capturable), in three parts around
// the sweep and the CG so that a batch can run every solver's parts and fuse
// the sweeps and the CGs.
//   pre:  wall coupling (Sec. II walls, lagged), T' kept for the residual,
//         (T', Qdot) gathered in level order;
//   mid:  residual words cleared, collision moment reduced (Eq. (5)) and
//         either applied (Eq. (6)) or turned into the synthetic rhs;
//   post: the synthetic update (Eq. (12)) and the residual words to the host.
template <typename R>
Src2Args<R> src2_args(nbte_solver* S) {
  Src2Args<R> a{};
  a.N = (int)S->mesh->m.n_cells;
  a.nfc = S->mesh->m.nfc;
  a.dim = S->mesh->m.dim;
  a.G = S->G;
  a.n_items = S->n_items;
  a.n_groups = S->n_groups;
  a.Bp = S->Bp;
  a.D = S->D;
  a.e = S->o2_e.as<R>();
  a.src2 = S->o2_src.as<R>();
  a.grad = S->o2_grad.as<R>();
  a.pos_cell = S->pos_cell.as<int32_t>();
  a.nb = S->rc_nb.as<int32_t>();
  a.twin = S->rc_twin.as<int32_t>();
  a.AnV = S->rc_AnV.as<R>();
  a.rc_a = S->rc_a.as<R>();
  a.gw = S->rc_gw.as<R>();
  a.rf = S->rc_rf.as<R>();
  a.dir_s = S->dir_s.as<double>();
  return a;
}

template <typename R>
cudaError_t enqueue_pre(nbte_solver* S, cudaStream_t st) {
  launch_walls<R>(wall_args<R>(S), st);
  // the gather also clears the residual words of this iteration's update
  cudaError_t e = launch_gather_tq<R>(S->rec.as<unsigned char>(), S->tq_dst.as<int2>(), S->srcTQ.as<R>(),
                                      (int64_t)S->D * S->mesh->m.n_cells, S->res.as<unsigned long long>(), st);
  if (e != cudaSuccess) return e;
  // second order: this sweep's reconstruction sources from the previous
  // sweep's distribution, one batch of directions at a time
  if (S->order == 2) {
    Src2Args<R> a = src2_args<R>(S);
    for (int d0 = 0; d0 < S->D && e == cudaSuccess; d0 += S->o2_db) {
      a.dir0 = d0;
      a.n_dirs = std::min(S->o2_db, S->D - d0);
      e = launch_src2<R>(a, st);
    }
  }
  return e;
}

template <typename R>
cudaError_t enqueue_mid(nbte_solver* S, int scheme, cudaStream_t st) {
  launch_update<R>(update_args<R>(S, scheme == 0 ? 0 : 3), st);
  return cudaGetLastError();
}

template <typename R>
cudaError_t enqueue_post(nbte_solver* S, int scheme, cudaStream_t st) {
  if (scheme != 0) launch_update<R>(update_args<R>(S, scheme == 1 ? 1 : 2), st);
  cudaError_t e = cudaMemcpyAsync(S->h_res, S->res.p, 24, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  // the CG's error word (synthetic schemes only)
  if (scheme != 0 && S->cg_err.p) e = cudaMemcpyAsync(S->h_misc, S->cg_err.p, 4, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// an FP32 coarse preconditioner suffices unless the correction is wanted to
// near FP64 rounding
inline bool coarse32(double cg_tol) { return cg_tol >= 1e-7; }

template <typename R>
cudaError_t enqueue_iteration(nbte_solver* S, int scheme, double cg_tol, int cg_max, cudaEvent_t ev0 = nullptr,
                              cudaEvent_t ev1 = nullptr) {
  cudaStream_t st = S->stream;
  cudaError_t e = enqueue_pre<R>(S, st);
  if (e != cudaSuccess) return e;
  if (ev0) cudaEventRecord(ev0, st);
  e = launch_sweep<R>(sweep_args<R>(S, 0), S->K, S->G, S->n_items, S->threads, S->smem, st);
  if (e != cudaSuccess) return e;
  if (ev1) cudaEventRecord(ev1, st);
  e = enqueue_mid<R>(S, scheme, st);
  if (e != cudaSuccess) return e;
  if (scheme != 0) {
    const bool c32 = coarse32(cg_tol);
    e = launch_cg(cg_args(S, cg_tol, cg_max), c32, S->cg_grid, S->cg_threads, cg_smem_for(S, c32), st);
    if (e != cudaSuccess) return e;
  }
  return enqueue_post<R>(S, scheme, st);
}

// T' from T_init (or T_ref), wall distributions at equilibrium with it, no
// synthetic correction carried yet
template <typename R>
int init_state(nbte_solver* S, const nbte_solve_opts& o) {
  const Mesh& m = S->mesh->m;
  const int64_t N = m.n_cells;
  cudaStream_t st = S->stream;
  std::vector<double> T0(N, 0.0);
  if (o.T_init) {
    for (int64_t c = 0; c < N; ++c) {
      const double t = o.T_init[m.perm[c]];
      if (!std::isfinite(t)) return fail(NBTE_ERR_ARG, "non-finite T_init");
      T0[c] = t - S->T_ref;
    }
  }
  NBTE_CK(cudaMemcpyAsync(S->T.p, T0.data(), N * 8, cudaMemcpyHostToDevice, st));
  if (o.init == 1) {
    // diffusion initial guess: L T' = Qdot V + sum_thermalizing g_f T'_w,
    // the synthetic correction's operator with the wall temperatures as
    // Dirichlet data, solved with the same CG to FP64 accuracy
    NBTE_CK(launch_fourier_rhs(S->rhs.as<double>(), S->Qd.as<double>(), S->Vd.as<double>(), S->fbc.as<double>(), N,
                               st));
    NBTE_CK(cudaMemsetAsync(S->cg_x.p, 0, N * 8, st));
    NBTE_CK(cudaMemsetAsync(S->cg_err.p, 0, 4, st));
    NBTE_CK(launch_cg(cg_args(S, 1e-12, 20000), false, S->cg_grid, S->cg_threads, cg_smem_for(S, false), st));
    NBTE_CK(cudaMemcpyAsync(S->T.p, S->delta.p, N * 8, cudaMemcpyDeviceToDevice, st));
    NBTE_CK(cudaMemsetAsync(S->cg_x.p, 0, N * 8, st));   // later corrections start from zero
    int32_t err = 0;
    NBTE_CK(cudaMemcpyAsync(&err, S->cg_err.p, 4, cudaMemcpyDeviceToHost, st));
    NBTE_CK(cudaStreamSynchronize(st));
    if (err != 0) {
      zero_now(S->cg_err.p, 16, S->stream);
      zero_now(S->cg_slots.p, S->cg_slots.bytes, S->stream);
      zero_now(S->cg_bar.p, 16, S->stream);
      return fail(NBTE_ERR_DEVICE_TIMEOUT, "a bounded device wait in the initial diffusion solve gave up");
    }
  }
  NBTE_CK(cudaMemsetAsync(S->Delta.p, 0, N * 8, st));
  NBTE_CK(cudaMemsetAsync(S->Tkin.p, 0, N * 8, st));
  if (S->order == 2) NBTE_CK(cudaMemsetAsync(S->o2_e.p, 0, S->o2_e.bytes, st));   // no reconstruction in sweep 1
  launch_fill_srcTQ<R>(S->srcTQ.as<R>(), S->T.as<double>(), S->Qd.as<double>(), (int)N, st);
  launch_init_exports<R>(S->expt.as<R>(), S->exp_cell.as<int32_t>(), S->T.as<double>(), S->band_CoW.as<double>(),
                         S->Bp, S->G, S->Gpad, S->n_exp, st);
  NBTE_CK(cudaGetLastError());
  NBTE_CK(cudaStreamSynchronize(st));
  return NBTE_OK;
}

// device time of one sweep of the current layout, on a scratch state
template <typename R>
int time_sweep(nbte_solver* S, const nbte_solve_opts& o, float* ms) {
  int rc = init_state<R>(S, o);
  if (rc) return rc;
  cudaStream_t st = S->stream;
  launch_walls<R>(wall_args<R>(S), st);
  NBTE_CK(launch_gather_tq<R>(S->rec.as<unsigned char>(), S->tq_dst.as<int2>(), S->srcTQ.as<R>(),
                              (int64_t)S->D * S->mesh->m.n_cells, nullptr, st));
  NBTE_CK(launch_sweep<R>(sweep_args<R>(S, 0), S->K, S->G, S->n_items, S->threads, S->smem, st));
  cudaEvent_t e0, e1;
  NBTE_CK(cudaEventCreate(&e0));
  NBTE_CK(cudaEventCreate(&e1));
  NBTE_CK(cudaEventRecord(e0, st));
  for (int k = 0; k < 2; ++k)
    NBTE_CK(launch_sweep<R>(sweep_args<R>(S, 0), S->K, S->G, S->n_items, S->threads, S->smem, st));
  NBTE_CK(cudaEventRecord(e1, st));
  NBTE_CK(cudaEventSynchronize(e1));
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  unsigned long long err = 0;
  NBTE_CK(cudaMemcpy(&err, S->res.as<unsigned long long>() + 2, 8, cudaMemcpyDeviceToHost));
  if (err) {
    zero_now(S->res.p, 32, S->stream);
    return sweep_error(err);
  }
  *ms = t / 2;
  return NBTE_OK;
}

// Autotuner: with band_group and cta_threads left at 0, time every feasible
// (band group, chunk length) layout once per (mesh plan, band table,
// precision) -- chunk lengths 64, 128, 256, 512, then a few multiples of 32
// around the best -- and keep the fastest.
int autotune(nbte_solver* S, const nbte_solve_opts& o) {
  if (o.band_group != 0 || o.cta_threads != 0 || o.ring != 0) return NBTE_OK;
  Tuned& tu = S->tuned[o.precision];
  if (tu.valid && tu.key == tune_key(S)) return NBTE_OK;
  tu.valid = false;
  const int maxG = o.precision ? 8 : 4;
  std::vector<int> Gs;
  for (int c : {8, 4, 2, 1}) {
    if (c > maxG) continue;
    const int ng = (S->B + c - 1) / c;
    if (c > 1 && (double)(ng * c - S->B) / S->B > 0.25) continue;   // too much padding
    Gs.push_back(c);
  }
  double best = 1e300;
  int bG = 0, bcap = 0;
  auto try_layout = [&](int G, int cap) -> int {
    nbte_solve_opts c = o;
    c.band_group = G;
    c.cta_threads = cap + 32;
    c.warm = 0;
    c.init = 0;
    if (ensure_layout(S, c) != NBTE_OK) return NBTE_OK;   // does not fit this mesh
    int rc = ensure_q(S);
    if (rc) return rc;
    float ms = 0.f;
    rc = o.precision ? time_sweep<float>(S, c, &ms) : time_sweep<double>(S, c, &ms);
    if (rc) return rc;
    if (ms < best) {
      best = ms;
      bG = G;
      bcap = cap;
    }
    return NBTE_OK;
  };
  // coarse: powers of two; then chunk lengths around the best, in steps of a warp
  for (int G : Gs)
    for (int cap : {64, 128, 256, 512}) {
      const int rc = try_layout(G, cap);
      if (rc) return rc;
    }
  if (bG != 0) {
    const int G = bG, c0 = bcap;
    for (int cap : {c0 - 32, c0 + 32, c0 + 64, c0 + c0 / 2}) {
      if (cap < 64 || cap > 512 || cap % 32 != 0 || cap == c0 || cap == 2 * c0) continue;
      const int rc = try_layout(G, cap);
      if (rc) return rc;
    }
  }
  if (bG == 0) return fail(NBTE_ERR_ARG, "no sweep layout fits shared memory for this mesh");
  tu.valid = true;
  tu.G = bG;
  tu.cap = bcap;
  tu.key = tune_key(S);
  tu.ms = best;
  S->layout_key.clear();
  S->have_state = false;
  set_error("");
  return NBTE_OK;
}

// One solve in progress: its options, iteration count and stopping state.
struct Run {
  nbte_solver* S = nullptr;
  nbte_solve_opts o{};
  double cg_tol = 1e-2;
  int cg_max = 5000;
  bool fixed = false;
  int limit = 0;
  int it = 0;                  // iterations enqueued
  double r = INFINITY;
  int status = NBTE_OK;
  IterationMonitor mon;        // stopping rule (iteration_monitor.h)
  int64_t kernels = 0;
  double sweep_ms = 0.0;
  int64_t sweeps_timed = 0;
  std::chrono::steady_clock::time_point t0, t1;

  int64_t kernels_per_iter() const {
    return (S->n_dbf > 0) + (S->n_imp > 0) + 2 + (o.scheme == 0 ? 1 : 3) +
           (S->order == 2 ? (S->mesh->m.nfc == 6 ? 2 : 1) * ((S->D + S->o2_db - 1) / S->o2_db) : 0);
  }
  // after an iteration's residual words reached the host: true to stop
  bool check() {
    // a wait that gave up leaves this iteration's fields incomplete: the
    // next solve starts from its initial state again (not warm)
    if (S->h_res[2] != 0) {
      status = sweep_error(S->h_res[2]);
      zero_now(S->res.p, 32, S->stream);
      S->have_state = false;
      return true;
    }
    if (S->h_misc[0] != 0 && o.scheme != 0) {
      status = fail(NBTE_ERR_DEVICE_TIMEOUT, "a bounded device wait in the CG correction gave up");
      zero_now(S->cg_err.p, 16, S->stream);
      zero_now(S->cg_slots.p, S->cg_slots.bytes, S->stream);
      zero_now(S->cg_bar.p, 16, S->stream);
      S->have_state = false;
      return true;
    }
    double dmax, tmax;
    std::memcpy(&dmax, &S->h_res[0], 8);
    std::memcpy(&tmax, &S->h_res[1], 8);
    mon.it = it - 1;   // the words are those of iteration `it`
    const IterationMonitor::Verdict v = mon.step(dmax, tmax);
    r = mon.r;
    if (v == IterationMonitor::DIVERGED) {
      status = fail(NBTE_ERR_DIVERGED, std::isfinite(r) ? "the temperature increment grew without bound: the iteration diverged"
                                                          : "non-finite temperature: the iteration diverged");
      S->have_state = false;
      return true;
    }
    return v != IterationMonitor::CONTINUE;
  }
  // the solve stopped where its options say it should (tolerance or floor
  // reached, or the fixed iteration count done)
  bool finished_ok() const {
    return fixed || mon.last == IterationMonitor::CONVERGED || mon.last == IterationMonitor::FLOOR;
  }
};

template <typename R>
int run_begin(Run& run, nbte_solver* S, const nbte_solve_opts& o) {
  run.S = S;
  run.o = o;
  run.cg_tol = o.cg_tol > 0 ? o.cg_tol : 1e-2;
  run.cg_max = o.cg_max_iter > 0 ? o.cg_max_iter : 5000;
  run.fixed = o.n_iter > 0;
  run.limit = run.fixed ? o.n_iter : o.max_iter;
  run.mon = IterationMonitor{};
  run.mon.tol = o.tol;
  run.mon.limit = run.limit;
  run.mon.fixed = run.fixed;
  run.mon.fp32 = S->prec != 0;
  cudaStream_t st = S->stream;
  if (!(o.warm && S->have_state)) {
    run.kernels += 2;
    int rc = init_state<R>(S, o);
    if (rc) return rc;
    S->have_state = true;
  } else {
    run.kernels += 1;
    launch_fill_srcTQ<R>(S->srcTQ.as<R>(), S->T.as<double>(), S->Qd.as<double>(), (int)S->mesh->m.n_cells, st);
  }
  if (S->cg_it.p) NBTE_CK(cudaMemsetAsync(S->cg_it.p, 0, 4, st));
  // the sweeps add into the collision-moment sums and the update clears them;
  // a timing sweep or a sweep that gave up leaves them dirty
  NBTE_CK(cudaMemsetAsync(S->acc.p, 0, (size_t)S->mesh->m.n_cells * 8, st));
  run.t0 = std::chrono::steady_clock::now();
  return NBTE_OK;
}

// results of a finished run: the last sweep replayed with the energy and
// flux moments on (unless skipped), the energy balance, the info record
template <typename R>
int run_finish(Run& run, nbte_solve_info* info) {
  nbte_solver* S = run.S;
  const nbte_solve_opts& o = run.o;
  const Mesh& m = S->mesh->m;
  const int64_t N = m.n_cells;
  cudaStream_t st = S->stream;
  run.t1 = std::chrono::steady_clock::now();
  int status = run.status;
  if (status == NBTE_OK && !run.finished_ok()) status = NBTE_ERR_NOT_CONVERGED;
  S->have_results = status == NBTE_OK || status == NBTE_ERR_NOT_CONVERGED;
  S->have_outputs = false;
  if ((status == NBTE_OK || status == NBTE_ERR_NOT_CONVERGED) && !o.skip_outputs) {
    run.kernels += 5;
    NBTE_CK(cudaMemsetAsync(S->accE.p, 0, N * 8, st));
    NBTE_CK(cudaMemsetAsync(S->accQ.p, 0, (size_t)N * m.dim * 8, st));
    launch_fill_srcTQ<R>(S->srcTQ_fin.as<R>(), S->Tprev.as<double>(), S->Qd.as<double>(), (int)N, st);
    NBTE_CK(launch_gather_tq<R>(S->rec.as<unsigned char>(), S->tq_dst.as<int2>(), S->srcTQ_fin.as<R>(), (int64_t)S->D * N,
                                nullptr, st));
    NBTE_CK(launch_sweep<R>(sweep_args<R>(S, 1), S->K, S->G, S->n_items, S->threads, S->smem, st));
    WallHeatArgs<R> wh{};
    wh.Bp = S->Bp;
    wh.G = S->G;
    wh.Gpad = S->Gpad;
    wh.n_exp = S->n_exp;
    wh.n_imp = S->n_imp;
    wh.n_wf = S->n_wf;
    wh.wf_ptr = S->wf_ptr.as<int64_t>();
    wh.wf_val = S->wf_val.as<int64_t>();
    wh.wf_coef = S->wf_coef.as<double>();
    wh.exp = S->expt.as<R>();
    wh.imp = S->impt.as<R>();
    wh.band_v = S->band_v64.as<double>();
    wh.heat = S->heat.as<double>();
    launch_wall_heat<R>(wh, st);
    NBTE_CK(cudaGetLastError());
    // wall heat per tag and the energy balance (FP64, on the device)
    const int n_tags = (int)S->tag_list.size();
    NBTE_CK(launch_wall_balance(S->heat.as<double>(), S->wf_tagidx.as<int32_t>(), S->tag_therm.as<int32_t>(), n_tags,
                                S->n_wf, S->Qd.as<double>(), S->Vd.as<double>(), N, S->balance.as<double>(), st));
    std::vector<double> bal(3 + n_tags, 0.0);
    NBTE_CK(cudaMemcpyAsync(bal.data(), S->balance.p, bal.size() * 8, cudaMemcpyDeviceToHost, st));
    NBTE_CK(cudaStreamSynchronize(st));
    S->have_outputs = true;
    S->last_energy_imbalance = bal[0];
    S->wall_heat_by_tag.assign(bal.begin() + 3, bal.end());
  }
  if (info) {
    info->iterations = run.it;
    info->residual = run.r;
    info->energy_imbalance = S->last_energy_imbalance;
    info->lagged_faces = S->lagged;
    info->seconds = std::chrono::duration<double>(run.t1 - run.t0).count();
    int32_t cgi = 0;
    if (S->cg_it.p && o.scheme != 0) cudaMemcpy(&cgi, S->cg_it.p, 4, cudaMemcpyDeviceToHost);
    info->cg_iterations = cgi;
    info->sweep_seconds = run.sweep_ms * 1e-3;
    info->sweep_launches = run.sweeps_timed;
    info->kernel_launches = run.kernels;
    info->status = status;
  }
  return status;
}

template <typename R>
int run_solve(nbte_solver* S, const nbte_solve_opts& o, nbte_solve_info* info) {
  Run run;
  int rc = run_begin<R>(run, S, o);
  if (rc) return rc;
  cudaStream_t st = S->stream;
  const int scheme = o.scheme;
  // ---- graph
  bool use_graph = o.use_graph != 0;
  const std::string gkey = S->layout_key + "/" + std::to_string(scheme) + "/" + std::to_string(run.cg_tol) + "/" +
                           std::to_string(run.cg_max) + "/" + std::to_string(S->lap_built) + "/" +
                           std::to_string(S->cg_part_key) + "/" + std::to_string((long long)(intptr_t)st) + "/" +
                           std::to_string(test_timeouts() ? 1 : 0);
  if (use_graph && (S->graph == nullptr || S->graph_key != gkey)) {
    drop_graph(S);
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t e = enqueue_iteration<R>(S, scheme, run.cg_tol, run.cg_max);
      cudaError_t e2 = cudaStreamEndCapture(st, &gr);
      if (e == cudaSuccess && e2 == cudaSuccess && gr &&
          cudaGraphInstantiate(&S->graph, gr, 0) == cudaSuccess) {
        S->graph_key = gkey;
      } else {
        S->graph = nullptr;
        use_graph = false;
      }
      if (gr) cudaGraphDestroy(gr);
    } else {
      use_graph = false;
    }
    cudaGetLastError();   // clear a failed capture
  }
  // ---- iterate
  const bool profile = o.profile != 0;
  if (profile) use_graph = false;   // events bracket each sweep launch
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (profile) {
    NBTE_CK(cudaEventCreate(&ev0));
    NBTE_CK(cudaEventCreate(&ev1));
  }
  // with a fixed iteration count the host only looks at the device once
  const bool check_each = !run.fixed || profile;
  while (run.it < run.limit) {
    if (use_graph) NBTE_CK(cudaGraphLaunch(S->graph, st));
    else NBTE_CK(enqueue_iteration<R>(S, scheme, run.cg_tol, run.cg_max, ev0, ev1));
    run.kernels += run.kernels_per_iter();
    ++run.it;
    if (!check_each) continue;
    NBTE_CK(cudaStreamSynchronize(st));
    if (profile) {
      float ms = 0.f;
      NBTE_CK(cudaEventElapsedTime(&ms, ev0, ev1));
      run.sweep_ms += ms;
      ++run.sweeps_timed;
    }
    if (run.check()) break;
  }
  if (!check_each) {
    NBTE_CK(cudaStreamSynchronize(st));
    run.check();
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  return run_finish<R>(run, info);
}

// ------------------------------------------------------------------ batches
// Device tables of one batch composition (the still-active solvers): for each
// sweep variant the solvers' SweepArgs and item prefix sums, and for the CG
// every synthetic solver's CGArgs and block prefix sums.
template <typename R>
struct BatchTables {
  struct SweepGroup {
    int K = 0, G = 0, threads = 0, items = 0;
    bool gr = false;
    bool o2 = false;
    size_t smem = 0;
    std::vector<int> members;
    DBuf args, start;
  };
  std::deque<SweepGroup> groups;   // deque: the device buffers never move
  std::vector<int> cg_members;
  DBuf cg_args_d, cg_start_d;
  int cg_blocks = 0, cg_threads = 0;
  size_t cg_smem = 0;
  cudaGraphExec_t graph = nullptr;
  ~BatchTables() {
    if (graph) cudaGraphExecDestroy(graph);
  }
};

template <typename R>
int batch_build(BatchTables<R>& bt, const std::vector<Run*>& act) {
  bt.groups.clear();
  for (int k = 0; k < (int)act.size(); ++k) {
    nbte_solver* S = act[k]->S;
    const bool gr = S->gring_stride > 0;
    const bool o2 = S->order == 2;
    typename BatchTables<R>::SweepGroup* grp = nullptr;
    for (auto& g : bt.groups)
      if (g.K == S->K && g.G == S->G && g.gr == gr && g.o2 == o2) grp = &g;
    if (!grp) {
      bt.groups.emplace_back();
      grp = &bt.groups.back();
      grp->K = S->K;
      grp->G = S->G;
      grp->gr = gr;
      grp->o2 = o2;
    }
    grp->members.push_back(k);
  }
  for (auto& g : bt.groups) {
    std::vector<SweepArgs<R>> args;
    std::vector<int32_t> start(1, 0);
    for (int k : g.members) {
      nbte_solver* S = act[k]->S;
      args.push_back(sweep_args<R>(S, 0));
      start.push_back(start.back() + S->n_items);
      g.threads = std::max(g.threads, S->threads);
      g.smem = std::max(g.smem, S->smem);
    }
    g.items = start.back();
    NBTE_CK(g.args.alloc(args.size() * sizeof(SweepArgs<R>)));
    NBTE_CK(cudaMemcpy(g.args.p, args.data(), args.size() * sizeof(SweepArgs<R>), cudaMemcpyHostToDevice));
    NBTE_CK(cudaStreamSynchronize(cudaStreamLegacy));
    NBTE_CK(upload(g.start, start));
  }
  // CG: every synthetic solver gets blocks in proportion to its cells (at
  // least one); one block per SM in all
  bt.cg_members.clear();
  bt.cg_blocks = 0;
  for (int k = 0; k < (int)act.size(); ++k)
    if (act[k]->o.scheme != 0) bt.cg_members.push_back(k);
  if (!bt.cg_members.empty()) {
    nbte_solver* S0 = act[bt.cg_members[0]]->S;
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, S0->device);
    const int n = (int)bt.cg_members.size();
    if (n > nsm) return fail(NBTE_ERR_ARG, "more synthetic solvers in one batch than SMs");
    double tot = 0;
    for (int k : bt.cg_members) tot += (double)act[k]->S->mesh->m.n_cells;
    std::vector<int> share(n);
    int used = 0;
    for (int j = 0; j < n; ++j) {
      nbte_solver* S = act[bt.cg_members[j]]->S;
      share[j] = std::max(1, (int)std::floor((nsm - n) * (double)S->mesh->m.n_cells / tot) + 1);
      share[j] = std::min(share[j], S->cg_Nc);
      used += share[j];
    }
    while (used > nsm) {   // rounding can overshoot by a few: trim the largest
      int jm = (int)(std::max_element(share.begin(), share.end()) - share.begin());
      --share[jm];
      --used;
    }
    int T = 0;
    for (int j = 0; j < n; ++j) {
      int rc = cg_partition(act[bt.cg_members[j]]->S, share[j], 0);
      if (rc) return rc;
      T = std::max(T, act[bt.cg_members[j]]->S->cg_threads);
    }
    std::vector<CGArgs> args;
    std::vector<int32_t> start(1, 0);
    bt.cg_smem = 0;
    const bool c32 = coarse32(act[bt.cg_members[0]]->cg_tol);
    for (int j = 0; j < n; ++j) {
      Run& run = *act[bt.cg_members[j]];
      int rc = cg_partition(run.S, share[j], T);
      if (rc) return rc;
      args.push_back(cg_args(run.S, run.cg_tol, run.cg_max));
      start.push_back(start.back() + run.S->cg_grid);
      bt.cg_smem = std::max(bt.cg_smem, cg_smem_for(run.S, c32));
    }
    bt.cg_blocks = start.back();
    bt.cg_threads = T;
    NBTE_CK(bt.cg_args_d.alloc(args.size() * sizeof(CGArgs)));
    NBTE_CK(cudaMemcpy(bt.cg_args_d.p, args.data(), args.size() * sizeof(CGArgs), cudaMemcpyHostToDevice));
    NBTE_CK(cudaStreamSynchronize(cudaStreamLegacy));
    NBTE_CK(upload(bt.cg_start_d, start));
  }
  if (bt.graph) {
    cudaGraphExecDestroy(bt.graph);
    bt.graph = nullptr;
  }
  return NBTE_OK;
}

template <typename R>
cudaError_t batch_enqueue(BatchTables<R>& bt, const std::vector<Run*>& act, cudaStream_t st) {
  const int scheme = act[0]->o.scheme;
  cudaError_t e;
  for (Run* run : act)
    if ((e = enqueue_pre<R>(run->S, st)) != cudaSuccess) return e;
  for (auto& g : bt.groups) {
    e = launch_sweep_batch<R>(g.args.template as<SweepArgs<R>>(), g.start.template as<int32_t>(), (int)g.members.size(), g.K, g.G,
                              g.gr, g.o2, g.items, g.threads, g.smem, st);
    if (e != cudaSuccess) return e;
  }
  for (Run* run : act)
    if ((e = enqueue_mid<R>(run->S, scheme, st)) != cudaSuccess) return e;
  if (!bt.cg_members.empty()) {
    e = launch_cg_batch(bt.cg_args_d.template as<CGArgs>(), bt.cg_start_d.template as<int32_t>(),
                        (int)bt.cg_members.size(), coarse32(act[bt.cg_members[0]]->cg_tol), bt.cg_blocks,
                        bt.cg_threads, bt.cg_smem, st);
    if (e != cudaSuccess) return e;
  }
  for (Run* run : act)
    if ((e = enqueue_post<R>(run->S, scheme, st)) != cudaSuccess) return e;
  return cudaSuccess;
}

// capture one batched iteration of the active set into bt.graph (left null
// if capture fails; the caller then enqueues directly)
template <typename R>
void batch_capture(BatchTables<R>& bt, const std::vector<Run*>& act, cudaStream_t st) {
  cudaGraph_t gr = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    cudaError_t e = batch_enqueue<R>(bt, act, st);
    cudaError_t e2 = cudaStreamEndCapture(st, &gr);
    if (!(e == cudaSuccess && e2 == cudaSuccess && gr && cudaGraphInstantiate(&bt.graph, gr, 0) == cudaSuccess))
      bt.graph = nullptr;
    if (gr) cudaGraphDestroy(gr);
  }
  cudaGetLastError();   // clear a failed capture
}

// Several solvers iterated together until each stops (see nbte_solve_batch).
template <typename R>
int run_batch(const std::vector<nbte_solver*>& Ss, const nbte_solve_opts& o, nbte_solve_info* infos) {
  const int n = (int)Ss.size();
  cudaStream_t st = Ss[0]->stream;
  std::vector<Run> runs(n);
  for (int k = 0; k < n; ++k) {
    int rc = run_begin<R>(runs[k], Ss[k], o);
    if (rc) return rc;
    NBTE_CK(cudaStreamSynchronize(Ss[k]->stream));
  }
  std::vector<Run*> active(n);
  for (int k = 0; k < n; ++k) active[k] = &runs[k];
  BatchTables<R> bt;
  bool rebuild = true;
  while (!active.empty()) {
    if (rebuild) {
      int rc = batch_build<R>(bt, active);
      if (rc) return rc;
      rebuild = false;
      if (o.use_graph) batch_capture<R>(bt, active, st);
    }
    if (bt.graph) NBTE_CK(cudaGraphLaunch(bt.graph, st));
    else NBTE_CK(batch_enqueue<R>(bt, active, st));
    NBTE_CK(cudaStreamSynchronize(st));
    std::vector<Run*> still;
    for (Run* run : active) {
      ++run->it;
      run->kernels += run->kernels_per_iter();
      if (run->check()) rebuild = true;
      else still.push_back(run);
    }
    active.swap(still);
  }
  int status = NBTE_OK;
  for (int k = 0; k < n; ++k) {
    const int rc = run_finish<R>(runs[k], infos ? infos + k : nullptr);
    if (rc != NBTE_OK && status == NBTE_OK) status = rc;
  }
  return status;
}

// the solver's device (the caller's current one), stream and pinned words
int ensure_device(nbte_solver* S) {
  if (S->device < 0) {
    NBTE_CK(cudaGetDevice(&S->device));
  }
  if (!S->own_stream) {
    DeviceGuard g(S->device);
    NBTE_CK(cudaStreamCreateWithFlags(&S->own_stream, cudaStreamNonBlocking));
    if (!S->stream) S->stream = S->own_stream;
    NBTE_CK(cudaMallocHost(&S->h_res, 32));
    NBTE_CK(cudaMallocHost(&S->h_misc, 16));
    S->h_misc[0] = 0;
  }
  return NBTE_OK;
}

// Device memory of the synthetic correction (estimate, before its setup).
size_t estimate_cg_bytes(const nbte_solver* S) {
  const size_t N = (size_t)S->mesh->m.n_cells, W = (size_t)S->mesh->m.nfc;
  const size_t Nc = std::min<size_t>(kMaxCoarse, std::max<size_t>(1, N <= 4096 ? N / 16 : std::min<size_t>(1536, N / 32)));
  const size_t Nc4 = (Nc + 3) / 4 * 4;
  return N * (W * 12 + 8 * 8 + 3 * 4) + Nc * Nc4 * 12 + Nc * 48;
}

// After a served solve: keep what the result getters read (T, the kinetic
// temperature, energy/flux moments, wall heat) and free everything the
// iteration held, so finished requests do not occupy the server's budget.
void shrink(nbte_solver* S) {
  DeviceGuard g(S->device);
  drop_graph(S);
  DBuf* big[] = {&S->rec_pos, &S->rec, &S->pos_cell, &S->gring, &S->e_scratch, &S->chunks, &S->chunk_off,
                 &S->chunk_doff, &S->chunk_dir, &S->chunk_sub_ptr, &S->chunk_sub_end, &S->tq_dst,
                 &S->expt, &S->impt, &S->srcTQ, &S->srcTQ_fin, &S->part, &S->acc, &S->Tprev, &S->Delta, &S->rhs,
                 &S->delta, &S->dsum, &S->cg_r, &S->cg_u, &S->cg_p, &S->cg_s, &S->cg_w, &S->cg_x, &S->cg_xw,
                 &S->cg_rw, &S->cg_rcx, &S->cg_scx, &S->cg_Ainv, &S->cg_Ainv64, &S->L_ecol, &S->L_eval,
                 &S->L_diag, &S->L_dinv, &S->cg_perm, &S->cg_agg_rel, &S->cg_agg_cell, &S->cg_blk_cell,
                 &S->cg_blk_agg, &S->cg_slots, &S->dinv, &S->o2_e, &S->o2_src, &S->o2_grad, &S->rc_nb,
                 &S->rc_twin, &S->rc_AnV, &S->rc_a, &S->rc_gw, &S->rc_rf, &S->pos_last, &S->chk_level,
                 &S->chk_last, &S->fbc};
  for (DBuf* b : big) b->release();
  S->rc_prec = -1;
  S->layout_key.clear();
  S->rec_key.clear();
  S->chunk_key.clear();
  S->blk_key.clear();
  S->lap_built = -1;
  S->cg_part_key = -1;
  S->have_state = false;
}

}  // namespace

// ------------------------------------------------------------------ serving
// A request queue in front of the batched iteration.  Submitted solves are
// planned on host threads, admitted to the device while their estimated
// memory fits the budget, and iterated together with every other admitted
// solve; arrivals join and converged solves leave between iterations.
struct ServedSolve {
  int64_t id = 0;
  nbte_solver* S = nullptr;
  int state = 0;   // 0 queued, 1 planned, 2 running, 3 done
  size_t bytes = 0;
  int status = NBTE_OK;
  nbte_solve_info info{};
  Run run;
  std::chrono::steady_clock::time_point t_submit, t_admit, t_done;
};

struct nbte_server {
  nbte_solve_opts opts{};
  int device = 0;
  size_t budget = 0, used = 0;
  int max_active = 64;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ServedSolve*> to_plan, planned;
  std::map<int64_t, std::unique_ptr<ServedSolve>> all;
  int64_t next_id = 1;
  bool stop = false;
  std::vector<std::thread> planners;
  std::thread worker;
  int64_t iterations = 0;   // batched iterations run

  void plan_loop();
  template <typename R>
  void work_loop();
};

void nbte_server::plan_loop() {
  cudaSetDevice(device);
  while (true) {
    ServedSolve* q = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !to_plan.empty(); });
      if (stop) return;
      q = to_plan.front();
      to_plan.pop_front();
    }
    nbte_solver* S = q->S;
    S->device = device;
    int rc = ensure_device(S);
    if (!rc) rc = ensure_plan(S);
    size_t b = 0;
    if (!rc) rc = ensure_layout(S, opts, &b);
    if (!rc && (opts.scheme != 0 || opts.init == 1)) {
      b += estimate_cg_bytes(S);
      rc = ensure_laplacian(S);   // host-heavy (aggregation, dense coarse inverse): off the GPU loop
    }
    std::lock_guard<std::mutex> lk(mu);
    if (rc) {
      q->status = rc;
      q->info.status = rc;
      q->state = 3;
      q->t_done = std::chrono::steady_clock::now();
      cv_done.notify_all();
    } else {
      q->bytes = b;
      q->state = 1;
      planned.push_back(q);
      cv_work.notify_all();
    }
  }
}

template <typename R>
void nbte_server::work_loop() {
  cudaSetDevice(device);
  std::vector<ServedSolve*> active;
  BatchTables<R> bt;
  bool rebuild = true;
  while (true) {
    std::vector<ServedSolve*> admit;
    {
      std::unique_lock<std::mutex> lk(mu);
      if (active.empty())
        cv_work.wait(lk, [&] { return stop || !planned.empty(); });
      if (stop) return;
      // admission in arrival order while the estimated memory fits (a solve
      // larger than the whole budget runs alone)
      while (!planned.empty() && (int)(active.size() + admit.size()) < max_active) {
        ServedSolve* q = planned.front();
        if (used + q->bytes > budget && !(active.empty() && admit.empty())) break;
        planned.pop_front();
        used += q->bytes;
        q->state = 2;
        q->t_admit = std::chrono::steady_clock::now();
        admit.push_back(q);
      }
    }
    for (ServedSolve* q : admit) {
      DeviceGuard g(q->S->device);
      int rc = ensure_layout(q->S, opts);
      if (!rc) rc = ensure_q(q->S);
      if (!rc && opts.init == 1) rc = cg_default_partition(q->S);
      if (!rc) rc = run_begin<R>(q->run, q->S, opts);
      if (!rc) rc = cudaStreamSynchronize(q->S->stream) == cudaSuccess ? NBTE_OK : NBTE_ERR_CUDA;
      if (rc) {
        shrink(q->S);
        std::lock_guard<std::mutex> lk(mu);
        used -= q->bytes;
        q->status = rc;
        q->info.status = rc;
        q->state = 3;
        q->t_done = std::chrono::steady_clock::now();
        cv_done.notify_all();
        continue;
      }
      active.push_back(q);
      rebuild = true;
    }
    if (active.empty()) continue;
    std::vector<Run*> act;
    for (ServedSolve* q : active) act.push_back(&q->run);
    if (rebuild) {
      if (batch_build<R>(bt, act) != NBTE_OK) {
        for (ServedSolve* q : active) q->run.status = NBTE_ERR_ARG;
      } else {
        rebuild = false;
        if (opts.use_graph) batch_capture<R>(bt, act, stream);
      }
    }
    cudaError_t e = cudaSuccess;
    if (rebuild) {
      e = cudaErrorInvalidValue;
    } else if (bt.graph) {
      e = cudaGraphLaunch(bt.graph, stream);
    } else {
      e = batch_enqueue<R>(bt, act, stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    ++iterations;
    std::vector<ServedSolve*> still, finished;
    for (ServedSolve* q : active) {
      Run& run = q->run;
      bool stop_it = true;
      if (e == cudaSuccess && run.status == NBTE_OK) {
        ++run.it;
        run.kernels += run.kernels_per_iter();
        stop_it = run.check();
      } else if (run.status == NBTE_OK) {
        run.status = fail(NBTE_ERR_CUDA, std::string("CUDA error in a served iteration: ") + cudaGetErrorString(e));
      }
      (stop_it ? finished : still).push_back(q);
    }
    for (ServedSolve* q : finished) {
      q->status = run_finish<R>(q->run, &q->info);
      shrink(q->S);
      std::lock_guard<std::mutex> lk(mu);
      used -= q->bytes;
      q->state = 3;
      q->t_done = std::chrono::steady_clock::now();
      rebuild = true;
    }
    if (!finished.empty()) cv_done.notify_all();
    active.swap(still);
  }
}

// ============================================================================ C ABI
extern "C" {

const char* nbte_last_error(void) { return g_err.c_str(); }

int nbte_test_timeouts(int32_t on) {
  g_test_timeouts.store(on ? 1 : 0, std::memory_order_relaxed);
  return NBTE_OK;
}
const char* nbte_version(void) { return "nanobte-b300 1.0 (sm_103a)"; }

int nbte_mesh_create(int dim, int64_t n_nodes, const double* xyz, int cell_type, int64_t n_cells,
                     const int64_t* cell_nodes, int64_t n_bfaces, const int64_t* bface_nodes,
                     const int32_t* bface_tag, nbte_mesh** out) {
  if (!out) return fail(NBTE_ERR_ARG, "out is NULL");
  *out = nullptr;
  std::unique_ptr<nbte_mesh> M(new (std::nothrow) nbte_mesh());
  if (!M) return fail(NBTE_ERR_OOM, "host allocation failed");
  try {
    Status st = build_mesh(dim, n_nodes, xyz, cell_type, n_cells, cell_nodes, n_bfaces, bface_nodes, bface_tag, M->m);
    if (!st.good()) return fail(st.code, st.msg);
  } catch (const std::bad_alloc&) {
    return fail(NBTE_ERR_OOM, "host allocation failed while building the mesh");
  }
  *out = M.release();
  return NBTE_OK;
}

int nbte_mesh_destroy(nbte_mesh* mesh) {
  delete mesh;
  return NBTE_OK;
}

int nbte_mesh_info(const nbte_mesh* mesh, int64_t* n_cells, double* volume) {
  if (!mesh) return fail(NBTE_ERR_ARG, "mesh is NULL");
  if (n_cells) *n_cells = mesh->m.n_cells;
  if (volume) *volume = mesh->m.volume;
  return NBTE_OK;
}

int nbte_solver_create(const nbte_mesh* mesh, double T_ref, nbte_solver** out) {
  if (!out) return fail(NBTE_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!mesh) return fail(NBTE_ERR_ARG, "mesh is NULL");
  if (!std::isfinite(T_ref) || T_ref <= 0) return fail(NBTE_ERR_ARG, "T_ref must be a positive temperature");
  std::unique_ptr<nbte_solver> S(new (std::nothrow) nbte_solver());
  if (!S) return fail(NBTE_ERR_OOM, "host allocation failed");
  S->mesh = mesh;
  S->T_ref = T_ref;
  // bind to the current device now if there is one; the stream and pinned
  // words are created on first device use, so argument checks of the set-up
  // calls work on a host without a GPU
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    cudaGetLastError();
    S->device = -1;
  }
  *out = S.release();
  return NBTE_OK;
}


int nbte_solver_destroy(nbte_solver* solver) {
  if (!solver) return NBTE_OK;
  if (solver->device >= 0) {
    DeviceGuard g(solver->device);
    if (solver->stream) cudaStreamSynchronize(solver->stream);
    delete solver;
  } else {
    delete solver;
  }
  return NBTE_OK;
}

int nbte_solver_set_stream(nbte_solver* S, void* cuda_stream) {
  if (!S) return fail(NBTE_ERR_ARG, "solver is NULL");
  int rc = ensure_device(S);
  if (rc) return rc;
  S->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : S->own_stream;
  drop_graph(S);
  return NBTE_OK;
}

int nbte_set_bands(nbte_solver* S, int n_bands, const double* C, const double* v, const double* tau) {
  if (!S) return fail(NBTE_ERR_ARG, "solver is NULL");
  if (n_bands <= 0 || n_bands > 4096) return fail(NBTE_ERR_ARG, "n_bands must be in [1, 4096]");
  if (!C || !v || !tau) return fail(NBTE_ERR_ARG, "null band array");
  for (int l = 0; l < n_bands; ++l)
    if (!(std::isfinite(C[l]) && C[l] > 0 && std::isfinite(v[l]) && v[l] > 0 && std::isfinite(tau[l]) && tau[l] > 0))
      return fail(NBTE_ERR_ARG, "band " + std::to_string(l) + ": C, v and tau must be positive and finite");
  S->B = n_bands;
  S->C.assign(C, C + n_bands);
  S->v.assign(v, v + n_bands);
  S->tau.assign(tau, tau + n_bands);
  S->version_bands++;
  S->have_results = false;
  return NBTE_OK;
}

int nbte_set_quadrature(nbte_solver* S, int n_dirs, const double* s, const double* w) {
  if (!S) return fail(NBTE_ERR_ARG, "solver is NULL");
  if (n_dirs <= 0 || n_dirs > 100000) return fail(NBTE_ERR_ARG, "n_dirs must be in [1, 100000]");
  if (!s || !w) return fail(NBTE_ERR_ARG, "null quadrature array");
  for (int i = 0; i < n_dirs; ++i) {
    const double n2 = s[3 * i] * s[3 * i] + s[3 * i + 1] * s[3 * i + 1] + s[3 * i + 2] * s[3 * i + 2];
    if (!std::isfinite(n2) || std::fabs(std::sqrt(n2) - 1.0) > 1e-9)
      return fail(NBTE_ERR_ARG, "direction " + std::to_string(i) + " is not a unit vector");
    if (!(std::isfinite(w[i]) && w[i] > 0)) return fail(NBTE_ERR_ARG, "weights must be positive and finite");
  }
  S->D = n_dirs;
  S->s.assign(s, s + 3 * n_dirs);
  S->w.assign(w, w + n_dirs);
  S->version_plan++;
  S->have_results = false;
  return NBTE_OK;
}

int nbte_set_boundaries(nbte_solver* S, int n, const nbte_boundary* bcs) {
  if (!S) return fail(NBTE_ERR_ARG, "solver is NULL");
  if (n <= 0 || !bcs) return fail(NBTE_ERR_ARG, "at least one boundary condition is required");
  std::vector<BC> v;
  bool therm = false;
  for (int k = 0; k < n; ++k) {
    const nbte_boundary& b = bcs[k];
    if (b.type < NBTE_THERMALIZING || b.type > NBTE_PARTIAL) return fail(NBTE_ERR_ARG, "unknown boundary type");
    for (auto& x : v)
      if (x.tag == b.tag) return fail(NBTE_ERR_ARG, "tag " + std::to_string(b.tag) + " given twice");
    if (b.type == NBTE_THERMALIZING && !(std::isfinite(b.T_wall) && b.T_wall > 0))
      return fail(NBTE_ERR_ARG, "thermalizing wall needs a positive T_wall");
    if (b.type == NBTE_PARTIAL && !(b.specularity >= 0.0 && b.specularity <= 1.0))
      return fail(NBTE_ERR_ARG, "specularity must be in [0, 1]");
    v.push_back({b.tag, b.type, b.T_wall, b.specularity});
  }
  for (int32_t t : S->mesh->m.tags_present) {
    bool found = false;
    for (auto& x : v) {
      if (x.tag == t) {
        found = true;
        if (x.type == NBTE_THERMALIZING) therm = true;
      }
    }
    if (!found) return fail(NBTE_ERR_ARG, "boundary tag " + std::to_string(t) + " has no condition");
  }
  if (!therm) return fail(NBTE_ERR_ARG, "no thermalizing wall: the steady problem has no unique solution");
  S->bcs = v;
  S->bcs_set = true;
  S->version_plan++;
  S->have_results = false;
  return NBTE_OK;
}

int nbte_set_heat_source(nbte_solver* S, const double* Qdot) {
  if (!S) return fail(NBTE_ERR_ARG, "solver is NULL");
  const int64_t N = S->mesh->m.n_cells;
  if (Qdot) {
    // non-finite <=> all exponent bits set; an integer OR-reduction that
    // vectorises, then one copy into pinned memory in the caller's order
    // (reordered on the device).  A rejected array leaves the old source.
    uint64_t bad = 0;
    for (int64_t k = 0; k < N; ++k) {
      uint64_t u;
      std::memcpy(&u, Qdot + k, 8);
      bad |= (uint64_t)((u & 0x7ff0000000000000ull) == 0x7ff0000000000000ull);
    }
    if (bad) return fail(NBTE_ERR_ARG, "non-finite heat source");
    if (!S->h_qc) {
      const size_t bytes = (size_t)std::max<int64_t>(N, 1) * 8;
      S->h_qc_pinned = cudaMallocHost(&S->h_qc, bytes) == cudaSuccess;
      if (!S->h_qc_pinned) {   // no device yet: plain memory, copied synchronously later
        cudaGetLastError();
        S->h_qc = static_cast<double*>(std::malloc(bytes));
        if (!S->h_qc) return fail(NBTE_ERR_OOM, "host allocation failed");
      }
    }
    std::memcpy(S->h_qc, Qdot, (size_t)N * 8);
  } else if (S->h_qc) {
    std::memset(S->h_qc, 0, (size_t)N * 8);
  }
  S->version_q++;
  S->have_results = false;
  return NBTE_OK;
}

int nbte_default_opts(nbte_solve_opts* o) {
  if (!o) return fail(NBTE_ERR_ARG, "opts is NULL");
  std::memset(o, 0, sizeof(*o));
  o->scheme = 0;
  o->precision = 0;
  o->tol = 1e-10;
  o->max_iter = 10000;
  return NBTE_OK;
}

static int check_opts(const nbte_solve_opts& o) {
  if (o.scheme < 0 || o.scheme > 2) return fail(NBTE_ERR_ARG, "scheme must be 0, 1 or 2");
  if (o.precision < 0 || o.precision > 1) return fail(NBTE_ERR_ARG, "precision must be 0 or 1");
  if (o.n_iter < 0) return fail(NBTE_ERR_ARG, "n_iter must be >= 0");
  if (o.n_iter == 0 && !(o.tol > 0 && std::isfinite(o.tol))) return fail(NBTE_ERR_ARG, "tol must be positive");
  if (o.n_iter == 0 && o.max_iter <= 0) return fail(NBTE_ERR_ARG, "max_iter must be positive");
  if (o.ring < 0 || o.ring > 2) return fail(NBTE_ERR_ARG, "ring must be 0, 1 or 2");
  if (o.init < 0 || o.init > 1) return fail(NBTE_ERR_ARG, "init must be 0 or 1");
  if (o.init == 1 && o.T_init) return fail(NBTE_ERR_ARG, "init = 1 (diffusion guess) excludes T_init");
  if (o.order < 0 || o.order > 2) return fail(NBTE_ERR_ARG, "order must be 0 (= 1), 1 or 2");
  if (o.deterministic < 0 || o.deterministic > 1) return fail(NBTE_ERR_ARG, "deterministic must be 0 or 1");
  return NBTE_OK;
}

int nbte_plan_stats(nbte_solver* S, const nbte_solve_opts* opts, int64_t stats[12]) {
  if (!S || !stats) return fail(NBTE_ERR_ARG, "null argument");
  nbte_solve_opts o;
  nbte_default_opts(&o);
  if (opts) o = *opts;
  int rc = check_opts(o);
  if (rc) return rc;
  rc = ensure_device(S);
  if (rc) return rc;
  DeviceGuard g(S->device);
  rc = ensure_plan(S);
  if (rc) return rc;
  if (S->B > 0 && S->D > 0 && S->bcs_set) {
    rc = autotune(S, o);
    if (rc) return rc;
  }
  rc = ensure_layout(S, o);
  if (rc) return rc;
  stats[0] = S->total_levels;
  stats[1] = S->max_levels;
  stats[2] = S->max_slots;
  stats[3] = S->lagged;
  stats[4] = S->n_items;
  stats[5] = S->G;
  stats[6] = S->gring_stride > 0 ? 2 : 1;
  stats[7] = (int64_t)device_bytes(S);
  stats[8] = S->K;
  stats[9] = S->n_exp;
  stats[10] = S->n_imp;
  stats[11] = S->threads;
  return NBTE_OK;
}

// prepare one solver for a solve with options o (plan, layout, heat source,
// Laplacian); shared by the single and the batched entry points
static int prepare(nbte_solver* S, const nbte_solve_opts& o) {
  if (S->B <= 0) return fail(NBTE_ERR_STATE, "nbte_set_bands must be called before solving");
  if (S->D <= 0) return fail(NBTE_ERR_STATE, "nbte_set_quadrature must be called before solving");
  if (!S->bcs_set) return fail(NBTE_ERR_STATE, "nbte_set_boundaries must be called before solving");
  int rc = ensure_device(S);
  if (rc) return rc;
  DeviceGuard g(S->device);
  rc = ensure_plan(S);
  if (rc) return rc;
  rc = autotune(S, o);
  if (rc) return rc;
  rc = ensure_layout(S, o);
  if (rc) return rc;
  rc = ensure_q(S);
  if (rc) return rc;
  if (o.scheme != 0 || o.init == 1) {
    rc = ensure_laplacian(S);
    if (rc) return rc;
    rc = cg_default_partition(S);
    if (rc) return rc;
  }
  return NBTE_OK;
}

int nbte_solve_steady(nbte_solver* S, const nbte_solve_opts* opts, nbte_solve_info* info) {
  if (!S) return fail(NBTE_ERR_ARG, "solver is NULL");
  nbte_solve_opts o;
  nbte_default_opts(&o);
  if (opts) o = *opts;
  int rc = check_opts(o);
  if (rc) return rc;
  try {
    rc = prepare(S, o);
    if (rc) return rc;
    DeviceGuard g(S->device);
    return S->prec ? run_solve<float>(S, o, info) : run_solve<double>(S, o, info);
  } catch (const std::bad_alloc&) {
    return fail(NBTE_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(NBTE_ERR_ARG, e.what());
  }
}

int nbte_solve_batch(nbte_solver* const* solvers, int32_t n, const nbte_solve_opts* opts, nbte_solve_info* infos) {
  if (!solvers || n < 1 || n > 148) return fail(NBTE_ERR_ARG, "n must be in [1, 148] with a solver array");
  nbte_solve_opts o;
  nbte_default_opts(&o);
  if (opts) o = *opts;
  int rc = check_opts(o);
  if (rc) return rc;
  if (o.T_init) return fail(NBTE_ERR_ARG, "T_init is not supported by nbte_solve_batch");
  if (o.profile) return fail(NBTE_ERR_ARG, "profile is not supported by nbte_solve_batch");
  std::vector<nbte_solver*> Ss(solvers, solvers + n);
  for (int k = 0; k < n; ++k) {
    if (!Ss[k]) return fail(NBTE_ERR_ARG, "null solver in the batch");
    for (int j = 0; j < k; ++j)
      if (Ss[j] == Ss[k]) return fail(NBTE_ERR_ARG, "a solver appears twice in the batch");
  }
  try {
    // the host-heavy set-up of every solver at once, one thread each (as the
    // server's planner threads do): direction plans and, for the synthetic
    // schemes, the correction's operator.  A failure here is left for the
    // serial preparation below to report on the calling thread.
    if (n > 1) {
      int dev = 0;
      NBTE_CK(cudaGetDevice(&dev));
      std::vector<std::thread> th;
      for (int k = 0; k < n; ++k)
        th.emplace_back([&, k] {
          nbte_solver* S = Ss[k];
          cudaSetDevice(S->device >= 0 ? S->device : dev);
          int r = ensure_device(S);
          if (!r) r = ensure_plan(S);
          if (!r && (o.scheme != 0 || o.init == 1)) ensure_laplacian(S);
        });
      for (auto& t : th) t.join();
    }
    for (int k = 0; k < n; ++k) {
      rc = prepare(Ss[k], o);
      if (rc) return rc;
      if (Ss[k]->device != Ss[0]->device) return fail(NBTE_ERR_ARG, "the solvers of a batch must share a device");
    }
    DeviceGuard g(Ss[0]->device);
    return o.precision ? run_batch<float>(Ss, o, infos) : run_batch<double>(Ss, o, infos);
  } catch (const std::bad_alloc&) {
    return fail(NBTE_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(NBTE_ERR_ARG, e.what());
  }
}

}  // extern "C"

// pinned host staging of n doubles for result read-back (grows on demand)
static double* host_stage(const nbte_solver* S, size_t n) {
  if (S->h_stage_n < n) {
    if (S->h_stage) cudaFreeHost(S->h_stage);
    S->h_stage = nullptr;
    S->h_stage_n = 0;
    if (cudaMallocHost(&S->h_stage, n * 8) != cudaSuccess) {
      S->h_stage = nullptr;
      return nullptr;
    }
    S->h_stage_n = n;
  }
  return S->h_stage;
}

// page-locked host memory (the device copies into it directly)
static bool host_pinned(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

// n doubles of the device staging buffer to the caller's out, directly when
// out is pinned
static int download(nbte_solver* S, double* out, size_t n) {
  if (host_pinned(out)) {
    NBTE_CK(cudaMemcpyAsync(out, S->io_d.p, n * 8, cudaMemcpyDeviceToHost, S->stream));
    NBTE_CK(cudaStreamSynchronize(S->stream));
    return NBTE_OK;
  }
  double* tmp = host_stage(S, n);
  if (!tmp) return fail(NBTE_ERR_OOM, "pinned host allocation failed");
  NBTE_CK(cudaMemcpyAsync(tmp, S->io_d.p, n * 8, cudaMemcpyDeviceToHost, S->stream));
  NBTE_CK(cudaStreamSynchronize(S->stream));
  std::memcpy(out, tmp, n * 8);
  return NBTE_OK;
}

extern "C" {

int nbte_get_temperature(const nbte_solver* S, int kind, double* out) {
  if (!S || !out) return fail(NBTE_ERR_ARG, "null argument");
  if (!S->have_results) return fail(NBTE_ERR_STATE, "no results: call nbte_solve_steady first");
  if (kind < 0 || kind > 2) return fail(NBTE_ERR_ARG, "kind must be 0, 1 or 2");
  if (kind == 1 && !S->have_outputs) return fail(NBTE_ERR_STATE, "the last solve skipped its outputs");
  DeviceGuard g(S->device);
  const Mesh& m = S->mesh->m;
  const int64_t N = m.n_cells;
  const DBuf& src = kind == 0 ? S->T : (kind == 1 ? S->accE : S->Tkin);
  nbte_solver* Sm = const_cast<nbte_solver*>(S);   // device staging only
  int rc = ensure_perm(Sm);
  if (rc) return rc;
  NBTE_CK(Sm->io_d.alloc(std::max<size_t>(Sm->io_d.bytes, (size_t)N * 8 * m.dim)));
  NBTE_CK(launch_to_caller(Sm->io_d.as<double>(), src.as<double>(), Sm->perm_d.as<int32_t>(), (int)N, 1,
                           kind == 1 ? 1.0 / S->Ctot : 1.0, S->T_ref, S->stream));
  return download(Sm, out, (size_t)N);
}

int nbte_get_heat_flux(const nbte_solver* S, double* out) {
  if (!S || !out) return fail(NBTE_ERR_ARG, "null argument");
  if (!S->have_results) return fail(NBTE_ERR_STATE, "no results: call nbte_solve_steady first");
  if (!S->have_outputs) return fail(NBTE_ERR_STATE, "the last solve skipped its outputs");
  DeviceGuard g(S->device);
  const Mesh& m = S->mesh->m;
  const int64_t N = m.n_cells;
  nbte_solver* Sm = const_cast<nbte_solver*>(S);   // device staging only
  int rc = ensure_perm(Sm);
  if (rc) return rc;
  NBTE_CK(Sm->io_d.alloc(std::max<size_t>(Sm->io_d.bytes, (size_t)N * 8 * m.dim)));
  NBTE_CK(launch_to_caller(Sm->io_d.as<double>(), S->accQ.as<double>(), Sm->perm_d.as<int32_t>(), (int)N, m.dim,
                           1.0, 0.0, S->stream));
  return download(Sm, out, (size_t)N * m.dim);
}

}  // extern "C"

// the last sweep's values of one work item, recomputed: its inputs (the
// gathered (T', Qdot) pairs and the import rows) are still resident and the
// sweep is deterministic, so re-running the item reproduces them exactly
template <typename R>
static int distribution(nbte_solver* S, int dir, int band, double* out) {
  const Mesh& m = S->mesh->m;
  const int64_t N = m.n_cells;
  const int G = S->G;
  cudaStream_t st = S->stream;
  NBTE_CK(S->e_scratch.alloc((size_t)N * G * sizeof(R)));
  SweepArgs<R> a = sweep_args<R>(S, 0);
  a.item0 = S->item_of[(size_t)dir * S->n_groups + band / G];
  a.e_out = S->e_scratch.as<R>();
  a.e_out_dstride = 0;
  a.e_out_gstride = 0;
  a.e_out_cstride = G;
  NBTE_CK(launch_sweep<R>(a, S->K, G, 1, S->threads, S->smem, st));
  std::vector<R> tmp((size_t)N * G);
  NBTE_CK(cudaMemcpyAsync(tmp.data(), S->e_scratch.p, tmp.size() * sizeof(R), cudaMemcpyDeviceToHost, st));
  unsigned long long err = 0;
  NBTE_CK(cudaMemcpyAsync(&err, S->res.as<unsigned long long>() + 2, 8, cudaMemcpyDeviceToHost, st));
  NBTE_CK(cudaStreamSynchronize(st));
  if (err) {
    zero_now(S->res.p, 32, S->stream);
    return sweep_error(err);
  }
  const int b = band % G;
  for (int64_t c = 0; c < N; ++c) out[m.perm[c]] = (double)tmp[(size_t)c * G + b];
  return NBTE_OK;
}

extern "C" {

int nbte_get_distribution(nbte_solver* S, int32_t direction, int32_t band, double* out) {
  if (!S || !out) return fail(NBTE_ERR_ARG, "null argument");
  if (!S->have_results || S->layout_key.empty())
    return fail(NBTE_ERR_STATE, "no results: call nbte_solve_steady first");
  if (direction < 0 || direction >= S->D) return fail(NBTE_ERR_ARG, "direction out of range");
  if (band < 0 || band >= S->B) return fail(NBTE_ERR_ARG, "band out of range");
  DeviceGuard g(S->device);
  return S->prec ? distribution<float>(S, direction, band, out) : distribution<double>(S, direction, band, out);
}

int nbte_get_wall_heat(const nbte_solver* S, int32_t tag, double* out) {
  if (!S || !out) return fail(NBTE_ERR_ARG, "null argument");
  if (!S->have_results) return fail(NBTE_ERR_STATE, "no results: call nbte_solve_steady first");
  if (!S->have_outputs) return fail(NBTE_ERR_STATE, "the last solve skipped its outputs");
  auto it = std::lower_bound(S->tag_list.begin(), S->tag_list.end(), tag);
  if (it == S->tag_list.end() || *it != tag || S->wall_heat_by_tag.size() != S->tag_list.size())
    return fail(NBTE_ERR_ARG, "no boundary face carries tag " + std::to_string(tag));
  *out = S->wall_heat_by_tag[it - S->tag_list.begin()];
  return NBTE_OK;
}

// ---------------------------------------------------------------- serving
int nbte_server_create(const nbte_solve_opts* opts, size_t budget_bytes, int32_t max_active, int32_t n_planners,
                       nbte_server** out) {
  if (!out) return fail(NBTE_ERR_ARG, "out is NULL");
  *out = nullptr;
  nbte_solve_opts o;
  nbte_default_opts(&o);
  if (opts) o = *opts;
  int rc = check_opts(o);
  if (rc) return rc;
  if (o.T_init) return fail(NBTE_ERR_ARG, "T_init is not supported by the server");
  if (o.profile) return fail(NBTE_ERR_ARG, "profile is not supported by the server");
  if (max_active < 1 || max_active > 148) return fail(NBTE_ERR_ARG, "max_active must be in [1, 148]");
  if (n_planners < 1 || n_planners > 64) return fail(NBTE_ERR_ARG, "n_planners must be in [1, 64]");
  std::unique_ptr<nbte_server> srv(new (std::nothrow) nbte_server());
  if (!srv) return fail(NBTE_ERR_OOM, "host allocation failed");
  srv->opts = o;
  NBTE_CK(cudaGetDevice(&srv->device));
  if (budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    NBTE_CK(cudaMemGetInfo(&fr, &tot));
    budget_bytes = fr / 10 * 8;
  }
  srv->budget = budget_bytes;
  srv->max_active = max_active;
  NBTE_CK(cudaStreamCreateWithFlags(&srv->stream, cudaStreamNonBlocking));
  nbte_server* p = srv.get();
  for (int k = 0; k < n_planners; ++k) p->planners.emplace_back([p] { p->plan_loop(); });
  if (o.precision) p->worker = std::thread([p] { p->work_loop<float>(); });
  else p->worker = std::thread([p] { p->work_loop<double>(); });
  *out = srv.release();
  return NBTE_OK;
}

int nbte_server_submit(nbte_server* srv, nbte_solver* solver, int64_t* request) {
  if (!srv || !solver || !request) return fail(NBTE_ERR_ARG, "null argument");
  if (solver->B <= 0 || solver->D <= 0 || !solver->bcs_set)
    return fail(NBTE_ERR_STATE, "bands, quadrature and boundaries must be set before submitting");
  std::lock_guard<std::mutex> lk(srv->mu);
  for (auto& kv : srv->all)
    if (kv.second->S == solver && kv.second->state != 3) return fail(NBTE_ERR_STATE, "solver already submitted");
  std::unique_ptr<ServedSolve> q(new ServedSolve());
  q->id = srv->next_id++;
  q->S = solver;
  q->t_submit = std::chrono::steady_clock::now();
  *request = q->id;
  srv->to_plan.push_back(q.get());
  srv->all[q->id] = std::move(q);
  srv->cv_work.notify_all();
  return NBTE_OK;
}

int nbte_server_poll(nbte_server* srv, int64_t request, int32_t* state, nbte_solve_info* info, double* seconds) {
  if (!srv || !state) return fail(NBTE_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->all.find(request);
  if (it == srv->all.end()) return fail(NBTE_ERR_ARG, "unknown request");
  const ServedSolve& q = *it->second;
  *state = q.state;
  if (q.state == 3) {
    if (info) *info = q.info;
    if (seconds) {
      seconds[0] = std::chrono::duration<double>(q.t_done - q.t_submit).count();
      seconds[1] = q.t_admit.time_since_epoch().count() ? std::chrono::duration<double>(q.t_admit - q.t_submit).count()
                                                        : seconds[0];
    }
    return q.status;
  }
  return NBTE_OK;
}

int nbte_server_drain(nbte_server* srv, double timeout_s) {
  if (!srv) return fail(NBTE_ERR_ARG, "null argument");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto done = [&] {
    for (auto& kv : srv->all)
      if (kv.second->state != 3) return false;
    return true;
  };
  if (timeout_s > 0) {
    if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done))
      return fail(NBTE_ERR_NOT_CONVERGED, "requests still running after the timeout");
  } else {
    srv->cv_done.wait(lk, done);
  }
  return NBTE_OK;
}

int nbte_server_stats(nbte_server* srv, int64_t stats[4]) {
  if (!srv || !stats) return fail(NBTE_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  int64_t done = 0;
  for (auto& kv : srv->all) done += kv.second->state == 3;
  stats[0] = srv->iterations;
  stats[1] = (int64_t)srv->all.size();
  stats[2] = done;
  stats[3] = (int64_t)srv->used;
  return NBTE_OK;
}

int nbte_server_destroy(nbte_server* srv) {
  if (!srv) return NBTE_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->planners) t.join();
  if (srv->worker.joinable()) srv->worker.join();
  if (srv->stream) {
    cudaStreamSynchronize(srv->stream);
    cudaStreamDestroy(srv->stream);
  }
  delete srv;
  return NBTE_OK;
}

}  // extern "C"

