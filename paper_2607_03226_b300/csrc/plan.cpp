// Direction planner: everything about a (mesh, direction set, walls) that does
// not change between outer iterations -- "precompute what is
// iteration-independent" (Sec. II, after Eq. (13)).
//
// For every direction i the first-order upwind system I/tau + v K_i of
// Eq. (13) is lower-triangular in a topological order of the upwind graph
// (edge u -> c when a face of c has s_i . An < 0 and u is across it), so its
// LU factorisation is the graph order itself and "triangular substitution" is
// a sweep.  The planner computes, per direction:
//
//  * Kahn levels of the upwind graph: cells of one level depend only on
//    earlier levels.  If no cell is ready (a cycle, possible on unstructured
//    3D meshes) the lowest-numbered unprocessed cell is released and its
//    inflow faces from unprocessed cells are marked "lagged": their upwind
//    value is taken from the previous iteration.  Structured and 2D meshes
//    have none.
//  * tilted fronts: where a direction's level fronts are wide (many cells
//    live at once), each cell may also be given a release level that grows
//    along the mesh's longest axis, level(c) = max(release(c), 1 + max over
//    upstream u of level(u)).  Any such assignment is a topological order of
//    the same graph, so the sweep computes the same values; the fronts lean
//    along the long axis and cross the mesh where it is narrow, which cuts
//    the live cells (ring slots) severalfold for a few more levels.  The
//    release slope is chosen per direction from a few candidates: fewest
//    live cells without more levels than the longest untilted direction.
//  * ring slots: a cell's value lives in shared memory from its own level to
//    the last level that reads it; slots are reused (interval colouring), so
//    a sweep needs only max-live-cells slots, not N.  A new value takes the
//    lowest free slot, which keeps the slots in use dense at the low end of
//    the ring (on the 1.14M-tet FinFET's global ring the sweep took 27.9 ms
//    with lowest-first reuse against 31.4 ms with the most recently freed
//    slot first).
//  * per-position records (cell, slot, diagonal G, inflow references and
//    coefficients |s.An|/V), in level order.
//  * exports (cells whose value is needed after the sweep: outgoing wall
//    faces and lagged upstream cells) and imports (wall and lagged inflow
//    values read by the sweep), with everything the wall kernel needs to
//    turn exports into imports.
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <functional>
#include <map>
#include <thread>

#include "nbte_internal.h"

namespace nbte {

namespace {

struct LocalImport {
  int32_t kind;
  int32_t dbf;        // diffuse face index
  int32_t src_dir;    // export direction (specular / partial / lag)
  int32_t src_cell;   // export cell
  double par;
};

struct DirOut {
  std::vector<int32_t> lp;          // level pointer
  int32_t n_slots = 0, max_width = 0;
  int64_t lagged = 0;
  std::vector<int32_t> exp_cells;   // sorted
  std::vector<LocalImport> imps;
  std::vector<std::pair<int64_t, int32_t>> bimp;  // (boundary half-face, local import), sorted
  std::string error;
};

constexpr double kTangent = 1e-12;   // |s.An| <= kTangent |An| counts as no flux
// directions with more live cells than this (untilted) try tilted fronts
constexpr int32_t kTiltLive = 4096;
// release slopes tried, in levels per cell length along the long axis
constexpr double kTiltSlopes[] = {1.0, 2.0, 3.0, 4.0, 6.0, 8.0, 12.0, 16.0};

}  // namespace

Status build_plan(const Mesh& m, int D, const double* s, const double* w, const std::vector<BC>& bcs,
                  double T_ref, Plan& P, int n_threads) {
  const int dim = m.dim, nfc = m.nfc;
  const int64_t N = m.n_cells, H = N * nfc;
  P = Plan();
  P.D = D;
  P.N = (int)N;
  // inflow entries per cell: at most nfc - 1 faces of a closed convex cell
  // face a given direction
  P.K = nfc - 1;
  const int K = P.K;

  std::map<int32_t, BC> bcmap;
  for (auto& b : bcs) bcmap[b.tag] = b;

  // boundary half-faces, their unit normals and diffuse-face numbering
  std::vector<int64_t> bhf;
  for (int64_t h = 0; h < H; ++h)
    if (m.nb[h] < 0) bhf.push_back(h);
  std::vector<int32_t> dbf_of_h(H, -1);
  std::vector<int64_t> dbf_h;
  for (int64_t h : bhf) {
    const BC& b = bcmap.at(m.tag[h]);
    if (b.type == NBTE_DIFFUSE || b.type == NBTE_PARTIAL) {
      dbf_of_h[h] = (int32_t)dbf_h.size();
      dbf_h.push_back(h);
    }
  }
  auto unit_normal = [&](int64_t h, double n[3]) {
    double a = 0;
    for (int d = 0; d < dim; ++d) a += m.An[h * dim + d] * m.An[h * dim + d];
    a = std::sqrt(a);
    n[0] = n[1] = n[2] = 0;
    for (int d = 0; d < dim; ++d) n[d] = m.An[h * dim + d] / a;
  };
  auto dotsa = [&](int i, int64_t h) {
    double a = 0;
    for (int d = 0; d < dim; ++d) a += s[i * 3 + d] * m.An[h * dim + d];
    return a;
  };
  std::vector<double> area(H);
  for (int64_t h = 0; h < H; ++h) {
    double a = 0;
    for (int d = 0; d < dim; ++d) a += m.An[h * dim + d] * m.An[h * dim + d];
    area[h] = std::sqrt(a);
  }
  auto cls = [&](double a, int64_t h) { return a > kTangent * area[h] ? 1 : (a < -kTangent * area[h] ? -1 : 0); };

  // mirror maps, cached per distinct normal: R[i] = direction nearest to
  // s_i - 2 (s_i . n) n among those leaving through the face
  std::map<std::array<long long, 3>, std::vector<int32_t>> mirror_cache;
  auto mirror_map = [&](int64_t h) -> const std::vector<int32_t>& {
    double n[3];
    unit_normal(h, n);
    std::array<long long, 3> key = {std::llround(n[0] * 1e12), std::llround(n[1] * 1e12), std::llround(n[2] * 1e12)};
    auto it = mirror_cache.find(key);
    if (it != mirror_cache.end()) return it->second;
    std::vector<int32_t> R(D);
    for (int i = 0; i < D; ++i) {
      const double sn = s[i * 3] * n[0] + s[i * 3 + 1] * n[1] + s[i * 3 + 2] * n[2];
      double mir[3];
      for (int d = 0; d < 3; ++d) mir[d] = s[i * 3 + d] - 2.0 * sn * n[d];
      int best = -1;
      double bd = 1e300;
      for (int j = 0; j < D; ++j) {
        const double sj = s[j * 3] * n[0] + s[j * 3 + 1] * n[1] + s[j * 3 + 2] * n[2];
        if (!(sj > kTangent)) continue;   // must leave through the wall
        double dd = 0;
        for (int d = 0; d < 3; ++d) dd += (s[j * 3 + d] - mir[d]) * (s[j * 3 + d] - mir[d]);
        if (dd < bd) { bd = dd; best = j; }
      }
      R[i] = best;
    }
    return mirror_cache.emplace(key, std::move(R)).first->second;
  };
  // fill the cache serially (it is read by the worker threads), and keep
  // each reflecting half-face's map
  std::vector<const std::vector<int32_t>*> mirror_of_h(H, nullptr);
  for (int64_t h : bhf) {
    const BC& b = bcmap.at(m.tag[h]);
    if (b.type == NBTE_SPECULAR || b.type == NBTE_PARTIAL) mirror_of_h[h] = &mirror_map(h);
  }

  P.pos_cell.assign((size_t)D * N, 0);
  P.pos_slot.assign((size_t)D * N, -1);
  P.pos_exp.assign((size_t)D * N, -1);
  if (kChecks) P.pos_last.assign((size_t)D * N, -1);
  P.pos_G.assign((size_t)D * N, 0.0);
  P.pos_ref.assign((size_t)D * K * N, 0);
  P.pos_coef.assign((size_t)D * K * N, 0.0);
  std::vector<DirOut> outs(D);

  // tilted fronts: the longest axis of the mesh's bounding box and a cell
  // length (the release level of cell c is slope * (x_c - x_min) / h along it,
  // x measured in the direction's own sense along the axis)
  // NBTE_PLAN_TILT: "0" plans untilted levels only; "force" (for testing)
  // tilts every direction, with the steepest slope within the level cap
  // whether or not it saves live cells
  const char* tilt_env = std::getenv("NBTE_PLAN_TILT");
  const bool tilt = !(tilt_env && tilt_env[0] == '0');
  const bool tilt_force = tilt_env && std::string(tilt_env) == "force";
  const int32_t tilt_live = tilt_force ? -1 : kTiltLive;
  int tilt_axis = 0;
  double bb_lo[3] = {0, 0, 0}, bb_hi[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) {
    bb_lo[d] = INFINITY;
    bb_hi[d] = -INFINITY;
    for (int64_t c = 0; c < N; ++c) {
      bb_lo[d] = std::min(bb_lo[d], m.xc[c * dim + d]);
      bb_hi[d] = std::max(bb_hi[d], m.xc[c * dim + d]);
    }
    if (bb_hi[d] - bb_lo[d] > bb_hi[tilt_axis] - bb_lo[tilt_axis]) tilt_axis = d;
  }
  const double hcell = std::pow(m.volume / (double)std::max<int64_t>(N, 1), 1.0 / dim);
  std::vector<int32_t> untilted_levels(D, 0);
  int32_t level_cap = 0;   // the longest untilted direction's level count

  // pass 0: Kahn level counts only (they set level_cap); pass 1: the plan
  auto work = [&](int tid, int nt, int pass) {
    std::vector<int32_t> indeg(N), level(N), slot(N), last_use(N), exp_local(N), cand, best, occ;
    std::vector<int32_t> up_off, up_list, dn_off, dn_list;
    std::vector<double> xr;
    std::vector<char> lagged(H);
    std::vector<signed char> fcls(H);
    std::vector<int32_t> order, cur, next, free_slots;
    std::vector<int32_t> rel_off, rel_cells, rel_fill;
    for (int i = tid; i < D; i += nt) {
      DirOut& o = outs[i];
      o = DirOut();
      // each half-face's class for this direction: inflow (-1), none, outflow
      if (dim == 3) {
        const double s0 = s[i * 3], s1 = s[i * 3 + 1], s2 = s[i * 3 + 2];
        for (int64_t h = 0; h < H; ++h) {
          const double a = s0 * m.An[h * 3] + s1 * m.An[h * 3 + 1] + s2 * m.An[h * 3 + 2];
          const double t = kTangent * area[h];
          fcls[h] = (signed char)(a > t ? 1 : (a < -t ? -1 : 0));
        }
      } else {
        for (int64_t h = 0; h < H; ++h) fcls[h] = (signed char)cls(dotsa(i, h), h);
      }
      std::fill(indeg.begin(), indeg.end(), 0);
      std::fill(level.begin(), level.end(), -1);
      std::fill(lagged.begin(), lagged.end(), 0);
      for (int64_t c = 0; c < N; ++c)
        for (int k = 0; k < nfc; ++k) {
          const int64_t h = c * nfc + k;
          if (m.nb[h] >= 0 && fcls[h] < 0) indeg[c]++;
        }
      // ---- Kahn levels with deterministic cycle breaking
      order.clear();
      cur.clear();
      o.lp.assign(1, 0);
      for (int64_t c = 0; c < N; ++c)
        if (indeg[c] == 0) cur.push_back((int32_t)c);
      int64_t processed = 0, scan = 0;
      while (processed < N) {
        if (cur.empty()) {
          while (level[scan] >= 0) ++scan;
          const int64_t c = scan;
          for (int k = 0; k < nfc; ++k) {
            const int64_t h = c * nfc + k;
            if (m.nb[h] >= 0 && level[m.nb[h]] < 0 && fcls[h] < 0) {
              lagged[h] = 1;
              o.lagged++;
            }
          }
          indeg[c] = 0;
          cur.push_back((int32_t)c);
        }
        const int32_t lev = (int32_t)o.lp.size() - 1;
        for (int32_t c : cur) {
          level[c] = lev;
          order.push_back(c);
        }
        processed += (int64_t)cur.size();
        o.max_width = std::max(o.max_width, (int32_t)cur.size());
        o.lp.push_back((int32_t)order.size());
        next.clear();
        for (int32_t u : cur)
          for (int k = 0; k < nfc; ++k) {
            const int64_t h = (int64_t)u * nfc + k;
            const int64_t v = m.nb[h];
            if (v < 0 || fcls[h] <= 0) continue;
            if (level[v] >= 0) continue;   // edge into an already released cell: lagged
            if (--indeg[v] == 0) next.push_back((int32_t)v);
          }
        // (the order within a level does not matter: the forced cell of a
        // cycle is found by index, and the level lists are rebuilt by cell
        // index below)
        cur.swap(next);
      }
      if (pass == 0) {
        untilted_levels[i] = (int32_t)o.lp.size() - 1;
        continue;
      }
      int L = (int)o.lp.size() - 1;
      // ---- tilted fronts (release levels along the long axis), see the
      // file comment.  `order` is topological for the non-lagged edges.
      // the direction's upwind graph without its lagged edges, compact:
      // upstream cells of each position (in topological order) and
      // downstream cells of each cell, and each position's coordinate along
      // the tilt axis (in the direction's sense, from the mesh's near end)
      const double sg = s[i * 3 + tilt_axis] >= 0 ? 1.0 : -1.0;
      const double x0 = sg > 0 ? bb_lo[tilt_axis] : -bb_hi[tilt_axis];
      up_off.assign(N + 1, 0);
      dn_off.assign(N + 1, 0);
      up_list.clear();
      dn_list.clear();
      xr.resize(N);
      for (int64_t p = 0; p < N; ++p) {
        const int32_t c = order[p];
        for (int k = 0; k < nfc; ++k) {
          const int64_t h = (int64_t)c * nfc + k;
          if (fcls[h] < 0 && m.nb[h] >= 0 && !lagged[h]) up_list.push_back((int32_t)m.nb[h]);
        }
        up_off[p + 1] = (int32_t)up_list.size();
        xr[p] = sg * m.xc[(int64_t)c * dim + tilt_axis] - x0;
      }
      for (int64_t c = 0; c < N; ++c) {
        for (int k = 0; k < nfc; ++k) {
          const int64_t h = c * nfc + k;
          const int64_t v = m.nb[h];
          if (v >= 0 && fcls[h] > 0 && !lagged[m.twin[h]]) dn_list.push_back((int32_t)v);
        }
        dn_off[c + 1] = (int32_t)dn_list.size();
      }
      // levels with release slope `slope` (0: none), then as late as
      // possible; returns the level count
      auto relevel = [&](double slope, std::vector<int32_t>& lev) -> int {
        lev.resize(N);
        for (int64_t p = 0; p < N; ++p) {
          int32_t l = slope > 0 ? (int32_t)std::floor(slope * xr[p] / hcell) : 0;
          for (int32_t e = up_off[p]; e < up_off[p + 1]; ++e) l = std::max(l, lev[up_list[e]] + 1);
          lev[order[p]] = l;
        }
        for (int64_t p = N - 1; p >= 0; --p) {
          const int32_t u = order[p];
          int32_t first = INT32_MAX;
          for (int32_t e = dn_off[u]; e < dn_off[u + 1]; ++e) first = std::min(first, lev[dn_list[e]]);
          if (first != INT32_MAX && first - 1 > lev[u]) lev[u] = first - 1;
        }
        // drop empty levels (release levels can leave gaps)
        int32_t top = 0;
        for (int64_t c = 0; c < N; ++c) top = std::max(top, lev[c]);
        occ.assign(top + 1, 0);
        for (int64_t c = 0; c < N; ++c) occ[lev[c]] = 1;
        int32_t used = 0;
        for (int32_t l = 0; l <= top; ++l) {
          const int32_t u = occ[l];
          occ[l] = used;
          used += u;
        }
        for (int64_t c = 0; c < N; ++c) lev[c] = occ[lev[c]];
        return used;
      };
      // most cells live at once (value written, a reader still to come)
      auto live_of = [&](const std::vector<int32_t>& lev, int nl) -> int32_t {
        occ.assign(nl + 1, 0);
        for (int64_t c = 0; c < N; ++c) {
          int32_t last = -1;
          for (int32_t e = dn_off[c]; e < dn_off[c + 1]; ++e) last = std::max(last, lev[dn_list[e]]);
          if (last >= 0) {
            occ[lev[c]]++;
            occ[last + 1]--;
          }
        }
        int32_t run = 0, mx = 0;
        for (int l = 0; l < nl; ++l) mx = std::max(mx, run += occ[l]);
        return mx;
      };
      if (tilt) {
        int nl0 = relevel(0.0, best);
        int32_t live_best = live_of(best, nl0);
        int nl_best = nl0;
        if (live_best > tilt_live) {
          for (double slope : kTiltSlopes) {
            const int nl = relevel(slope, cand);
            if (nl > level_cap) break;
            const int32_t lv = live_of(cand, nl);
            if (lv < live_best || tilt_force) {
              live_best = lv;
              nl_best = nl;
              best.swap(cand);
            }
          }
        }
        std::copy(best.begin(), best.end(), level.begin());
        L = nl_best;
        // level lists (stable in topological order within a level)
        std::vector<int32_t> cnt(L + 1, 0);
        for (int64_t c = 0; c < N; ++c) cnt[level[c] + 1]++;
        for (int l = 0; l < L; ++l) cnt[l + 1] += cnt[l];
        o.lp.assign(cnt.begin(), cnt.end());
        std::vector<int32_t> reord(N);
        for (int64_t p = 0; p < N; ++p) reord[cnt[level[order[p]]]++] = order[p];
        order.swap(reord);
      }
      // ---- push producers down to just before their first consumer (as
      // late as possible), visiting cells in reverse level order: a value then
      // lives in the ring for fewer levels, and the dependency order is kept
      // because every consumer's final level is already fixed
      {
        for (int64_t p = N - 1; p >= 0; --p) {
          const int32_t u = order[p];
          int32_t first = INT32_MAX;
          for (int k = 0; k < nfc; ++k) {
            const int64_t h = (int64_t)u * nfc + k;
            const int64_t v = m.nb[h];
            if (v < 0 || fcls[h] <= 0 || lagged[m.twin[h]]) continue;
            first = std::min(first, level[v]);
          }
          if (first != INT32_MAX && first - 1 > level[u]) level[u] = first - 1;
        }
        // rebuild the level lists (stable in cell index within a level)
        std::vector<int32_t> cnt(L + 1, 0);
        for (int64_t c = 0; c < N; ++c) cnt[level[c] + 1]++;
        for (int l = 0; l < L; ++l) cnt[l + 1] += cnt[l];
        for (int l = 0; l <= L; ++l) o.lp[l] = cnt[l];
        for (int64_t c = 0; c < N; ++c) order[cnt[level[c]]++] = (int32_t)c;
        o.max_width = 0;
        for (int l = 0; l < L; ++l) o.max_width = std::max(o.max_width, o.lp[l + 1] - o.lp[l]);
      }
      // ---- ring slots
      std::fill(last_use.begin(), last_use.end(), -1);
      for (int64_t c = 0; c < N; ++c)
        for (int k = 0; k < nfc; ++k) {
          const int64_t h = c * nfc + k;
          const int64_t v = m.nb[h];
          if (v < 0 || fcls[h] <= 0) continue;
          if (lagged[m.twin[h]]) continue;
          last_use[c] = std::max(last_use[c], level[v]);
        }
      // cells whose slot frees at each level (counting sort by that level,
      // cell order kept within one)
      rel_off.assign(L + 2, 0);
      for (int64_t c = 0; c < N; ++c)
        if (last_use[c] >= 0) rel_off[(last_use[c] + 1 <= L ? last_use[c] + 1 : L) + 1]++;
      for (int l = 0; l <= L; ++l) rel_off[l + 1] += rel_off[l];
      rel_cells.resize(rel_off[L + 1]);
      rel_fill.assign(rel_off.begin(), rel_off.end() - 1);
      for (int64_t c = 0; c < N; ++c)
        if (last_use[c] >= 0) rel_cells[rel_fill[last_use[c] + 1 <= L ? last_use[c] + 1 : L]++] = (int32_t)c;
      free_slots.clear();
      int32_t next_new = 1;   // slot 0 is the permanent zero slot
      for (int l = 0; l < L; ++l) {
        for (int32_t e = rel_off[l]; e < rel_off[l + 1]; ++e) {
          const int32_t c = rel_cells[e];
          free_slots.push_back(slot[c]);
          std::push_heap(free_slots.begin(), free_slots.end(), std::greater<int32_t>());
        }
        for (int32_t p = o.lp[l]; p < o.lp[l + 1]; ++p) {
          const int32_t c = order[p];
          if (last_use[c] >= 0) {
            if (!free_slots.empty()) {
              std::pop_heap(free_slots.begin(), free_slots.end(), std::greater<int32_t>());
              slot[c] = free_slots.back();
              free_slots.pop_back();
            } else {
              slot[c] = next_new++;
            }
          } else {
            slot[c] = -1;
          }
        }
      }
      o.n_slots = next_new - 1;
      // ---- exports: outgoing wall faces and upstream ends of lagged faces
      std::fill(exp_local.begin(), exp_local.end(), -1);
      o.exp_cells.clear();
      std::vector<char> is_exp(N, 0);
      for (int64_t h : bhf)
        if (fcls[h] > 0) is_exp[h / nfc] = 1;
      for (int64_t h = 0; h < H; ++h)
        if (lagged[h]) is_exp[m.nb[h]] = 1;
      for (int64_t c = 0; c < N; ++c)
        if (is_exp[c]) {
          exp_local[c] = (int32_t)o.exp_cells.size();
          o.exp_cells.push_back((int32_t)c);
        }
      // ---- records in level order, imports on first use
      o.imps.clear();
      const size_t base = (size_t)i * N;
      for (int32_t p = 0; p < (int32_t)N; ++p) {
        const int32_t c = order[p];
        P.pos_cell[base + p] = c;
        P.pos_slot[base + p] = slot[c];
        P.pos_exp[base + p] = exp_local[c];
        if (kChecks) P.pos_last[base + p] = last_use[c];
        double G = 0.0;
        int kk = 0;
        for (int k = 0; k < nfc; ++k) {
          const int64_t h = (int64_t)c * nfc + k;
          const double a = dotsa(i, h);
          const int cl = cls(a, h);
          if (cl >= 0) continue;
          G -= a;   // G = sum over inflow faces of |s.An| (= outflow sum for a closed cell)
          int32_t ref;
          if (m.nb[h] >= 0 && !lagged[h]) {
            ref = slot[m.nb[h]];
            if (ref < 1) { o.error = "internal: upstream cell without a ring slot"; return; }
          } else {
            LocalImport im{};
            if (m.nb[h] >= 0) {
              im.kind = IMP_LAG;
              im.src_dir = i;
              im.src_cell = (int32_t)m.nb[h];
            } else {
              const BC& b = bcmap.at(m.tag[h]);
              im.dbf = dbf_of_h[h];
              if (b.type == NBTE_THERMALIZING) {
                im.kind = IMP_THERM;
                im.par = b.T_wall - T_ref;
              } else if (b.type == NBTE_DIFFUSE) {
                im.kind = IMP_DIFFUSE;
              } else {
                im.kind = b.type == NBTE_SPECULAR ? IMP_SPECULAR : IMP_PARTIAL;
                im.par = b.p;
                im.src_dir = (*mirror_of_h[h])[i];
                im.src_cell = c;
                if (im.src_dir < 0) { o.error = "no direction leaves through a specular wall"; return; }
              }
            }
            ref = -(1 + (int32_t)o.imps.size());
            if (m.nb[h] < 0) o.bimp.emplace_back(h, (int32_t)o.imps.size());
            o.imps.push_back(im);
          }
          if (kk >= K) { o.error = "internal: more inflow faces than K"; return; }
          P.pos_ref[((size_t)i * K + kk) * N + p] = ref;
          P.pos_coef[((size_t)i * K + kk) * N + p] = -a / m.V[c];
          ++kk;
        }
        P.pos_G[base + p] = G / m.V[c];
      }
      std::sort(o.bimp.begin(), o.bimp.end());
    }
  };
  n_threads = std::max(1, std::min(n_threads, D));
  for (int pass = tilt ? 0 : 1; pass < 2; ++pass) {
    std::vector<std::thread> th;
    for (int t = 1; t < n_threads; ++t) th.emplace_back(work, t, n_threads, pass);
    work(0, n_threads, pass);
    for (auto& t : th) t.join();
    if (pass == 0) level_cap = *std::max_element(untilted_levels.begin(), untilted_levels.end());
  }
  for (auto& o : outs)
    if (!o.error.empty()) return Status::err(NBTE_ERR_MESH, o.error);

  // ---- flatten per-direction results
  P.lvl_off.assign(D + 1, 0);
  P.exp_off.assign(D + 1, 0);
  P.imp_off.assign(D + 1, 0);
  P.n_slots.resize(D);
  P.max_width.resize(D);
  for (int i = 0; i < D; ++i) {
    const DirOut& o = outs[i];
    P.lvl_off[i + 1] = P.lvl_off[i] + (int64_t)o.lp.size();
    P.exp_off[i + 1] = P.exp_off[i] + (int64_t)o.exp_cells.size();
    P.imp_off[i + 1] = P.imp_off[i] + (int64_t)o.imps.size();
    P.n_slots[i] = o.n_slots;
    P.max_width[i] = o.max_width;
    P.lagged_faces += o.lagged;
    const int L = (int)o.lp.size() - 1;
    P.total_levels += L;
    P.max_levels = std::max(P.max_levels, L);
    P.max_slots = std::max(P.max_slots, o.n_slots);
    P.max_width_all = std::max(P.max_width_all, o.max_width);
  }
  P.level_ptr.resize(P.lvl_off[D]);
  P.exp_cell.resize(P.exp_off[D]);
  for (int i = 0; i < D; ++i) {
    std::copy(outs[i].lp.begin(), outs[i].lp.end(), P.level_ptr.begin() + P.lvl_off[i]);
    std::copy(outs[i].exp_cells.begin(), outs[i].exp_cells.end(), P.exp_cell.begin() + P.exp_off[i]);
  }
  auto export_index = [&](int dir, int32_t cell) -> int64_t {
    const auto& v = outs[dir].exp_cells;
    auto it = std::lower_bound(v.begin(), v.end(), cell);
    if (it == v.end() || *it != cell) return -1;
    return P.exp_off[dir] + (it - v.begin());
  };
  const int64_t n_imp = P.imp_off[D];
  P.imp_kind.resize(n_imp);
  P.imp_dbf.resize(n_imp);
  P.imp_src.resize(n_imp);
  P.imp_par.resize(n_imp);
  for (int i = 0; i < D; ++i)
    for (size_t k = 0; k < outs[i].imps.size(); ++k) {
      const LocalImport& im = outs[i].imps[k];
      const int64_t x = P.imp_off[i] + (int64_t)k;
      P.imp_kind[x] = im.kind;
      P.imp_dbf[x] = im.dbf;
      P.imp_par[x] = im.par;
      P.imp_src[x] = -1;
      if (im.kind == IMP_SPECULAR || im.kind == IMP_PARTIAL || im.kind == IMP_LAG) {
        P.imp_src[x] = export_index(im.src_dir, im.src_cell);
        if (P.imp_src[x] < 0) return Status::err(NBTE_ERR_MESH, "internal: missing export for a wall/lag import");
      }
    }

  // ---- diffuse re-emission weights per diffuse/partial face
  P.dif_ptr.assign(dbf_h.size() + 1, 0);
  for (size_t f = 0; f < dbf_h.size(); ++f) {
    const int64_t h = dbf_h[f];
    double n[3];
    unit_normal(h, n);
    double denom = 0.0;
    for (int j = 0; j < D; ++j) {
      const double sn = s[j * 3] * n[0] + s[j * 3 + 1] * n[1] + s[j * 3 + 2] * n[2];
      if (cls(dotsa(j, h), h) < 0) denom += w[j] * (-sn);
    }
    for (int j = 0; j < D; ++j) {
      if (cls(dotsa(j, h), h) <= 0) continue;
      const double sn = s[j * 3] * n[0] + s[j * 3 + 1] * n[1] + s[j * 3 + 2] * n[2];
      const int64_t e = export_index(j, (int32_t)(h / nfc));
      if (e < 0) return Status::err(NBTE_ERR_MESH, "internal: missing export for a diffuse wall");
      P.dif_src.push_back(e);
      P.dif_wt.push_back(w[j] * sn / denom);
    }
    P.dif_ptr[f + 1] = (int64_t)P.dif_src.size();
  }

  // ---- wall heat table: every boundary half-face, every non-tangent
  // direction: the upwind value on the face (export when leaving, import when
  // entering) and its weight w_i (s_i . An)
  P.wf_ptr.assign(1, 0);
  for (int64_t h : bhf) {
    const int64_t c = h / nfc;
    P.wf_tag.push_back(m.tag[h]);
    P.wf_cell.push_back((int32_t)c);
    for (int i = 0; i < D; ++i) {
      const double a = dotsa(i, h);
      const int cl = cls(a, h);
      if (cl == 0) continue;
      int64_t val;
      if (cl > 0) {
        val = export_index(i, (int32_t)c);
        if (val < 0) return Status::err(NBTE_ERR_MESH, "internal: missing wall export");
      } else {
        const auto& v = outs[i].bimp;
        auto it = std::lower_bound(v.begin(), v.end(), std::make_pair(h, (int32_t)INT32_MIN));
        if (it == v.end() || it->first != h) return Status::err(NBTE_ERR_MESH, "internal: missing wall import");
        val = -(1 + (P.imp_off[i] + it->second));
      }
      P.wf_val.push_back(val);
      P.wf_coef.push_back(w[i] * a);
    }
    P.wf_ptr.push_back((int64_t)P.wf_val.size());
  }
  return Status::ok();
}

void build_laplacian(const Mesh& m, const std::vector<BC>& bcs, double kappa_bulk, double k1, Laplacian& L) {
  const int dim = m.dim, nfc = m.nfc;
  const int64_t N = m.n_cells;
  std::map<int32_t, int> type;
  std::map<int32_t, double> twall;
  for (auto& b : bcs) {
    type[b.tag] = b.type;
    twall[b.tag] = b.T_wall;
  }
  L.row_ptr.assign(N + 1, 0);
  L.col.clear();
  L.val.clear();
  L.diag.assign(N, 0.0);
  L.bc_g.assign(N, 0.0);
  L.bc_gT.assign(N, 0.0);
  for (int64_t c = 0; c < N; ++c) {
    double dg = 0.0;
    for (int k = 0; k < nfc; ++k) {
      const int64_t h = c * nfc + k;
      double area = 0;
      for (int d = 0; d < dim; ++d) area += m.An[h * dim + d] * m.An[h * dim + d];
      area = std::sqrt(area);
      const int64_t v = m.nb[h];
      if (v >= 0) {
        double dist = 0;
        for (int d = 0; d < dim; ++d) dist += (m.xc[v * dim + d] - m.xc[c * dim + d]) * m.An[h * dim + d] / area;
        dist = std::fabs(dist);
        const double g = (kappa_bulk + k1 * dist) * area / dist;
        dg += g;
        L.col.push_back((int32_t)v);
        L.val.push_back(-g);
      } else if (type.at(m.tag[h]) == NBTE_THERMALIZING) {
        double dist = 0;
        for (int d = 0; d < dim; ++d) dist += (m.xf[h * dim + d] - m.xc[c * dim + d]) * m.An[h * dim + d] / area;
        dist = std::fabs(dist);
        const double gw = (kappa_bulk + k1 * 2.0 * dist) * area / dist;
        dg += gw;
        L.bc_g[c] += gw;
        L.bc_gT[c] += gw * twall.at(m.tag[h]);
      }
    }
    L.col.push_back((int32_t)c);
    L.val.push_back(dg);
    L.diag[c] = dg;
    L.row_ptr[c + 1] = (int64_t)L.col.size();
  }
}

namespace {
// eigenvalues lam and eigenvectors (columns of U, row-major) of a symmetric
// n x n matrix (n <= 3) by cyclic Jacobi rotations
void sym_eigen(int n, double A[3][3], double lam[3], double U[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) U[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i][j] * A[i][j];
        if (i != j) off += A[i][j] * A[i][j];
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (A[p][q] == 0.0) continue;
        // rotation angle that zeroes A[p][q]
        const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {   // A <- A J
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - sn * akq;
          A[k][q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // A <- J^T A
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - sn * aqk;
          A[q][k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {   // U <- U J
          const double ukp = U[k][p], ukq = U[k][q];
          U[k][p] = c * ukp - sn * ukq;
          U[k][q] = sn * ukp + c * ukq;
        }
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[i][i];
}
}  // namespace

void build_reconstruction(const Mesh& m, Reconstruction& rc) {
  const int64_t N = m.n_cells;
  const int nf = m.nfc, dim = m.dim;
  rc.nb.assign((size_t)N * nf, -1);
  rc.twin.assign((size_t)N * nf, -1);
  rc.AnV.assign((size_t)N * nf * 3, 0.0);
  rc.a.assign((size_t)N * nf * nf, 0.0);
  rc.gw.assign((size_t)N * nf * 3, 0.0);
  rc.rf.assign((size_t)N * nf * 3, 0.0);
  rc.cells_with_gradient = 0;
  for (int64_t c = 0; c < N; ++c) {
    int n_nb = 0;
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double r[6][3] = {};
    for (int k = 0; k < nf; ++k) {
      const int64_t h = c * nf + k;
      for (int d = 0; d < dim; ++d) rc.AnV[h * 3 + d] = m.An[h * dim + d] / m.V[c];
      for (int d = 0; d < dim; ++d) rc.rf[h * 3 + d] = m.xf[h * dim + d] - m.xc[c * dim + d];
      const int64_t nk = m.nb[h];
      if (nk < 0) continue;
      rc.nb[h] = (int32_t)nk;
      rc.twin[h] = (int32_t)(m.twin[h] - nk * nf);
      ++n_nb;
      for (int d = 0; d < dim; ++d) r[k][d] = m.xc[nk * dim + d] - m.xc[c * dim + d];
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) M[i][j] += r[k][i] * r[k][j];
    }
    // exactly determined stencils (fewer than dim + 1 neighbours) get no gradient
    if (n_nb < dim + 1) continue;
    double lam[3], U[3][3];
    sym_eigen(dim, M, lam, U);
    double lmax = 0.0;
    for (int i = 0; i < dim; ++i) lmax = std::max(lmax, lam[i]);
    // P = pseudo-inverse of M (eigenvalues at or below 1e-9 lmax dropped)
    double P[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int e = 0; e < dim; ++e) {
      if (!(lam[e] > 1e-9 * lmax)) continue;
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) P[i][j] += U[i][e] * U[j][e] / lam[e];
    }
    ++rc.cells_with_gradient;
    for (int mm = 0; mm < nf; ++mm) {
      if (m.nb[c * nf + mm] < 0) continue;
      double g[3] = {0, 0, 0};   // P r_m
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) g[i] += P[i][j] * r[mm][j];
      for (int d = 0; d < dim; ++d) rc.gw[((size_t)c * nf + mm) * 3 + d] = g[d];
      for (int k = 0; k < nf; ++k) {
        const int64_t h = c * nf + k;
        double w = 0.0;
        for (int d = 0; d < dim; ++d) w += g[d] * (m.xf[h * dim + d] - m.xc[c * dim + d]);
        rc.a[(size_t)h * nf + mm] = w;
      }
    }
  }
}

}  // namespace nbte
