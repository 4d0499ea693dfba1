// Mesh building: faces, outward face vectors, volumes, centroids, boundary
// tags, and the internal (Morton) cell order.
//
// The finite-volume geometry follows the paper's "cell-face connectivity ...
// constructed once from the mesh" (Sec. II, after Eq. (13)).
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>

#include "nbte_internal.h"

namespace nbte {

namespace {

struct LocalFaces {
  int nfc, nvf;
  int f[6][4];
};

bool local_faces(int ct, LocalFaces& lf, int& nvc, int& dim) {
  switch (ct) {
    case NBTE_TRI: lf = {3, 2, {{0, 1}, {1, 2}, {2, 0}}}; nvc = 3; dim = 2; return true;
    case NBTE_QUAD: lf = {4, 2, {{0, 1}, {1, 2}, {2, 3}, {3, 0}}}; nvc = 4; dim = 2; return true;
    case NBTE_TET: lf = {4, 3, {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}}}; nvc = 4; dim = 3; return true;
    case NBTE_HEX:
      lf = {6, 4, {{0, 3, 2, 1}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}}};
      nvc = 8; dim = 3; return true;
    default: return false;
  }
}

inline uint64_t spread2(uint64_t x) {  // 32 -> interleave with zeros (2D)
  x &= 0xffffffffull;
  x = (x | (x << 16)) & 0x0000ffff0000ffffull;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

inline uint64_t spread3(uint64_t x) {  // 21 bits -> every third bit (3D)
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

struct FaceKey {
  std::array<int64_t, 4> k;
  int64_t hf;
  bool operator<(const FaceKey& o) const { return k < o.k || (k == o.k && hf < o.hf); }
};

}  // namespace

Status build_mesh(int dim, int64_t n_nodes, const double* xyz, int cell_type, int64_t n_cells,
                  const int64_t* cell_nodes, int64_t n_bfaces, const int64_t* bface_nodes,
                  const int32_t* bface_tag, Mesh& m) {
  LocalFaces lf;
  int nvc = 0, cdim = 0;
  if (!local_faces(cell_type, lf, nvc, cdim)) return Status::err(NBTE_ERR_ARG, "unknown cell_type");
  if (dim != cdim) return Status::err(NBTE_ERR_ARG, "dim does not match cell_type");
  if (n_nodes <= 0 || n_cells <= 0 || n_bfaces < 0)
    return Status::err(NBTE_ERR_ARG, "n_nodes and n_cells must be positive, n_bfaces >= 0");
  if (!xyz || !cell_nodes || (n_bfaces > 0 && (!bface_nodes || !bface_tag)))
    return Status::err(NBTE_ERR_ARG, "null array");
  if (n_cells > (int64_t)INT32_MAX / 8) return Status::err(NBTE_ERR_ARG, "too many cells");
  for (int64_t i = 0; i < n_nodes * dim; ++i)
    if (!std::isfinite(xyz[i])) return Status::err(NBTE_ERR_ARG, "non-finite node coordinate");
  for (int64_t i = 0; i < n_cells * nvc; ++i)
    if (cell_nodes[i] < 0 || cell_nodes[i] >= n_nodes) return Status::err(NBTE_ERR_MESH, "cell node index out of range");
  for (int64_t i = 0; i < n_bfaces * lf.nvf; ++i)
    if (bface_nodes[i] < 0 || bface_nodes[i] >= n_nodes) return Status::err(NBTE_ERR_MESH, "boundary face node index out of range");

  m.dim = dim; m.cell_type = cell_type; m.nvc = nvc; m.nfc = lf.nfc; m.nvf = lf.nvf;
  m.n_nodes = n_nodes; m.n_cells = n_cells; m.n_bfaces = n_bfaces;
  const int64_t N = n_cells;

  // ---- internal order: Morton code of the vertex-average centroid
  std::vector<double> cu(N * dim, 0.0);
  for (int64_t c = 0; c < N; ++c)
    for (int a = 0; a < nvc; ++a)
      for (int d = 0; d < dim; ++d) cu[c * dim + d] += xyz[cell_nodes[c * nvc + a] * dim + d] / nvc;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t c = 0; c < N; ++c)
    for (int d = 0; d < dim; ++d) { lo[d] = std::min(lo[d], cu[c * dim + d]); hi[d] = std::max(hi[d], cu[c * dim + d]); }
  double ext = 0;
  for (int d = 0; d < dim; ++d) ext = std::max(ext, hi[d] - lo[d]);
  if (!(ext > 0)) ext = 1.0;
  std::vector<uint64_t> code(N);
  const double scale = (dim == 2 ? 4294967295.0 : 2097151.0) / ext;
  for (int64_t c = 0; c < N; ++c) {
    uint64_t q[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) q[d] = (uint64_t)std::llround((cu[c * dim + d] - lo[d]) * scale);
    code[c] = dim == 2 ? (spread2(q[0]) | (spread2(q[1]) << 1))
                       : (spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2));
  }
  m.perm.resize(N);
  std::iota(m.perm.begin(), m.perm.end(), 0);
  std::stable_sort(m.perm.begin(), m.perm.end(), [&](int64_t a, int64_t b) { return code[a] < code[b]; });
  m.iperm.resize(N);
  for (int64_t c = 0; c < N; ++c) m.iperm[m.perm[c]] = c;

  // ---- half faces and their neighbours
  const int nfc = lf.nfc, nvf = lf.nvf;
  const int64_t H = N * nfc;
  std::vector<FaceKey> keys(H);
  auto face_node = [&](int64_t c, int k, int a) { return cell_nodes[m.perm[c] * nvc + lf.f[k][a]]; };
  for (int64_t c = 0; c < N; ++c)
    for (int k = 0; k < nfc; ++k) {
      FaceKey& fk = keys[c * nfc + k];
      fk.k = {-1, -1, -1, -1};
      for (int a = 0; a < nvf; ++a) fk.k[a] = face_node(c, k, a);
      std::sort(fk.k.begin(), fk.k.begin() + nvf);
      fk.hf = c * nfc + k;
    }
  std::sort(keys.begin(), keys.end());
  m.nb.assign(H, -1);
  for (int64_t i = 0; i < H;) {
    int64_t j = i + 1;
    while (j < H && keys[j].k == keys[i].k) ++j;
    if (j - i > 2) return Status::err(NBTE_ERR_MESH, "a face is shared by more than two cells");
    if (j - i == 2) {
      m.nb[keys[i].hf] = keys[i + 1].hf / nfc;
      m.nb[keys[i + 1].hf] = keys[i].hf / nfc;
    }
    i = j;
  }

  // ---- boundary tags
  std::vector<FaceKey> bkeys(n_bfaces);
  for (int64_t b = 0; b < n_bfaces; ++b) {
    bkeys[b].k = {-1, -1, -1, -1};
    for (int a = 0; a < nvf; ++a) bkeys[b].k[a] = bface_nodes[b * nvf + a];
    std::sort(bkeys[b].k.begin(), bkeys[b].k.begin() + nvf);
    bkeys[b].hf = b;
  }
  std::sort(bkeys.begin(), bkeys.end());
  for (int64_t b = 1; b < n_bfaces; ++b)
    if (bkeys[b].k == bkeys[b - 1].k) return Status::err(NBTE_ERR_MESH, "duplicate boundary face");
  m.tag.assign(H, 0);
  std::vector<char> used(n_bfaces, 0);
  std::vector<int32_t> present;
  for (int64_t h = 0; h < H; ++h) {
    if (m.nb[h] >= 0) continue;
    FaceKey q;
    q.k = {-1, -1, -1, -1};
    for (int a = 0; a < nvf; ++a) q.k[a] = face_node(h / nfc, (int)(h % nfc), a);
    std::sort(q.k.begin(), q.k.begin() + nvf);
    q.hf = -1;
    auto it = std::lower_bound(bkeys.begin(), bkeys.end(), q);
    if (it == bkeys.end() || it->k != q.k) return Status::err(NBTE_ERR_MESH, "untagged exterior face");
    used[it->hf] = 1;
    m.tag[h] = bface_tag[it->hf];
    present.push_back(m.tag[h]);
  }
  for (int64_t b = 0; b < n_bfaces; ++b)
    if (!used[b]) return Status::err(NBTE_ERR_MESH, "a tagged boundary face is not an exterior face");
  std::sort(present.begin(), present.end());
  present.erase(std::unique(present.begin(), present.end()), present.end());
  m.tags_present = present;

  // ---- geometry
  m.xc.assign(N * dim, 0.0);
  m.V.assign(N, 0.0);
  m.An.assign(H * dim, 0.0);
  m.xf.assign(H * dim, 0.0);
  m.volume = 0.0;
  for (int64_t c = 0; c < N; ++c) {
    for (int d = 0; d < dim; ++d) m.xc[c * dim + d] = cu[m.perm[c] * dim + d];
    double vol = 0.0;
    for (int k = 0; k < nfc; ++k) {
      const int64_t h = c * nfc + k;
      double P[4][3] = {};
      for (int a = 0; a < nvf; ++a)
        for (int d = 0; d < dim; ++d) P[a][d] = xyz[face_node(c, k, a) * dim + d];
      double xf[3] = {0, 0, 0}, A[3] = {0, 0, 0};
      for (int a = 0; a < nvf; ++a)
        for (int d = 0; d < dim; ++d) xf[d] += P[a][d] / nvf;
      if (dim == 2) {
        A[0] = P[1][1] - P[0][1];
        A[1] = -(P[1][0] - P[0][0]);
      } else {
        double u[3], v[3];
        if (nvf == 3) {
          for (int d = 0; d < 3; ++d) { u[d] = P[1][d] - P[0][d]; v[d] = P[2][d] - P[0][d]; }
        } else {
          for (int d = 0; d < 3; ++d) { u[d] = P[2][d] - P[0][d]; v[d] = P[3][d] - P[1][d]; }
        }
        A[0] = 0.5 * (u[1] * v[2] - u[2] * v[1]);
        A[1] = 0.5 * (u[2] * v[0] - u[0] * v[2]);
        A[2] = 0.5 * (u[0] * v[1] - u[1] * v[0]);
      }
      double dot = 0, na = 0, nr = 0;
      for (int d = 0; d < dim; ++d) {
        const double r = xf[d] - m.xc[c * dim + d];
        dot += r * A[d];
        na += A[d] * A[d];
        nr += r * r;
      }
      if (dot < 0) {
        for (int d = 0; d < dim; ++d) A[d] = -A[d];
        dot = -dot;
      }
      if (!(dot > 1e-9 * std::sqrt(na * nr)))
        return Status::err(NBTE_ERR_MESH, "degenerate or non-convex cell (cell " +
                                              std::to_string(m.perm[c]) + ")");
      vol += dot / dim;
      for (int d = 0; d < dim; ++d) {
        m.An[h * dim + d] = A[d];
        m.xf[h * dim + d] = xf[d];
      }
    }
    m.V[c] = vol;
    m.volume += vol;
  }
  // the two half-faces of an interior face carry exactly opposite vectors, so
  // every direction classifies the face as outflow on one side and inflow on
  // the other (or as tangential on both)
  m.twin.assign(H, -1);
  for (int64_t i = 0; i + 1 < H; ++i) {
    if (keys[i].k != keys[i + 1].k) continue;
    const int64_t h1 = keys[i].hf, h2 = keys[i + 1].hf;
    m.twin[h1] = h2;
    m.twin[h2] = h1;
    for (int d = 0; d < dim; ++d) {
      m.An[h2 * dim + d] = -m.An[h1 * dim + d];
      m.xf[h2 * dim + d] = m.xf[h1 * dim + d];
    }
  }
  return Status::ok();
}

}  // namespace nbte
