// Data layouts shared by the host set-up code and the device kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#ifdef __CUDACC__
#define NBTE_HD __host__ __device__
#else
#define NBTE_HD
#endif

namespace nbte {

// Wall/lag import and export tables: band-group major, every row padded to a
// multiple of 16 bytes so one work item's rows are one contiguous, aligned
// range (bulk-copy friendly).  Value of (entry x, band b) for n entries:
//   [(g * n + x) * Gpad + (b - g * G)],  g = b / G.
NBTE_HD inline size_t io_index(int64_t x, int b, int64_t n, int G, int Gpad) {
  const int g = b / G;
  return ((size_t)g * (size_t)n + (size_t)x) * (size_t)Gpad + (size_t)(b - g * G);
}

NBTE_HD constexpr int padded_group(int G, int elem_bytes) {
  const int per16 = 16 / elem_bytes;
  return ((G + per16 - 1) / per16) * per16;
}

// Packed position record (one per direction and position, level order):
//   int32 cell, int32 slot, int32 export, [pad], R G, int32 ref[K], [pad], R coef[K]
// padded to an ODD multiple of 16 bytes: a warp reads records of consecutive
// positions with 16-byte shared-memory loads, eight threads per wavefront,
// and an odd stride (in 16-byte units) puts those eight in distinct banks.
struct RecLayout {
  int size, off_G, off_ref, off_coef;
};

NBTE_HD constexpr RecLayout rec_layout(int elem_bytes, int K) {
  RecLayout L{0, 0, 0, 0};
  int off = 12;
  off = (off + elem_bytes - 1) / elem_bytes * elem_bytes;
  L.off_G = off;
  off += elem_bytes;
  L.off_ref = off;
  off += 4 * K;
  off = (off + elem_bytes - 1) / elem_bytes * elem_bytes;
  L.off_coef = off;
  off += elem_bytes * K;
  int n16 = (off + 15) / 16;
  if (n16 % 2 == 0) ++n16;
  L.size = 16 * n16;
  return L;
}

// Bytes of a chunk's (T', Qdot) pairs behind its records, padded to 16 (the
// next chunk's block starts 16-byte aligned; records are multiples of 16).
NBTE_HD constexpr unsigned chunk_tq_bytes(int len, int elem_bytes) {
  return (unsigned)((len * 2 * elem_bytes + 15) / 16 * 16);
}

// A chunk: up to CAP consecutive positions of one direction, either whole
// consecutive levels or a piece of one level wider than CAP.
struct Chunk {
  int32_t pos;       // first position (relative to the direction)
  int32_t len;       // positions
  int32_t imp;       // first import (relative to the direction)
  int32_t nimp_end;  // bits 0-15: imports in the chunk; bits 16-29: levels in the
                     // chunk; bit 30: the chunk ends a level
};
constexpr int kChunkMaxImports = 0xffff;
constexpr int kChunkMaxLevels = 0x3fff;
NBTE_HD constexpr int32_t chunk_flags(int n_imports, int n_levels, bool level_end) {
  return (int32_t)(n_imports | (n_levels << 16) | (level_end ? (1 << 30) : 0));
}
NBTE_HD constexpr int chunk_imports(int32_t f) { return f & 0xffff; }
NBTE_HD constexpr int chunk_levels(int32_t f) { return (f >> 16) & 0x3fff; }
NBTE_HD constexpr bool chunk_level_end(int32_t f) { return (f & (1 << 30)) != 0; }
// A chunk block starts with a header: int32 level count, then each level's
// end (relative to the chunk's first position), padded to 16 bytes.
NBTE_HD constexpr unsigned chunk_header_bytes(int n_levels) {
  return (unsigned)(((n_levels + 1) * 4 + 15) / 16 * 16);
}

}  // namespace nbte
