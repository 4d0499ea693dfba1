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

// A chunk: up to CAP consecutive positions of one direction inside one level.
struct Chunk {
  int32_t pos;       // first position (relative to the direction)
  int32_t len;       // positions
  int32_t imp;       // first import (relative to the direction)
  int32_t nimp_end;  // number of imports in the chunk (low 30 bits); bit 30: last chunk of its level
};

}  // namespace nbte
