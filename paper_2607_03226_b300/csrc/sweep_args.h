// Arguments of the transport sweep kernels and the device error codes their
// bounded waits report (internal; no torch types).
#pragma once

#include <cstdint>

#include "layout.h"

namespace nbte {

// device error word values (written by bounded waits, read by the host)
enum DevError : int32_t { DEV_OK = 0, DEV_BARRIER_TIMEOUT = 1, DEV_QUEUE_TIMEOUT = 2, DEV_CHECK_FAILED = 3 };

// Polls of an mbarrier before a sweep wait gives up.  A poll that finds the
// phase incomplete suspends the thread for a few microseconds (measured about
// 3.9 us on B300), so this is about a second.  The bound is a compile-time
// constant: a run-time bound in the producer's wait loop made the 2D fin's
// sweep 1.8x slower (same-box A/B).
constexpr unsigned long long kSweepWaitPolls = 1ull << 18;

// shared-memory budget of one sweep CTA (the rest of the SM's 228 KB stays
// free for a second CTA when the ring is small)
constexpr int kSweepSmemMax = 227 * 1024;

template <typename R>
struct SweepArgs {
  int N, dim;
  int full;                      // also accumulate E and q (atomics): selects the output-sweep
                                 // kernel variant of launch_sweep; launch_sweep_batch ignores it
  int Gpad;                      // padded row length of the import/export tables
  int n_stages;                  // shared-memory stages of the copy pipeline
  int stage_bytes, off_ring, off_stage, off_imp, off_den, off_src2;   // shared-memory layout
  const R* dinv;                 // FP64 only: [n_items*N*G] denominators 1/(1/tau + v G), else null
  const R* src2;                 // second-order upwind: [n_items*N*G] per position, the
                                 // reconstruction's extra source (sum over faces), else null
  int64_t n_exp, n_imp;
  const int32_t* item_dir;       // [n_items] direction of the CTA's work item
  const int32_t* item_grp;       // [n_items] band group of the CTA's work item
  int n_groups;                  // band groups per direction: per-item tables (dinv, src2, part) are
                                 // indexed direction-major, i * n_groups + g
  const int64_t* chunk_off;      // [D+1]
  const Chunk* chunks;
  const unsigned char* rec;      // per chunk: its packed position records, then its (T', Qdot) pairs
  const int64_t* chunk_doff;     // [chunks] byte offset of each chunk's block in rec
  const int64_t* exp_off;        // [D+1]
  const int64_t* imp_off;
  const R* imp;                  // band-group-major import rows
  R* exp;                        // band-group-major export rows
  const R* band_v;               // [Bp]
  const R* band_inv_tau;
  const R* band_cw;              // C / W
  const R* band_aQ;              // C / (C_tot W)
  const double* dir_w;           // [D]
  const double* dir_s;           // [D*3]
  int item0;                     // first work item of the launch (block b runs item item0 + b)
  R* e_out;                      // null, or every cell's outgoing values of the item's bands at
                                 // e_out + i * e_out_dstride + g * e_out_gstride + cell * e_out_cstride
                                 // (written by second-order sweeps and by launch_sweep's
                                 // e_out variant; the first-order batched launch ignores it)
  int64_t e_out_dstride, e_out_gstride, e_out_cstride;   // (direction i, band group g)
  R* gring;                      // global-memory value rings, or null for the shared-memory ring
  int64_t gring_stride;          // elements per CTA's global ring
  R* part;                       // [n_items*N] collision-moment partials of e - e0 (deterministic
                                 // form), or null: then
  double* acc;                   // [N] the collision moment summed over every work item by FP64
                                 // atomic adds (the update kernel reads and clears it)
  double* accE;                  // [N]   (full)
  double* accQ;                  // [N*dim] (full)
  int32_t* err;                  // device error word
  int32_t hold_copies;           // nonzero: the producer issues no copy, so every consumer wait runs
                                 // out (the timeout test of nbte_test_timeouts)
  // consistency checks (NBTE_CHECKS builds only; null otherwise): per work
  // item and ring slot the level that last wrote the slot and the last level
  // that may read it, and per position the last level reading its value
  int32_t* chk_level;
  int32_t* chk_last;
  const int32_t* pos_last;       // [D*N]
  int32_t ring_slots;            // slots of one work item's value ring (zero slot included)
};

}  // namespace nbte
