// The transport sweep (sm_103a): per (direction, band group) work item, the
// first-order upwind solve of Eq. (4) in the topological (level) order of the
// direction's upwind graph -- the triangular substitution of the factorised
// system of Eq. (13) -- fused with the collision moment of Eq. (5) and, on
// request, the energy and flux moments of Eq. (7).
//
// Warp-specialised pipeline, one CTA per work item:
//  * warp 0 (one elected lane) is the producer.  It walks the direction's
//    chunks (whole consecutive levels of at most CAP positions together, or a
//    piece of one wider level) and, several chunks ahead of the consumers,
//    bulk-copies (cp.async.bulk, completion counted on an mbarrier) each
//    chunk's block -- a header of level ends, the packed position records and
//    the pre-gathered (T', Qdot) pairs -- and its slice of wall/lag import
//    values into a ring of shared-memory stages;
//  * the other warps are consumers: they wait on a stage's "full" barrier,
//    compute one position per thread from shared memory and the value ring,
//    release the stage on its "empty" barrier, and meet on a named barrier
//    only at the end of a level (so the next level sees the ring writes).
// The value ring holds the outgoing values of the direction's live cells
// (slots assigned by the planner).  It lives in shared memory when it fits
// (GR = false); otherwise (GR = true, large 3D meshes whose sweep front has
// tens of thousands of live cells) in a per-CTA global-memory region, where
// the concurrently running CTAs' live windows stay mostly in L2.  Every wait
// is bounded (kSweepWaitPolls polls, about a second): on timeout the error
// word is set, a consumer warp any of whose lanes gave up stops computing
// but keeps the barrier sequence, the producer waits for the copies it
// issued, and the CTA leaves.
//
// Per cell and band the balance is solved for the deviation from the cell's
// own equilibrium e0 = C T'/W (Eq. (11)):
//   e = e0 + (Qdot C/(C_tot W) + v sum_in c_k (e_up,k - e0) + v src2) / (1/tau + v G),
//   c_k = |s.An_k|/V,  G = sum_in c_k  (= sum_out (s.An)/V for a closed cell),
// src2 = 0 for first-order upwind; with second-order face values it is the
// reconstruction increment of every interior face taken from the previous
// iteration's gradients (deferred correction, see launch_src2).
// Each position adds its collision-moment share sum_l w_i (e - e0)/tau_l to
// the cell's FP64 sum over all work items (one atomic add), or writes it as
// the (work item, cell) partial of the deterministic form; the equilibrium
// part sums to beta T' exactly and is added back in FP64 by the update kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "layout.h"
#include "vecio.cuh"

namespace nbte {

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait (at most kSweepWaitPolls polls, about a second); false on
// timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (unsigned long long k = 0; k < kSweepWaitPolls; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void consumer_barrier(int count) {
  asm volatile("bar.sync 1, %0;" ::"r"(count) : "memory");
}
// FP32: the hardware approximate reciprocal (relative error below 2^-22,
// under the FP32 sweep's own rounding); FP64: a correctly rounded division
__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// exact FP32 -> FP64 widening by the IEEE-754 field layout (8-bit exponent
// rebiased by 1023 - 127, 23-bit fraction shifted into the 52-bit one) in
// integer instructions: the conversion instruction would run on the FP64
// pipe, which has a small fraction of the FP32 rate on this part.  Zero and
// FP32 subnormals (below 1.2e-38, far under any collision moment) give a
// signed zero; infinities and NaNs keep their class.
__device__ __forceinline__ double widen(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t ex = (u >> 23) & 0xffu;
  const uint32_t sg = u & 0x80000000u;
  uint32_t hi = sg | ((ex + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  uint32_t lo = u << 29;
  if (ex == 0u) {
    hi = sg;
    lo = 0u;
  } else if (ex == 0xffu) {
    hi |= 0x7ff00000u;
  }
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen(double x) { return x; }

// word idx (4-byte units) of a record held in registers; idx is a
// compile-time constant after unrolling, so this folds to a register move
template <int NQ>
__device__ __forceinline__ uint32_t rec_word(const uint4 (&w)[NQ], int idx) {
  const uint4 v = w[idx >> 2];
  switch (idx & 3) {
    case 0: return v.x;
    case 1: return v.y;
    case 2: return v.z;
    default: return v.w;
  }
}
template <typename R>
struct RecField;
template <>
struct RecField<float> {
  template <int NQ>
  __device__ __forceinline__ static float get(const uint4 (&w)[NQ], int byte_off) {
    return __uint_as_float(rec_word(w, byte_off / 4));
  }
};
template <>
struct RecField<double> {
  template <int NQ>
  __device__ __forceinline__ static double get(const uint4 (&w)[NQ], int byte_off) {
    return __hiloint2double((int)rec_word(w, byte_off / 4 + 1), (int)rec_word(w, byte_off / 4));
  }
};

}  // namespace

// One work item (direction i, band group g) of one solver; the whole CTA.
// MODE selects the outputs beyond the collision moment: 0 none, 1 every
// outgoing value to e_out, 2 the energy and flux moments.  Second order
// always writes e_out (the next iteration's gradients read it).  They are
// compile-time switches: behind runtime flags the compiler evaluated their
// address arithmetic and FP64 products ahead of the branches, for every
// position of every sweep (the FP64 products on the FP64 pipe, a small
// fraction of the FP32 rate on this part).  The global-ring variants keep
// the e_out store behind its runtime null check: measured on the 1.14M-tet
// FinFET, their sweep is faster with it (38.3 against 43.1 ms).
template <typename R, int K, int G, bool GR, bool O2, int MODE>
__device__ __forceinline__ void sweep_item(const SweepArgs<R>& a, const int item, unsigned char* smem) {
  constexpr bool EOUT = O2 || MODE == 1 || GR;
  const int NS = a.n_stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + NS;
  Chunk* meta = reinterpret_cast<Chunk*>(smem + 16 * NS);
  R* ring = GR ? a.gring + (size_t)item * (size_t)a.gring_stride : reinterpret_cast<R*>(smem + a.off_ring);
  unsigned char* stages = smem + a.off_stage;
  constexpr RecLayout RL = rec_layout((int)sizeof(R), K);
  constexpr int NQ = RL.size / 16;
  constexpr int GP = padded_group(G, (int)sizeof(R));   // row length of the import/export tables

  const int i = a.item_dir[item];
  const int g = a.item_grp[item];
  const int64_t di = (int64_t)i * a.n_groups + g;   // direction-major index of the per-item tables
  const int ncons = blockDim.x - 32;
  const int64_t ch0 = a.chunk_off[i];
  const int nch = (int)(a.chunk_off[i + 1] - ch0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, ncons / 32);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (threadIdx.x < 32) {
    // ------------------------------------------------------------ producer
    if (a.hold_copies) return;   // timeout test: no copy, every consumer wait runs out
    // the warp fetches chunk descriptors 32 at a time, one batch ahead; lane
    // 0 waits for free stages and issues the copies
    const int lane = threadIdx.x;
    auto fetch = [&](int base) {
      int4 v = make_int4(0, 0, 0, 0);
      if (base + lane < nch) v = *reinterpret_cast<const int4*>(a.chunks + ch0 + base + lane);
      return v;
    };
    auto fetch_off = [&](int base) {
      return base + lane < nch ? a.chunk_doff[ch0 + base + lane] : (int64_t)0;
    };
    int4 cur = fetch(0), nxt = fetch(32);
    int64_t cur_off = fetch_off(0), nxt_off = fetch_off(32);
    int issued = 0;
    bool ok = true;
    // stage of chunk c and the parity of its round, kept incrementally (the
    // stage count is not a compile-time constant, so c % NS would divide)
    int sp = 0;
    unsigned php = 0;
    for (int c = 0; c < nch; ++c) {
      if (c > 0 && (c & 31) == 0) {
        cur = nxt;
        nxt = fetch(c + 32);
        cur_off = nxt_off;
        nxt_off = fetch_off(c + 32);
      }
      const int64_t doff = __shfl_sync(0xffffffffu, cur_off, c & 31);
      Chunk m;
      m.pos = __shfl_sync(0xffffffffu, cur.x, c & 31);
      m.len = __shfl_sync(0xffffffffu, cur.y, c & 31);
      m.imp = __shfl_sync(0xffffffffu, cur.z, c & 31);
      m.nimp_end = __shfl_sync(0xffffffffu, cur.w, c & 31);
      if (lane == 0) {
        const int s = sp;
        if (c >= NS && !mbar_wait(empty + s, php ^ 1u)) {
          atomicExch(a.err, (int32_t)DEV_QUEUE_TIMEOUT);
          ok = false;
        }
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) break;
      if (lane == 0) {
        const int s = sp;
        meta[s] = m;
        unsigned char* st = stages + (size_t)s * a.stage_bytes;
        // the chunk's header, records and (T', Qdot) pairs: one contiguous
        // block, one copy
        const unsigned rec_bytes = chunk_header_bytes(chunk_levels(m.nimp_end)) + (unsigned)(m.len * RL.size) +
                                   chunk_tq_bytes(m.len, (int)sizeof(R));
        const int nimp = chunk_imports(m.nimp_end);
        const unsigned imp_bytes = (unsigned)nimp * (unsigned)(a.Gpad * sizeof(R));
        // FP64: the chunk's denominators, a 16-byte aligned superset
        unsigned den_bytes = 0;
        int64_t da = 0;
        if constexpr (sizeof(R) == 8) {
          constexpr int dper16 = G == 1 ? 2 : 1;   // positions per 16 bytes
          const int64_t d0 = di * a.N + m.pos;
          da = d0 / dper16 * dper16;
          const int64_t de = (d0 + m.len + dper16 - 1) / dper16 * dper16;
          den_bytes = (unsigned)((de - da) * G * 8);
        }
        // second order: the chunk's reconstruction sources, a 16-byte aligned superset
        unsigned s2_bytes = 0;
        int64_t sa = 0;
        if constexpr (O2) {
          constexpr int sper16 = (int)(16 / (G * sizeof(R))) > 1 ? (int)(16 / (G * sizeof(R))) : 1;
          const int64_t s0 = di * a.N + m.pos;
          sa = s0 / sper16 * sper16;
          const int64_t se = (s0 + m.len + sper16 - 1) / sper16 * sper16;
          s2_bytes = (unsigned)((se - sa) * G * sizeof(R));
        }
        mbar_arrive_expect_tx(full + s, rec_bytes + imp_bytes + den_bytes + s2_bytes);
        bulk_copy(st, a.rec + doff, rec_bytes, full + s);
        if (den_bytes) bulk_copy(st + a.off_den, a.dinv + (size_t)da * G, den_bytes, full + s);
        if constexpr (O2) bulk_copy(st + a.off_src2, a.src2 + (size_t)sa * G, s2_bytes, full + s);
        if (nimp > 0)
          bulk_copy(st + a.off_imp, a.imp + ((size_t)g * a.n_imp + a.imp_off[i] + m.imp) * a.Gpad, imp_bytes,
                    full + s);
      }
      ++issued;
      if (++sp == NS) {
        sp = 0;
        php ^= 1u;
      }
    }
    // every copy issued must land before the CTA leaves
    if (lane == 0)
      for (int c = issued - NS > 0 ? issued - NS : 0; c < issued; ++c) mbar_wait(full + (c % NS), (c / NS) & 1);
    return;
  }

  // ------------------------------------------------------------ consumers
  const int ct = threadIdx.x - 32;
  for (int t = ct; t < G; t += ncons) ring[t] = R(0);   // zero slot
  const double wi = a.dir_w[i];
  const int band0 = g * G;
  R vb[G], itau[G], cw[G], aQ[G], wt[G];
#pragma unroll
  for (int b = 0; b < G; ++b) {
    vb[b] = a.band_v[band0 + b];
    itau[b] = a.band_inv_tau[band0 + b];
    cw[b] = a.band_cw[band0 + b];
    aQ[b] = a.band_aQ[band0 + b];
    wt[b] = (R)(wi * (double)itau[b]);
  }
  R* part = a.part ? a.part + di * a.N : nullptr;
  double* acc = a.acc;
  R* exp_g = a.exp + ((size_t)g * a.n_exp + a.exp_off[i]) * GP;
#ifdef NBTE_CHECKS
  // every slot of this item's ring: not written yet, no reader left
  const size_t chk0 = (size_t)item * a.ring_slots;
  for (int t = ct; t < a.ring_slots; t += ncons) {
    a.chk_level[chk0 + t] = -1;
    a.chk_last[chk0 + t] = -1;
  }
  const int64_t n_exp_i = a.exp_off[i + 1] - a.exp_off[i];
  int next_level = 0;        // level index of the next chunk's first level
#endif
  consumer_barrier(ncons);

  int sc = 0;          // stage of chunk c, and the parity of its round
  unsigned phc = 0;
  int c = 0;
  for (; c < nch; ++c) {
    const int s = sc;
    // a warp any of whose lanes' waits gave up leaves this loop (below)
    if (__any_sync(0xffffffffu, !mbar_wait(full + s, phc))) {
      if ((ct & 31) == 0) atomicExch(a.err, (int32_t)DEV_QUEUE_TIMEOUT);
      break;
    }
    const Chunk m = meta[s];
    const int n_lev = chunk_levels(m.nimp_end);
#ifdef NBTE_CHECKS
    const int level0 = next_level;
    next_level = level0 + n_lev - (chunk_level_end(m.nimp_end) ? 0 : 1);
    const int nimp_chunk = chunk_imports(m.nimp_end);
#endif
    const unsigned char* st = stages + (size_t)s * a.stage_bytes;
    // the block: header (level count, level ends), records, (T', Qdot) pairs
    const int32_t* lev_end = reinterpret_cast<const int32_t*>(st) + 1;
    const unsigned char* recs = st + chunk_header_bytes(n_lev);
    using R2 = typename Vec2<R>::T;
    const R2* tqs = reinterpret_cast<const R2*>(recs + (size_t)m.len * RL.size);
    const R* imps = reinterpret_cast<const R*>(st + a.off_imp);
    const int imp0 = m.imp;
    // FP64: this chunk's precomputed denominators (superset starts d_shift early)
    const R* dens = reinterpret_cast<const R*>(st + a.off_den);
    const int d_shift = sizeof(R) == 8 && G == 1 ? (int)((di * a.N + m.pos) % 2) : 0;
    // second order: this chunk's reconstruction sources (superset starts s_shift early)
    constexpr int sper16 = (int)(16 / (G * sizeof(R))) > 1 ? (int)(16 / (G * sizeof(R))) : 1;
    const R* s2 = reinterpret_cast<const R*>(st + a.off_src2);
    const int s_shift = O2 ? (int)((di * a.N + m.pos) % sper16) : 0;
    // the chunk's levels in order, a named barrier between them (each sees
    // the ring values the previous one wrote)
    int lb = 0;
    for (int lv = 0; lv < n_lev; ++lv) {
      const int le = lev_end[lv];
      for (int j = lb + ct; j < le; j += ncons) {
        uint4 w[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) w[q] = reinterpret_cast<const uint4*>(recs)[j * NQ + q];
        const int cell = (int)rec_word(w, 0);
        const int slot = (int)rec_word(w, 1);
        const int ex = (int)rec_word(w, 2);
        const R Gc = RecField<R>::get(w, RL.off_G);
#ifdef NBTE_CHECKS
        // indices in range, every upstream value written in an earlier level
        // and still owned by its cell, a slot reused only after its last reader
        {
          const int lvl = level0 + lv;
          bool bad = cell < 0 || cell >= a.N || slot < -1 || slot == 0 || slot >= a.ring_slots || ex < -1 ||
                     ex >= n_exp_i;
          for (int k = 0; k < K && !bad; ++k) {
            const int ref = (int)rec_word(w, RL.off_ref / 4 + k);
            if (ref >= a.ring_slots) bad = true;
            else if (ref > 0) bad = !(a.chk_level[chk0 + ref] >= 0 && a.chk_level[chk0 + ref] < lvl &&
                                      lvl <= a.chk_last[chk0 + ref]);
            else if (ref < 0) bad = (-1 - ref) - imp0 < 0 || (-1 - ref) - imp0 >= nimp_chunk;
          }
          if (!bad && slot > 0) bad = a.chk_last[chk0 + slot] >= lvl;
          if (bad) {
            atomicExch(a.err, (int32_t)DEV_CHECK_FAILED);
            continue;
          }
          if (slot > 0) {
            a.chk_level[chk0 + slot] = lvl;
            a.chk_last[chk0 + slot] = a.pos_last[(size_t)i * a.N + m.pos + j];
          }
        }
#endif
        const R2 tq = tqs[j];
        const R T = tq.x;
        const R Q = tq.y;
        R e0[G], up[G];
#pragma unroll
        for (int b = 0; b < G; ++b) {
          e0[b] = cw[b] * T;
          up[b] = R(0);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int ref = (int)rec_word(w, RL.off_ref / 4 + k);
          const R cf = RecField<R>::get(w, RL.off_coef + k * (int)sizeof(R));
          const R* src = ref >= 0 ? ring + ref * G : imps + ((-1 - ref) - imp0) * GP;
          R eu[G];
          load_vals<R, G>(src, eu);
#pragma unroll
          for (int b = 0; b < G; ++b) up[b] += cf * (eu[b] - e0[b]);
        }
        if constexpr (O2) {
#pragma unroll
          for (int b = 0; b < G; ++b) up[b] += s2[(j + s_shift) * G + b];
        }
        R e[G];
        R nl = R(0);
#pragma unroll
        for (int b = 0; b < G; ++b) {
          R den;
          if constexpr (sizeof(R) == 8) den = dens[(j + d_shift) * G + b];
          else den = recip(itau[b] + vb[b] * Gc);
          const R phi = (aQ[b] * Q + vb[b] * up[b]) * den;
          e[b] = e0[b] + phi;
          nl += wt[b] * phi;
        }
        if (slot >= 0) store_vals<R, G>(ring + slot * G, e);
        if (ex >= 0) store_vals<R, G>(exp_g + (size_t)ex * GP, e);
        if constexpr (EOUT) {
          if (a.e_out)
            store_vals<R, G>(a.e_out + (size_t)i * a.e_out_dstride + (size_t)g * a.e_out_gstride +
                                 (size_t)cell * a.e_out_cstride,
                             e);
        }
        // the collision moment of Eq. (5) (the output sweep, MODE 2, does not
        // need it): one FP64 atomic add per position into the cell's sum over
        // every (direction, band group), or, in the deterministic form, one
        // partial per (work item, cell) that the update kernel sums in a
        // fixed order
        if constexpr (MODE != 2) {
          if (part) part[cell] = nl;
          else atomicAdd(acc + cell, widen(nl));
        }
        // energy and flux moments, Eq. (7): the output sweep only
        if constexpr (MODE == 2) {
          R es = R(0), evs = R(0);
#pragma unroll
          for (int b = 0; b < G; ++b) {
            es += e[b];
            evs += vb[b] * e[b];
          }
          atomicAdd(a.accE + cell, wi * (double)es);
          for (int d = 0; d < a.dim; ++d)
            atomicAdd(a.accQ + (int64_t)cell * a.dim + d, wi * a.dir_s[i * 3 + d] * (double)evs);
        }
      }
      if (lv + 1 < n_lev) consumer_barrier(ncons);
      lb = le;
    }
    __syncwarp();
    if ((ct & 31) == 0) mbar_arrive(empty + s);
    if (chunk_level_end(m.nimp_end)) consumer_barrier(ncons);
    if (++sc == NS) {
      sc = 0;
      phc ^= 1u;
    }
  }
  // A warp whose wait gave up computes nothing more and releases no stage,
  // but keeps the barrier sequence of the remaining chunks (read from the
  // chunk descriptors in global memory), so no other consumer is left
  // waiting at a level barrier.
  for (; c < nch; ++c) {
    const Chunk m = a.chunks[ch0 + c];
    for (int lv = 0; lv + 1 < chunk_levels(m.nimp_end); ++lv) consumer_barrier(ncons);
    if (chunk_level_end(m.nimp_end)) consumer_barrier(ncons);
  }
}

template <typename R, int K, int G, bool GR, bool O2, int MODE>
__global__ void __launch_bounds__(544) sweep_kernel(const SweepArgs<R> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  sweep_item<R, K, G, GR, O2, MODE>(a, blockIdx.x + a.item0, smem);
}

// Work items of several solvers in one launch: block b runs item
// b - item_start[s] of solver s, item_start[s] <= b < item_start[s+1].  The
// solvers share (R, K, G, ring placement); each brings its own tables, value
// rings and shared-memory layout (the launch takes the largest).
template <typename R, int K, int G, bool GR, bool O2>
__global__ void __launch_bounds__(544) sweep_batch_kernel(const SweepArgs<R>* args, const int32_t* item_start,
                                                          int n_solvers) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ SweepArgs<R> sa;
  __shared__ int s_item;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n_solvers - 1;
    while (lo < hi) {   // last solver whose first item is <= blockIdx.x
      const int mid = (lo + hi + 1) / 2;
      if (item_start[mid] <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    sa = args[lo];
    s_item = (int)blockIdx.x - item_start[lo];
  }
  __syncthreads();
  sweep_item<R, K, G, GR, O2, 0>(sa, s_item, smem);
}

template <typename R, int K, int G, bool GR, bool O2>
static cudaError_t launch_one(const SweepArgs<R>& a, int n_items, int threads, size_t smem, cudaStream_t st) {
  auto kern = a.full ? sweep_kernel<R, K, G, GR, O2, 2> : sweep_kernel<R, K, G, GR, O2, 0>;
  if constexpr (!O2) {
    if (!a.full && a.e_out) kern = sweep_kernel<R, K, G, GR, O2, 1>;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_items, threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename R, int K, bool GR, bool O2>
static cudaError_t launch_k(const SweepArgs<R>& a, int G, int n_items, int threads, size_t smem, cudaStream_t st) {
  switch (G) {
    case 1: return launch_one<R, K, 1, GR, O2>(a, n_items, threads, smem, st);
    case 2: return launch_one<R, K, 2, GR, O2>(a, n_items, threads, smem, st);
    case 4: return launch_one<R, K, 4, GR, O2>(a, n_items, threads, smem, st);
    case 8:
      if constexpr (sizeof(R) == 4) return launch_one<R, K, 8, GR, O2>(a, n_items, threads, smem, st);
      return cudaErrorInvalidConfiguration;
    default:
      return cudaErrorInvalidConfiguration;
  }
}

template <typename R, bool GR, bool O2>
static cudaError_t launch_gr(const SweepArgs<R>& a, int K, int G, int n_items, int threads, size_t smem,
                             cudaStream_t st) {
  switch (K) {
    case 1: return launch_k<R, 1, GR, O2>(a, G, n_items, threads, smem, st);
    case 2: return launch_k<R, 2, GR, O2>(a, G, n_items, threads, smem, st);
    case 3: return launch_k<R, 3, GR, O2>(a, G, n_items, threads, smem, st);
    case 4: return launch_k<R, 4, GR, O2>(a, G, n_items, threads, smem, st);
    case 5: return launch_k<R, 5, GR, O2>(a, G, n_items, threads, smem, st);
    default: return cudaErrorInvalidConfiguration;
  }
}

template <typename R, int K, int G, bool GR, bool O2>
static cudaError_t launch_batch_one(const SweepArgs<R>* args, const int32_t* item_start, int n_solvers,
                                    int n_items, int threads, size_t smem, cudaStream_t st) {
  auto kern = sweep_batch_kernel<R, K, G, GR, O2>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_items, threads, smem, st>>>(args, item_start, n_solvers);
  return cudaGetLastError();
}

template <typename R, int K, bool GR, bool O2>
static cudaError_t launch_batch_k(const SweepArgs<R>* args, const int32_t* item_start, int n_solvers, int G,
                                  int n_items, int threads, size_t smem, cudaStream_t st) {
  switch (G) {
    case 1: return launch_batch_one<R, K, 1, GR, O2>(args, item_start, n_solvers, n_items, threads, smem, st);
    case 2: return launch_batch_one<R, K, 2, GR, O2>(args, item_start, n_solvers, n_items, threads, smem, st);
    case 4: return launch_batch_one<R, K, 4, GR, O2>(args, item_start, n_solvers, n_items, threads, smem, st);
    case 8:
      if constexpr (sizeof(R) == 4)
        return launch_batch_one<R, K, 8, GR, O2>(args, item_start, n_solvers, n_items, threads, smem, st);
      return cudaErrorInvalidConfiguration;
    default:
      return cudaErrorInvalidConfiguration;
  }
}

template <typename R>
cudaError_t launch_sweep_batch(const SweepArgs<R>* args, const int32_t* item_start, int n_solvers, int K, int G,
                               bool global_ring, bool order2, int n_items, int threads, size_t smem,
                               cudaStream_t st) {
  if (n_solvers < 1 || n_items < 1) return cudaSuccess;
#define NBTE_BK(Kv)                                                                                               \
  case Kv:                                                                                                        \
    if (order2)                                                                                                   \
      return global_ring                                                                                          \
                 ? launch_batch_k<R, Kv, true, true>(args, item_start, n_solvers, G, n_items, threads, smem, st)  \
                 : launch_batch_k<R, Kv, false, true>(args, item_start, n_solvers, G, n_items, threads, smem, st); \
    return global_ring                                                                                            \
               ? launch_batch_k<R, Kv, true, false>(args, item_start, n_solvers, G, n_items, threads, smem, st)   \
               : launch_batch_k<R, Kv, false, false>(args, item_start, n_solvers, G, n_items, threads, smem, st);
  switch (K) {
    NBTE_BK(1) NBTE_BK(2) NBTE_BK(3) NBTE_BK(4) NBTE_BK(5)
    default:
      return cudaErrorInvalidConfiguration;
  }
#undef NBTE_BK
}

template <typename R>
cudaError_t launch_sweep(const SweepArgs<R>& a, int K, int G, int n_items, int threads, size_t smem, cudaStream_t st) {
  // second-order sources (src2) select their own kernel variant, so the
  // first-order sweep carries none of their per-chunk work
  if (a.src2)
    return a.gring ? launch_gr<R, true, true>(a, K, G, n_items, threads, smem, st)
                   : launch_gr<R, false, true>(a, K, G, n_items, threads, smem, st);
  return a.gring ? launch_gr<R, true, false>(a, K, G, n_items, threads, smem, st)
                 : launch_gr<R, false, false>(a, K, G, n_items, threads, smem, st);
}

template cudaError_t launch_sweep<float>(const SweepArgs<float>&, int, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_sweep_batch<float>(const SweepArgs<float>*, const int32_t*, int, int, int, bool, bool, int,
                                               int, size_t, cudaStream_t);
template cudaError_t launch_sweep_batch<double>(const SweepArgs<double>*, const int32_t*, int, int, int, bool, bool,
                                                int, int, size_t, cudaStream_t);
template cudaError_t launch_sweep<double>(const SweepArgs<double>&, int, int, int, int, size_t, cudaStream_t);
}  // namespace nbte
