// The transport sweep (sm_103a): per (direction, band group) work item, the
// first-order upwind solve of Eq. (4) in the topological (level) order of the
// direction's upwind graph -- the triangular substitution of the factorised
// system of Eq. (13) -- fused with the collision moment of Eq. (5) and, on
// request, the energy and flux moments of Eq. (7).
//
// Warp-specialised pipeline, one CTA per work item:
//  * warp 0 (one elected lane) is the producer.  It walks the direction's
//    chunks (up to CAP consecutive positions of one level) and, several chunks
//    ahead of the consumers, bulk-copies (cp.async.bulk, completion counted on
//    an mbarrier) each chunk's packed position records, its pre-gathered
//    (T', Qdot) pairs and its slice of wall/lag import values into a ring of
//    shared-memory stages;
//  * the other warps are consumers: they wait on a stage's "full" barrier,
//    compute one position per thread from shared memory and the value ring,
//    release the stage on its "empty" barrier, and meet on a named barrier
//    only at the end of a level (so the next level sees the ring writes).
// The value ring holds the outgoing values of the direction's live cells
// (slots assigned by the planner).  It lives in shared memory when it fits
// (GR = false); otherwise (GR = true, large 3D meshes whose sweep front has
// tens of thousands of live cells) in a per-CTA global-memory region, where
// the concurrently running CTAs' live windows stay mostly in L2.  Every wait
// is bounded: on timeout the error word is set, the producer waits (bounded)
// for the copies it issued, and the CTA leaves.
//
// Per cell and band the balance is solved for the deviation from the cell's
// own equilibrium e0 = C T'/W (Eq. (11)):
//   e = e0 + (Qdot C/(C_tot W) + v sum_in c_k (e_up,k - e0) + v src2) / (1/tau + v G),
//   c_k = |s.An_k|/V,  G = sum_in c_k  (= sum_out (s.An)/V for a closed cell),
// src2 = 0 for first-order upwind; with second-order face values it is the
// reconstruction increment of every interior face taken from the previous
// iteration's gradients (deferred correction, see launch_src2).
// The collision-moment partial is sum_l w_i (e - e0)/tau_l; the equilibrium
// part sums to beta T' exactly and is added back in FP64 by the update kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "layout.h"

namespace nbte {

namespace {

constexpr unsigned long long kWaitLimit = 1ull << 26;

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
// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (unsigned long long k = 0; k < kWaitLimit; ++k)
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

template <typename R>
struct Vec2;
template <>
struct Vec2<float> { using T = float2; };
template <>
struct Vec2<double> { using T = double2; };

template <typename R, int BPT>
__device__ __forceinline__ void load_vals(const R* p, R (&v)[BPT]) {
  if constexpr (sizeof(R) == 4 && BPT % 4 == 0) {
#pragma unroll
    for (int b = 0; b < BPT; b += 4) {
      const float4 t = *reinterpret_cast<const float4*>(p + b);
      v[b] = t.x; v[b + 1] = t.y; v[b + 2] = t.z; v[b + 3] = t.w;
    }
  } else if constexpr (BPT % 2 == 0) {
#pragma unroll
    for (int b = 0; b < BPT; b += 2) {
      const typename Vec2<R>::T t = *reinterpret_cast<const typename Vec2<R>::T*>(p + b);
      v[b] = t.x; v[b + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int b = 0; b < BPT; ++b) v[b] = p[b];
  }
}

template <typename R, int BPT>
__device__ __forceinline__ void store_vals(R* p, const R (&v)[BPT]) {
  if constexpr (sizeof(R) == 4 && BPT % 4 == 0) {
#pragma unroll
    for (int b = 0; b < BPT; b += 4) *reinterpret_cast<float4*>(p + b) = make_float4(v[b], v[b + 1], v[b + 2], v[b + 3]);
  } else if constexpr (BPT % 2 == 0) {
#pragma unroll
    for (int b = 0; b < BPT; b += 2) {
      typename Vec2<R>::T t;
      t.x = v[b]; t.y = v[b + 1];
      *reinterpret_cast<typename Vec2<R>::T*>(p + b) = t;
    }
  } else {
#pragma unroll
    for (int b = 0; b < BPT; ++b) p[b] = v[b];
  }
}

// FP32: the hardware approximate reciprocal (relative error below 2^-22,
// under the FP32 sweep's own rounding); FP64: a correctly rounded division
__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

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
template <typename R, int K, int G, bool GR, bool O2>
__device__ __forceinline__ void sweep_item(const SweepArgs<R>& a, const int item, unsigned char* smem) {
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
          const int64_t d0 = (int64_t)item * a.N + m.pos;
          da = d0 / dper16 * dper16;
          const int64_t de = (d0 + m.len + dper16 - 1) / dper16 * dper16;
          den_bytes = (unsigned)((de - da) * G * 8);
        }
        // second order: the chunk's reconstruction sources, a 16-byte aligned superset
        unsigned s2_bytes = 0;
        int64_t sa = 0;
        if constexpr (O2) {
          constexpr int sper16 = (int)(16 / (G * sizeof(R))) > 1 ? (int)(16 / (G * sizeof(R))) : 1;
          const int64_t s0 = (int64_t)item * a.N + m.pos;
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
  R* part = a.part + (int64_t)item * a.N;
  R* exp_g = a.exp + ((size_t)g * a.n_exp + a.exp_off[i]) * GP;
  consumer_barrier(ncons);

  int sc = 0;          // stage of chunk c, and the parity of its round
  unsigned phc = 0;
  for (int c = 0; c < nch; ++c) {
    const int s = sc;
    if (!mbar_wait(full + s, phc)) {
      atomicExch(a.err, (int32_t)DEV_QUEUE_TIMEOUT);
      break;
    }
    const Chunk m = meta[s];
    const unsigned char* st = stages + (size_t)s * a.stage_bytes;
    // the block: header (level count, level ends), records, (T', Qdot) pairs
    const int n_lev = chunk_levels(m.nimp_end);
    const int32_t* lev_end = reinterpret_cast<const int32_t*>(st) + 1;
    const unsigned char* recs = st + chunk_header_bytes(n_lev);
    using R2 = typename Vec2<R>::T;
    const R2* tqs = reinterpret_cast<const R2*>(recs + (size_t)m.len * RL.size);
    const R* imps = reinterpret_cast<const R*>(st + a.off_imp);
    const int imp0 = m.imp;
    // FP64: this chunk's precomputed denominators (superset starts d_shift early)
    const R* dens = reinterpret_cast<const R*>(st + a.off_den);
    const int d_shift = sizeof(R) == 8 && G == 1 ? (int)(((int64_t)item * a.N + m.pos) % 2) : 0;
    // second order: this chunk's reconstruction sources (superset starts s_shift early)
    constexpr int sper16 = (int)(16 / (G * sizeof(R))) > 1 ? (int)(16 / (G * sizeof(R))) : 1;
    const R* s2 = reinterpret_cast<const R*>(st + a.off_src2);
    const int s_shift = O2 ? (int)(((int64_t)item * a.N + m.pos) % sper16) : 0;
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
        if (a.e_out)
          store_vals<R, G>(a.e_out + (size_t)i * a.e_out_dstride + (size_t)g * a.e_out_gstride +
                               (size_t)cell * a.e_out_cstride,
                           e);
        part[cell] = nl;
        if (a.full) {
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
}

template <typename R, int K, int G, bool GR, bool O2>
__global__ void __launch_bounds__(544) sweep_kernel(const SweepArgs<R> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  sweep_item<R, K, G, GR, O2>(a, blockIdx.x + a.item0, smem);
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
  sweep_item<R, K, G, GR, O2>(sa, s_item, smem);
}

template <typename R, int K, int G, bool GR, bool O2>
static cudaError_t launch_one(const SweepArgs<R>& a, int n_items, int threads, size_t smem, cudaStream_t st) {
  auto kern = sweep_kernel<R, K, G, GR, O2>;
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

// One block per chunk: its positions' records (multiples of 16 bytes, copied
// as 16-byte words) to the chunk's block, and each position's pair index
__global__ void pack_blocks_kernel(unsigned char* blk, uint32_t* tq_dst, const unsigned char* rec_pos,
                                   const Chunk* chunks, const int64_t* chunk_doff, const int32_t* chunk_dir,
                                   const int64_t* sub_ptr, const int32_t* sub_end, int64_t N, int rec_size,
                                   int pair_bytes) {
  const int64_t c = blockIdx.x;
  const Chunk ch = chunks[c];
  const int64_t doff = chunk_doff[c];
  const int64_t q0 = (int64_t)chunk_dir[c] * N + ch.pos;
  const int n_lev = chunk_levels(ch.nimp_end);
  int32_t* hdr = reinterpret_cast<int32_t*>(blk + doff);
  for (int t = threadIdx.x; t <= n_lev; t += blockDim.x) hdr[t] = t == 0 ? n_lev : sub_end[sub_ptr[c] + t - 1];
  const int64_t roff = doff + chunk_header_bytes(n_lev);
  const int w16 = rec_size / 16;
  const uint4* src = reinterpret_cast<const uint4*>(rec_pos + (size_t)q0 * rec_size);
  uint4* dst = reinterpret_cast<uint4*>(blk + roff);
  for (int t = threadIdx.x; t < ch.len * w16; t += blockDim.x) dst[t] = src[t];
  const uint32_t tq0 = (uint32_t)((roff + (int64_t)ch.len * rec_size) / pair_bytes);
  for (int j = threadIdx.x; j < ch.len; j += blockDim.x) tq_dst[q0 + j] = tq0 + (uint32_t)j;
}

cudaError_t launch_pack_blocks(unsigned char* blk, uint32_t* tq_dst, const unsigned char* rec_pos,
                               const Chunk* chunks, const int64_t* chunk_doff, const int32_t* chunk_dir,
                               const int64_t* sub_ptr, const int32_t* sub_end, int64_t n_chunks, int64_t N,
                               int rec_size, int pair_bytes, cudaStream_t st) {
  if (n_chunks == 0) return cudaSuccess;
  if (rec_size % 16 != 0 || n_chunks > 0x7fffffff) return cudaErrorInvalidValue;
  pack_blocks_kernel<<<(unsigned)n_chunks, 128, 0, st>>>(blk, tq_dst, rec_pos, chunks, chunk_doff, chunk_dir,
                                                         sub_ptr, sub_end, N, rec_size, pair_bytes);
  return cudaGetLastError();
}

// FP64 denominators of every (work item, position); one thread per pair
__global__ void fill_dinv_kernel(double* dinv, const double* pos_G, const double* band_v, const double* band_inv_tau,
                                 int D, int ng, int G, int64_t N) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)D * ng * N) return;
  const int64_t item = t / N, pos = t - item * N;
  const int i = (int)(item / ng), g = (int)(item - (int64_t)i * ng);
  const double Gc = pos_G[(size_t)i * N + pos];
  for (int b = 0; b < G; ++b) dinv[t * G + b] = 1.0 / (band_inv_tau[g * G + b] + band_v[g * G + b] * Gc);
}

cudaError_t launch_fill_dinv(double* dinv, const double* pos_G, const double* band_v, const double* band_inv_tau,
                             int D, int n_groups, int G, int64_t N, cudaStream_t st) {
  const int64_t n = (int64_t)D * n_groups * N;
  if (n == 0) return cudaSuccess;
  fill_dinv_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dinv, pos_G, band_v, band_inv_tau, D, n_groups, G,
                                                                N);
  return cudaGetLastError();
}

// (T', Qdot) of every position's cell, in each direction's level order, so
// the sweep's producer can bulk-copy them with the position records
template <typename R>
__global__ void gather_tq_kernel(R* data, const uint32_t* tq_dst, const int32_t* pos_cell, const R* srcTQ,
                                 int64_t n) {
  using R2 = typename Vec2<R>::T;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  reinterpret_cast<R2*>(data)[__ldcs(tq_dst + q)] = __ldg(reinterpret_cast<const R2*>(srcTQ) + __ldcs(pos_cell + q));
}

// Second-order upwind sources.  One thread per (direction, position): it
// resolves the cell's faces once -- upwind cell, its neighbours and the
// reconstruction weights toward the face -- and keeps them in registers
// while it walks the band groups along each needed row of the direction's
// distribution (N*Bp values, L2-resident while the direction's blocks run).
// Consecutive threads take consecutive positions, so each band group's
// results are stored as one contiguous run of the [item][position][G]
// layout the sweep copies.  Wall faces get d = 0 and read the cell itself;
// a wall neighbour of the upwind cell reads the upwind cell (zero difference,
// zero weight): no branches between the loads.
template <typename R, int G, int NF>
__global__ void __launch_bounds__(256, NF > 4 ? 3 : 1) src2_kernel(const Src2Args<R> a) {
  const int i = blockIdx.y;   // direction (a 2D grid: no division by N)
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.N) return;
  const int c = __ldg(a.pos_cell + (int64_t)i * a.N + p);
  const R sx = (R)a.dir_s[i * 3], sy = (R)a.dir_s[i * 3 + 1], sz = (R)a.dir_s[i * 3 + 2];
  // hexahedra (36 weights and neighbours) re-read the tables from L1 per band
  // group instead of holding them in registers
  constexpr bool kHold = NF <= 4;
  constexpr int NH = kHold ? NF : 1;
  R d[NF], w[NH][NH];
  int u[NF], h[NF], nbu[NH][NH];
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const int nk = __ldg(a.nb + (int64_t)c * NF + k);
    const int tw = __ldg(a.twin + (int64_t)c * NF + k);
    const R* An = a.AnV + ((int64_t)c * NF + k) * 3;
    R dk = sx * __ldg(An) + sy * __ldg(An + 1) + sz * __ldg(An + 2);
    if (nk < 0) dk = R(0);
    const bool in = dk < R(0);
    d[k] = dk;
    u[k] = in ? nk : c;
    h[k] = in ? tw : k;
    if constexpr (kHold) {
#pragma unroll
      for (int m2 = 0; m2 < NF; ++m2) {
        const int nm = __ldg(a.nb + (int64_t)u[k] * NF + m2);
        nbu[k][m2] = nm >= 0 ? nm : u[k];
        w[k][m2] = __ldg(a.rc_a + ((int64_t)u[k] * NF + h[k]) * NF + m2);
      }
    }
  }
  const R* e = a.e + (size_t)i * a.N * a.Bp;
  R* out = a.src2 + ((size_t)i * a.n_groups * a.N + p) * G;
  for (int g = 0; g < a.n_groups; ++g) {
    const R* eg = e + g * G;
    R acc[G];
#pragma unroll
    for (int b = 0; b < G; ++b) acc[b] = R(0);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      R eu[G], inc[G];
      load_vals<R, G>(eg + (size_t)u[k] * a.Bp, eu);
#pragma unroll
      for (int b = 0; b < G; ++b) inc[b] = R(0);
#pragma unroll
      for (int m2 = 0; m2 < NF; ++m2) {
        int nm;
        R wm;
        if constexpr (kHold) {
          nm = nbu[k][m2];
          wm = w[k][m2];
        } else {
          nm = __ldg(a.nb + (int64_t)u[k] * NF + m2);
          nm = nm >= 0 ? nm : u[k];
          wm = __ldg(a.rc_a + ((int64_t)u[k] * NF + h[k]) * NF + m2);
        }
        R en[G];
        load_vals<R, G>(eg + (size_t)nm * a.Bp, en);
#pragma unroll
        for (int b = 0; b < G; ++b) inc[b] += wm * (en[b] - eu[b]);
      }
#pragma unroll
      for (int b = 0; b < G; ++b) acc[b] -= d[k] * inc[b];
    }
    store_vals<R, G>(out + (size_t)g * a.N * G, acc);
  }
}

template <typename R, int G>
static cudaError_t launch_src2_g(const Src2Args<R>& a, cudaStream_t st) {
  const dim3 grid((unsigned)((a.N + 255) / 256), (unsigned)a.D);
  switch (a.nfc) {
    case 3: src2_kernel<R, G, 3><<<grid, 256, 0, st>>>(a); break;
    case 4: src2_kernel<R, G, 4><<<grid, 256, 0, st>>>(a); break;
    case 6: src2_kernel<R, G, 6><<<grid, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_src2(const Src2Args<R>& a, cudaStream_t st) {
  if ((int64_t)a.n_items * a.N == 0) return cudaSuccess;
  if (a.Bp != a.n_groups * a.G || a.D > 65535) return cudaErrorInvalidValue;
  switch (a.G) {
    case 1: return launch_src2_g<R, 1>(a, st);
    case 2: return launch_src2_g<R, 2>(a, st);
    case 4: return launch_src2_g<R, 4>(a, st);
    case 8:
      if constexpr (sizeof(R) == 4) return launch_src2_g<R, 8>(a, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_gather_tq(unsigned char* data, const uint32_t* tq_dst, const int32_t* pos_cell, const R* srcTQ,
                             int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  gather_tq_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<R*>(data), tq_dst, pos_cell,
                                                                    srcTQ, n);
  return cudaGetLastError();
}

template cudaError_t launch_sweep<float>(const SweepArgs<float>&, int, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_sweep_batch<float>(const SweepArgs<float>*, const int32_t*, int, int, int, bool, bool, int,
                                               int, size_t, cudaStream_t);
template cudaError_t launch_sweep_batch<double>(const SweepArgs<double>*, const int32_t*, int, int, int, bool, bool,
                                                int, int, size_t, cudaStream_t);
template cudaError_t launch_sweep<double>(const SweepArgs<double>&, int, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_src2<float>(const Src2Args<float>&, cudaStream_t);
template cudaError_t launch_src2<double>(const Src2Args<double>&, cudaStream_t);
template cudaError_t launch_gather_tq<float>(unsigned char*, const uint32_t*, const int32_t*, const float*, int64_t,
                                             cudaStream_t);
template cudaError_t launch_gather_tq<double>(unsigned char*, const uint32_t*, const int32_t*, const double*, int64_t,
                                              cudaStream_t);

}  // namespace nbte
