// Vector loads and stores of a few consecutive values (shared by the sweep
// and its data-preparation kernels).  Callers keep p aligned to the vector
// width they request: 16 bytes for groups of 4 floats, 8 or 16 bytes for
// pairs.
#pragma once

#include <cuda_runtime.h>

namespace nbte {

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

}  // namespace nbte
