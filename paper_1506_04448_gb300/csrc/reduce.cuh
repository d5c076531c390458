// Warp and block reductions, and the small-sample median used for the B sketches.
#pragma once

#include "common.cuh"

namespace tsk {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over a block of NT threads (NT a multiple of 32).  `red` holds >= 33 floats of shared
// memory.  Every thread receives the total; `red` may be reused after return.
template <int NT>
__device__ __forceinline__ float block_sum(float v, float* red) {
  static_assert(NT % 32 == 0, "block of whole warps");
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float r = (threadIdx.x < NT / 32) ? red[threadIdx.x] : 0.f;
    r = warp_sum(r);
    if (threadIdx.x == 0) red[32] = r;
  }
  __syncthreads();
  const float total = red[32];
  __syncthreads();
  return total;
}

// Median of x[0..cnt) (cnt >= 1) by insertion sort in place; mean of the two middle values
// when cnt is even (the even-B reading of Alg. 1's median).
template <typename V>
__device__ __forceinline__ V small_median(V* x, int cnt) {
  for (int a = 1; a < cnt; ++a) {
    const V key = x[a];
    int c = a - 1;
    while (c >= 0 && x[c] > key) {
      x[c + 1] = x[c];
      --c;
    }
    x[c + 1] = key;
  }
  return (cnt & 1) ? x[cnt / 2] : (V)0.5 * (x[cnt / 2 - 1] + x[cnt / 2]);
}

// small_median on cnt values spaced `stride` apart (a column of a shared-memory scratch array,
// so that the threads of a warp sort in different banks).
__device__ __forceinline__ float small_median_strided(float* x, int cnt, int stride) {
  for (int a = 1; a < cnt; ++a) {
    const float key = x[a * stride];
    int c = a - 1;
    while (c >= 0 && x[c * stride] > key) {
      x[(c + 1) * stride] = x[c * stride];
      --c;
    }
    x[(c + 1) * stride] = key;
  }
  const int h = cnt / 2;
  return (cnt & 1) ? x[h * stride] : 0.5f * (x[(h - 1) * stride] + x[h * stride]);
}

}  // namespace tsk
