// Block-wide exclusive scan for 256-thread blocks (stable compactions).
#pragma once

#include "gs2d_common.cuh"

namespace gs2d {

// Exclusive prefix of one value per thread over a 256-thread block (int, or
// uint32_t for sums modulo 2^32); *total receives the block sum.  s_w: shared
// scratch of 8 values.  Every thread of the block must call it.
template <typename T>
__device__ __forceinline__ T block_exscan256(T v, T* s_w, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < 8 ? s_w[lane] : T(0);
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    if (lane < 8) s_w[lane] = w;
  }
  __syncthreads();
  const T pre = (warp ? s_w[warp - 1] : T(0)) + x - v;
  *total = s_w[7];
  __syncthreads();
  return pre;
}

}  // namespace gs2d
