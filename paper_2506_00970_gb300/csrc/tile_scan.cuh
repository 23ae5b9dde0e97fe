// Tile ranges from per-tile pair counts, by one block: exclusive scan of the
// counts -> [start, end) of every tile's segment, K = the total and the
// capacity check (GS2D_ERR_CAPACITY in the gate), and the list of tiles whose
// segment exceeds long_len keys.  Used by the binning's tile-scan kernel and
// by the last block of the projection kernel when projection and counting
// are fused.  blockDim.x: a multiple of 32, at most 1024.
#pragma once

#include "gs2d_common.cuh"

namespace gs2d {

__device__ __forceinline__ void tile_scan_block(const uint32_t* __restrict__ tile_count,
                                                int n_tiles, int32_t* __restrict__ ranges,
                                                int32_t* __restrict__ n_isect, long long capacity,
                                                uint32_t* __restrict__ long_list,
                                                uint32_t* __restrict__ n_long, int long_len,
                                                int32_t* __restrict__ gate, uint32_t* s_w,
                                                uint32_t* s_carry) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) *s_carry = 0;
  __syncthreads();
  for (int base = 0; base < n_tiles; base += blockDim.x) {
    const int t = base + (int)threadIdx.x;
    // counters written by other blocks: read past L1
    const uint32_t c = t < n_tiles ? __ldcg(tile_count + t) : 0u;
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
      const uint32_t x = lane < nw ? s_w[lane] : 0u;
      uint32_t xi = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, xi, o);
        if (lane >= o) xi += v;
      }
      if (lane < nw) s_w[lane] = xi - x;
    }
    __syncthreads();
    const uint32_t start = *s_carry + s_w[w] + inc - c;
    if (t < n_tiles) {
      ranges[2 * t] = (int32_t)start;
      ranges[2 * t + 1] = (int32_t)(start + c);
      if (c > (uint32_t)long_len) long_list[atomicAdd(n_long, 1u)] = (uint32_t)t;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) *s_carry = start + c;
    __syncthreads();
  }
  // K and the capacity check (ranges beyond the capacity are never read)
  if (threadIdx.x == 0) {
    const unsigned long long K = *s_carry;
    *n_isect = (int32_t)min(K, (unsigned long long)0x7FFFFFFF);
    if (K > (unsigned long long)capacity) atomicExch(gate, (int32_t)GS2D_ERR_CAPACITY);
  }
}

}  // namespace gs2d
