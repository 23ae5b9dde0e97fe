// Tile ranges from per-tile pair counts, by one block: exclusive scan of the
// counts -> [start, end) of every tile's segment, K = the total and the
// capacity check (GS2D_ERR_CAPACITY in the gate), and the list of tiles whose
// segment exceeds long_len keys.  Used by the binning's tile-scan kernel and
// by the last block of the projection kernel when projection and counting
// are fused.  blockDim.x: a multiple of 32, at most 1024.
#pragma once

#include "gs2d_common.cuh"
#include "scan.cuh"

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

// Bucket of a tile in the launch order: 256 buckets linear in
// count / max count, bucket 0 holding the longest segments.
__device__ __forceinline__ int order_bucket(uint32_t c, unsigned long long mx) {
  return 255 - (int)((unsigned long long)c * 255ull / mx);
}

// Launch order of the tiles by decreasing segment length, by one 256-thread
// block: a counting sort of the counts into the 256 buckets of
// order_bucket, order[0 .. n_tiles) a permutation of the tile ids.  Ties
// within a bucket land in arrival order: the order only schedules blocks,
// every result stays indexed by tile.  s_n: shared scratch of 257 words;
// s_w: 8 words.
__device__ __forceinline__ void tile_order_block(const uint32_t* __restrict__ tile_count,
                                                 int n_tiles, int32_t* __restrict__ order,
                                                 uint32_t* s_n, uint32_t* s_w) {
  const int tid = threadIdx.x;
  s_n[tid] = 0u;
  if (tid == 0) s_n[256] = 0u;
  __syncthreads();
  uint32_t m = 0u;
  for (int t = tid; t < n_tiles; t += 256) m = max(m, __ldcg(tile_count + t));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) atomicMax(s_n + 256, m);
  __syncthreads();
  const unsigned long long mx = max(s_n[256], 1u);
  for (int t = tid; t < n_tiles; t += 256)
    atomicAdd(s_n + order_bucket(__ldcg(tile_count + t), mx), 1u);
  __syncthreads();
  uint32_t total;
  const uint32_t off = block_exscan256<uint32_t>(s_n[tid], s_w, &total);
  s_n[tid] = off;
  __syncthreads();
  for (int t = tid; t < n_tiles; t += 256)
    order[atomicAdd(s_n + order_bucket(__ldcg(tile_count + t), mx), 1u)] = t;
}

// tile_scan_block and tile_order_block for at most 256 kPer tiles by one
// 256-thread block, with the counts held in registers: thread i owns the
// consecutive tiles [i per, (i + 1) per), per = ceil(n_tiles / 256), so the
// counts are read once, in one round of loads, and scanned by one block-wide
// prefix (same ranges, K, long list and gate as tile_scan_block).
// order may be NULL.  s_n: shared scratch of 257 words; s_w: 8 words.
template <int kPer>
__device__ __forceinline__ void tile_scan_order_small(
    const uint32_t* __restrict__ tile_count, int n_tiles, int32_t* __restrict__ ranges,
    int32_t* __restrict__ n_isect, long long capacity, uint32_t* __restrict__ long_list,
    uint32_t* __restrict__ n_long, int long_len, int32_t* __restrict__ gate,
    int32_t* __restrict__ order, uint32_t* s_n, uint32_t* s_w) {
  const int tid = threadIdx.x;
  const int per = (n_tiles + 255) / 256;
  const int t0 = tid * per;
  uint32_t c[kPer];
  uint32_t sum = 0u, m = 0u;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int t = t0 + k;
    // counters written by other blocks: read past L1
    c[k] = (k < per && t < n_tiles) ? __ldcg(tile_count + t) : 0u;
  }
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    sum += c[k];
    m = max(m, c[k]);
  }
  uint32_t K;
  uint32_t run = block_exscan256<uint32_t>(sum, s_w, &K);
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int t = t0 + k;
    if (k < per && t < n_tiles) {
      ranges[2 * t] = (int32_t)run;
      ranges[2 * t + 1] = (int32_t)(run + c[k]);
      if (c[k] > (uint32_t)long_len) long_list[atomicAdd(n_long, 1u)] = (uint32_t)t;
      run += c[k];
    }
  }
  // K and the capacity check (ranges beyond the capacity are never read)
  if (tid == 0) {
    *n_isect = (int32_t)min((unsigned long long)K, (unsigned long long)0x7FFFFFFF);
    if ((unsigned long long)K > (unsigned long long)capacity)
      atomicExch(gate, (int32_t)GS2D_ERR_CAPACITY);
  }
  if (!order) return;
  s_n[tid] = 0u;
  if (tid == 0) s_n[256] = 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  __syncthreads();
  if ((tid & 31) == 0) atomicMax(s_n + 256, m);
  __syncthreads();
  const unsigned long long mx = max(s_n[256], 1u);
#pragma unroll
  for (int k = 0; k < kPer; ++k)
    if (k < per && t0 + k < n_tiles) atomicAdd(s_n + order_bucket(c[k], mx), 1u);
  __syncthreads();
  uint32_t total;
  const uint32_t off = block_exscan256<uint32_t>(s_n[tid], s_w, &total);
  s_n[tid] = off;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kPer; ++k)
    if (k < per && t0 + k < n_tiles) order[atomicAdd(s_n + order_bucket(c[k], mx), 1u)] = t0 + k;
}

}  // namespace gs2d
