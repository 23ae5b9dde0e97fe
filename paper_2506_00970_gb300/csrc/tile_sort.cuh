// Device code of the per-tile depth sort (step 4 of the binning in sort.cu),
// shared by the binning's sort kernels and by the fused tracking kernel,
// whose blocks sort their own tile's segment before rendering it: a segment
// of at most kSegSmem keys is sorted in shared memory by a bitonic network;
// a longer one in kSegSmem-key chunks whose sorted runs are then merged in
// global memory.
#pragma once

#include "gs2d_common.cuh"

namespace gs2d {

constexpr int kSegSmem = 2048;  // keys sorted in shared memory (16 KB)

struct Rect {
  int tx0, ty0, tx1, ty1;
};
__device__ __forceinline__ Rect load_rect(const float4* proj, uint32_t id) {
  const float4 rc = proj[(size_t)id * (kProjFloats / 4) + 7];
  const uint32_t r01 = __float_as_uint(rc.x), r23 = __float_as_uint(rc.y);
  return Rect{(int)(r01 & 0xFFFF), (int)(r01 >> 16), (int)(r23 & 0xFFFF), (int)(r23 >> 16)};
}

// Per-tile sort of a segment and the binning's outputs.  The flip-form
// bitonic network sorts ascending with the smaller key to the lower index;
// comparisons whose partner lies past the end are skipped (a virtual +inf).
__device__ __forceinline__ void cmp_swap(unsigned long long* a, int i, int j) {
  const unsigned long long x = a[i], y = a[j];
  if (y < x) {
    a[i] = y;
    a[j] = x;
  }
}
__device__ inline void bitonic_sort(unsigned long long* a, int len) {
  int lg = 0;
  while ((1 << lg) < len) ++lg;
  const int pairs = (1 << lg) >> 1;
  for (int ls = 1; ls <= lg; ++ls) {
    // flip step: i pairs with its mirror i ^ (size - 1) inside each block of
    // size = 2^ls (the index arithmetic in shifts: sizes are powers of two)
    const int lh = ls - 1;
    for (int q = threadIdx.x; q < pairs; q += blockDim.x) {
      const int i = ((q >> lh) << ls) | (q & ((1 << lh) - 1));
      const int j = i ^ ((1 << ls) - 1);
      if (j < len) cmp_swap(a, i, j);
    }
    __syncthreads();
    for (int lst = ls - 2; lst >= 0; --lst) {
      for (int q = threadIdx.x; q < pairs; q += blockDim.x) {
        const int i = ((q >> lst) << (lst + 1)) | (q & ((1 << lst) - 1));
        const int j = i + (1 << lst);
        if (j < len) cmp_swap(a, i, j);
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ void write_outputs(const unsigned long long* a, int len, int start, int t,
                                              int tiles_x, int n, const float4* __restrict__ proj,
                                              const uint32_t* __restrict__ surfel_off,
                                              uint32_t* __restrict__ vals, uint32_t* __restrict__ emit,
                                              unsigned long long* __restrict__ keys64) {
  const int tx = t % tiles_x, ty = t / tiles_x;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const unsigned long long key = a[i];
    const uint32_t id = min((uint32_t)(key & 0xFFFFFFFFull), (uint32_t)(n - 1));
    vals[start + i] = id;
    if (emit) {
      const Rect r = load_rect(proj, id);
      const int rw = max(r.tx1 - r.tx0 + 1, 1);
      emit[start + i] = surfel_off[id] + (uint32_t)((ty - r.ty0) * rw + (tx - r.tx0));
    }
    if (keys64) keys64[start + i] = ((unsigned long long)t << 32) | (key >> 32);
  }
}

// Position in the merge of sorted runs A[0, la) and B[0, lb) (unique keys):
// the number i of elements taken from A among the first d outputs.
__device__ __forceinline__ int co_rank(const unsigned long long* A, int la, const unsigned long long* B,
                                       int lb, int d) {
  int lo = max(0, d - lb), hi = min(d, la);
  while (lo < hi) {
    const int i = (lo + hi) >> 1;  // i from A, d - i from B
    if (A[i] < B[d - i - 1])
      lo = i + 1;
    else
      hi = i;
  }
  return lo;
}

// Segments longer than kSegSmem: chunks of kLongChunk keys are sorted in
// shared memory by 1024 threads, then adjacent sorted runs are merged in
// global memory (seg_keys <-> seg_tmp), each thread producing a contiguous
// span of the output located by a co-rank search.
// One long segment (tile t) by the whole block.
template <int kChunkKeys>
__device__ void sort_long_segment(int t, const float4* __restrict__ proj, int n, int tiles_x,
                                  const int32_t* __restrict__ ranges,
                                  unsigned long long* __restrict__ seg_keys,
                                  unsigned long long* __restrict__ seg_tmp,
                                  const uint32_t* __restrict__ surfel_off, uint32_t* __restrict__ vals,
                                  uint32_t* __restrict__ emit, unsigned long long* __restrict__ keys64,
                                  long long capacity, unsigned long long* s_keys) {
  const int start = ranges[2 * t];
  const int end = (int)min((long long)ranges[2 * t + 1], capacity);
  const int len = end - start;
  if (len <= kSegSmem) return;
  unsigned long long* src = seg_keys + start;
  unsigned long long* dst = seg_tmp + start;
  const int chunks = (len + kChunkKeys - 1) / kChunkKeys;
  for (int c = 0; c < chunks; ++c) {
    const int c0 = c * kChunkKeys, cl = min(kChunkKeys, len - c0);
    for (int i = threadIdx.x; i < cl; i += blockDim.x) s_keys[i] = src[c0 + i];
    __syncthreads();
    bitonic_sort(s_keys, cl);
    if (chunks == 1) {
      write_outputs(s_keys, len, start, t, tiles_x, n, proj, surfel_off, vals, emit, keys64);
      return;
    }
    for (int i = threadIdx.x; i < cl; i += blockDim.x) src[c0 + i] = s_keys[i];
    __syncthreads();
  }
  const int span = (len + blockDim.x - 1) / blockDim.x;
  for (int w = kChunkKeys; w < len; w <<= 1) {
    const int p0 = min(len, (int)threadIdx.x * span), p1 = min(len, p0 + span);
    int p = p0;
    while (p < p1) {
      // the run pair holding output position p
      const int lo = (p / (2 * w)) * (2 * w);
      const int mid = min(lo + w, len), hi = min(lo + 2 * w, len);
      const unsigned long long* A = src + lo;
      const unsigned long long* B = src + mid;
      const int la = mid - lo, lb = hi - mid;
      int i = co_rank(A, la, B, lb, p - lo);
      int j = (p - lo) - i;
      const int stop = min(p1, hi);
      for (; p < stop; ++p) {
        if (j >= lb || (i < la && A[i] < B[j]))
          dst[p] = A[i++];
        else
          dst[p] = B[j++];
      }
    }
    __syncthreads();
    unsigned long long* x = src;
    src = dst;
    dst = x;
  }
  write_outputs(src, len, start, t, tiles_x, n, proj, surfel_off, vals, emit, keys64);
}

}  // namespace gs2d
