// Device helpers shared by the gs2d CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs2d.h"

#define GS2D_CUDA_TRY(expr)                       \
  do {                                            \
    cudaError_t e_ = (expr);                      \
    if (e_ != cudaSuccess) return GS2D_ERR_CUDA;  \
  } while (0)

#define GS2D_LAUNCH_CHECK()                                   \
  do {                                                        \
    if (cudaPeekAtLastError() != cudaSuccess) {               \
      cudaGetLastError();                                     \
      return GS2D_ERR_CUDA;                                   \
    }                                                         \
  } while (0)

namespace gs2d {

constexpr int kProjFloats = GS2D_PROJ_FLOATS;

// slots of the projected record (see gs2d.h)
enum ProjSlot {
  kC0 = 0, kC1 = 3, kC2 = 6, kDet = 9, kAlpha = 10, kRgb = 11, kTn = 14, kNrm = 17, kDu = 20,
  kDv = 23, kDepth = 26, kRect01 = 28, kRect23 = 29
};
constexpr int kFwdVec4 = 5;  // float4s of a record the forward pass reads (slots 0-19)
constexpr int kBwdVec4 = 7;  // float4s the backward pass reads (slots 0-27)

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves a workspace into aligned sub-buffers (host side).
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

struct F3 {
  float x, y, z;
};
__device__ __forceinline__ F3 f3(float x, float y, float z) { return F3{x, y, z}; }
__device__ __forceinline__ F3 operator+(F3 a, F3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ F3 operator*(float s, F3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(F3 a, F3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ F3 cross3(F3 a, F3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Rows of a 3x3 matrix; m[r*3+c].
__device__ __forceinline__ F3 mat_mul(const float* m, F3 v) {
  return f3(fmaf(m[0], v.x, fmaf(m[1], v.y, m[2] * v.z)), fmaf(m[3], v.x, fmaf(m[4], v.y, m[5] * v.z)),
            fmaf(m[6], v.x, fmaf(m[7], v.y, m[8] * v.z)));
}
__device__ __forceinline__ F3 mat_tmul(const float* m, F3 v) {
  return f3(fmaf(m[0], v.x, fmaf(m[3], v.y, m[6] * v.z)), fmaf(m[1], v.x, fmaf(m[4], v.y, m[7] * v.z)),
            fmaf(m[2], v.x, fmaf(m[5], v.y, m[8] * v.z)));
}

__host__ __device__ inline int tiles_along(int px, int tile) { return (px + tile - 1) / tile; }


// Sum over a 256-thread block (fixed order); the result is valid in thread 0.
// s: shared scratch of 8 floats.  Every thread must call it.
__device__ __forceinline__ float block_sum256(float v, float* s) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < 8; ++w) t += s[w];
  return t;
}


// Unit quaternion (w, x, y, z) of a rotation matrix D (row-major [9]), by
// the branch of the largest of w, x, y, z (no division by a small number);
// returned as float4 (x = w, y = x, z = y, w = z).
__device__ __forceinline__ float4 quat_from_matrix(const float* D) {
  const float tr = D[0] + D[4] + D[8];
  float w, x, y, z;
  if (tr >= D[0] && tr >= D[4] && tr >= D[8]) {
    const float s = 2.f * sqrtf(fmaxf(1.f + tr, 1e-30f));   // s = 4 w
    w = 0.25f * s;
    x = (D[7] - D[5]) / s;
    y = (D[2] - D[6]) / s;
    z = (D[3] - D[1]) / s;
  } else if (D[0] >= D[4] && D[0] >= D[8]) {
    const float s = 2.f * sqrtf(fmaxf(1.f + D[0] - D[4] - D[8], 1e-30f));   // s = 4 x
    w = (D[7] - D[5]) / s;
    x = 0.25f * s;
    y = (D[1] + D[3]) / s;
    z = (D[2] + D[6]) / s;
  } else if (D[4] >= D[8]) {
    const float s = 2.f * sqrtf(fmaxf(1.f + D[4] - D[0] - D[8], 1e-30f));   // s = 4 y
    w = (D[2] - D[6]) / s;
    x = (D[1] + D[3]) / s;
    y = 0.25f * s;
    z = (D[5] + D[7]) / s;
  } else {
    const float s = 2.f * sqrtf(fmaxf(1.f + D[8] - D[0] - D[4], 1e-30f));   // s = 4 z
    w = (D[3] - D[1]) / s;
    x = (D[2] + D[6]) / s;
    y = (D[5] + D[7]) / s;
    z = 0.25f * s;
  }
  const float qn = rsqrtf(w * w + x * x + y * y + z * z);
  return make_float4(w * qn, x * qn, y * qn, z * qn);
}

}  // namespace gs2d
