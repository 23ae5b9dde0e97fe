// SSIM term of the mapping loss (Sec. III-E, L_c with L_SSIM; SSIM of Wang
// et al. 2004 with the 11 x 11 Gaussian window, sigma 1.5, C1 = 0.01^2,
// C2 = 0.03^2 for images in [0, 1]) and its gradient, in one fused pass.
//
// Per channel and pixel p, with the window w (zero padding at the border),
// the usual statistics mu_x = w * x, mu_y, sigma_x^2 = w * x^2 - mu_x^2,
// sigma_y^2, sigma_xy give
//   S = (2 mu_x mu_y + C1)(2 sigma_xy + C2) /
//       ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)).
// FP32 loses that form to cancellation where x ~ y (the numerator and the
// denominator agree to many digits, and so do the terms of its gradient),
// so the kernel works with the difference image d = x - y: with
// mu_d = w * d and sigma_d^2 = w * d^2 - mu_d^2 (identities:
// 2 mu_x mu_y + C1 = b1 - mu_d^2, 2 sigma_xy + C2 = b2 - sigma_d^2),
//   S = (1 - mu_d^2 / b1)(1 - sigma_d^2 / b2),
//   b1 = mu_x^2 + mu_y^2 + C1,  b2 = sigma_x^2 + sigma_y^2 + C2,
// so 1 - S = p + q - p q with p = mu_d^2 / b1, q = sigma_d^2 / b2 and the
// partial derivatives w.r.t. the moments (mu_x, mu_d, E_xx, E_yy, E_dd)
// have no large cancelling terms.  The loss adds
// weight / |Omega| sum_p (1 - mean_c S_c(p)); with G_* the partials of S
// times the upstream -weight / (3 |Omega|), the gradient w.r.t. x is
//   w * (G_mux + G_mud) + 2 x (w * G_xx) + 2 d (w * G_dd)
// (the window is symmetric, so the adjoint filter is the same filter).
//
// One block per 32 x 32 output tile and channel.  It stages x and y on the
// tile plus a 10-pixel ring in shared memory, filters the five moment maps
// separably (rows, then columns) on the tile plus a 5-pixel ring, evaluates
// S and the three G maps there (zero outside the image), filters those
// separably down to the tile and writes the gradient.  Everything between
// the image reads and the gradient write stays in shared memory: per pixel
// and channel the kernel reads x and y and adds one gradient value.  The
// per-block loss sums are reduced in a fixed order (deterministic).
#include <cmath>

#include "gs2d_common.cuh"
#include "gs2d_internal.h"

namespace gs2d {

constexpr int kSsimT = 32;                 // output tile edge
constexpr int kSsimR = 5;                  // window radius
constexpr int kSsimA = kSsimT + 4 * kSsimR;  // 52: staged edge (two rings)
constexpr int kSsimB = kSsimT + 2 * kSsimR;  // 42: moment / G map edge
constexpr int kSsimThreads = 256;
constexpr float kSsimC1 = 0.0001f, kSsimC2 = 0.0009f;

struct SsimWin {
  float g[2 * kSsimR + 1];  // normalised 1D Gaussian; the window is g g^T
};

// Shared memory (floats).  Region A: x and y (2 x 52 x 52, rows of 52), later
// the three G maps (3 x 42 rows of 44).  Region B: the five row-filtered
// moment maps (5 x 52 rows of 44), later the three row-filtered G maps
// (3 x 42 rows of 32).  Row strides are multiples of 4 floats so a thread
// reads 16 consecutive taps as four float4; each region has a little slack
// for the taps past the last row that only padding outputs use.
constexpr int kSsimBP = 44;                       // padded row of the 42-wide maps
constexpr int kSsimSmemA = 3 * kSsimB * kSsimBP + 16;
constexpr int kSsimSmemB = 5 * kSsimA * kSsimBP + 2 * kSsimBP + 16;
constexpr size_t kSsimSmemBytes = (size_t)(kSsimSmemA + kSsimSmemB) * sizeof(float);
static_assert(2 * kSsimA * kSsimA + 16 <= kSsimSmemA, "x and y fit region A");
static_assert(3 * kSsimB * kSsimT <= kSsimSmemB, "filtered G maps fit region B");
constexpr int kSsimRB = 4;                        // outputs per thread along a row or column

__device__ __forceinline__ void load16(const float* p, float (&v)[16]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 t = q[i];
    v[4 * i] = t.x;
    v[4 * i + 1] = t.y;
    v[4 * i + 2] = t.z;
    v[4 * i + 3] = t.w;
  }
}

__global__ void __launch_bounds__(kSsimThreads) ssim_kernel(const float* __restrict__ x,
                                                           const float* __restrict__ y, int H,
                                                           int W, float weight, SsimWin win,
                                                           float* __restrict__ g_x,
                                                           float* __restrict__ part) {
  extern __shared__ float4 smem4[];
  float* sa = reinterpret_cast<float*>(smem4);    // x, y [52][52]  ->  G [3][42][44]
  float* sb = sa + kSsimSmemA;                    // M [5][52][44]  ->  F [3][42][32]
  __shared__ float s_red[kSsimThreads / 32];
  const int c = blockIdx.z;
  const int tx0 = blockIdx.x * kSsimT, ty0 = blockIdx.y * kSsimT;
  const int ax0 = tx0 - 2 * kSsimR, ay0 = ty0 - 2 * kSsimR;   // staged origin
  // stage x, y (zero outside the image) and clear the slack; unrolled so
  // that several loads of each thread are in flight
#pragma unroll 4
  for (int e = threadIdx.x; e < kSsimA * kSsimA; e += kSsimThreads) {
    const int r = e / kSsimA, q = e % kSsimA;
    const int py = ay0 + r, px = ax0 + q;
    float vx = 0.f, vy = 0.f;
    if (px >= 0 && py >= 0 && px < W && py < H) {
      const size_t i = ((size_t)py * W + px) * 3 + c;
      vx = x[i];
      vy = y[i];
    }
    sa[e] = vx;
    sa[kSsimA * kSsimA + e] = vy;
  }
  if (threadIdx.x < 16) sa[2 * kSsimA * kSsimA + threadIdx.x] = 0.f;
  __syncthreads();
  // row filter of the five moments (x, d = x - y, x^2, y^2, d^2): outputs
  // M[k][r][q0 .. q0 + 3], r in [0, 52), q0 = 4 g, g in [0, 11)
  constexpr int kG1 = (kSsimB + kSsimRB - 1) / kSsimRB;   // 11 groups along a row
  for (int e = threadIdx.x; e < kSsimA * kG1; e += kSsimThreads) {
    const int r = e / kG1, q0 = (e % kG1) * kSsimRB;
    float xa[16], ya[16];
    load16(sa + r * kSsimA + q0, xa);
    load16(sa + kSsimA * kSsimA + r * kSsimA + q0, ya);
    float m[5][kSsimRB];
#pragma unroll
    for (int o = 0; o < kSsimRB; ++o) {
      float mx = 0.f, md = 0.f, exx = 0.f, eyy = 0.f, edd = 0.f;
#pragma unroll
      for (int t = 0; t <= 2 * kSsimR; ++t) {
        const float a = xa[o + t], b = ya[o + t], w = win.g[t];
        const float d = a - b;
        const float wa = w * a, wb = w * b, wd = w * d;
        mx += wa;
        md += wd;
        exx = fmaf(wa, a, exx);
        eyy = fmaf(wb, b, eyy);
        edd = fmaf(wd, d, edd);
      }
      m[0][o] = mx;
      m[1][o] = md;
      m[2][o] = exx;
      m[3][o] = eyy;
      m[4][o] = edd;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k)
      *reinterpret_cast<float4*>(sb + (k * kSsimA + r) * kSsimBP + q0) =
          make_float4(m[k][0], m[k][1], m[k][2], m[k][3]);
  }
  __syncthreads();
  // column filter, S and the G maps on the 42 x 42 region (origin tile - 5):
  // rows r0 .. r0 + 3 of column q per thread; x and y are dead, so the G
  // maps take region A
  const float up = -weight / (3.f * (float)H * (float)W);
  float loss = 0.f;
  for (int e = threadIdx.x; e < kSsimB * kG1; e += kSsimThreads) {
    const int q = e % kSsimB, r0 = (e / kSsimB) * kSsimRB;
    float m[5][kSsimRB];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float* col = sb + (k * kSsimA + r0) * kSsimBP + q;
      float v[kSsimRB + 2 * kSsimR];
#pragma unroll
      for (int t = 0; t < kSsimRB + 2 * kSsimR; ++t) v[t] = col[t * kSsimBP];
#pragma unroll
      for (int o = 0; o < kSsimRB; ++o) {
        float a = 0.f;
#pragma unroll
        for (int t = 0; t <= 2 * kSsimR; ++t) a = fmaf(win.g[t], v[o + t], a);
        m[k][o] = a;
      }
    }
#pragma unroll
    for (int o = 0; o < kSsimRB; ++o) {
      const int r = r0 + o;
      if (r >= kSsimB) break;
      const int py = ty0 - kSsimR + r, px = tx0 - kSsimR + q;
      float g0 = 0.f, g1 = 0.f, g2 = 0.f;
      if (px >= 0 && py >= 0 && px < W && py < H) {
        const float mx = m[0][o], md = m[1][o], my = mx - md;
        const float b1 = fmaf(mx, mx, fmaf(my, my, kSsimC1));
        const float b2 = (m[2][o] - mx * mx) + (m[3][o] - my * my) + kSsimC2;
        const float vd = m[4][o] - md * md;
        const float ib1 = 1.f / b1, ib2 = 1.f / b2;
        const float p1 = md * md * ib1, q1 = vd * ib2;   // 1 - P, 1 - Q
        const float P = 1.f - p1, Q = 1.f - q1;
        if (r >= kSsimR && r < kSsimR + kSsimT && q >= kSsimR && q < kSsimR + kSsimT)
          loss += p1 + q1 - p1 * q1;                      // 1 - S
        const float dmx = 2.f * (mx + my) * (Q * p1 * ib1 - P * q1 * ib2);
        const float dmd = Q * (-2.f * ib1) * (md + my * p1) + P * (2.f * ib2) * (md + my * q1);
        g0 = up * (dmx + dmd);
        g1 = up * P * q1 * ib2;
        g2 = -up * P * ib2;
      }
      sa[(0 * kSsimB + r) * kSsimBP + q] = g0;
      sa[(1 * kSsimB + r) * kSsimBP + q] = g1;
      sa[(2 * kSsimB + r) * kSsimBP + q] = g2;
    }
  }
  __syncthreads();
  // row filter of the G maps: F[k][r][q0 .. q0 + 3], r in [0, 42), q0 = 4 g
  constexpr int kG2 = kSsimT / kSsimRB;   // 8 groups along an output row
  for (int e = threadIdx.x; e < kSsimB * kG2; e += kSsimThreads) {
    const int r = e / kG2, q0 = (e % kG2) * kSsimRB;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float v[16];
      load16(sa + (k * kSsimB + r) * kSsimBP + q0, v);
      float f[kSsimRB];
#pragma unroll
      for (int o = 0; o < kSsimRB; ++o) {
        float a = 0.f;
#pragma unroll
        for (int t = 0; t <= 2 * kSsimR; ++t) a = fmaf(win.g[t], v[o + t], a);
        f[o] = a;
      }
      *reinterpret_cast<float4*>(sb + (k * kSsimB + r) * kSsimT + q0) =
          make_float4(f[0], f[1], f[2], f[3]);
    }
  }
  __syncthreads();
  // column filter to the tile (rows r0 .. r0 + 3 of column q) and the gradient
  if (g_x) {
    for (int e = threadIdx.x; e < kSsimT * kG2; e += kSsimThreads) {
      const int q = e % kSsimT, r0 = (e / kSsimT) * kSsimRB;
      const int px = tx0 + q;
      float f[3][kSsimRB];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float* col = sb + (k * kSsimB + r0) * kSsimT + q;
        float v[kSsimRB + 2 * kSsimR];
#pragma unroll
        for (int t = 0; t < kSsimRB + 2 * kSsimR; ++t) v[t] = col[t * kSsimT];
#pragma unroll
        for (int o = 0; o < kSsimRB; ++o) {
          float a = 0.f;
#pragma unroll
          for (int t = 0; t <= 2 * kSsimR; ++t) a = fmaf(win.g[t], v[o + t], a);
          f[k][o] = a;
        }
      }
      if (px >= W) continue;
#pragma unroll
      for (int o = 0; o < kSsimRB; ++o) {
        const int py = ty0 + r0 + o;
        if (py >= H) break;
        const size_t i = ((size_t)py * W + px) * 3 + c;
        const float xv = x[i], yv = y[i];
        g_x[i] += fmaf(2.f * xv, f[1][o], fmaf(2.f * (xv - yv), f[2][o], f[0][o]));
      }
    }
  }
  const float t = block_sum256(loss, s_red);
  if (threadIdx.x == 0)
    part[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
}

// loss[0] += scale * (fixed-order sum of the block partials)
__global__ void ssim_sum_kernel(const float* __restrict__ part, int n, float scale,
                                float* __restrict__ loss) {
  __shared__ float s_red[kSsimThreads / 32];
  float a = 0.f;
  for (int i = threadIdx.x; i < n; i += kSsimThreads) a += part[i];
  const float t = block_sum256(a, s_red);
  if (threadIdx.x == 0) loss[0] += scale * t;
}

SsimWin ssim_window() {
  SsimWin w;
  double g[2 * kSsimR + 1], s = 0.0;
  for (int t = 0; t <= 2 * kSsimR; ++t) {
    const double d = t - kSsimR;
    g[t] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
    s += g[t];
  }
  for (int t = 0; t <= 2 * kSsimR; ++t) w.g[t] = (float)(g[t] / s);
  return w;
}

size_t ssim_ws_bytes(int height, int width) {
  const size_t nb = (size_t)((width + kSsimT - 1) / kSsimT) * ((height + kSsimT - 1) / kSsimT) * 3;
  return align_up(nb * sizeof(float), 256);
}

int ssim_launch(const float* x, const float* y, int height, int width, float weight, float* g_x,
                float* loss, void* workspace, size_t ws_bytes, size_t* ws_needed,
                cudaStream_t st) {
  if (height <= 0 || width <= 0 || !x || !y || !loss) return GS2D_ERR_INVALID_ARG;
  const size_t need = ssim_ws_bytes(height, width);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(ssim_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSsimSmemBytes) != cudaSuccess)
      return GS2D_ERR_CUDA;
    attr_set = true;
  }
  const dim3 grid((width + kSsimT - 1) / kSsimT, (height + kSsimT - 1) / kSsimT, 3);
  float* part = static_cast<float*>(workspace);
  ssim_kernel<<<grid, kSsimThreads, kSsimSmemBytes, st>>>(x, y, height, width, weight,
                                                          ssim_window(), g_x, part);
  GS2D_LAUNCH_CHECK();
  ssim_sum_kernel<<<1, kSsimThreads, 0, st>>>(part, (int)(grid.x * grid.y * grid.z),
                                              weight / (3.f * (float)height * (float)width), loss);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

}  // namespace gs2d

using namespace gs2d;

extern "C" {

size_t gs2d_ssim_workspace(int height, int width) { return ssim_ws_bytes(height, width); }

int gs2d_ssim_loss(const float* x, const float* y, int height, int width, float weight,
                   float* g_x, float* loss, void* workspace, size_t ws_bytes, size_t* ws_needed,
                   gs2d_stream stream) {
  return ssim_launch(x, y, height, width, weight, g_x, loss, workspace, ws_bytes, ws_needed,
                     (cudaStream_t)stream);
}

}  // extern "C"
