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

// Shared memory (floats): region A holds x and y (2 x 52 x 52), later the
// three G maps (3 x 42 x 42); region B holds the five row-filtered moment
// maps (5 x 52 x 42), later the three row-filtered G maps (3 x 42 x 32).
constexpr int kSsimSmemA = 2 * kSsimA * kSsimA;
constexpr int kSsimSmemB = 5 * kSsimA * kSsimB;
constexpr size_t kSsimSmemBytes = (size_t)(kSsimSmemA + kSsimSmemB) * sizeof(float);
static_assert(3 * kSsimB * kSsimB <= kSsimSmemA, "G maps fit region A");
static_assert(3 * kSsimB * kSsimT <= kSsimSmemB, "filtered G maps fit region B");

__global__ void __launch_bounds__(kSsimThreads) ssim_kernel(const float* __restrict__ x,
                                                           const float* __restrict__ y, int H,
                                                           int W, float weight, SsimWin win,
                                                           float* __restrict__ g_x,
                                                           float* __restrict__ part) {
  extern __shared__ float smem[];
  float* sa = smem;                 // x [52][52], y [52][52]  ->  G [3][42][42]
  float* sb = smem + kSsimSmemA;    // M [5][52][42]           ->  F [3][42][32]
  __shared__ float s_red[kSsimThreads / 32];
  const int c = blockIdx.z;
  const int tx0 = blockIdx.x * kSsimT, ty0 = blockIdx.y * kSsimT;
  const int ax0 = tx0 - 2 * kSsimR, ay0 = ty0 - 2 * kSsimR;   // staged origin
  // stage x, y (zero outside the image)
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
  __syncthreads();
  // row filter of the five moments: M[k][r][q], r in [0,52), q in [0,42)
  for (int e = threadIdx.x; e < kSsimA * kSsimB; e += kSsimThreads) {
    const int r = e / kSsimB, q = e % kSsimB;
    const float* rx = sa + r * kSsimA + q;
    const float* ry = rx + kSsimA * kSsimA;
    float mx = 0.f, md = 0.f, exx = 0.f, eyy = 0.f, edd = 0.f;
#pragma unroll
    for (int t = 0; t <= 2 * kSsimR; ++t) {
      const float a = rx[t], b = ry[t], w = win.g[t];
      const float d = a - b;
      const float wa = w * a, wb = w * b, wd = w * d;
      mx += wa;
      md += wd;
      exx = fmaf(wa, a, exx);
      eyy = fmaf(wb, b, eyy);
      edd = fmaf(wd, d, edd);
    }
    sb[e] = mx;
    sb[kSsimA * kSsimB + e] = md;
    sb[2 * kSsimA * kSsimB + e] = exx;
    sb[3 * kSsimA * kSsimB + e] = eyy;
    sb[4 * kSsimA * kSsimB + e] = edd;
  }
  __syncthreads();
  // column filter, S and the G maps on the 42 x 42 region (origin tile - 5);
  // x and y are no longer needed, so the G maps take region A
  const float up = -weight / (3.f * (float)H * (float)W);
  float loss = 0.f;
  for (int e = threadIdx.x; e < kSsimB * kSsimB; e += kSsimThreads) {
    const int r = e / kSsimB, q = e % kSsimB;
    float m[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float* col = sb + k * kSsimA * kSsimB + r * kSsimB + q;
      float s = 0.f;
#pragma unroll
      for (int t = 0; t <= 2 * kSsimR; ++t) s = fmaf(win.g[t], col[t * kSsimB], s);
      m[k] = s;
    }
    const int py = ty0 - kSsimR + r, px = tx0 - kSsimR + q;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (px >= 0 && py >= 0 && px < W && py < H) {
      const float mx = m[0], md = m[1], my = mx - md;
      const float b1 = fmaf(mx, mx, fmaf(my, my, kSsimC1));
      const float b2 = (m[2] - mx * mx) + (m[3] - my * my) + kSsimC2;
      const float vd = m[4] - md * md;
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
    sa[e] = g0;
    sa[kSsimB * kSsimB + e] = g1;
    sa[2 * kSsimB * kSsimB + e] = g2;
  }
  __syncthreads();
  // row filter of the G maps: F[k][r][q], r in [0,42), q in [0,32)
  for (int e = threadIdx.x; e < kSsimB * kSsimT; e += kSsimThreads) {
    const int r = e / kSsimT, q = e % kSsimT;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float* row = sa + k * kSsimB * kSsimB + r * kSsimB + q;
      float s = 0.f;
#pragma unroll
      for (int t = 0; t <= 2 * kSsimR; ++t) s = fmaf(win.g[t], row[t], s);
      sb[k * kSsimB * kSsimT + e] = s;
    }
  }
  __syncthreads();
  // column filter to the tile and the gradient
  if (g_x) {
    for (int e = threadIdx.x; e < kSsimT * kSsimT; e += kSsimThreads) {
      const int r = e / kSsimT, q = e % kSsimT;
      const int py = ty0 + r, px = tx0 + q;
      if (px >= W || py >= H) continue;
      float f[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float* col = sb + k * kSsimB * kSsimT + r * kSsimT + q;
        float s = 0.f;
#pragma unroll
        for (int t = 0; t <= 2 * kSsimR; ++t) s = fmaf(win.g[t], col[t * kSsimT], s);
        f[k] = s;
      }
      const size_t i = ((size_t)py * W + px) * 3 + c;
      const float xv = x[i], yv = y[i];
      g_x[i] += fmaf(2.f * xv, f[1], fmaf(2.f * (xv - yv), f[2], f[0]));
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
