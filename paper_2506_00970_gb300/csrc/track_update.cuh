// Pose update of the tracking loop (Sec. III-D): fixed-order reduction of
// the tiles' loss and pose partials, AdamW on tau = (rho, theta) and the
// left retraction T <- Exp(tau) T.  Included by the fused tile kernel, whose
// last block runs it.
#pragma once

#include <math.h>

#include "gs2d_common.cuh"

namespace gs2d {

constexpr int32_t kConverged = 256;  // status value after early stopping

// SE(3) exponential of tau = (rho, theta): R = I + A K + B K^2,
// t = (I + B K + C K^2) rho with K = [theta]_x, A = sin t / t,
// B = (1 - cos t) / t^2, C = (t - sin t) / t^3 (series for small angles).
__device__ __forceinline__ void se3_exp_f(const float tau[6], float R[9], float t[3]) {
  const float wx = tau[3], wy = tau[4], wz = tau[5];
  const float th2 = wx * wx + wy * wy + wz * wz;
  const float th = sqrtf(th2);
  float A, B, C;
  if (th < 1e-2f) {
    A = 1.f - th2 / 6.f + th2 * th2 / 120.f;
    B = 0.5f - th2 / 24.f + th2 * th2 / 720.f;
    C = 1.f / 6.f - th2 / 120.f + th2 * th2 / 5040.f;
  } else {
    const float s = sinf(th), c = cosf(th);
    A = s / th;
    B = (1.f - c) / th2;
    C = (th - s) / (th2 * th);
  }
  const float K[9] = {0.f, -wz, wy, wz, 0.f, -wx, -wy, wx, 0.f};
  float K2[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      K2[3 * r + c] = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
  for (int k = 0; k < 9; ++k) {
    const float I = (k % 4 == 0) ? 1.f : 0.f;
    R[k] = I + A * K[k] + B * K2[k];
  }
  for (int r = 0; r < 3; ++r) {
    float acc = 0.f;
    for (int c = 0; c < 3; ++c) {
      const float V = ((r == c) ? 1.f : 0.f) + B * K[3 * r + c] + C * K2[3 * r + c];
      acc += V * tau[c];
    }
    t[r] = acc;
  }
}

// Records the history of an iteration that is skipped after convergence:
// the previous loss, the unchanged pose and a zero gradient (none is formed).
__device__ __forceinline__ void record_converged(const float* __restrict__ pose,
                                                 float* __restrict__ loss_hist,
                                                 float* __restrict__ pose_hist,
                                                 float* __restrict__ grad_hist, int iter) {
  if (loss_hist) loss_hist[iter] = loss_hist[iter > 0 ? iter - 1 : 0];
  if (pose_hist)
    for (int k = 0; k < 12; ++k) pose_hist[12 * iter + k] = pose[k];
  if (grad_hist)
    for (int k = 0; k < 6; ++k) grad_hist[6 * iter + k] = 0.f;
}

// Block-wide (256 threads): sum the n_part partials in a fixed order (L1 is
// bypassed: other blocks wrote them), then thread 0 takes the AdamW step
// (tau is zero before the step, so weight decay has no effect) and retracts.
// Records the loss and the gradient at the pre-update pose and the updated
// pose.  A non-finite loss or gradient leaves the pose and the moments as
// they were and records GS2D_ERR_NONFINITE.  adam = m[6], v[6], step, done.
__device__ __forceinline__ void reduce_and_step(const float* __restrict__ pose_part,
                                const float* __restrict__ loss_part, int n_part,
                                float* __restrict__ pose, float* __restrict__ adam,
                                const gs2d_track_params& prm, float* __restrict__ loss_hist,
                                float* __restrict__ pose_hist, float* __restrict__ grad_hist,
                                int iter, int32_t* __restrict__ status, float (*s)[256]) {
  float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int b = threadIdx.x; b < n_part; b += 256) {
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += __ldcg(pose_part + (size_t)b * 6 + c);
    acc[6] += __ldcg(loss_part + b);
  }
#pragma unroll
  for (int c = 0; c < 7; ++c) s[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int c = 0; c < 7; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  bool finite = isfinite(s[6][0]);
  for (int k = 0; k < 6; ++k) finite = finite && isfinite(s[k][0]);
  if (loss_hist) loss_hist[iter] = s[6][0];
  if (grad_hist)
    for (int k = 0; k < 6; ++k) grad_hist[6 * iter + k] = s[k][0];
  if (!finite) {
    *status = GS2D_ERR_NONFINITE;
    return;
  }
  const float step = adam[12] + 1.f;
  adam[12] = step;
  const float bc1 = 1.f - powf(prm.beta1, step), bc2 = 1.f - powf(prm.beta2, step);
  float tau[6];
  float nrm2 = 0.f;
  for (int k = 0; k < 6; ++k) {
    const float g = s[k][0];
    const float m = prm.beta1 * adam[k] + (1.f - prm.beta1) * g;
    const float v = prm.beta2 * adam[6 + k] + (1.f - prm.beta2) * g * g;
    adam[k] = m;
    adam[6 + k] = v;
    tau[k] = -prm.lr * (m / bc1) / (sqrtf(v / bc2) + prm.eps);
    nrm2 += tau[k] * tau[k];
  }
  float dR[9], dt[3];
  se3_exp_f(tau, dR, dt);
  float R[9], t[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c)
      R[3 * r + c] = dR[3 * r] * pose[c] + dR[3 * r + 1] * pose[3 + c] + dR[3 * r + 2] * pose[6 + c];
    t[r] = dR[3 * r] * pose[9] + dR[3 * r + 1] * pose[10] + dR[3 * r + 2] * pose[11] + dt[r];
  }
  for (int k = 0; k < 9; ++k) pose[k] = R[k];
  for (int k = 0; k < 3; ++k) pose[9 + k] = t[k];
  if (pose_hist)
    for (int k = 0; k < 12; ++k) pose_hist[12 * iter + k] = pose[k];
  if (sqrtf(nrm2) < prm.stop_tol) {
    adam[13] = 1.f;
    *status = kConverged;
  }
}

}  // namespace gs2d
