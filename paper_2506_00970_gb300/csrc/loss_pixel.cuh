// Per-pixel tracking loss and its gradient (Eq. tracking_loss with the masks
// of Eq. normal_mask and opacity_mask), shared by the standalone loss kernel
// and the fused tracking kernel so both compute identical numbers.
#pragma once

#include "gs2d_common.cuh"

namespace gs2d {

__device__ __forceinline__ float sgnf(float v) { return (float)((v > 0.f) - (v < 0.f)); }

struct PixLoss {
  float loss;        // M_n M_o (|I_r - I|_1 + lambda_d |D_r - D|) (not yet / |Omega|)
  float g_rgb[3];    // dL/d rendered colour (with the 1/|Omega| factor)
  float g_depth;     // dL/d literal depth D = sum w z
  float g_opac;      // dL/d opacity O
};

// rx, ry: the pixel ray's (x - cx)/fx, (y - cy)/fy; its length does not
// change the sign of N_r . r.  depth_mode 1: D_r = D / max(O, 1e-6).
// Sub-gradient sign(0) = 0; the masks carry no gradient.
__device__ __forceinline__ PixLoss tracking_pixel_loss(F3 rgb, float D, F3 N, float O, F3 obs,
                                                       float obs_d, float rx, float ry, float inv,
                                                       const gs2d_track_params& prm) {
  PixLoss r;
  r.loss = 0.f;
  r.g_rgb[0] = r.g_rgb[1] = r.g_rgb[2] = 0.f;
  r.g_depth = 0.f;
  r.g_opac = 0.f;
  const float nr = N.x * rx + N.y * ry + N.z;
  if (!((nr > 0.f) && (O > prm.opacity_thresh))) return r;
  const float Oc = fmaxf(O, 1e-6f);
  const float Dh = prm.depth_mode ? D / Oc : D;
  const float d0 = rgb.x - obs.x, d1 = rgb.y - obs.y, d2 = rgb.z - obs.z;
  const float dd = Dh - obs_d;
  r.loss = fabsf(d0) + fabsf(d1) + fabsf(d2) + prm.lambda_d * fabsf(dd);
  r.g_rgb[0] = sgnf(d0) * inv;
  r.g_rgb[1] = sgnf(d1) * inv;
  r.g_rgb[2] = sgnf(d2) * inv;
  const float sd = prm.lambda_d * sgnf(dd) * inv;
  if (prm.depth_mode) {
    r.g_depth = sd / Oc;
    r.g_opac = O > 1e-6f ? -sd * D / (O * O) : 0.f;
  } else {
    r.g_depth = sd;
  }
  return r;
}

}  // namespace gs2d
