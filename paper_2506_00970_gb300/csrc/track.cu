// gs2d_track_step: frame-to-map camera tracking (Sec. III-D) as one device-
// resident launch sequence.  Each iteration projects and bins the map at the
// current pose, then one fused kernel per tile renders it, evaluates the
// masked tracking loss (Eq. tracking_loss) and back-propagates it to the pose
// tangent only (Sec. III-B; the map is frozen during tracking), and a last
// kernel reduces the tiles' partials and takes an AdamW step on
// tau = (rho, theta) followed by the retraction T <- Exp(tau) T with tau reset
// to zero (the moments are kept across iterations of the frame).
// Four launches per iteration: project, bin_sort (5 kernels), fused tile
// kernel, reduce + AdamW -- 8 kernels.
#include <math.h>

#include "gs2d_common.cuh"
#include "gs2d_internal.h"

namespace gs2d {

constexpr int32_t kConverged = 256;  // gate value after early stopping

// Optional timing of the fused tile kernel (see gs2d_profile_track_kernel).
struct KernelTimer {
  cudaEvent_t* start = nullptr;
  cudaEvent_t* stop = nullptr;
  int capacity = 0;
  int used = 0;
};
KernelTimer g_timer;

__global__ void track_reset_kernel(float* adam, int32_t* status) {
  if (threadIdx.x < 16) adam[threadIdx.x] = 0.f;
  if (threadIdx.x == 0) *status = 0;
}

// SE(3) exponential of tau = (rho, theta): R = I + A K + B K^2,
// t = (I + B K + C K^2) rho with K = [theta]_x, A = sin t / t,
// B = (1 - cos t) / t^2, C = (t - sin t) / t^3 (series for small angles).
__device__ void se3_exp_f(const float tau[6], float R[9], float t[3]) {
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

// Fixed-order reduction of the tiles' loss and pose partials, then AdamW on
// tau (zero before the step, so weight decay has no effect) and the left
// retraction.  Records the loss at the pre-update pose and the updated pose.
// adam = m[6], v[6], step, done.
__global__ void __launch_bounds__(256) adam_retract_kernel(
    const float* __restrict__ pose_part, const float* __restrict__ loss_part, int n_part,
    float* __restrict__ pose, float* __restrict__ adam, gs2d_track_params prm,
    float* __restrict__ loss_hist, float* __restrict__ pose_hist, int iter,
    int32_t* __restrict__ status) {
  __shared__ float s[7][256];
  const int32_t st = *status;
  if (st != 0 && st != kConverged) return;
  if (st == kConverged) {
    if (threadIdx.x == 0) {
      if (loss_hist) loss_hist[iter] = loss_hist[iter > 0 ? iter - 1 : 0];
      if (pose_hist)
        for (int k = 0; k < 12; ++k) pose_hist[12 * iter + k] = pose[k];
    }
    return;
  }
  float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int b = threadIdx.x; b < n_part; b += 256) {
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += pose_part[(size_t)b * 6 + c];
    acc[6] += loss_part[b];
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
  const float step = adam[12] + 1.f;
  adam[12] = step;
  const float bc1 = 1.f - powf(prm.beta1, step), bc2 = 1.f - powf(prm.beta2, step);
  float tau[6];
  float nrm2 = 0.f;
  bool finite = true;
  for (int k = 0; k < 6; ++k) {
    const float g = s[k][0];
    finite = finite && isfinite(g);
    const float m = prm.beta1 * adam[k] + (1.f - prm.beta1) * g;
    const float v = prm.beta2 * adam[6 + k] + (1.f - prm.beta2) * g * g;
    adam[k] = m;
    adam[6 + k] = v;
    tau[k] = -prm.lr * (m / bc1) / (sqrtf(v / bc2) + prm.eps);
    nrm2 += tau[k] * tau[k];
  }
  if (loss_hist) loss_hist[iter] = s[6][0];
  if (!finite) {
    *status = GS2D_ERR_NONFINITE;
    return;
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

struct TrackWs {
  float* proj;
  int32_t* tiles;
  uint32_t *vals, *emit, *soff;
  int32_t *ranges, *n_isect;
  void* sort_ws;
  size_t sort_bytes;
  float *loss_part, *pose_part, *adam;
  size_t bytes;
};

TrackWs carve_track_ws(void* base, int n, size_t cap, const gs2d_camera* cam,
                       const gs2d_config* cfg) {
  Carver c(base);
  TrackWs w;
  const size_t nn = n > 0 ? n : 1;
  const size_t cc = cap > 0 ? cap : 1;
  const int nt = gs2d_tiles_x(cam, cfg) * gs2d_tiles_y(cam, cfg);
  w.proj = c.take<float>(nn * kProjFloats);
  w.tiles = c.take<int32_t>(nn);
  w.vals = c.take<uint32_t>(cc);
  w.emit = c.take<uint32_t>(cc);
  w.soff = c.take<uint32_t>(nn);
  w.ranges = c.take<int32_t>(2 * (size_t)nt);
  w.n_isect = c.take<int32_t>(1);
  w.sort_bytes = gs2d_bin_sort_workspace(n, cap);
  w.sort_ws = c.take<char>(w.sort_bytes);
  w.loss_part = c.take<float>((size_t)nt);
  w.pose_part = c.take<float>((size_t)nt * 6);
  w.adam = c.take<float>(16);
  w.bytes = align_up(c.off, 256);
  return w;
}

}  // namespace gs2d

using namespace gs2d;

extern "C" {

size_t gs2d_track_workspace(int n, size_t capacity, const gs2d_camera* cam,
                            const gs2d_config* cfg) {
  if (!cam || !cfg) return 0;
  // the first 256 bytes hold the status word at a size-independent address
  return 256 + carve_track_ws(nullptr, n, capacity, cam, cfg).bytes;
}

int gs2d_profile_track_kernel(void* const* start_events, void* const* stop_events, int n) {
  if (n < 0 || (n > 0 && (!start_events || !stop_events))) return GS2D_ERR_INVALID_ARG;
  g_timer.start = reinterpret_cast<cudaEvent_t*>(const_cast<void**>(start_events));
  g_timer.stop = reinterpret_cast<cudaEvent_t*>(const_cast<void**>(stop_events));
  g_timer.capacity = n;
  g_timer.used = 0;
  return GS2D_OK;
}

int gs2d_profile_track_kernel_count(void) { return g_timer.used; }

int32_t* gs2d_track_status(void* workspace) {
  return workspace ? reinterpret_cast<int32_t*>(workspace) : nullptr;
}

int gs2d_track_step(const gs2d_surfels* s, const gs2d_camera* cam, const gs2d_config* cfg,
                    const gs2d_track_params* prm, float* pose, const float* obs_rgb, const float* obs_depth, int n_iter, size_t capacity,
                    float* loss_hist, float* pose_hist, void* workspace, size_t ws_bytes,
                    size_t* ws_needed, gs2d_stream stream) {
  if (!s || !cam || !cfg || !prm || !pose || !obs_rgb || !obs_depth || n_iter < 0)
    return GS2D_ERR_INVALID_ARG;
  if (capacity >= (size_t)0x3FFFFFFF) return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_track_workspace(s->n, capacity, cam, cfg);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  // byte 0..255: the status word (stable address for gs2d_track_status)
  int32_t* status = reinterpret_cast<int32_t*>(workspace);
  const TrackWs w = carve_track_ws(static_cast<char*>(workspace) + 256, s->n, capacity, cam, cfg);
  track_reset_kernel<<<1, 32, 0, st>>>(w.adam, status);
  GS2D_LAUNCH_CHECK();
  gs2d_bins bins;
  bins.keys = nullptr;
  bins.vals = w.vals;
  bins.isect_emit = w.emit;
  bins.surfel_off = w.soff;
  bins.tile_ranges = w.ranges;
  bins.n_isect = w.n_isect;
  bins.status = status;
  bins.capacity = capacity;
  const int n_tiles = gs2d_tiles_x(cam, cfg) * gs2d_tiles_y(cam, cfg);
  for (int it = 0; it < n_iter; ++it) {
    int r = project_launch(s, cam, pose, cfg, w.proj, w.tiles, status, st);
    if (r) return r;
    r = gs2d_bin_sort(w.proj, w.tiles, s->n, cam, cfg, w.sort_ws, w.sort_bytes, nullptr, &bins,
                      stream);
    if (r) return r;
    const bool timed = g_timer.used < g_timer.capacity;
    if (timed) GS2D_CUDA_TRY(cudaEventRecord(g_timer.start[g_timer.used], st));
    r = track_tile_launch(w.proj, &bins, cam, cfg, obs_rgb, obs_depth, prm, w.loss_part,
                          w.pose_part, status, st);
    if (r) return r;
    if (timed) GS2D_CUDA_TRY(cudaEventRecord(g_timer.stop[g_timer.used++], st));
    adam_retract_kernel<<<1, 256, 0, st>>>(w.pose_part, w.loss_part, n_tiles, pose, w.adam, *prm,
                                           loss_hist, pose_hist, it, status);
    GS2D_LAUNCH_CHECK();
  }
  return GS2D_OK;
}

}  // extern "C"
