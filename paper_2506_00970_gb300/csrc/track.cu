// gs2d_track_step: frame-to-map camera tracking (Sec. III-D) as one device-
// resident launch sequence.  Each iteration projects and bins the map at the
// current pose, then one fused kernel per tile renders it, evaluates the
// masked tracking loss (Eq. tracking_loss) and back-propagates it to the pose
// tangent only (Sec. III-B; the map is frozen during tracking), and a last
// block of that kernel reduces the tiles' partials and takes an AdamW step on
// tau = (rho, theta) followed by the retraction T <- Exp(tau) T with tau reset
// to zero (the moments are kept across iterations of the frame, in the
// caller's AdamW state when one is given, so a frame may span several calls).
// Kernels per iteration: the projection (which also counts, scans and --
// for up to 2048 tiles -- scatters the tile pairs; otherwise the binning's
// scatter kernel follows) and the fused tile kernel (which first sorts its
// tile's segment by depth) -- 2 or 3.
#include <math.h>

#include "gs2d_common.cuh"
#include "gs2d_internal.h"
#include "track_update.cuh"

namespace gs2d {


// Optional timing of the fused tile kernel (see gs2d_profile_track_kernel).
struct KernelTimer {
  cudaEvent_t* start = nullptr;
  cudaEvent_t* stop = nullptr;
  int capacity = 0;
  int used = 0;
  int every = 1;  // bracket the launches of iterations it % every == 0
};
KernelTimer g_timer;

// Records a timing event; inside a stream capture it becomes an event-record
// node of the graph (cudaEventRecordExternal), so replays record it.
cudaError_t record_timing_event(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  return cudaEventRecordWithFlags(
      ev, st, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// Start of a call: zero the completion counter, the status word and the
// binning counters, and the moments when they live in the workspace (a
// caller-owned AdamW state is left as the caller passed it).
__global__ void track_reset_kernel(float* adam, uint32_t* counter, int32_t* status,
                                   uint32_t* sort_zero, size_t sort_zero_words) {
  if (adam && threadIdx.x < 16) adam[threadIdx.x] = 0.f;
  if (threadIdx.x == 0) {
    *counter = 0u;
    *status = 0;
  }
  for (size_t i = threadIdx.x; i < sort_zero_words; i += blockDim.x) sort_zero[i] = 0u;
}

struct TrackWs {
  float* proj;
  int32_t* tiles;
  uint32_t *vals, *emit, *soff;
  int32_t *ranges, *n_isect, *order;
  void* sort_ws;
  size_t sort_bytes;
  float *loss_part, *pose_part, *adam;
  uint32_t* counter;
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
  w.order = c.take<int32_t>((size_t)nt);
  w.sort_bytes = gs2d_bin_sort_workspace(n, cap);
  w.sort_ws = c.take<char>(w.sort_bytes);
  w.loss_part = c.take<float>((size_t)nt);
  w.pose_part = c.take<float>((size_t)nt * 6);
  w.adam = c.take<float>(16);
  w.counter = c.take<uint32_t>(1);
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

int gs2d_profile_track_kernel_every(int every) {
  if (every < 1) return GS2D_ERR_INVALID_ARG;
  g_timer.every = every;
  return GS2D_OK;
}

int32_t* gs2d_track_status(void* workspace) {
  return workspace ? reinterpret_cast<int32_t*>(workspace) : nullptr;
}

const int32_t* gs2d_track_tile_order(void* workspace, int n, size_t capacity,
                                     const gs2d_camera* cam, const gs2d_config* cfg) {
  if (!workspace || !cam || !cfg) return nullptr;
  return carve_track_ws(static_cast<char*>(workspace) + 256, n, capacity, cam, cfg).order;
}

int gs2d_track_step(const gs2d_surfels* s, const gs2d_camera* cam, const gs2d_config* cfg,
                    const gs2d_track_params* prm, float* pose, float* adam_state,
                    const float* obs_rgb, const float* obs_depth, int n_iter, size_t capacity,
                    float* loss_hist, float* pose_hist, float* grad_hist, void* workspace,
                    size_t ws_bytes, size_t* ws_needed, gs2d_stream stream) {
  if (!s || !cam || !cfg || !prm || !pose || !obs_rgb || !obs_depth || n_iter < 0)
    return GS2D_ERR_INVALID_ARG;
  if (capacity >= (size_t)0x3FFFFFFF) return GS2D_ERR_INVALID_ARG;
  if (adam_state && (reinterpret_cast<uintptr_t>(adam_state) & 3)) return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_track_workspace(s->n, capacity, cam, cfg);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  // byte 0..255: the status word (stable address for gs2d_track_status)
  int32_t* status = reinterpret_cast<int32_t*>(workspace);
  const TrackWs w = carve_track_ws(static_cast<char*>(workspace) + 256, s->n, capacity, cam, cfg);
  // binning counters: zeroed here for the first iteration and by the fused
  // kernel's last block for every later one (no init launch per iteration)
  uint32_t* zero_begin = nullptr;
  size_t zero_words = 0;
  sort_zero_region(w.sort_ws, s->n, capacity, gs2d_tiles_x(cam, cfg) * gs2d_tiles_y(cam, cfg),
                   &zero_begin, &zero_words);
  float* adam = adam_state ? adam_state : w.adam;
  track_reset_kernel<<<1, 256, 0, st>>>(adam_state ? nullptr : w.adam, w.counter, status,
                                        zero_begin, zero_words);
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
  // projection, tile counts and tile scan in one launch, and every block of
  // the fused tile kernel sorts its own tile's segment
  const int tiles_x = gs2d_tiles_x(cam, cfg);
  SortFuse fuse = sort_fuse_args(w.sort_ws, s->n, &bins, tiles_x,
                                 tiles_x * gs2d_tiles_y(cam, cfg));
  // the projection's last block also orders the tiles by decreasing list
  // length; the fused tile kernel launches them in that order
  fuse.order = w.order;
  unsigned long long *seg_keys = nullptr, *seg_tmp = nullptr;
  sort_seg_args(w.sort_ws, s->n, capacity, tiles_x * gs2d_tiles_y(cam, cfg), &seg_keys, &seg_tmp);
  // up to 2048 tiles the projection also scatters the pairs into the tile
  // segments (a cooperative launch with a grid barrier); beyond, the
  // binning's scatter kernel does
  const bool fused_scatter = project_can_fuse_scatter(fuse.n_tiles);
  if (fused_scatter) fuse.seg_keys = seg_keys;
  for (int it = 0; it < n_iter; ++it) {
    int r = project_launch(s, cam, pose, cfg, w.proj, w.tiles, status, st, &fuse);
    if (r) return r;
    if (!fused_scatter) {
      r = bin_sort_launch(w.proj, w.tiles, s->n, cam, cfg, w.sort_ws, w.sort_bytes, nullptr,
                          &bins, false, st, kSortPreZeroed | kSortPreScanned | kSortInTileKernel);
      if (r) return r;
    }
    const bool timed = g_timer.used < g_timer.capacity && it % g_timer.every == 0;
    if (timed) GS2D_CUDA_TRY(record_timing_event(g_timer.start[g_timer.used], st));
    TrackStep ts{pose, adam, loss_hist, pose_hist, grad_hist, it, w.counter, zero_begin,
                 zero_words, w.order, seg_keys, seg_tmp, s->n};
    r = track_tile_launch(w.proj, &bins, cam, cfg, obs_rgb, obs_depth, prm, w.loss_part,
                          w.pose_part, ts, status, st);
    if (r) return r;
    if (timed) GS2D_CUDA_TRY(record_timing_event(g_timer.stop[g_timer.used++], st));
  }
  return GS2D_OK;
}

}  // extern "C"
