// Internal launchers shared between translation units.  Each takes a device
// "gate" word: its kernels return immediately while *gate != 0 (an error, or
// a converged tracking loop), which keeps a captured launch sequence valid
// without host round trips.
#pragma once

#include <cuda_runtime.h>

#include "gs2d.h"

namespace gs2d {

// Binning state a fused projection fills: tile counts (shared-memory
// histograms flushed with global atomics), then, by its last block, the tile
// ranges, K, the capacity check and the long-tile list.
struct SortFuse {
  uint32_t* tile_count;
  int32_t* ranges;
  int32_t* n_isect;
  long long capacity;
  uint32_t* long_list;
  uint32_t* n_long;
  uint32_t* done;   // block completion counter (zeroed before the launch)
  int tiles_x, n_tiles, long_len;
  int32_t* order;   // [n_tiles] launch order of the tiles, longest lists first (or NULL)
  // scatter fused into the projection (NULL: not fused): after a grid-wide
  // barrier every block writes its own pairs' keys into the tile segments
  unsigned long long* seg_keys;
  uint32_t* cursor;  // [n_tiles] slots claimed per tile (zeroed before the launch)
  uint32_t* bar;     // grid barrier counter (zeroed before the launch)
};
// Whether the projection can also scatter the pairs (its tile histograms
// fit in shared memory).
bool project_can_fuse_scatter(int n_tiles);

// Per-surfel projection; with fuse, also the binning's tile counts and scan
// (the binning then runs with kSortPreScanned).
int project_launch(const gs2d_surfels* s, const gs2d_camera* cam, const float* pose,
                   const gs2d_config* cfg, float* proj_out, int32_t* tiles_per_surfel_out,
                   const int32_t* gate, cudaStream_t st, const SortFuse* fuse = nullptr);

// gs2d_bin_sort; with need_emit false the emission offsets and indices
// (used only by the full backward) are not computed.  flags:
// kSortPreZeroed -- the caller has zeroed the counter region
// (sort_zero_region) since the last binning, so no init launch;
// kSortLongInBlock -- tiles with segments over 2048 keys are sorted by their
// own 256-thread block (chunks + merges) instead of a separate launch.
// kSortPreScanned -- a fused projection already counted and scanned the
// tiles (implies pre-zeroed counters; no emission offsets);
// kSortInTileKernel -- no per-tile sort launch: the tile kernel that reads
// the bins sorts each tile's segment itself (sort_seg_args).
constexpr unsigned kSortPreZeroed = 1u, kSortLongInBlock = 2u, kSortPreScanned = 4u,
                   kSortInTileKernel = 8u;
// Binning of several views, one launch per stage (sort.cu): the workspace
// is a 256-byte header followed by each view's gs2d_bin_sort workspace.
size_t bin_sort_batch_bytes(const gs2d_view* views, int n_views, int n);
size_t bin_sort_batch_header();
size_t bin_sort_batch_view_bytes(int m, size_t capacity);
int bin_sort_batch_launch(const gs2d_view* views, int n_views, int n, void* workspace,
                          size_t ws_bytes, size_t* ws_needed, cudaStream_t st);
int bin_sort_launch(const float* proj, const int32_t* tiles_per_surfel, int n,
                    const gs2d_camera* cam, const gs2d_config* cfg, void* workspace,
                    size_t ws_bytes, size_t* ws_needed, const gs2d_bins* bins, bool need_emit,
                    cudaStream_t st, unsigned flags = 0u);
// Pointers of a sort workspace for a fused projection.
SortFuse sort_fuse_args(void* workspace, int n, const gs2d_bins* bins, int tiles_x, int n_tiles);
// The unsorted segment keys and the merge buffer of a sort workspace.
void sort_seg_args(void* workspace, int n, size_t capacity, int n_tiles,
                   unsigned long long** seg_keys, unsigned long long** seg_tmp);
// The counter region of a sort workspace that every binning needs zeroed.
void sort_zero_region(void* workspace, int n, size_t capacity, int n_tiles, uint32_t** begin,
                      size_t* words);

// Camera and tile configuration check shared by the tile kernels' entry
// points (GS2D_OK or GS2D_ERR_INVALID_ARG).
int validate_tile_cfg(const gs2d_camera* cam, const gs2d_config* cfg);

// SSIM term (weight / |Omega| sum_p (1 - mean_c SSIM_c(p)) added to *loss,
// its gradient added to g_x): x, y [H*W*3].
size_t ssim_ws_bytes(int height, int width);
int ssim_launch(const float* x, const float* y, int height, int width, float weight, float* g_x,
                float* loss, void* workspace, size_t ws_bytes, size_t* ws_needed,
                cudaStream_t st);

int render_fwd_launch(const float* proj, const gs2d_bins* bins, const gs2d_camera* cam,
                      const gs2d_config* cfg, float* rgb, float* depth, float* normal,
                      float* opacity, float* t_final, uint32_t* n_last, const int32_t* gate,
                      cudaStream_t st);

// The pose-update state the fused tracking kernel's last block works on.
struct TrackStep {
  float* pose;       // [12] in/out
  float* adam;       // [16] m, v, step, done
  float* loss_hist;  // [n_iter] or NULL
  float* pose_hist;  // [n_iter * 12] or NULL
  float* grad_hist;  // [n_iter * 6] or NULL
  int iter;
  uint32_t* counter; // blocks finished in this iteration (reset by the last)
  uint32_t* sort_zero;   // binning counters the last block zeroes for the next
  size_t sort_zero_words;  // iteration's binning (kSortPreZeroed)
  const int32_t* order;    // block b runs tile order[b] (or b when NULL)
  // the binning's unsorted tile segments (kSortInTileKernel): each block
  // sorts its own tile's keys; seg_tmp is the merge buffer of long segments
  unsigned long long* seg_keys;
  unsigned long long* seg_tmp;
  int n;  // surfels (ids are clamped below it)
};

// Fused tracking iteration per tile (forward, tracking loss, pose backward)
// with the pose update in the last block: loss_part [n_tiles] (already
// divided by the pixel count), pose_part [n_tiles * 6].  status is the gate.
int track_tile_launch(const float* proj, const gs2d_bins* bins, const gs2d_camera* cam,
                      const gs2d_config* cfg, const float* obs_rgb, const float* obs_depth,
                      const gs2d_track_params* prm, float* loss_part, float* pose_part,
                      const TrackStep& ts, int32_t* status, cudaStream_t st);

size_t render_bwd_ws_bytes(int n, size_t cap, int n_tiles, bool full, int Q);
int render_bwd_launch(const float* proj, const gs2d_bins* bins, const int32_t* tiles_per_surfel,
                      const gs2d_surfels* s, const float* pose, const gs2d_camera* cam,
                      const gs2d_config* cfg, const float* t_final, const uint32_t* n_last,
                      const float* d_rgb, const float* d_depth, const float* d_normal,
                      const float* d_opacity, float* d_mu, float* d_quat, float* d_scale,
                      float* d_opac, float* d_rgb_out, float* d_pose6, void* workspace,
                      size_t ws_bytes, size_t* ws_needed, const int32_t* gate, cudaStream_t st);

size_t loss_ws_bytes(const gs2d_camera* cam);
int tracking_loss_launch(const float* rgb, const float* depth, const float* normal,
                         const float* opacity, const float* obs_rgb, const float* obs_depth,
                         const gs2d_camera* cam, const gs2d_track_params* prm, float* g_rgb,
                         float* g_depth, float* g_opacity, float* loss_out, void* workspace,
                         size_t ws_bytes, size_t* ws_needed, const int32_t* gate, cudaStream_t st);

// Per-surfel reduction of one view's (tile, region, surfel) partials, Q
// region slots per tile, with the view's projected records proj (record i
// is surfel active[i] or i; accumulate adds into the outputs) and the block partials of that view's pose gradient;
// fixed-order pose reduction.
int surfel_grad_launch(const gs2d_surfels* s, const int32_t* active, int m, int accumulate,
                       const float* pose, const int32_t* tiles, const uint32_t* surfel_off, int Q,
                       const float* proj, const float* partials, float* d_mu, float* d_quat,
                       float* d_scale, float* d_opac, float* d_rgb, float* pose_part,
                       const int32_t* gate, cudaStream_t st);
int pose_reduce_launch(const float* part, int n_part, float* out, const int32_t* gate,
                       cudaStream_t st);

}  // namespace gs2d
