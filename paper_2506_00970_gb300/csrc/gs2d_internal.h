// Internal launchers shared between translation units.  Each takes a device
// "gate" word: its kernels return immediately while *gate != 0 (an error, or
// a converged tracking loop), which keeps a captured launch sequence valid
// without host round trips.
#pragma once

#include <cuda_runtime.h>

#include "gs2d.h"

namespace gs2d {

int project_launch(const gs2d_surfels* s, const gs2d_camera* cam, const float* pose,
                   const gs2d_config* cfg, float* proj_out, int32_t* tiles_per_surfel_out,
                   const int32_t* gate, cudaStream_t st);

int render_fwd_launch(const float* proj, const gs2d_bins* bins, const gs2d_camera* cam,
                      const gs2d_config* cfg, float* rgb, float* depth, float* normal,
                      float* opacity, float* t_final, uint32_t* n_last, const int32_t* gate,
                      cudaStream_t st);

// Fused tracking iteration (forward, tracking loss, pose backward) per tile:
// loss_part [n_tiles] (already divided by the pixel count), pose_part
// [n_tiles * 6].
int track_tile_launch(const float* proj, const gs2d_bins* bins, const gs2d_camera* cam,
                      const gs2d_config* cfg, const float* obs_rgb, const float* obs_depth,
                      const gs2d_track_params* prm, float* loss_part, float* pose_part,
                      const int32_t* gate, cudaStream_t st);

size_t render_bwd_ws_bytes(int n, size_t cap, int n_tiles, bool full);
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

}  // namespace gs2d
