/* Map state of 2DGS-SLAM on the GPU: the per-surfel bookkeeping of Eq. map
 * (Sec. III-C), its update after each keyframe (Sec. III-F), the map
 * correction after pose graph optimisation (Sec. IV-C) and the removal of
 * occluded surfels (Sec. III-F), as C-ABI calls on caller-owned device
 * memory.
 *
 * Eq. map extends every surfel g_i with
 *   delta_i  active flag: 1 = active map M_A, 0 = inactive map M_I;
 *   t^c_i    id of the keyframe that observed g_i at the closest distance
 *            (the keyframe g_i follows in the map correction);
 *   d^c_i    that closest distance;
 *   t^l_i    id of the last keyframe that observed g_i.
 * "Observed" is the visibility of Sec. III-D: contribution (Eq.
 * contribution, gs2d_render_contrib) above 0.5.
 *
 * Layouts: surfel arrays as in gs2d.h (mu [n*3], quat [n*4] (w, x, y, z),
 * scale [n*2], opacity [n], rgb [n*3]); state arrays [n].  Poses are
 * world-to-camera T_cw, 12 floats: row-major R then t.  All pointers are
 * device memory owned by the caller; every call is asynchronous on the given
 * stream and returns a gs2d_status (GS2D_ERR_INVALID_ARG for a NULL pointer,
 * a negative size or a misaligned vector array, GS2D_ERR_WORKSPACE with the
 * needed size in *ws_needed when the workspace is too small).
 */
#ifndef GS2D_MAP_H_
#define GS2D_MAP_H_

#include <stddef.h>
#include <stdint.h>

#include "gs2d.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint8_t* delta;   /* [n] 1 = active, 0 = inactive       */
  int32_t* t_c;     /* [n] closest observing keyframe id   */
  float* d_c;       /* [n] closest observing distance (m)  */
  int32_t* t_l;     /* [n] last observing keyframe id      */
} gs2d_map_state;

typedef struct {
  float vis_threshold;  /* visibility: contribution > this (0.5)                  */
  int inactive_after;   /* an active surfel turns inactive once kf_id - t^l > this */
  int reactivate;       /* 1 within the T keyframes that follow a loop closure    */
  int loop_h;           /* id of the loop closure's historical keyframe K_h       */
} gs2d_state_params;

/* State update for keyframe kf_id with world-to-camera pose pose_cw (device
 * [12]) and the contributions contrib [n] of its view (0 for surfels not
 * rendered), Sec. III-F, per surfel i in this order:
 *   if delta_i = 1 (active on entry):
 *     if visible: t^l_i = kf_id; d = |mu_i - c| with c = -R^T t the
 *       keyframe's camera centre; if d < d^c_i: d^c_i = d, t^c_i = kf_id;
 *     if kf_id - t^l_i > inactive_after: delta_i = 0;
 *   else if reactivate and visible and t^c_i > loop_h: delta_i = 1,
 *     t^l_i = kf_id.
 * counts (device uint32 [4], may be NULL; zeroed here): visible active
 * surfels, closest-distance updates, deactivations, reactivations. */
int gs2d_map_observe(const float* contrib, const float* mu, int n, const float* pose_cw,
                     int kf_id, const gs2d_state_params* prm, const gs2d_map_state* st,
                     uint32_t* counts, gs2d_stream stream);

/* Map correction (Sec. IV-C): keyframe j's pose increment
 * dT_j = T^o_j T_j^-1 with T_j, T^o_j its camera-to-world poses before and
 * after pose graph optimisation, i.e. dT_j = (T^o_cw,j)^-1 T_cw,j from the
 * world-to-camera poses given here (poses_old, poses_new: device
 * [n_kf * 12]); every surfel i with 0 <= t^c_i < n_kf becomes
 * mu_i <- dR mu_i + dt and R_i <- dR R_i (quat_i <- q(dR) quat_i, the
 * quaternion's norm kept); other surfels are left as they are and counted
 * in *n_skipped (device int32 [1], may be NULL).  Workspace:
 * gs2d_map_correct_workspace(n_kf) bytes (the increments). */
size_t gs2d_map_correct_workspace(int n_kf);
int gs2d_map_correct(float* mu, float* quat, const int32_t* t_c, int n, const float* poses_old,
                     const float* poses_new, int n_kf, void* workspace, size_t ws_bytes,
                     size_t* ws_needed, int32_t* n_skipped, gs2d_stream stream);

/* Removal test of Sec. III-F for a sampled keyframe r: keep[i] = 0 when
 * t^c_i = r and contrib[i] < vis_threshold (occluded by its neighbours),
 * else 1 (device uint8 [n]). */
int gs2d_map_prune(const float* contrib, const int32_t* t_c, int n, int r, float vis_threshold,
                   uint8_t* keep, gs2d_stream stream);

/* Stable compaction of the map by keep [n] (uint8, nonzero = keep): every
 * kept surfel's parameters and state are copied, in index order, to the
 * *_out arrays (sized for n; they must not overlap the inputs);
 * new_index [n] (int32, may be NULL) receives each surfel's new index or -1;
 * *n_out (device int32 [1]) the kept count.  Any state array pointer may be
 * NULL in both st and st_out (that array is skipped).  Workspace:
 * gs2d_map_compact_workspace(n) bytes. */
size_t gs2d_map_compact_workspace(int n);
int gs2d_map_compact(const uint8_t* keep, int n, const gs2d_surfels* s, const gs2d_map_state* st,
                     float* mu_out, float* quat_out, float* scale_out, float* opacity_out,
                     float* rgb_out, const gs2d_map_state* st_out, int32_t* new_index,
                     int32_t* n_out, void* workspace, size_t ws_bytes, size_t* ws_needed,
                     gs2d_stream stream);

/* Back from a compacted subset to the whole map: out[i] = vals[new_index[i]]
 * when new_index[i] >= 0, else fill (new_index as gs2d_map_compact writes
 * it); e.g. the contributions of a view of the active map M_A, rendered from
 * its compacted copy, indexed by the whole map's surfel ids. */
int gs2d_map_expand_values(const float* vals, const int32_t* new_index, int n, float fill,
                           float* out, gs2d_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* GS2D_MAP_H_ */
