/* Map expansion of 2DGS-SLAM on the GPU (Sec. III-E): new surfels from a
 * keyframe's RGB-D image, gated by a voxel hash table of the occupied space
 * of the active map.
 *
 * Steps of gs2d_expand, in the paper's order:
 *   1. the RGB-D image becomes a coloured point cloud P: every pixel with a
 *      valid depth (finite, > 0) back-projected, X_c = D(p) r(p) with
 *      r = ((x - cx)/fx, (y - cy)/fy, 1) at the pixel centre;
 *   2. random downsampling: P_s keeps pixel p when u_keep[p] < ratio
 *      (u_keep: caller-drawn uniforms in [0, 1), one per pixel);
 *   3. P_s goes to world space, X_w = R^T (X_c - t) for T_cw = (R, t);
 *   4. every point of P_s whose pixel has a normal in N_D (Eq. normal_fromD
 *      of the observed depth: central differences of the back-projected
 *      points, the pixel and its four neighbours valid, image interior) and
 *      whose voxel (floor(X_w / voxel) per axis) is not in the table becomes
 *      a surfel: centre X_w, scales s_u = s_v = the distance to its nearest
 *      neighbour in P_s (max_scale when P_s has no other point), opacity
 *      prm->opacity (0.99 in the paper), colour rgb(p), normal
 *      t_n = R^T N_D(p), tangents t_u = cos(phi) b1 + sin(phi) b2,
 *      t_v = t_n x t_u with phi = 2 pi u_angle[p] and (b1, b2) the
 *      orthonormal basis of t_n's plane of Duff et al., "Building an
 *      Orthonormal Basis, Revisited" (JCGT 2017); the quaternion of
 *      [t_u, t_v, t_n]; state delta = 1, t^c = t^l = kf_id, d^c = the
 *      distance to the keyframe's viewpoint (Sec. III-E, Eq. map);
 *   5. with insert_new, the new surfels' voxels are added to the table.
 * New surfels are written in pixel order at indices n_map .. n_map + k - 1
 * of the caller's map arrays (capacity entries); *n_new (device int32)
 * receives k.  When n_map + k > capacity nothing is written, *n_new still
 * receives k and the table's status word GS2D_ERR_CAPACITY.
 *
 * Voxel table: open addressing of 64-bit voxel keys (21 bits per axis,
 * voxel indices clamped to [-2^20, 2^20)), linear probing bounded by the
 * capacity (a power of two); a full table sets status to GS2D_ERR_CAPACITY
 * (the insert gives up, nothing hangs).  The table is rebuilt from the
 * active map (gs2d_voxel_clear, then gs2d_voxel_insert with the active
 * flags as mask) whenever surfels change state (Sec. III-E).
 *
 * All pointers are caller-owned device memory; images are H x W (x 3 for
 * colour), channel-last; calls are asynchronous on the stream and return a
 * gs2d_status (GS2D_ERR_INVALID_ARG for NULL pointers, bad sizes or a
 * capacity that is not a power of two; GS2D_ERR_WORKSPACE with the needed
 * size in *ws_needed).
 */
#ifndef GS2D_EXPAND_H_
#define GS2D_EXPAND_H_

#include <stddef.h>
#include <stdint.h>

#include "gs2d.h"
#include "gs2d_map.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint64_t* keys;     /* [capacity] voxel keys, all ones = empty          */
  uint32_t capacity;  /* power of two                                     */
  float voxel;        /* voxel edge r_h (m)                               */
  int32_t* status;    /* [1] device status word (GS2D_ERR_CAPACITY: full) */
} gs2d_voxel_table;

/* Empties the table and zeroes its status word. */
int gs2d_voxel_clear(const gs2d_voxel_table* t, gs2d_stream stream);

/* Inserts the voxels of points [m*3] (world coordinates) where mask[i] is
 * nonzero (mask may be NULL: all points). */
int gs2d_voxel_insert(const gs2d_voxel_table* t, const float* points, const uint8_t* mask, int m,
                      gs2d_stream stream);

/* occupied[i] = 1 when the voxel of points[i] is in the table, else 0. */
int gs2d_voxel_query(const gs2d_voxel_table* t, const float* points, int m, uint8_t* occupied,
                     gs2d_stream stream);

typedef struct {
  float ratio;      /* keep probability of random downsampling, (0, 1]     */
  float opacity;    /* initial opacity (0.99)                              */
  float max_scale;  /* scale of a point without a neighbour in P_s (m)     */
  int kf_id;        /* id of the keyframe                                  */
  int insert_new;   /* 1: add the new surfels' voxels to the table         */
} gs2d_expand_params;

size_t gs2d_expand_workspace(const gs2d_camera* cam);
int gs2d_expand(const float* rgb, const float* depth, const gs2d_camera* cam, const float* pose_cw,
                const float* u_keep, const float* u_angle, const gs2d_voxel_table* table,
                const gs2d_expand_params* prm, int n_map, int capacity, float* mu, float* quat,
                float* scale, float* opacity, float* rgb_out, const gs2d_map_state* st,
                int32_t* n_new, void* workspace, size_t ws_bytes, size_t* ws_needed,
                gs2d_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* GS2D_EXPAND_H_ */
