/*
 * gs2d.h -- C ABI of the GB300-native differentiable 2D Gaussian surfel
 * rasterizer (the data-parallel hot path of 2DGS-SLAM, arXiv 2506.00970).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * All array arguments are DEVICE pointers owned by the caller.  The library
 *    never allocates or frees device memory and never synchronises the host;
 *    every call only enqueues kernels on `stream`.
 *  * Return value: GS2D_OK if all kernels were enqueued, GS2D_ERR_INVALID_ARG
 *    for a NULL/ill-sized argument (nothing is launched), GS2D_ERR_WORKSPACE
 *    if the workspace is NULL or too small (the required size is written to
 *    *ws_needed when that pointer is non-NULL; nothing is launched),
 *    GS2D_ERR_CUDA if a launch failed.  Conditions only the device can see
 *    (intersection capacity overflow, non-finite pose) are reported through
 *    the device status word of `gs2d_bins.status` (GS2D_ERR_CAPACITY,
 *    GS2D_ERR_NONFINITE); later kernels that read it skip their work.
 *  * Layouts: surfel arrays are structure-of-arrays, C-contiguous FP32;
 *    images are H x W row-major, channel-last (rgb and normal are H x W x 3).
 *  * Poses are world->camera T_cw as 12 device floats: R row-major (9) then
 *    t (3), x_c = R x_w + t; camera axes x right, y down, z forward.
 *  * Surfel parameters are *activated*: opacity in (0,1), scales > 0.  The
 *    quaternion (w, x, y, z) need not be normalised; the kernels normalise it
 *    and gradients are w.r.t. the raw quaternion.
 *
 * The operations follow the paper's statement of the problem:
 *  surfel g = (mu, R = [t_u t_v t_n], s_u, s_v, c, alpha) (Sec. III-A,
 *  Eq. Puv), camera-space splat H_c = T_cw H (Eq. hc), pixel ray
 *  x = (xz, yz, z, 1) = W T_cw H (u, v, 0, 1) (Eq. homo, wth), front-to-back
 *  alpha blending of colour, depth, normal and opacity (Eq. alpha_blending),
 *  gradients to the pose through the left perturbation Exp(tau) o T_cw,
 *  tau = (rho, theta) (Sec. III-B, Eq. derivatives), the masked tracking loss
 *  (Eq. tracking_loss) and AdamW pose tracking (Sec. III-D).
 */
#ifndef GS2D_H_
#define GS2D_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gs2d_stream; /* a cudaStream_t (NULL = legacy default stream) */

typedef enum {
  GS2D_OK = 0,
  GS2D_ERR_INVALID_ARG = 1,
  GS2D_ERR_WORKSPACE = 2,
  GS2D_ERR_CAPACITY = 3,
  GS2D_ERR_CUDA = 4,
  GS2D_ERR_TIMEOUT = 5,
  GS2D_ERR_NONFINITE = 6
} gs2d_status;

/* Pinhole intrinsics (the camera-to-image matrix W of Eq. homo).  Pixel
 * (i, j) has its centre at (i + 0.5, j + 0.5); near_z culls surfel centres
 * and ray intersections at camera depth <= near_z. */
typedef struct {
  float fx, fy, cx, cy;
  int width, height;
  float near_z;
} gs2d_camera;

/* Surfel map, structure of arrays (Sec. III-A): mu [n*3], quat [n*4]
 * (w,x,y,z), scale [n*2] (s_u, s_v), opacity [n], rgb [n*3]. */
typedef struct {
  const float* mu;
  const float* quat;
  const float* scale;
  const float* opacity;
  const float* rgb;
  int n;
} gs2d_surfels;

/* Tiling and compositing constants.  The paper leaves the numerical rules
 * of its blending open; the defaults (gs2d_default_config) are
 * alpha_min = 1/255 (skip), alpha_max = 0.99 (clamp), t_min = 1e-4 (stop
 * before the transmittance would fall below it) and cutoff_r2 = 9
 * (u^2 + v^2 beyond three standard deviations is skipped).  tile_w x tile_h
 * and px_per_thread P describe a tile of 256 P pixels handled by a 256-thread
 * block, P in {1, 2, 3, 4}: thread t owns P pixels 4 rows apart and each warp
 * an 8 x 4P block, so tile_w is a multiple of 8 and tile_h of 4P (P = 1:
 * 16x16, 8x32, 32x8; P = 2: 16x32, 32x16, 8x64, 64x8; P = 3: 64x12, 32x24,
 * 16x48, 8x96; P = 4: 32x32, 16x64, 64x16).  Other shapes return GS2D_ERR_INVALID_ARG.  The batch autotuner
 * picks the shape per resolution class and P per batch; every view of one
 * batched call must share P. */
typedef struct {
  int tile_w, tile_h, px_per_thread;
  float alpha_min, alpha_max, t_min, cutoff_r2;
} gs2d_config;

/* Per-surfel projected record written by gs2d_project: 32 floats (128 B,
 * 16-byte aligned).  Image coordinates x' = x - cx, y' = y - cy are relative
 * to the principal point.  Float slots:
 *   0-1   (x0, y0): projected centre of the surfel (x', y')
 *   2     p2c = det / mu_c.z
 *   3-8   c1, c2: the homogeneous (u, v, 1) of the ray through (x', y') is
 *         p = (x' - x0) c1 + (y' - y0) c2 + (0, 0, p2c) (the inverse of the
 *         homography of Eq. wth up to scale): u = p0/p2, v = p1/p2
 *   9     det (intersection depth z = det / p2)      10  alpha
 *   11-13 rgb          14-16 t_nc (camera-space normal)
 *   17-19 n = s_u t_uc x s_v t_vc   20-22 dual tangent d_u   23-25 dual d_v
 *         (d_u . s_u t_uc = 1, d_u . s_v t_vc = 0, d_u . n = 0; d_v alike)
 *   26    centre depth mu_c.z (the sort key)          27  unused
 *   28    uint32 tx0 | ty0 << 16,  29  uint32 tx1 | ty1 << 16  (inclusive tile
 *         rectangle; tx0 > tx1 marks a culled surfel)
 *   30    uint32 i0 | i1 << 16,    31  uint32 j0 | j1 << 16  (inclusive pixel
 *         columns / rows of the footprint). */
#define GS2D_PROJ_FLOATS 32

/* Binning output of gs2d_bin_sort.  capacity bounds the number of
 * (tile, surfel) intersections K.  keys may be NULL. */
typedef struct {
  uint64_t* keys;        /* [capacity] tile << 32 | float bits of mu_c.z       */
  uint32_t* vals;        /* [capacity] surfel id per sorted position            */
  uint32_t* isect_emit;  /* [capacity] emission index of each sorted position   */
  uint32_t* surfel_off;  /* [n] first emission index of surfel i (its k_i
                            intersections are emission indices off..off+k_i-1);
                            both may be NULL (gs2d_bin_sort then skips the
                            emission scan): bins for gs2d_render_fwd only --
                            the full gs2d_render_bwd and gs2d_render_contrib
                            need them */
  int32_t* tile_ranges;  /* [2 * n_tiles] [start, end) of each tile's list       */
  int32_t* n_isect;      /* [1] K (the needed count when K > capacity)          */
  int32_t* status;       /* [1] device status word (gs2d_status)                */
  size_t capacity;
} gs2d_bins;

/* Tracking hyper-parameters (Sec. III-D).  The paper names AdamW and
 * n_iter = 120 (Table I) but not lr, betas or the stop rule; defaults:
 * lr 1e-3, betas (0.9, 0.999), eps 1e-8, weight decay 0, stop when
 * |tau| < 1e-5, lambda_d 1, opacity mask 0.95 (Eq. opacity_mask),
 * depth_mode 1 (depth loss on D/O). */
typedef struct {
  float lambda_d, lr, beta1, beta2, eps, weight_decay, stop_tol, opacity_thresh;
  int depth_mode;
} gs2d_track_params;

gs2d_config gs2d_default_config(void);
gs2d_track_params gs2d_default_track_params(void);
const char* gs2d_status_string(int status);
/* Tiles per row / column for a camera and config. */
int gs2d_tiles_x(const gs2d_camera* cam, const gs2d_config* cfg);
int gs2d_tiles_y(const gs2d_camera* cam, const gs2d_config* cfg);

/* Per-surfel projection (Eq. hc, homo, wth; footprint bound of the 3-sigma
 * disc).  pose: device [12].  proj_out: device [n * GS2D_PROJ_FLOATS] floats;
 * tiles_per_surfel_out: device int32 [n], the number of tiles of the
 * surfel's rectangle (0 if culled).  One thread per surfel. */
int gs2d_project(const gs2d_surfels* s, const gs2d_camera* cam, const float* pose,
                 const gs2d_config* cfg, float* proj_out, int32_t* tiles_per_surfel_out,
                 gs2d_stream stream);

/* Tile binning and depth ordering (the per-tile depth sort of Sec. III-A): every
 * surfel with k_i > 0 emits one intersection per tile of its rectangle; the
 * intersections are ordered by (tile, mu_c.z bits, surfel id) -- the order
 * of a stable sort by tile of the depth-ordered emission -- by binning the
 * pairs into per-tile segments and sorting every segment by (depth bits, id)
 * in shared memory (hand-written bitonic networks; long segments in chunks
 * merged in global memory), so the result is unique and deterministic.
 * This replaces the global LSD radix sort on (tile, depth) keys of the first
 * design (four 8-bit passes over the depth keys, then one or two over the
 * tile keys): the per-tile sort gives the identical order in fewer passes
 * and took a 100-iteration 640x480 tracking frame from 28.1 to 24.1 ms.
 * proj: device [n * GS2D_PROJ_FLOATS] (only slots 26, 28, 29 are read).
 * tiles_per_surfel: device [n], must equal the rectangle's tile count.
 * Workspace: gs2d_bin_sort_workspace(n, capacity) bytes.  The emission
 * offsets are an exclusive scan whose blocks wait (boundedly) on their
 * predecessors' published sums; a wait that runs out records
 * GS2D_ERR_TIMEOUT in the status word, keeps every write in bounds and
 * makes every later kernel skip (see gs2d_set_lookback_wait). */
size_t gs2d_bin_sort_workspace(int n, size_t capacity);
int gs2d_bin_sort(const float* proj, const int32_t* tiles_per_surfel, int n,
                  const gs2d_camera* cam, const gs2d_config* cfg, void* workspace,
                  size_t ws_bytes, size_t* ws_needed, const gs2d_bins* bins, gs2d_stream stream);

/* Look-back waits of gs2d_bin_sort's emission scan (diagnostic; no
 * counterpart in the paper).  spin_limit: how many polls a scan block makes
 * for a predecessor's published sum before it records GS2D_ERR_TIMEOUT and
 * finishes with a partial prefix (0 restores the default of 2^22 polls, a
 * second or more).  withheld_chunk: for tests of that failure path, the scan
 * block (4096 surfels each) that never publishes its sum, so that the next
 * block's wait runs out (-1 = none, the default).  Process-wide, read at
 * each launch (a captured graph keeps the values it was captured with); not
 * thread-safe against launches from other host threads. */
void gs2d_set_lookback_wait(int spin_limit, int withheld_chunk);

/* gs2d_bin_sort without a workspace argument: it allocates nothing.  The
 * paper has no counterpart; this serves callers that cannot allocate device
 * memory when they bin -- code inside a CUDA stream capture (cudaMalloc is
 * not allowed there), real-time loops with a no-allocation rule, or host
 * frameworks that own all device memory and pass only inputs and outputs.
 * Scratch is a file-scope __device__ array of GS2D_SORT_STATIC_SCRATCH_BYTES
 * that every GPU loading the library holds until the process exits.  Sizes
 * whose gs2d_bin_sort_workspace(n, bins->capacity) exceeds it are rejected
 * with GS2D_ERR_WORKSPACE before anything is launched (about 200k surfels
 * with a capacity of 1M intersections fit).  The first call on each device
 * looks up that device's copy of the array (cudaGetSymbolAddress, with the
 * device current) and caches it; make that first call before any stream
 * capture.  The cached address belongs to the device's context at that
 * first call: cudaDeviceReset on that device afterwards is not supported
 * (the array may move in the new context; a later call would pass the old
 * address).  All calls on a device share the one array: calls whose kernels
 * may overlap on the GPU (different streams without ordering) race and must
 * be serialised by the caller.  Results equal gs2d_bin_sort's. */
#define GS2D_SORT_STATIC_SCRATCH_BYTES (32u << 20)
int gs2d_bin_sort_static(const float* proj, const int32_t* tiles_per_surfel, int n,
                         const gs2d_camera* cam, const gs2d_config* cfg, const gs2d_bins* bins,
                         gs2d_stream stream);

/* Front-to-back compositing (Eq. alpha_blending) of colour (rgb [H*W*3]),
 * literal depth D = sum w z ([H*W]), normal sum w t_nc ([H*W*3]) and opacity
 * O = 1 - T ([H*W]); also the final transmittance t_final [H*W] and n_last
 * [H*W] (one past the last blended position in the pixel's tile list), the
 * state the backward pass replays from.  One thread block per tile. */
int gs2d_render_fwd(const float* proj, const gs2d_bins* bins, const gs2d_camera* cam,
                    const gs2d_config* cfg, float* rgb, float* depth, float* normal,
                    float* opacity, float* t_final, uint32_t* n_last, gs2d_stream stream);

/* Work counter of gs2d_render_fwd (diagnostic, same loop and culling):
 * counts[0] = evaluated (pixel, surfel) pairs, counts[1] = pairs inside the
 * cutoff radius, counts[2] = blended pairs, counts[3] / counts[4] = the
 * evaluated pairs / those inside the cutoff up to each pixel's last blended
 * pair (the pairs a backward replay evaluates); device uint64 [5], zeroed
 * here.  The roofline of the compositing kernels is stated per these counts. */
int gs2d_render_count(const float* proj, const gs2d_bins* bins, const gs2d_camera* cam,
                      const gs2d_config* cfg, unsigned long long* counts, gs2d_stream stream);

/* Scheduling of the one-pixel-per-thread tile kernels of gs2d_render_fwd and
 * gs2d_track_step (no counterpart in the paper; results do not depend on
 * it): a tile grid of at most max_tiles tiles runs the grouped form of the
 * compositing loops, which keeps four (pixel, surfel) evaluations in flight
 * per thread at two blocks per SM -- for images too small to fill the GPU
 * (160x120 has 80 tiles of 16x16), where each pixel's serial walk over its
 * tile's list is the bound.  -1 (the default) = twice the device's SM count;
 * 0 = never.  Process-wide; read at each launch (so a captured graph keeps
 * the form it was captured with).  Not thread-safe against concurrent
 * launches from other host threads. */
void gs2d_set_grouped_tiles(int max_tiles);

/* Backward of gs2d_render_fwd (Sec. III-B): replays compositing back to
 * front from (t_final, n_last) and returns dL/d(mu, quat, scale, opacity,
 * rgb) per surfel and dL/dtau (rho, theta) of the pose (Eq. derivatives)
 * given dL/d(rgb, depth, normal, opacity) of the images (d_normal and
 * d_opacity may be NULL = zero).  Per-(tile, surfel) partial sums are formed
 * with warp shuffles and written once; a second, fixed-order pass reduces
 * them per surfel, so the result is deterministic.  If d_mu, d_quat,
 * d_scale, d_opac and d_rgb are all NULL only d_pose6 is computed (tracking
 * mode: no per-surfel partials).  pose: device [12]; d_pose6: device [6] or
 * NULL.  Workspace: gs2d_render_bwd_workspace(n, capacity, n_tiles). */
size_t gs2d_render_bwd_workspace(int n, size_t capacity, int n_tiles);
int gs2d_render_bwd(const float* proj, const gs2d_bins* bins, const int32_t* tiles_per_surfel,
                    const gs2d_surfels* s, const float* pose, const gs2d_camera* cam,
                    const gs2d_config* cfg, const float* t_final, const uint32_t* n_last,
                    const float* d_rgb, const float* d_depth, const float* d_normal,
                    const float* d_opacity, float* d_mu, float* d_quat, float* d_scale,
                    float* d_opac, float* d_rgb_out, float* d_pose6, void* workspace,
                    size_t ws_bytes, size_t* ws_needed, gs2d_stream stream);

/* Per-surfel contribution of a view (Sec. III-D, Eq. weight and Eq.
 * contribution): contrib[i] = sum over all pixels p of w_i(p) = a_i(p) T_i(p),
 * the blending weight record i receives in gs2d_render_fwd's compositing
 * (same clamp, skip and stop rules; records culled or never reached get 0).
 * Summed per (tile, surfel) pair and then per surfel in emission order:
 * deterministic.  A surfel is visible from the view when contrib > 0.5.
 * Inputs as gs2d_render_fwd plus tiles_per_surfel [n] and the emission
 * arrays of bins (as gs2d_bin_sort fills them); contrib: device [n] FP32.
 * Workspace: gs2d_render_contrib_workspace(bins->capacity) bytes. */
size_t gs2d_render_contrib_workspace(size_t capacity);
int gs2d_render_contrib(const float* proj, const gs2d_bins* bins, const int32_t* tiles_per_surfel,
                        int n, const gs2d_camera* cam, const gs2d_config* cfg, float* contrib,
                        void* workspace, size_t ws_bytes, size_t* ws_needed, gs2d_stream stream);

/* Covisibility of two views A and B (Sec. III-D): with the visible sets
 * G_X = {i : contrib_X[i] > vis_threshold} (0.5 in the paper),
 * counts[0] = |G_A n G_B|, counts[1] = |G_A u G_B| (device uint32 [2]),
 * score = counts[0] / counts[1] (0 when both are empty; device [1], may be
 * NULL) and the keyframe rule is_keyframe = score < c_k or
 * |t_A - t_B| > d_k, t the translation of each world-to-camera pose
 * (device [12] each; c_k = 0.9 and d_k = 0.15 m in Table I; device int32
 * [1], may be NULL, then the poses may be NULL).  contrib_a / contrib_b:
 * device [n], both indexed by the same surfel ids. */
int gs2d_covisibility(const float* contrib_a, const float* contrib_b, int n, float vis_threshold,
                      const float* pose_a, const float* pose_b, float c_k, float d_k,
                      uint32_t* counts, float* score, int32_t* is_keyframe, gs2d_stream stream);

/* ------------------------------------------------------------------------
 * Batches of views (the mapping window of Sec. III-E renders several
 * keyframes per iteration, each over the active map M_A of Sec. III-C; the
 * tracking of several frames is the same pattern).  Every view carries its
 * camera, tile configuration, pose, optional active-surfel subset and its own
 * caller-owned buffers; up to GS2D_MAX_VIEWS views per call.  The render
 * passes are single persistent launches over all (view, tile) work items,
 * taken from an atomic queue (no waiting), so views of different sizes
 * share the GPU; the view table travels by value in the kernel parameters,
 * so the calls can be captured in a CUDA graph.  Results per view equal the
 * single-view entry points'. */
#define GS2D_MAX_VIEWS 32
typedef struct {
  gs2d_camera cam;
  gs2d_config cfg;            /* per view: tile shape may differ per resolution */
  const float* pose;          /* device [12] world->camera                          */
  const int32_t* active;      /* device [n_active] surfel ids drawn, or NULL = all  */
  int n_active;
  float* proj;                /* [m * GS2D_PROJ_FLOATS], m = active ? n_active : n  */
  int32_t* tiles_per_surfel;  /* [m]                                                */
  gs2d_bins bins;             /* vals / isect_emit [capacity], surfel_off [m], ...  */
  float* rgb;                 /* forward outputs: H x W x 3, H x W, H x W x 3,     */
  float* depth;               /*   H x W, H x W, H x W (as gs2d_render_fwd)        */
  float* normal;
  float* opacity;
  float* t_final;
  uint32_t* n_last;
  const float* d_rgb;         /* backward inputs (d_normal, d_opacity may be NULL)  */
  const float* d_depth;
  const float* d_normal;
  const float* d_opacity;
  float* d_pose6;             /* [6] this view's pose gradient, or NULL             */
} gs2d_view;

/* Projection of every view (one launch; record j of a view is surfel
 * active[j], or j).  Binning of every view, equal to gs2d_bin_sort's on the
 * same view bit for bit: up to 8 views each on its own side stream of the
 * device (forked from and joined back to `stream` by events -- parallel
 * branches when captured into a CUDA graph; the side streams are created by
 * the first call with several views on each device, so make that call before
 * any stream capture), more views in one launch per stage (the stage's blocks
 * split over the views); every view has its own slice of the workspace
 * after a 256-byte header, its own counters and its own bins.status, which
 * must be 0 on entry.  The
 * forward pass of every view in one persistent launch.  The backward pass of
 * every view in one persistent launch, then the per-surfel reductions view by
 * view in a fixed order: d_* (device [n*3], [n*4], [n*2], [n], [n*3]) receive
 * the sum over views (surfels outside every subset get zero). */
int gs2d_project_batch(const gs2d_surfels* s, const gs2d_view* views, int n_views,
                       gs2d_stream stream);
size_t gs2d_bin_sort_batch_workspace(const gs2d_view* views, int n_views, int n);
int gs2d_bin_sort_batch(const gs2d_view* views, int n_views, int n, void* workspace,
                        size_t ws_bytes, size_t* ws_needed, gs2d_stream stream);
size_t gs2d_render_batch_workspace(const gs2d_view* views, int n_views, int n);
int gs2d_render_fwd_batch(const gs2d_view* views, int n_views, void* workspace, size_t ws_bytes,
                          size_t* ws_needed, gs2d_stream stream);
int gs2d_render_bwd_batch(const gs2d_view* views, int n_views, const gs2d_surfels* s, float* d_mu,
                          float* d_quat, float* d_scale, float* d_opac, float* d_rgb,
                          void* workspace, size_t ws_bytes, size_t* ws_needed, gs2d_stream stream);

/* Tracking loss L_t (Eq. tracking_loss with the masks of Eq. normal_mask and
 * opacity_mask) of rendered images against an observed RGB-D frame, and its
 * gradient w.r.t. the rendered rgb, depth and opacity (g_* [H*W*3], [H*W],
 * [H*W]; the masks carry no gradient).  loss_out: device [1].  Per-block
 * partial sums are reduced in a fixed order. */
int gs2d_tracking_loss(const float* rgb, const float* depth, const float* normal,
                       const float* opacity, const float* obs_rgb, const float* obs_depth,
                       const gs2d_camera* cam, const gs2d_track_params* prm, float* g_rgb,
                       float* g_depth, float* g_opacity, float* loss_out, void* workspace,
                       size_t ws_bytes, size_t* ws_needed, gs2d_stream stream);

/* Mapping loss of Sec. III-E without the SSIM term:
 * 1/|Omega| sum (|I_r - I|_1 + w_d |D_r/O - D| + w_n (1 - N_{D_r} . N_r)),
 * N_{D_r} from Eq. normal_fromD on the back-projected rendered depth with
 * central differences (interior pixels whose own and 4-neighbour opacity
 * exceed 0.5).  Gradients w.r.t. rendered rgb, depth, normal, opacity. */
int gs2d_mapping_loss(const float* rgb, const float* depth, const float* normal,
                      const float* opacity, const float* obs_rgb, const float* obs_depth,
                      const gs2d_camera* cam, float w_d, float w_n, float* g_rgb, float* g_depth,
                      float* g_normal, float* g_opacity, float* loss_out, void* workspace,
                      size_t ws_bytes, size_t* ws_needed, gs2d_stream stream);

/* gs2d_mapping_loss of several views in one launch (the mapping window of
 * Sec. III-E renders every keyframe; each view's loss is its own mean over
 * its pixels).  View v's images and gradients are device buffers laid out as
 * for gs2d_mapping_loss at its own resolution; every pointer non-NULL.  The
 * gradients are bit-identical to gs2d_mapping_loss on the same view; the
 * loss (loss_out: device [n_views]) equals it up to the order of the FP32
 * sum (per-warp partials of each 32 x 8 tile, added in a fixed order).
 * 1 <= n_views <= GS2D_MAX_VIEWS; workspace
 * gs2d_mapping_loss_batch_workspace(views, n_views) bytes (0 for invalid
 * views).  GS2D_ERR_INVALID_ARG / GS2D_ERR_WORKSPACE before any launch. */
typedef struct {
  gs2d_camera cam;
  const float* rgb;      /* rendered H x W x 3, H x W, H x W x 3, H x W */
  const float* depth;
  const float* normal;
  const float* opacity;
  const float* obs_rgb;  /* observed H x W x 3, H x W                    */
  const float* obs_depth;
  float* g_rgb;          /* gradient outputs, shaped as the rendered     */
  float* g_depth;
  float* g_normal;
  float* g_opacity;
} gs2d_loss_view;
size_t gs2d_mapping_loss_batch_workspace(const gs2d_loss_view* views, int n_views);
int gs2d_mapping_loss_batch(const gs2d_loss_view* views, int n_views, float w_d, float w_n,
                            float* loss_out, void* workspace, size_t ws_bytes, size_t* ws_needed,
                            gs2d_stream stream);

/* The full mapping loss of Sec. III-E, L_m = 1/|Omega| sum_p (L_c + w_d L_D
 * + w_n L_n) with L_c = (1 - w_ssim) |I_r - I|_1 + w_ssim (1 - SSIM(p)),
 * SSIM(p) the mean over the three channels of the SSIM of Wang et al. 2004
 * (11 x 11 Gaussian window, sigma 1.5, C1 = 0.01^2, C2 = 0.03^2, zero
 * padding at the border) of the rendered against the observed colour.
 * Table I gives the SSIM term the weight 0.125 (w_ssim; the equation's
 * lambda_c weights the L1 term, so lambda_c = 1 - w_ssim).  w_ssim = 0 is
 * gs2d_mapping_loss.  w_ssim in [0, 1]; arguments otherwise as
 * gs2d_mapping_loss; workspace gs2d_mapping_loss_ssim_workspace(cam). */
size_t gs2d_mapping_loss_ssim_workspace(const gs2d_camera* cam);
int gs2d_mapping_loss_ssim(const float* rgb, const float* depth, const float* normal,
                           const float* opacity, const float* obs_rgb, const float* obs_depth,
                           const gs2d_camera* cam, float w_ssim, float w_d, float w_n,
                           float* g_rgb, float* g_depth, float* g_normal, float* g_opacity,
                           float* loss_out, void* workspace, size_t ws_bytes, size_t* ws_needed,
                           gs2d_stream stream);

/* The SSIM term alone: *loss += weight / (H W) sum_p (1 - mean_c SSIM_c(p))
 * of x against y (device [H*W*3], channel-last, SSIM as above) and, if g_x
 * is not NULL, g_x += its gradient w.r.t. x.  One fused pass (moments,
 * SSIM, adjoint filtering in shared memory); the block sums are reduced in
 * a fixed order.  loss: device [1].  Workspace gs2d_ssim_workspace(H, W). */
size_t gs2d_ssim_workspace(int height, int width);
int gs2d_ssim_loss(const float* x, const float* y, int height, int width, float weight,
                   float* g_x, float* loss, void* workspace, size_t ws_bytes, size_t* ws_needed,
                   gs2d_stream stream);

/* Frame-to-map tracking (Sec. III-D): n_iter iterations of
 * project -> bin_sort -> render_fwd -> tracking loss -> pose-only backward
 * -> AdamW on tau -> T <- Exp(tau) T with tau reset to 0.  Once
 * |tau| < stop_tol the remaining iterations only copy the history.
 * Everything stays on the device.
 *   pose        [12] in/out (world->camera, as everywhere).
 *   adam_state  [16] AdamW state m[6], v[6], step, done flag (1 once the stop
 *               rule fired), 2 unused; owned by the caller, read and updated
 *               in place, never reset here: zero it to start a frame, and
 *               pass it again to continue one (a frame split over several
 *               calls gives the same bits as one call).  NULL = moments kept
 *               in the workspace and zeroed at the start of every call.
 *   loss_hist   [n_iter]: the loss at the pose before each update;
 *   pose_hist   [n_iter * 12]: the pose after it;
 *   grad_hist   [n_iter * 6]: dL/dtau (rho, theta) at the pose before each
 *               update, the vector AdamW receives (zero for the iterations
 *               skipped after convergence).  Each may be NULL.
 * capacity bounds K per iteration.  The status word
 * (gs2d_track_status(workspace)) ends as GS2D_OK, 256 (converged early) or
 * an error: GS2D_ERR_CAPACITY (raise capacity and retry), GS2D_ERR_NONFINITE
 * (a non-finite loss or gradient, e.g. from a non-finite observation: the
 * pose and the AdamW state keep the values they had before that iteration,
 * whose loss_hist / grad_hist entries record what was found), or
 * GS2D_ERR_TIMEOUT; every later kernel of the call then skips its work.
 * Workspace: gs2d_track_workspace(n, capacity, cam, cfg). */
size_t gs2d_track_workspace(int n, size_t capacity, const gs2d_camera* cam,
                            const gs2d_config* cfg);
int gs2d_track_step(const gs2d_surfels* s, const gs2d_camera* cam, const gs2d_config* cfg,
                    const gs2d_track_params* prm, float* pose, float* adam_state,
                    const float* obs_rgb, const float* obs_depth, int n_iter, size_t capacity,
                    float* loss_hist, float* pose_hist, float* grad_hist, void* workspace,
                    size_t ws_bytes, size_t* ws_needed, gs2d_stream stream);
/* Device pointer of the status word inside a track workspace (int32). */
int32_t* gs2d_track_status(void* workspace);

/* Device pointer of the tile launch order inside a track workspace (int32
 * [n_tiles], the same n, capacity, cam and cfg as gs2d_track_workspace):
 * after an iteration, a permutation of the tile ids by decreasing tile list
 * length (256 buckets linear in length / the longest length; arrival order
 * within a bucket), the order in which the fused tile kernel launched the
 * tiles.  A diagnostic; NULL for a NULL argument. */
const int32_t* gs2d_track_tile_order(void* workspace, int n, size_t capacity,
                                     const gs2d_camera* cam, const gs2d_config* cfg);

/* Diagnostic timing of the fused tile kernel of gs2d_track_step: while set,
 * every later launch of that kernel (in any gs2d_track_step call, in launch
 * order) is bracketed by records of start_events[i] and stop_events[i] on
 * the call's stream (event-record nodes when the stream is being captured
 * into a CUDA graph, so every replay records them), until n launches have
 * been recorded.  The events are caller-created cudaEvent_t handles
 * that must stay alive meanwhile.  n = 0 switches it off.  No work is
 * skipped or reordered.  gs2d_profile_track_kernel_count() = launches
 * recorded so far.  Not thread safe. */
int gs2d_profile_track_kernel(void* const* start_events, void* const* stop_events, int n);
int gs2d_profile_track_kernel_count(void);
/* Bracket only the launches of iterations it with it % every == 0 of each
 * gs2d_track_step call (default 1: every launch), so a timed frame carries
 * fewer event records; every < 1 returns GS2D_ERR_INVALID_ARG. */
int gs2d_profile_track_kernel_every(int every);

#ifdef __cplusplus
}
#endif
#endif /* GS2D_H_ */
