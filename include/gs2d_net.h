/* Learned tracking-pose proposal: BF16 tensor-core network kernels.
 *
 * Not in the paper.  The tracking loop of Sec. III-D starts each frame from
 * the previous frame's pose and refines it by gradient steps on the tracking
 * loss (Eq. tracking_loss); this network proposes a better starting pose
 * from the rendered and the observed RGB-D images, and the same loop then
 * refines it (and judges it: a proposal that raises the tracking loss is
 * discarded by the caller).
 *
 * Network (input 120 x 160, 8 channels, channels-last NHWC bfloat16):
 *   six convolutions 3x3, stride 2, zero padding 1, each + bias + ReLU,
 *   channels 8 -> 32 -> 64 -> 128 -> 256 -> 256 -> 256, spatial
 *   120x160 -> 60x80 -> 30x40 -> 15x20 -> 8x10 -> 4x5 -> 2x3; output pixel
 *   (oy, ox) reads input pixel (2 oy - 1 + ky, 2 ox - 1 + kx);
 *   flatten (h, w, c) -> 1536; FC 1536 -> 256 + ReLU; FC 256 -> 6.
 * The 6 outputs y, scaled by GS2D_NET_TAU_SCALE, are a twist (rho, theta)
 * applied on the left: T <- Exp(y * scale) T (the left perturbation of
 * Sec. III-B).  Training target y* = Log(T_gt T^-1) / scale, loss
 * L = 1/(2B) sum_b |y_b - y*_b|^2.
 *
 * Flat parameter vector (float32, caller-owned, device): for each conv layer
 * W [c_out][3][3][c_in] then b [c_out]; then FC1 W [256][1536], b [256];
 * then FC2 W [6][256], b [6] (gs2d_net_layout gives the offsets).
 *
 * Precision: the input, a bfloat16 copy of the weights and every stored
 * activation and activation gradient are bfloat16 (round to nearest even);
 * every product accumulates in FP32 on the tensor cores (mma m16n8k16);
 * biases, outputs, loss, weight gradients, AdamW moments and the master
 * weights are FP32.  All reductions have a fixed order (deterministic).
 *
 * Every call is asynchronous on the given stream and returns a gs2d_status
 * (GS2D_ERR_INVALID_ARG for a bad size or a pointer that is NULL or not
 * 16-byte aligned; GS2D_ERR_WORKSPACE when ws_bytes < the needed size,
 * which is written to *ws_needed when that is not NULL).
 */
#ifndef GS2D_NET_H_
#define GS2D_NET_H_

#include <stddef.h>
#include <stdint.h>

#include "gs2d.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GS2D_NET_IN_H 120
#define GS2D_NET_IN_W 160
#define GS2D_NET_IN_C 8
#define GS2D_NET_OUT 6
#define GS2D_NET_LAYERS 8            /* 6 convolutions + 2 fully connected */
#define GS2D_NET_TAU_SCALE 0.03f     /* metres (rho) and radians (theta) per unit output */
#define GS2D_NET_DEPTH_OFFSET 2.5f   /* metres subtracted from valid input depths */

/* Number of floats of the flat parameter vector. */
size_t gs2d_net_param_count(void);

/* Offsets (in floats) of every layer's weights and bias in the flat vector,
 * and each layer's fan-in (c_in * 9, or the FC input width); arrays of
 * GS2D_NET_LAYERS entries. */
int gs2d_net_layout(size_t* w_off, size_t* b_off, int* fan_in);

/* Workspace bytes for gs2d_net_forward / gs2d_net_grad at this batch. */
size_t gs2d_net_workspace(int batch);

/* Network input from images of one size: rendered colour r_rgb [B*H*W*3],
 * rendered accumulated depth r_depth and opacity r_opacity [B*H*W] (as
 * gs2d_render_fwd writes them), observed colour o_rgb and depth o_depth.
 * x [B*H*W*8] bfloat16 (raw uint16 bits): channels rendered rgb, rendered
 * expected depth D/O - GS2D_NET_DEPTH_OFFSET (0 where O <= 0.5), observed
 * rgb, observed depth - offset (0 where it is not positive).  H and W must
 * equal GS2D_NET_IN_H and GS2D_NET_IN_W for the network. */
int gs2d_net_pack_input(const float* r_rgb, const float* r_depth, const float* r_opacity,
                        const float* o_rgb, const float* o_depth, int batch, int height,
                        int width, uint16_t* x, gs2d_stream stream);

/* The network's view of a full-resolution observation: rgb [H*W*3] and
 * depth [H*W] box-downsampled by an integer factor (H and W multiples of
 * it) to rgb_out [(H/f)*(W/f)*3] (block mean) and depth_out [(H/f)*(W/f)]
 * (mean of the block's valid depths, 0 if none); e.g. 640 x 480 -> 160 x 120
 * with f = 4, the camera's fx, fy, cx, cy divided by f. */
int gs2d_net_downsample_rgbd(const float* rgb, const float* depth, int height, int width,
                             int factor, float* rgb_out, float* depth_out, gs2d_stream stream);

/* Forward pass: y [batch * 6] (FP32) from x [batch * 120 * 160 * 8]. */
int gs2d_net_forward(const float* params, const uint16_t* x, int batch, float* y,
                     void* workspace, size_t ws_bytes, size_t* ws_needed, gs2d_stream stream);

/* Inference with fixed weights: gs2d_net_prepare writes the bfloat16 copy of
 * the weights into a workspace sized for this batch; gs2d_net_forward_prepared
 * is gs2d_net_forward without that cast, valid while the weights and the
 * workspace are unchanged since the last gs2d_net_prepare with this batch
 * (params still supplies the FP32 biases). */
int gs2d_net_prepare(const float* params, int batch, void* workspace, size_t ws_bytes,
                     size_t* ws_needed, gs2d_stream stream);
int gs2d_net_forward_prepared(const float* params, const uint16_t* x, int batch, float* y,
                              void* workspace, size_t ws_bytes, size_t* ws_needed,
                              gs2d_stream stream);

/* Forward + loss + backward: loss [1] (FP32) against target [batch * 6] and
 * the flat gradient grad [gs2d_net_param_count()] (FP32, overwritten);
 * y [batch * 6] may be NULL. */
int gs2d_net_grad(const float* params, const uint16_t* x, const float* target, int batch,
                  float* loss, float* grad, float* y, void* workspace, size_t ws_bytes,
                  size_t* ws_needed, gs2d_stream stream);

/* AdamW (Loshchilov & Hutter) on n parameters, decoupled weight decay:
 * p <- p (1 - lr wd); m <- b1 m + (1 - b1) g; v <- b2 v + (1 - b2) g^2;
 * p <- p - lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * step >= 1 counts this update. */
int gs2d_net_adamw(float* params, const float* grad, float* m, float* v, size_t n, int step,
                   float lr, float beta1, float beta2, float eps, float weight_decay,
                   gs2d_stream stream);

/* Applies proposals: poses [batch * 12] (row-major R then t, world to
 * camera) <- Exp(y * GS2D_NET_TAU_SCALE) pose, y [batch * 6]. */
int gs2d_net_apply(const float* y, int batch, float* poses, gs2d_stream stream);

/* Training targets: target [batch * 6] = Log(T_gt T_init^-1) /
 * GS2D_NET_TAU_SCALE (rho then theta), so that Exp(target * scale) T_init =
 * T_gt; poses [batch * 12] as above; rotation angles below pi. */
int gs2d_net_target(const float* poses_init, const float* poses_gt, int batch, float* target,
                    gs2d_stream stream);

/* The proposal's fallback: for every b, pose[b] <- proposal[b] when
 * loss_prop[b] <= loss_init[b] (the tracking loss, Eq. tracking_loss, at
 * the proposed and at the current pose), else pose[b] is kept; accepted
 * [batch] (int32, may be NULL) records the choice. */
int gs2d_net_accept(const float* loss_prop, const float* loss_init, const float* proposal,
                    int batch, float* poses, int32_t* accepted, gs2d_stream stream);

/* gs2d_net_accept that also keeps what the kept pose's next proposal pass
 * needs, so the network can refine its own proposal without rendering the
 * kept pose again: where proposal b is taken, its rendered images (prop_rgb
 * [n_px*3], prop_depth and prop_opacity [n_px] per element, as
 * gs2d_render_fwd writes them) are copied over kept_rgb / kept_depth /
 * kept_opacity (the images of the current pose), and loss_prop[b] over
 * loss_init[b]; elsewhere both stay as they are.  Renders are deterministic,
 * so the kept images equal a new render at the kept pose bit for bit.  The
 * copy runs before the poses and losses change (two kernels in stream
 * order). */
int gs2d_net_accept_keep(const float* loss_prop, float* loss_init, const float* proposal, int batch,
                         float* poses, int32_t* accepted, size_t n_px, const float* prop_rgb,
                         const float* prop_depth, const float* prop_opacity, float* kept_rgb,
                         float* kept_depth, float* kept_opacity, gs2d_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* GS2D_NET_H_ */
