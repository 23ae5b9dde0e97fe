// Per-pixel loss kernels of tracking (Sec. III-D) and mapping (Sec. III-E):
// value and gradient w.r.t. the rendered images in one pass, per-block
// partial sums of the loss reduced in a fixed order.
#include "gs2d_common.cuh"
#include "gs2d_internal.h"
#include "loss_pixel.cuh"

namespace gs2d {

constexpr int kLossBlocks = 4 * 152;
constexpr int kLossThreads = 256;

// L_t = 1/|Omega| sum M_n M_o (|I_r - I|_1 + lambda_d |D_r - D|), Eq.
// tracking_loss; M_n = [N_r . r > 0] (Eq. normal_mask; r's length does not
// change the sign), M_o = [O > thresh] (Eq. opacity_mask); D_r = D/O in
// depth_mode 1.  Sub-gradient sign(0) = 0; the masks carry no gradient.
__global__ void __launch_bounds__(kLossThreads) tracking_loss_kernel(
    const float* __restrict__ rgb, const float* __restrict__ depth, const float* __restrict__ normal,
    const float* __restrict__ opac, const float* __restrict__ obs_rgb,
    const float* __restrict__ obs_depth, gs2d_camera cam, gs2d_track_params prm,
    float* __restrict__ g_rgb, float* __restrict__ g_depth, float* __restrict__ g_opac,
    float* __restrict__ part, const int32_t* __restrict__ gate) {
  __shared__ float s[kLossThreads / 32];
  if (gate && *gate) return;
  const int P = cam.width * cam.height;
  const float inv = 1.f / (float)P;
  float acc = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const float x = (i % cam.width) + 0.5f, y = (i / cam.width) + 0.5f;
    const float rx = (x - cam.cx) / cam.fx, ry = (y - cam.cy) / cam.fy;
    const PixLoss L = tracking_pixel_loss(
        f3(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2]), depth[i],
        f3(normal[3 * i], normal[3 * i + 1], normal[3 * i + 2]), opac[i],
        f3(obs_rgb[3 * i], obs_rgb[3 * i + 1], obs_rgb[3 * i + 2]), obs_depth[i], rx, ry, inv, prm);
    acc += L.loss;
    g_rgb[3 * i] = L.g_rgb[0];
    g_rgb[3 * i + 1] = L.g_rgb[1];
    g_rgb[3 * i + 2] = L.g_rgb[2];
    g_depth[i] = L.g_depth;
    g_opac[i] = L.g_opac;
  }
  const float t = block_sum256(acc, s);
  if (threadIdx.x == 0) part[blockIdx.x] = t * inv;
}

__global__ void __launch_bounds__(256) sum_parts_kernel(const float* __restrict__ part, int n,
                                                        float* __restrict__ out,
                                                        const int32_t* __restrict__ gate) {
  __shared__ float s[256];
  if (gate && *gate) return;
  float v = 0.f;
  for (int i = threadIdx.x; i < n; i += 256) v += part[i];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// ---------------------------------------------------------------------------
// Mapping loss (Sec. III-E, colour term without SSIM):
//   per pixel |I_r - I|_1 + w_d |D_r/O - D| + w_n (1 - N_D . N_r),
// N_D = normalised cross product of the central differences of the
// back-projected points X = (D_r/O) r (Eq. normal_fromD), counted at interior
// pixels whose own and 4-neighbour opacities exceed 0.5.  The normal term's
// gradient w.r.t. the depth of pixel q collects the four stencils that use
// q, recomputed here (a gather, so no atomics).
// Tiles of 32 x 8 pixels; a block strides over tiles in a fixed order.
// Phase 0 stages D/O and O of the tile and a two-pixel ring in shared
// memory; phase 1 evaluates the normal term once for every position of the
// tile and its one-pixel edge ring (the four neighbours' stencils read it);
// phase 2 forms each pixel's outputs, gathering the neighbours' gradients
// w.r.t. its back-projected point from there.
constexpr int kMapTW = 32, kMapTH = 8;
constexpr int kMapRW = kMapTW + 2, kMapRH = kMapTH + 2;  // with the ring
constexpr int kMapSW = kMapTW + 4, kMapSH = kMapTH + 4;  // with two rings
struct MapSmem {
  float dh[kMapSH][kMapSW];     // D / max(O, 1e-6); 0 outside the image
  float op[kMapSH][kMapSW];     // O; 0 outside the image
  float g[kMapRH][kMapRW][12];  // dL_n / dX of the four stencil points
  float ln[kMapTH][kMapTW];     // L_n of the tile's own pixels
  float gn[kMapTH][kMapTW][3];  // dL_n / dN_r of the tile's own pixels
  bool ok[kMapRH][kMapRW];
};

// Pixel ray (x', y', 1) of pixel (px, py) with the reciprocal focal lengths
// (ifx, ify) = (1/fx, 1/fy) taken once per kernel.
__device__ __forceinline__ F3 ray_of(const gs2d_camera& cam, float ifx, float ify, int px, int py) {
  return f3((px + 0.5f - cam.cx) * ifx, (py + 0.5f - cam.cy) * ify, 1.f);
}
// Normal term at pixel (px, py), staged at (sx, sy) of the two-ring arrays:
// returns L_n (false if invalid: border pixel, own or a 4-neighbour's
// opacity <= 0.5, degenerate cross product) and the gradients of L_n w.r.t.
// X(p+ex), X(p-ex), X(p+ey), X(p-ey) and N_r(p).
__device__ bool ln_eval(const MapSmem& sm, const float* __restrict__ normal,
                        const gs2d_camera& cam, float ifx, float ify, int px, int py, int sx,
                        int sy, float& Ln, F3 g[4], F3& gNr) {
  const int W = cam.width, H = cam.height;
  if (px < 1 || py < 1 || px > W - 2 || py > H - 2) return false;
  if (!(sm.op[sy][sx] > 0.5f && sm.op[sy][sx - 1] > 0.5f && sm.op[sy][sx + 1] > 0.5f &&
        sm.op[sy - 1][sx] > 0.5f && sm.op[sy + 1][sx] > 0.5f))
    return false;
  const int i = py * W + px;
  const F3 Xr = sm.dh[sy][sx + 1] * ray_of(cam, ifx, ify, px + 1, py);
  const F3 Xl = sm.dh[sy][sx - 1] * ray_of(cam, ifx, ify, px - 1, py);
  const F3 Xd = sm.dh[sy + 1][sx] * ray_of(cam, ifx, ify, px, py + 1);
  const F3 Xu = sm.dh[sy - 1][sx] * ray_of(cam, ifx, ify, px, py - 1);
  const F3 gx = 0.5f * (Xr - Xl), gy = 0.5f * (Xd - Xu);
  const F3 n = cross3(gx, gy);
  const float n2 = dot3(n, n);
  if (!(n2 > 0.f)) return false;
  const float inn = rsqrtf(n2);  // 1 / |n|
  const F3 ND = inn * n;
  const F3 Nr = f3(normal[3 * i], normal[3 * i + 1], normal[3 * i + 2]);
  const float dp = dot3(ND, Nr);
  Ln = 1.f - dp;
  gNr = (-1.f) * ND;
  // dLn/dn = -(Nr - ND (ND . Nr)) / |n|
  const F3 gn = (-inn) * (Nr - dp * ND);
  const F3 ggx = cross3(gy, gn), ggy = cross3(gn, gx);
  g[0] = 0.5f * ggx;
  g[1] = (-0.5f) * ggx;
  g[2] = 0.5f * ggy;
  g[3] = (-0.5f) * ggy;
  return true;
}

// One 32 x 8 tile of the mapping loss at (x0, y0): gradients written for
// its pixels, this thread's pixel's loss terms added to acc (unscaled).
__device__ __forceinline__ void mapping_loss_tile(
    MapSmem& sm, int x0, int y0, const float* __restrict__ rgb, const float* __restrict__ depth,
    const float* __restrict__ normal, const float* __restrict__ opac,
    const float* __restrict__ obs_rgb, const float* __restrict__ obs_depth,
    const gs2d_camera& cam, float ifx, float ify, float inv, float w_l1, float w_d, float w_n,
    float* __restrict__ g_rgb, float* __restrict__ g_depth, float* __restrict__ g_normal,
    float* __restrict__ g_opac, float& acc) {
  const int W = cam.width, H = cam.height;
  __syncthreads();
  // phase 0: D/O and O on the tile and two rings
  for (int e = threadIdx.x; e < kMapSW * kMapSH; e += blockDim.x) {
    const int sy = e / kMapSW, sx = e % kMapSW;
    const int px = x0 + sx - 2, py = y0 + sy - 2;
    float d = 0.f, o = 0.f;
    if (px >= 0 && py >= 0 && px < W && py < H) {
      const int i = py * W + px;
      o = opac[i];
      d = depth[i] / fmaxf(o, 1e-6f);
    }
    sm.dh[sy][sx] = d;
    sm.op[sy][sx] = o;
  }
  __syncthreads();
  // phase 1: the normal term on the tile and its ring
  for (int e = threadIdx.x; e < kMapRW * kMapRH; e += blockDim.x) {
    const int ry = e / kMapRW, rx = e % kMapRW;
    const int px = x0 + rx - 1, py = y0 + ry - 1;
    const bool tile_px = rx >= 1 && rx <= kMapTW && ry >= 1 && ry <= kMapTH;
    const bool ring = !tile_px && !((rx == 0 || rx == kMapRW - 1) && (ry == 0 || ry == kMapRH - 1));
    float Ln = 0.f;
    F3 g4[4], gNr = f3(0.f, 0.f, 0.f);
    bool ok = false;
    if ((tile_px || ring) && px >= 0 && py >= 0 && px < W && py < H)
      ok = ln_eval(sm, normal, cam, ifx, ify, px, py, rx + 1, ry + 1, Ln, g4, gNr);
    sm.ok[ry][rx] = ok;
    if (ok)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        sm.g[ry][rx][3 * k] = g4[k].x;
        sm.g[ry][rx][3 * k + 1] = g4[k].y;
        sm.g[ry][rx][3 * k + 2] = g4[k].z;
      }
    if (tile_px) {
      sm.ln[ry - 1][rx - 1] = ok ? Ln : 0.f;
      sm.gn[ry - 1][rx - 1][0] = ok ? gNr.x : 0.f;
      sm.gn[ry - 1][rx - 1][1] = ok ? gNr.y : 0.f;
      sm.gn[ry - 1][rx - 1][2] = ok ? gNr.z : 0.f;
    }
  }
  __syncthreads();
  // phase 2: one pixel per thread
  const int lx = threadIdx.x % kMapTW, ly = threadIdx.x / kMapTW;
  const int px = x0 + lx, py = y0 + ly;
  if (px < W && py < H) {
    const int i = py * W + px;
    const float O = sm.op[ly + 2][lx + 2];
    const float Oc = fmaxf(O, 1e-6f);
    const float D = depth[i];
    const float Dh = sm.dh[ly + 2][lx + 2];
    const float d0 = rgb[3 * i] - obs_rgb[3 * i];
    const float d1 = rgb[3 * i + 1] - obs_rgb[3 * i + 1];
    const float d2 = rgb[3 * i + 2] - obs_rgb[3 * i + 2];
    const float dd = Dh - obs_depth[i];
    acc += w_l1 * (fabsf(d0) + fabsf(d1) + fabsf(d2)) + w_d * fabsf(dd);
    const float sl = w_l1 * inv;
    g_rgb[3 * i] = sgnf(d0) * sl;
    g_rgb[3 * i + 1] = sgnf(d1) * sl;
    g_rgb[3 * i + 2] = sgnf(d2) * sl;
    float gDh = w_d * sgnf(dd) * inv;
    // own normal term
    const int ry = ly + 1, rx = lx + 1;
    if (sm.ok[ry][rx]) acc += w_n * sm.ln[ly][lx];
    const float sn = w_n * inv;
    g_normal[3 * i] = sn * sm.gn[ly][lx][0];
    g_normal[3 * i + 1] = sn * sm.gn[ly][lx][1];
    g_normal[3 * i + 2] = sn * sm.gn[ly][lx][2];
    // stencils of the four neighbours that read X(q): p = q-ex uses X(p+ex)
    // (slot 0), p = q+ex uses X(p-ex) (1), p = q-ey uses X(p+ey) (2),
    // p = q+ey uses X(p-ey) (3)
    const F3 rq = ray_of(cam, ifx, ify, px, py);
    const int nb[4][3] = {{rx - 1, ry, 0}, {rx + 1, ry, 1}, {rx, ry - 1, 2}, {rx, ry + 1, 3}};
    F3 gX = f3(0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int qx = nb[k][0], qy = nb[k][1], sl2 = nb[k][2];
      if (sm.ok[qy][qx])
        gX = gX + f3(sm.g[qy][qx][3 * sl2], sm.g[qy][qx][3 * sl2 + 1], sm.g[qy][qx][3 * sl2 + 2]);
    }
    gDh += w_n * inv * dot3(gX, rq);
    g_depth[i] = gDh / Oc;
    g_opac[i] = O > 1e-6f ? -gDh * D / (O * O) : 0.f;
  }
}

__global__ void __launch_bounds__(kLossThreads) mapping_loss_kernel(
    const float* __restrict__ rgb, const float* __restrict__ depth, const float* __restrict__ normal,
    const float* __restrict__ opac, const float* __restrict__ obs_rgb,
    const float* __restrict__ obs_depth, gs2d_camera cam, float w_l1, float w_d, float w_n,
    float* __restrict__ g_rgb, float* __restrict__ g_depth, float* __restrict__ g_normal,
    float* __restrict__ g_opac, float* __restrict__ part) {
  __shared__ float s[kLossThreads / 32];
  __shared__ MapSmem sm;
  const int W = cam.width, H = cam.height, P = W * H;
  const float inv = 1.f / (float)P;
  const int tiles_x = (W + kMapTW - 1) / kMapTW, tiles_y = (H + kMapTH - 1) / kMapTH;
  const float ifx = 1.f / cam.fx, ify = 1.f / cam.fy;
  float acc = 0.f;
  for (int tile = blockIdx.x; tile < tiles_x * tiles_y; tile += gridDim.x)
    mapping_loss_tile(sm, (tile % tiles_x) * kMapTW, (tile / tiles_x) * kMapTH, rgb, depth, normal,
                      opac, obs_rgb, obs_depth, cam, ifx, ify, inv, w_l1, w_d, w_n, g_rgb,
                      g_depth, g_normal, g_opac, acc);
  const float t = block_sum256(acc, s);
  if (threadIdx.x == 0) part[blockIdx.x] = t * inv;
}

// The mapping loss of many views in one launch: work items are the views'
// 32 x 8 tiles in view order; each tile's loss terms are summed per warp
// into part[item * 8 + warp] (no block barrier beyond the tile's own), and
// mapping_loss_batch_sum_kernel adds each view's items in order.
struct LossViewDev {
  gs2d_camera cam;
  const float *rgb, *depth, *normal, *opac, *obs_rgb, *obs_depth;
  float *g_rgb, *g_depth, *g_normal, *g_opac;
  int tiles_x, item0, n_items;
};
struct LossTable {
  int n_views, n_items;
  LossViewDev v[GS2D_MAX_VIEWS];
};
constexpr int kLossWarps = kLossThreads / 32;

__global__ void __launch_bounds__(kLossThreads) mapping_loss_batch_kernel(const LossTable tab,
                                                                          float w_d, float w_n,
                                                                          float* __restrict__ part) {
  __shared__ MapSmem sm;
  for (int item = blockIdx.x; item < tab.n_items; item += gridDim.x) {
    int v = 0;
    while (v + 1 < tab.n_views && item >= tab.v[v + 1].item0) ++v;
    const LossViewDev& V = tab.v[v];
    const int tile = item - V.item0;
    const float inv = 1.f / (float)(V.cam.width * V.cam.height);
    float acc = 0.f;
    mapping_loss_tile(sm, (tile % V.tiles_x) * kMapTW, (tile / V.tiles_x) * kMapTH, V.rgb, V.depth,
                      V.normal, V.opac, V.obs_rgb, V.obs_depth, V.cam, 1.f / V.cam.fx,
                      1.f / V.cam.fy, inv, 1.f, w_d, w_n, V.g_rgb, V.g_depth, V.g_normal, V.g_opac,
                      acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) part[(size_t)item * kLossWarps + (threadIdx.x >> 5)] = acc;
  }
}

// loss_out[v] = inv_v x the sum of view v's per-warp partials: thread t adds
// entries t, t + 256, ... in order, then a fixed tree over the threads.
__global__ void __launch_bounds__(256) mapping_loss_batch_sum_kernel(const LossTable tab,
                                                                     const float* __restrict__ part,
                                                                     float* __restrict__ loss_out) {
  __shared__ float s[256];
  const LossViewDev& V = tab.v[blockIdx.x];
  const float* p = part + (size_t)V.item0 * kLossWarps;
  const int n = V.n_items * kLossWarps;
  float a = 0.f;
#pragma unroll 8
  for (int e = threadIdx.x; e < n; e += 256) a += p[e];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_out[blockIdx.x] = s[0] / (float)(V.cam.width * V.cam.height);
}

size_t loss_ws_bytes(const gs2d_camera* cam) {
  (void)cam;
  return align_up(kLossBlocks * sizeof(float), 256);
}

int tracking_loss_launch(const float* rgb, const float* depth, const float* normal,
                         const float* opacity, const float* obs_rgb, const float* obs_depth,
                         const gs2d_camera* cam, const gs2d_track_params* prm, float* g_rgb,
                         float* g_depth, float* g_opacity, float* loss_out, void* workspace,
                         size_t ws_bytes, size_t* ws_needed, const int32_t* gate, cudaStream_t st) {
  if (!rgb || !depth || !normal || !opacity || !obs_rgb || !obs_depth || !cam || !prm || !g_rgb ||
      !g_depth || !g_opacity || !loss_out)
    return GS2D_ERR_INVALID_ARG;
  if (cam->width <= 0 || cam->height <= 0) return GS2D_ERR_INVALID_ARG;
  const size_t need = loss_ws_bytes(cam);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  float* part = static_cast<float*>(workspace);
  tracking_loss_kernel<<<kLossBlocks, kLossThreads, 0, st>>>(rgb, depth, normal, opacity, obs_rgb,
                                                             obs_depth, *cam, *prm, g_rgb, g_depth,
                                                             g_opacity, part, gate);
  GS2D_LAUNCH_CHECK();
  sum_parts_kernel<<<1, 256, 0, st>>>(part, kLossBlocks, loss_out, gate);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

}  // namespace gs2d

using namespace gs2d;

extern "C" {

int gs2d_tracking_loss(const float* rgb, const float* depth, const float* normal,
                       const float* opacity, const float* obs_rgb, const float* obs_depth,
                       const gs2d_camera* cam, const gs2d_track_params* prm, float* g_rgb,
                       float* g_depth, float* g_opacity, float* loss_out, void* workspace,
                       size_t ws_bytes, size_t* ws_needed, gs2d_stream stream) {
  return tracking_loss_launch(rgb, depth, normal, opacity, obs_rgb, obs_depth, cam, prm, g_rgb,
                              g_depth, g_opacity, loss_out, workspace, ws_bytes, ws_needed, nullptr,
                              (cudaStream_t)stream);
}

int gs2d_mapping_loss(const float* rgb, const float* depth, const float* normal,
                      const float* opacity, const float* obs_rgb, const float* obs_depth,
                      const gs2d_camera* cam, float w_d, float w_n, float* g_rgb, float* g_depth,
                      float* g_normal, float* g_opacity, float* loss_out, void* workspace,
                      size_t ws_bytes, size_t* ws_needed, gs2d_stream stream) {
  return gs2d_mapping_loss_ssim(rgb, depth, normal, opacity, obs_rgb, obs_depth, cam, 0.f, w_d,
                                w_n, g_rgb, g_depth, g_normal, g_opacity, loss_out, workspace,
                                ws_bytes, ws_needed, stream);
}

size_t gs2d_mapping_loss_batch_workspace(const gs2d_loss_view* views, int n_views) {
  if (!views || n_views <= 0 || n_views > GS2D_MAX_VIEWS) return 0;
  size_t items = 0;
  for (int v = 0; v < n_views; ++v) {
    const gs2d_camera& c = views[v].cam;
    if (c.width <= 0 || c.height <= 0) return 0;
    items += (size_t)((c.width + kMapTW - 1) / kMapTW) * ((c.height + kMapTH - 1) / kMapTH);
  }
  return align_up(items * kLossWarps * sizeof(float), 256);
}

int gs2d_mapping_loss_batch(const gs2d_loss_view* views, int n_views, float w_d, float w_n,
                            float* loss_out, void* workspace, size_t ws_bytes, size_t* ws_needed,
                            gs2d_stream stream) {
  if (!views || n_views <= 0 || n_views > GS2D_MAX_VIEWS || !loss_out) return GS2D_ERR_INVALID_ARG;
  LossTable tab;
  tab.n_views = n_views;
  long long items = 0;
  for (int v = 0; v < n_views; ++v) {
    const gs2d_loss_view& x = views[v];
    if (!x.rgb || !x.depth || !x.normal || !x.opacity || !x.obs_rgb || !x.obs_depth || !x.g_rgb ||
        !x.g_depth || !x.g_normal || !x.g_opacity)
      return GS2D_ERR_INVALID_ARG;
    if (x.cam.width <= 0 || x.cam.height <= 0) return GS2D_ERR_INVALID_ARG;
    LossViewDev& d = tab.v[v];
    d.cam = x.cam;
    d.rgb = x.rgb;
    d.depth = x.depth;
    d.normal = x.normal;
    d.opac = x.opacity;
    d.obs_rgb = x.obs_rgb;
    d.obs_depth = x.obs_depth;
    d.g_rgb = x.g_rgb;
    d.g_depth = x.g_depth;
    d.g_normal = x.g_normal;
    d.g_opac = x.g_opacity;
    d.tiles_x = (x.cam.width + kMapTW - 1) / kMapTW;
    d.item0 = (int)items;
    d.n_items = d.tiles_x * ((x.cam.height + kMapTH - 1) / kMapTH);
    items += d.n_items;
    if (items > 0x7FFFFFFF / kLossWarps) return GS2D_ERR_INVALID_ARG;
  }
  tab.n_items = (int)items;
  const size_t need = gs2d_mapping_loss_batch_workspace(views, n_views);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  float* part = static_cast<float*>(workspace);
  // a resident grid (the partials are per item, so the result does not
  // depend on it)
  static int slots[64] = {};
  int dev = 0;
  GS2D_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return GS2D_ERR_CUDA;
  if (!slots[dev]) {
    int per_sm = 0, sms = 0;
    GS2D_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mapping_loss_batch_kernel,
                                                                kLossThreads, 0));
    GS2D_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    slots[dev] = max(1, per_sm) * max(1, sms);
  }
  mapping_loss_batch_kernel<<<min(slots[dev], tab.n_items), kLossThreads, 0, st>>>(tab, w_d, w_n,
                                                                                  part);
  GS2D_LAUNCH_CHECK();
  mapping_loss_batch_sum_kernel<<<n_views, 256, 0, st>>>(tab, part, loss_out);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

size_t gs2d_mapping_loss_ssim_workspace(const gs2d_camera* cam) {
  if (!cam || cam->width <= 0 || cam->height <= 0) return 0;
  return loss_ws_bytes(cam) + ssim_ws_bytes(cam->height, cam->width);
}

int gs2d_mapping_loss_ssim(const float* rgb, const float* depth, const float* normal,
                           const float* opacity, const float* obs_rgb, const float* obs_depth,
                           const gs2d_camera* cam, float w_ssim, float w_d, float w_n,
                           float* g_rgb, float* g_depth, float* g_normal, float* g_opacity,
                           float* loss_out, void* workspace, size_t ws_bytes, size_t* ws_needed,
                           gs2d_stream stream) {
  if (!rgb || !depth || !normal || !opacity || !obs_rgb || !obs_depth || !cam || !g_rgb ||
      !g_depth || !g_normal || !g_opacity || !loss_out)
    return GS2D_ERR_INVALID_ARG;
  if (cam->width <= 0 || cam->height <= 0 || !(w_ssim >= 0.f && w_ssim <= 1.f))
    return GS2D_ERR_INVALID_ARG;
  const size_t base = loss_ws_bytes(cam);
  const size_t need = w_ssim > 0.f ? base + ssim_ws_bytes(cam->height, cam->width) : base;
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  float* part = static_cast<float*>(workspace);
  mapping_loss_kernel<<<kLossBlocks, kLossThreads, 0, st>>>(
      rgb, depth, normal, opacity, obs_rgb, obs_depth, *cam, 1.f - w_ssim, w_d, w_n, g_rgb,
      g_depth, g_normal, g_opacity, part);
  GS2D_LAUNCH_CHECK();
  sum_parts_kernel<<<1, 256, 0, st>>>(part, kLossBlocks, loss_out, nullptr);
  GS2D_LAUNCH_CHECK();
  if (w_ssim > 0.f)
    return ssim_launch(rgb, obs_rgb, cam->height, cam->width, w_ssim, g_rgb, loss_out,
                       static_cast<char*>(workspace) + base, ws_bytes - base, nullptr, st);
  return GS2D_OK;
}

}  // extern "C"
