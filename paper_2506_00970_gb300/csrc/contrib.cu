// gs2d_render_contrib / gs2d_covisibility: per-surfel rendering contribution
// (Eq. weight and Eq. contribution, Sec. III-D keyframe selection) and the
// covisibility score of two views with the keyframe rule.
//
// Contribution: the forward compositing of gs2d_render_fwd replayed front to
// back (same staging, same culling, same skip and stop decisions, so every
// blending weight w_k(p) = a_k T_k is the forward's), and instead of images
// the weights are summed per surfel.  Per staged batch each warp walks its
// hit list in chunks of 16 surfels: every lane stores its pixels' weight sum
// for each surfel of the chunk in a 16 x 32 shared-memory table (one row per
// surfel, padded to 33 columns: conflict-free both ways), then each row is
// summed by two half-warps in a fixed order and combined with one shuffle.
// The 8 warps' sums of a staged surfel are added in warp order and written
// once per (tile, surfel) pair at the pair's emission index; a second kernel
// adds each surfel's partials in emission order.  Deterministic, no atomics.
#include "gs2d_common.cuh"
#include "gs2d_internal.h"
#include "tile_loops.cuh"

namespace gs2d {

constexpr int kCtbVec4 = 4;    // c0t|c1.x, c1.yz|c2.xy, c2.z|det|alpha, footprint
constexpr int kCtbChunk = 16;  // surfels per transpose chunk

struct CtbSmem {
  float4 rec[kTileThreads][kCtbVec4];
  HitLists hl;
  float tr[kTileThreads / 32][kCtbChunk][33];
  float wsum[kTileThreads / 32][kTileThreads];
};

template <int P>
__global__ void __launch_bounds__(kTileThreads, P == 1 ? 4 : (P == 2 ? 3 : 2)) contrib_tile_kernel(
    const float4* __restrict__ proj, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ emit, const int32_t* __restrict__ ranges, gs2d_camera cam,
    gs2d_config cfg, int tiles_x, float* __restrict__ partials, const int32_t* __restrict__ gate) {
  __shared__ CtbSmem sm;
  if (gate && *gate) return;
  const int tile = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TilePix<P> tp = tile_pixel<P>(tile, tiles_x, cfg.tile_w, cfg.tile_h);
  const int tile_x0 = (tile % tiles_x) * cfg.tile_w, tile_y0 = (tile / tiles_x) * cfg.tile_h;
  const float xt = (float)tile_x0 + 0.5f - cam.cx;
  const float yt = (float)tile_y0 + 0.5f - cam.cy;
  const int start = ranges[2 * tile], end = ranges[2 * tile + 1];
  float T[P], lyk[P];
  bool done[P];
  bool all_done = true;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    T[k] = 1.f;
    lyk[k] = k ? tp.ly + 4.f * k : tp.ly;
    done[k] = !(tp.px < cam.width && tp.py + 4 * k < cam.height);
    all_done = all_done && done[k];
  }
  int b = start;
  for (; b < end; b += kTileThreads) {
    if (__syncthreads_count(!all_done) == 0) break;
    const int idx = b + (int)threadIdx.x;
    if (idx < end) {
      const float4* src = proj + (size_t)vals[idx] * (kProjFloats / 4);
      const float4 r0 = src[0], r1 = src[1], r2 = src[2], r7 = src[7];
      sm.rec[threadIdx.x][0] = stage_c0(r0, r1, r2, xt, yt);
      sm.rec[threadIdx.x][1] = r1;
      sm.rec[threadIdx.x][2] = r2;
      sm.rec[threadIdx.x][3] = make_float4(r7.z, r7.w, 0.f, 0.f);
      sm.hl.mask[threadIdx.x] = footprint_mask<P>(r7.z, r7.w, tile_x0, tile_y0, cfg.tile_w);
    }
    __syncthreads();
    const int cnt_b = min(kTileThreads, end - b);
    const int nh = warp_hit_list(sm.hl.mask, sm.hl.list[warp], cnt_b, warp, lane);
    for (int base = 0; base < nh; base += kCtbChunk) {
      const int m = min(kCtbChunk, nh - base);
      if (__all_sync(0xffffffffu, all_done)) {
        // the warp's pixels have all stopped: zero weight for the rest
        for (int i = base + lane; i < nh; i += 32) sm.wsum[warp][sm.hl.list[warp][i]] = 0.f;
        break;
      }
      for (int i = 0; i < m; ++i) {
        const int j = sm.hl.list[warp][base + i];
        const float4 r0 = sm.rec[j][0], r1 = sm.rec[j][1], r2 = sm.rec[j][2];
        float w = 0.f;
#pragma unroll
        for (int k = 0; k < P; ++k) {
          if (done[k]) continue;
          Eval e;
          if (!eval_pair(r0, r1, r2, tp.lx, lyk[k], cam.near_z, cfg.cutoff_r2, cfg.alpha_min,
                         cfg.alpha_max, e))
            continue;
          const float Tn = T[k] * (1.f - e.a);
          if (Tn < cfg.t_min) {
            done[k] = true;
            continue;
          }
          w += e.a * T[k];
          T[k] = Tn;
        }
        sm.tr[warp][i][lane] = w;
      }
      all_done = true;
#pragma unroll
      for (int k = 0; k < P; ++k) all_done = all_done && done[k];
      __syncwarp();
      // row r = surfel base + r; half-warp h sums columns 16h .. 16h + 15
      const int r = lane & 15, h = lane >> 4;
      float s = 0.f;
      if (r < m) {
#pragma unroll
        for (int c = 0; c < 16; ++c) s += sm.tr[warp][r][16 * h + c];
      }
      s += __shfl_xor_sync(0xffffffffu, s, 16);
      if (h == 0 && r < m) sm.wsum[warp][sm.hl.list[warp][base + r]] = s;
      __syncwarp();
    }
    __syncthreads();
    if (idx < end) {
      const uint32_t mk = sm.hl.mask[threadIdx.x];
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < kTileThreads / 32; ++w)
        if ((mk >> w) & 1u) s += sm.wsum[w][threadIdx.x];
      partials[emit[idx]] = s;
    }
  }
  // the rest of the list was not reached by any pixel
  for (int idx = b + (int)threadIdx.x; idx < end; idx += kTileThreads) partials[emit[idx]] = 0.f;
}

// contrib[i] = sum of surfel i's partials in emission order.
__global__ void __launch_bounds__(256) contrib_reduce_kernel(const int32_t* __restrict__ tiles,
                                                             const uint32_t* __restrict__ surfel_off,
                                                             const float* __restrict__ partials,
                                                             int n, float* __restrict__ contrib,
                                                             const int32_t* __restrict__ gate) {
  if (gate && *gate) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = tiles[i];
  float s = 0.f;
  if (k > 0) {
    const float* p = partials + surfel_off[i];
    for (int e = 0; e < k; ++e) s += p[e];
  }
  contrib[i] = s;
}

// Covisibility counts |G_A n G_B| and |G_A u G_B| (integers, so the atomic
// order does not matter).
__global__ void __launch_bounds__(256) covis_count_kernel(const float* __restrict__ ca,
                                                          const float* __restrict__ cb, int n,
                                                          float thr, uint32_t* __restrict__ counts) {
  uint32_t inter = 0, uni = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const bool a = ca[i] > thr, b = cb[i] > thr;
    inter += (a && b) ? 1u : 0u;
    uni += (a || b) ? 1u : 0u;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    inter += __shfl_xor_sync(0xffffffffu, inter, off);
    uni += __shfl_xor_sync(0xffffffffu, uni, off);
  }
  if ((threadIdx.x & 31) == 0 && (inter || uni)) {
    atomicAdd(counts, inter);
    atomicAdd(counts + 1, uni);
  }
}

// S_cov = |G_A n G_B| / |G_A u G_B| (0 when both sets are empty) and the
// keyframe rule: S_cov < c_k or |t_A - t_B| > d_k, t the translation of the
// world-to-camera pose T_cw.
__global__ void covis_final_kernel(const uint32_t* __restrict__ counts,
                                   const float* __restrict__ pose_a,
                                   const float* __restrict__ pose_b, float c_k, float d_k,
                                   float* __restrict__ score, int32_t* __restrict__ is_kf) {
  const uint32_t inter = counts[0], uni = counts[1];
  const float s = uni ? (float)((double)inter / (double)uni) : 0.f;
  if (score) *score = s;
  if (is_kf) {
    const float dx = pose_a[9] - pose_b[9], dy = pose_a[10] - pose_b[10],
                dz = pose_a[11] - pose_b[11];
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    *is_kf = (s < c_k || d2 > d_k * d_k) ? 1 : 0;
  }
}

}  // namespace gs2d

using namespace gs2d;

extern "C" {

size_t gs2d_render_contrib_workspace(size_t capacity) {
  return align_up((capacity > 0 ? capacity : 1) * sizeof(float), 256);
}

int gs2d_render_contrib(const float* proj, const gs2d_bins* bins, const int32_t* tiles_per_surfel,
                        int n, const gs2d_camera* cam, const gs2d_config* cfg, float* contrib,
                        void* workspace, size_t ws_bytes, size_t* ws_needed, gs2d_stream stream) {
  if (!bins || n < 0) return GS2D_ERR_INVALID_ARG;
  const int v = validate_tile_cfg(cam, cfg);
  if (v) return v;
  const size_t need = gs2d_render_contrib_workspace(bins->capacity);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  if (n == 0) return GS2D_OK;
  if (!proj || !bins->vals || !bins->isect_emit || !bins->surfel_off || !bins->tile_ranges ||
      !tiles_per_surfel || !contrib)
    return GS2D_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(proj) & 15) return GS2D_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  float* partials = static_cast<float*>(workspace);
  const int tx = gs2d_tiles_x(cam, cfg), ty = gs2d_tiles_y(cam, cfg);
  GS2D_DISPATCH_P(cfg->px_per_thread, contrib_tile_kernel<P><<<tx * ty, kTileThreads, 0, st>>>(
      reinterpret_cast<const float4*>(proj), bins->vals, bins->isect_emit, bins->tile_ranges, *cam,
      *cfg, tx, partials, bins->status));
  GS2D_LAUNCH_CHECK();
  contrib_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(tiles_per_surfel, bins->surfel_off,
                                                         partials, n, contrib, bins->status);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int gs2d_covisibility(const float* contrib_a, const float* contrib_b, int n, float vis_threshold,
                      const float* pose_a, const float* pose_b, float c_k, float d_k,
                      uint32_t* counts, float* score, int32_t* is_keyframe, gs2d_stream stream) {
  if (n < 0 || !counts || (n > 0 && (!contrib_a || !contrib_b))) return GS2D_ERR_INVALID_ARG;
  if (is_keyframe && (!pose_a || !pose_b)) return GS2D_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(counts, 0, 2 * sizeof(uint32_t), st) != cudaSuccess) return GS2D_ERR_CUDA;
  if (n > 0) {
    const int blocks = min((n + 255) / 256, 152 * 8);
    covis_count_kernel<<<blocks, 256, 0, st>>>(contrib_a, contrib_b, n, vis_threshold, counts);
    GS2D_LAUNCH_CHECK();
  }
  if (score || is_keyframe) {
    covis_final_kernel<<<1, 1, 0, st>>>(counts, pose_a, pose_b, c_k, d_k, score, is_keyframe);
    GS2D_LAUNCH_CHECK();
  }
  return GS2D_OK;
}

}  // extern "C"
