// gs2d_render_fwd / gs2d_render_bwd: tile-based front-to-back compositing of
// 2D Gaussian surfels (Eq. alpha_blending) and its reverse mode to the surfel
// parameters and to the camera pose (Sec. III-B, Eq. derivatives), plus the
// fused tracking kernel (forward, tracking loss and pose backward per tile).
//
// Forward: one 256-thread block per image tile, one pixel per thread, each
// warp an 8 x 4 pixel block.  The tile's depth-ordered surfel list is staged
// through shared memory in batches of 256 records, the record's linear
// intersection map re-based on the tile's first pixel (c0t); a warp skips a
// surfel whose footprint misses its block, and every thread evaluates
// u = p0/p2, v = p1/p2, z = det/p2 with p = c0t + lx c1 + ly c2,
// G = exp(-(u^2+v^2)/2), a = min(alpha G, alpha_max), skips a < alpha_min or
// u^2+v^2 > cutoff or z <= near, blends colour, depth z, normal t_nc and
// opacity, and stops before the transmittance would fall below t_min.  The
// block leaves the list once every pixel has stopped.
//
// Backward: each pixel replays its list back to front from the stored
// (T_final, n_last): T_i = T_{i+1} / (1 - a_i), and with the running suffix
// S = sum_{j>i} w_j (c_j . gC + z_j gD + t_nc,j . gN) the blending gradient is
//   dL/da_i = T_i (c_i . gC + z_i gD + t_nc,i . gN) - (S - gO T_final) / (1 - a_i).
// Through the intersection, with q = gu d_u + gv d_v (dual tangents) and
// beta = (q . r + gz) / (n . r) (r the pixel ray, n = m_u x m_v), the
// gradient of one (pixel, surfel) pair w.r.t. the camera-space splat is
// rank one:
//   dL/dmu_c = Gv,  dL/d(s_u t_uc) = u Gv,  dL/d(s_v t_vc) = v Gv,  Gv = beta n - q,
// (moving the plane along n shifts the hit point along the ray; moving it
// in-plane shifts (u, v) through the dual basis).  The left pose perturbation
// moves every splat by (rho, theta x .), so the pair's pose gradient is
// (Gv, X x Gv) with X = z r the hit point, plus t_nc x dL/dt_nc from the
// normal image -- the Jacobians [I, -mu_c^x] and [0, -R_c,:,i^x] of Sec. III-B
// contracted with these rank-one gradients.
//
// Full mode: per batch each warp sums its 32 pixels' 16 per-pair values with
// a butterfly reduce-scatter (16 shuffles per surfel instead of 80), the 8
// warps are summed through shared memory, and one 64-byte partial per
// (tile, surfel) pair is written at the pair's emission index.  A second
// kernel adds each surfel's partials in emission order (deterministic),
// chains to world space, scales and the quaternion, and forms the pose term.
// Tracking mode: pixels accumulate the 6-vector pose gradient directly; one
// partial per tile, reduced in a fixed order.
#include "bwd_warp.cuh"
#include "gs2d_common.cuh"
#include "gs2d_internal.h"
#include "loss_pixel.cuh"
#include "tile_loops.cuh"
#include "tile_sort.cuh"
#include "track_update.cuh"

namespace gs2d {

// Blocks per SM of the tile kernels: with P pixels per thread, and for the
// grouped one-pixel loops (kG > 1: kG evaluations in flight per thread,
// meant for grids too small to fill the GPU, where registers are plentiful
// and the per-pixel walk's latency is the bound).
constexpr int kGroup = 4;  // evaluations in flight of the grouped loops

template <int P, int kG>
constexpr int tile_blocks_per_sm() {
  return kG > 1 ? 2 : (P == 1 ? 4 : (P == 2 ? 3 : 2));
}

template <bool kCount, int P, int kG = 1>
__global__ void __launch_bounds__(kTileThreads, tile_blocks_per_sm<P, kG>()) render_fwd_kernel(
    const float4* __restrict__ proj, const uint32_t* __restrict__ vals,
    const int32_t* __restrict__ ranges, gs2d_camera cam, gs2d_config cfg, int tiles_x,
    float* __restrict__ out_rgb, float* __restrict__ out_depth, float* __restrict__ out_normal,
    float* __restrict__ out_opac, float* __restrict__ out_T, uint32_t* __restrict__ out_nlast,
    unsigned long long* __restrict__ counts, const int32_t* __restrict__ gate) {
  __shared__ float4 s_rec[kTileThreads][kFwdVec4];
  __shared__ HitLists hl;
  if (gate && *gate) return;
  const int tile = blockIdx.x;
  const TilePix<P> tp = tile_pixel<P>(tile, tiles_x, cfg.tile_w, cfg.tile_h);
  bool inside[P];
#pragma unroll
  for (int k = 0; k < P; ++k) inside[k] = tp.px < cam.width && tp.py + 4 * k < cam.height;
  const int tile_x0 = (tile % tiles_x) * cfg.tile_w, tile_y0 = (tile / tiles_x) * cfg.tile_h;
  const float xt = (float)tile_x0 + 0.5f - cam.cx;
  const float yt = (float)tile_y0 + 0.5f - cam.cy;
  uint32_t cnt[5] = {0u, 0u, 0u, 0u, 0u};
  FwdState st[P];
  fwd_tile<kFwdVec4, kCount, P, kG>(proj, vals + ranges[2 * tile], ranges[2 * tile], ranges[2 * tile + 1], xt, yt,
                                    tile_x0, tile_y0, tp, inside, cam, cfg, s_rec, hl, cnt, st);
  if (kCount) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      unsigned long long v = cnt[k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if ((threadIdx.x & 31) == 0) atomicAdd(counts + k, v);
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < P; ++k) {
    if (!inside[k]) continue;
    const size_t p = (size_t)(tp.py + 4 * k) * cam.width + tp.px;
    out_rgb[3 * p] = st[k].C.x;
    out_rgb[3 * p + 1] = st[k].C.y;
    out_rgb[3 * p + 2] = st[k].C.z;
    out_depth[p] = st[k].D;
    out_normal[3 * p] = st[k].N.x;
    out_normal[3 * p + 1] = st[k].N.y;
    out_normal[3 * p + 2] = st[k].N.z;
    out_opac[p] = 1.f - st[k].T;
    out_T[p] = st[k].T;
    out_nlast[p] = st[k].last;
  }
}

// Upstream gradients and compositing state of the thread's P pixels.
template <int P>
__device__ __forceinline__ void load_pix_grads(const TilePix<P>& tp, const bool (&inside)[P],
                                               const gs2d_camera& cam, const float* T_final,
                                               const uint32_t* n_last, const float* g_rgb,
                                               const float* g_depth, const float* g_normal,
                                               const float* g_opac, PixGrad (&pg)[P]) {
#pragma unroll
  for (int k = 0; k < P; ++k) {
    pg[k].Tf = 1.f;
    pg[k].nl = 0;
    pg[k].gC = f3(0.f, 0.f, 0.f);
    pg[k].gN = f3(0.f, 0.f, 0.f);
    pg[k].gD = 0.f;
    pg[k].gO = 0.f;
    if (!inside[k]) continue;
    const size_t p = (size_t)(tp.py + 4 * k) * cam.width + tp.px;
    pg[k].Tf = T_final[p];
    pg[k].nl = n_last[p];
    pg[k].gC = f3(g_rgb[3 * p], g_rgb[3 * p + 1], g_rgb[3 * p + 2]);
    pg[k].gD = g_depth[p];
    if (g_normal) pg[k].gN = f3(g_normal[3 * p], g_normal[3 * p + 1], g_normal[3 * p + 2]);
    if (g_opac) pg[k].gO = g_opac[p];
  }
}

// Pose-only backward (the full backward is render_bwd_warp_kernel): the
// tile's pose 6-vector partial.
template <int P>
__global__ void __launch_bounds__(kTileThreads, P == 1 ? 4 : (P == 2 ? 3 : 2)) render_bwd_kernel(
    const float4* __restrict__ proj, const uint32_t* __restrict__ vals,
    const int32_t* __restrict__ ranges, gs2d_camera cam, gs2d_config cfg, int tiles_x,
    const float* __restrict__ T_final, const uint32_t* __restrict__ n_last,
    const float* __restrict__ g_rgb, const float* __restrict__ g_depth,
    const float* __restrict__ g_normal, const float* __restrict__ g_opac,
    float* __restrict__ pose_part, const int32_t* __restrict__ gate) {
  __shared__ BwdSmem sm;
  __shared__ HitLists hl;
  __shared__ float s_pose[kTileThreads / 32][6];
  if (gate && *gate) return;
  const int tile = blockIdx.x;
  const TilePix<P> tp = tile_pixel<P>(tile, tiles_x, cfg.tile_w, cfg.tile_h);
  bool inside[P];
#pragma unroll
  for (int k = 0; k < P; ++k) inside[k] = tp.px < cam.width && tp.py + 4 * k < cam.height;
  const int tile_x0 = (tile % tiles_x) * cfg.tile_w, tile_y0 = (tile / tiles_x) * cfg.tile_h;
  const float xt = (float)tile_x0 + 0.5f - cam.cx;
  const float yt = (float)tile_y0 + 0.5f - cam.cy;
  const float rx = (tp.px + 0.5f - cam.cx) / cam.fx, ry = (tp.py + 0.5f - cam.cy) / cam.fy;
  PixGrad pg[P];
  load_pix_grads<P>(tp, inside, cam, T_final, n_last, g_rgb, g_depth, g_normal, g_opac, pg);
  float pr[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (g_normal)
    bwd_tile_pose<true, P>(proj, vals + ranges[2 * tile], ranges[2 * tile], ranges[2 * tile + 1], xt, yt, tile_x0,
                           tile_y0, tp, inside, rx, ry, cam, cfg, pg, sm, hl, pr);
  else
    bwd_tile_pose<false, P>(proj, vals + ranges[2 * tile], ranges[2 * tile], ranges[2 * tile + 1], xt, yt, tile_x0,
                            tile_y0, tp, inside, rx, ry, cam, cfg, pg, sm, hl, pr);
  block_sum6(pr, s_pose, pose_part + (size_t)tile * 6);
}

// Full backward: one warp per (tile, region) work item, kBwdWarps warps per
// block and no block barrier (bwd_warp.cuh).
template <int R>
__global__ void __launch_bounds__(kBwdWarps * 32, kBwdWarpBlocks) render_bwd_warp_kernel(
    const float4* __restrict__ proj, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ emit, const int32_t* __restrict__ ranges, gs2d_camera cam,
    gs2d_config cfg, int tiles_x, int Q, int n_units, const float* __restrict__ T_final,
    const uint32_t* __restrict__ n_last, const float* __restrict__ g_rgb,
    const float* __restrict__ g_depth, const float* __restrict__ g_normal,
    const float* __restrict__ g_opac, float* __restrict__ partials,
    const int32_t* __restrict__ gate) {
  __shared__ WarpBwdSmem<R> sm[kBwdWarps];
  if (gate && *gate) return;
  const int warp = threadIdx.x >> 5;
  const int unit = blockIdx.x * kBwdWarps + warp;
  if (unit >= n_units) return;
  const int tile = unit / Q, region = unit - tile * Q;
  bwd_region<R>(proj, vals, emit, ranges[2 * tile], ranges[2 * tile + 1],
                         (tile % tiles_x) * cfg.tile_w, (tile / tiles_x) * cfg.tile_h, region, Q,
                         cam, cfg, T_final, n_last, g_rgb, g_depth, g_normal, g_opac, partials,
                         sm[warp]);
}

// Fused tracking iteration on one tile: the depth sort of the tile's
// segment, forward compositing, the tracking loss and its image gradient per
// pixel (in registers), and the pose-only backward replay -- the images never
// leave the chip.  Writes the tile's loss partial (already divided by
// |Omega|) and pose 6-vector partial.  A segment of at most kSegSmem keys is
// sorted in shared memory and its ids stay there; a longer one is sorted in
// chunks merged in global memory and its ids written to vals, which this
// block then reads back (coherent loads: vals is written in this launch).
template <int P, int kG = 1>
__global__ void __launch_bounds__(kTileThreads, tile_blocks_per_sm<P, kG>()) track_tile_kernel(
    const float4* __restrict__ proj, uint32_t* vals,
    const int32_t* __restrict__ ranges, gs2d_camera cam, gs2d_config cfg, int tiles_x,
    const float* __restrict__ obs_rgb, const float* __restrict__ obs_depth, gs2d_track_params prm,
    float* __restrict__ loss_part, float* __restrict__ pose_part, TrackStep ts,
    int32_t* __restrict__ status) {
  __shared__ BwdSmem sm;
  __shared__ HitLists hl;
  __shared__ float s_pose[kTileThreads / 32][6];
  __shared__ float s_loss[kTileThreads / 32];
  __shared__ bool s_last;
  __shared__ uint32_t s_ids[kSegSmem];
  {
    const int32_t g = *status;
    if (g != 0) {
      if (g == kConverged && blockIdx.x == 0 && threadIdx.x == 0)
        record_converged(ts.pose, ts.loss_hist, ts.pose_hist, ts.grad_hist, ts.iter);
      return;
    }
  }
  // longest lists first: the blocks of the heaviest tiles start in the first
  // wave instead of trailing the grid (partials stay indexed by tile)
  const int tile = ts.order ? ts.order[blockIdx.x] : (int)blockIdx.x;
  const TilePix<P> tp = tile_pixel<P>(tile, tiles_x, cfg.tile_w, cfg.tile_h);
  bool inside[P];
#pragma unroll
  for (int k = 0; k < P; ++k) inside[k] = tp.px < cam.width && tp.py + 4 * k < cam.height;
  const int tile_x0 = (tile % tiles_x) * cfg.tile_w, tile_y0 = (tile / tiles_x) * cfg.tile_h;
  const float xt = (float)tile_x0 + 0.5f - cam.cx;
  const float yt = (float)tile_y0 + 0.5f - cam.cy;
  const float rx = (tp.px + 0.5f - cam.cx) / cam.fx, ry = (tp.py + 0.5f - cam.cy) / cam.fy;
  const int start = ranges[2 * tile], end = ranges[2 * tile + 1];
  // the segment's depth order, keys (depth bits << 32 | id) sorted in the
  // record staging area before any record is staged
  const uint32_t* ids;
  {
    const int len = end - start;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(&sm.rec[0][0]);
    static_assert(sizeof(sm.rec) >= kSegSmem * sizeof(unsigned long long), "sort area");
    if (len <= kTileThreads) {
      // one key per thread: its rank among the segment's (distinct) keys is
      // its position -- two barriers instead of a bitonic network's stages
      unsigned long long ki = 0ull;
      if ((int)threadIdx.x < len) ki = keys[threadIdx.x] = ts.seg_keys[start + threadIdx.x];
      __syncthreads();
      if ((int)threadIdx.x < len) {
        int rank = 0, j = 0;
        for (; j + 1 < len; j += 2) {
          const ulonglong2 kk = *reinterpret_cast<const ulonglong2*>(keys + j);
          rank += (int)(kk.x < ki) + (int)(kk.y < ki);
        }
        if (j < len) rank += (int)(keys[j] < ki);
        s_ids[rank] = min((uint32_t)(ki & 0xFFFFFFFFull), (uint32_t)(ts.n - 1));
      }
      __syncthreads();
      ids = s_ids;
    } else if (len <= kSegSmem) {
      for (int i = threadIdx.x; i < len; i += kTileThreads) keys[i] = ts.seg_keys[start + i];
      __syncthreads();
      bitonic_sort(keys, len);
      for (int i = threadIdx.x; i < len; i += kTileThreads)
        s_ids[i] = min((uint32_t)(keys[i] & 0xFFFFFFFFull), (uint32_t)(ts.n - 1));
      __syncthreads();
      ids = s_ids;
    } else {
      sort_long_segment<kSegSmem>(tile, proj, ts.n, tiles_x, ranges, ts.seg_keys, ts.seg_tmp,
                                  nullptr, vals, nullptr, nullptr, (long long)end, keys);
      __syncthreads();
      ids = vals + start;
    }
  }
  FwdState st[P];
  fwd_tile<kBwdVec4, false, P, kG>(proj, ids, start, end, xt, yt, tile_x0, tile_y0, tp, inside,
                                   cam, cfg, sm.rec, hl, nullptr, st);
  float pr[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const float inv = 1.f / (float)(cam.width * cam.height);
  PixGrad pg[P];
  float loss = 0.f;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    PixLoss L;
    L.loss = 0.f;
    L.g_rgb[0] = L.g_rgb[1] = L.g_rgb[2] = 0.f;
    L.g_depth = L.g_opac = 0.f;
    if (inside[k]) {
      const size_t p = (size_t)(tp.py + 4 * k) * cam.width + tp.px;
      L = tracking_pixel_loss(st[k].C, st[k].D, st[k].N, 1.f - st[k].T,
                              f3(obs_rgb[3 * p], obs_rgb[3 * p + 1], obs_rgb[3 * p + 2]),
                              obs_depth[p], rx, ry + (4.f * k) / cam.fy, inv, prm);
    }
    loss += L.loss * inv;
    pg[k].Tf = st[k].T;
    pg[k].nl = st[k].last;
    pg[k].gC = f3(L.g_rgb[0], L.g_rgb[1], L.g_rgb[2]);
    pg[k].gN = f3(0.f, 0.f, 0.f);
    pg[k].gD = L.g_depth;
    pg[k].gO = L.g_opac;
  }
  {
    float v = loss;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < kTileThreads / 32; ++w) t += s_loss[w];
      loss_part[tile] = t;
    }
  }
  // a list of at most one batch is still staged with its hit lists
  bwd_tile_pose<false, P, kG>(proj, ids, start, end, xt, yt, tile_x0, tile_y0, tp, inside, rx, ry,
                              cam, cfg, pg, sm, hl, pr, end - start <= kTileThreads);
  block_sum6(pr, s_pose, pose_part + (size_t)tile * 6);
  // the last block to finish reduces every tile's partials and updates the pose
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ts.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  float(*s_red)[256] = reinterpret_cast<float(*)[256]>(&sm.rec[0][0]);  // 7 x 256 floats fit
  reduce_and_step(pose_part, loss_part, gridDim.x, ts.pose, ts.adam, prm, ts.loss_hist,
                  ts.pose_hist, ts.grad_hist, ts.iter, status, s_red);
  if (threadIdx.x == 0) *ts.counter = 0u;
  // the next iteration's binning starts from zeroed counters (its kernels
  // run after this one; this iteration's binning finished before it)
  if (ts.sort_zero)
    for (size_t i = threadIdx.x; i < ts.sort_zero_words; i += blockDim.x) ts.sort_zero[i] = 0u;
}

// Per-surfel reduction of the (tile, region, surfel) partials in emission
// order (Q region slots per tile) and the chain rule to world-space
// parameters; pose term per block.
// Record i is surfel active[i] (or i); with accumulate the gradients are
// added to the outputs (several views, one after another).
__global__ void __launch_bounds__(256) surfel_grad_kernel(
    const float* __restrict__ mu, const float* __restrict__ quat, const float* __restrict__ scale,
    int n, const int32_t* __restrict__ active, int accumulate, const float* __restrict__ pose,
    const int32_t* __restrict__ tiles, const uint32_t* __restrict__ surfel_off,
    int Q, const float* __restrict__ proj, const float* __restrict__ partials,
    float* __restrict__ d_mu,
    float* __restrict__ d_quat, float* __restrict__ d_scale, float* __restrict__ d_opac,
    float* __restrict__ d_rgb, float* __restrict__ pose_part, int n_all,
    const int32_t* __restrict__ gate) {
  __shared__ float sp[12];
  __shared__ float s_pose[8][6];
  if (gate && *gate) return;
  if (threadIdx.x < 12) sp[threadIdx.x] = pose[threadIdx.x];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float pr[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (i < n) {
    float S[kRedVals];
#pragma unroll
    for (int c = 0; c < kRedVals; ++c) S[c] = 0.f;
    const int k = tiles[i] * Q;
    if (k > 0) {
      const float4* p = reinterpret_cast<const float4*>(partials) + (size_t)surfel_off[i] * Q * 4;
      for (int e = 0; e < k; ++e) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float4 t = p[(size_t)e * 4 + c];
          S[4 * c] += t.x;
          S[4 * c + 1] += t.y;
          S[4 * c + 2] += t.z;
          S[4 * c + 3] += t.w;
        }
      }
    }
    const float* R = sp;
    const int sid = active ? min(max(active[i], 0), n_all - 1) : i;
    const float4 q4 = reinterpret_cast<const float4*>(quat)[sid];
    const float qn2 = fmaf(q4.x, q4.x, fmaf(q4.y, q4.y, fmaf(q4.z, q4.z, q4.w * q4.w)));
    const float qinv = rsqrtf(qn2);
    const float w = q4.x * qinv, x = q4.y * qinv, y = q4.z * qinv, z = q4.w * qinv;
    const F3 tu = f3(1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y));
    const F3 tv = f3(2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x));
    const F3 tn = f3(2.f * (x * z + w * y), 2.f * (y * z - w * x), 1.f - 2.f * (x * x + y * y));
    const F3 mu_c = mat_mul(R, f3(mu[3 * sid], mu[3 * sid + 1], mu[3 * sid + 2])) + f3(sp[9], sp[10], sp[11]);
    const F3 tuc = mat_mul(R, tu), tvc = mat_mul(R, tv), tnc = mat_mul(R, tn);
    const float su = scale[2 * sid], sv = scale[2 * sid + 1];
    // sum Gv, sum u Gv, sum v Gv from the moment sums and the record's
    // n, d_u, d_v and opacity (a surfel in no tile has all sums zero)
    F3 g_muc = f3(0.f, 0.f, 0.f), g_mu = g_muc, g_mv = g_muc;
    if (k > 0) {
      const float* rec = proj + (size_t)i * kProjFloats;
      const F3 nrm = f3(rec[kNrm], rec[kNrm + 1], rec[kNrm + 2]);
      const F3 du = f3(rec[kDu], rec[kDu + 1], rec[kDu + 2]);
      const F3 dv = f3(rec[kDv], rec[kDv + 1], rec[kDv + 2]);
      const float op = rec[kAlpha];
      g_muc = S[0] * nrm + op * (S[4] * du + S[5] * dv);
      g_mu = S[1] * nrm + op * (S[6] * du + S[7] * dv);
      g_mv = S[2] * nrm + op * (S[7] * du + S[8] * dv);
    }
    const F3 g_tnc = f3(S[12], S[13], S[14]);
    const F3 g_tuc = su * g_mu, g_tvc = sv * g_mv;
    // o(p, v): write, or add when accumulating over views
    auto o = [&](float* p, float v) { *p = accumulate ? *p + v : v; };
    o(d_scale + 2 * sid, dot3(tuc, g_mu));
    o(d_scale + 2 * sid + 1, dot3(tvc, g_mv));
    o(d_opac + sid, S[3]);
    o(d_rgb + 3 * sid, S[9]);
    o(d_rgb + 3 * sid + 1, S[10]);
    o(d_rgb + 3 * sid + 2, S[11]);
    const F3 th = cross3(mu_c, g_muc) + cross3(tuc, g_tuc) + cross3(tvc, g_tvc) + cross3(tnc, g_tnc);
    pr[0] = g_muc.x; pr[1] = g_muc.y; pr[2] = g_muc.z;
    pr[3] = th.x; pr[4] = th.y; pr[5] = th.z;
    const F3 gmw = mat_tmul(R, g_muc);
    o(d_mu + 3 * sid, gmw.x);
    o(d_mu + 3 * sid + 1, gmw.y);
    o(d_mu + 3 * sid + 2, gmw.z);
    // world-space column gradients G[:,0..2] = R^T g_t{u,v,n}c
    const F3 G0 = mat_tmul(R, g_tuc), G1 = mat_tmul(R, g_tvc), G2 = mat_tmul(R, g_tnc);
    // d/dq of the rotation matrix of a unit quaternion, contracted with G
    // (G_rc = gradient of entry (r, c); column c of R is t_u, t_v, t_n)
    const float G00 = G0.x, G10 = G0.y, G20 = G0.z;
    const float G01 = G1.x, G11 = G1.y, G21 = G1.z;
    const float G02 = G2.x, G12 = G2.y, G22 = G2.z;
    const float gw = 2.f * (z * (G10 - G01) + y * (G02 - G20) + x * (G21 - G12));
    const float gx = 2.f * (y * (G10 + G01) + z * (G02 + G20) + w * (G21 - G12)) - 4.f * x * (G11 + G22);
    const float gy = 2.f * (x * (G10 + G01) + z * (G12 + G21) + w * (G02 - G20)) - 4.f * y * (G00 + G22);
    const float gz = 2.f * (x * (G02 + G20) + y * (G12 + G21) + w * (G10 - G01)) - 4.f * z * (G00 + G11);
    // unit quaternion -> raw quaternion: (I - q q^T) / |q|
    const float qd = w * gw + x * gx + y * gy + z * gz;
    o(d_quat + 4 * sid, (gw - w * qd) * qinv);
    o(d_quat + 4 * sid + 1, (gx - x * qd) * qinv);
    o(d_quat + 4 * sid + 2, (gy - y * qd) * qinv);
    o(d_quat + 4 * sid + 3, (gz - z * qd) * qinv);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float v = pr[c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) s_pose[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    float v = 0.f;
    for (int ww = 0; ww < 8; ++ww) v += s_pose[ww][threadIdx.x];
    pose_part[(size_t)blockIdx.x * 6 + threadIdx.x] = v;
  }
}

// Fixed-order sum of per-block 6-vector partials.
__global__ void __launch_bounds__(256) pose_reduce_kernel(const float* __restrict__ part, int n_part,
                                                          float* __restrict__ out,
                                                          const int32_t* __restrict__ gate) {
  __shared__ float s[6][256];
  if (gate && *gate) return;
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int b = threadIdx.x; b < n_part; b += 256)
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += part[(size_t)b * 6 + c];
#pragma unroll
  for (int c = 0; c < 6; ++c) s[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int c = 0; c < 6; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 6) out[threadIdx.x] = s[threadIdx.x][0];
}

struct BwdWs {
  float* partials;
  float* pose_part;
  size_t bytes;
};
BwdWs carve_bwd_ws(void* base, int n, size_t cap, int n_tiles, bool full, int Q) {
  Carver c(base);
  BwdWs w;
  w.partials = c.take<float>(full ? (cap > 0 ? cap : 1) * Q * kRedVals : 1);
  const int nb = max(n_tiles, (n + 255) / 256);
  w.pose_part = c.take<float>((size_t)max(nb, 1) * 6);
  w.bytes = align_up(c.off, 256);
  return w;
}

int validate_tile_cfg(const gs2d_camera* cam, const gs2d_config* cfg) {
  if (!cam || !cfg) return GS2D_ERR_INVALID_ARG;
  // P pixels per thread; warps cover 8 x 4P pixel blocks of the tile
  if (!tile_cfg_ok(*cfg)) return GS2D_ERR_INVALID_ARG;
  if (cam->width <= 0 || cam->height <= 0) return GS2D_ERR_INVALID_ARG;
  const long long nt = (long long)gs2d_tiles_x(cam, cfg) * gs2d_tiles_y(cam, cfg);
  if (nt > 65535) return GS2D_ERR_INVALID_ARG;
  return GS2D_OK;
}

// Tile grids of at most this many tiles run the grouped one-pixel loops
// (-1: twice the device's SM count, i.e. at most two blocks per SM).
static int g_grouped_max_tiles = -1;

// Whether a one-pixel tile kernel over n_tiles tiles takes the grouped loops.
static bool use_grouped(int px_per_thread, int n_tiles) {
  if (px_per_thread != 1) return false;
  int limit = g_grouped_max_tiles;
  if (limit < 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return false;
    limit = 2 * sms;
  }
  return n_tiles <= limit;
}

int render_fwd_launch(const float* proj, const gs2d_bins* bins, const gs2d_camera* cam,
                      const gs2d_config* cfg, float* rgb, float* depth, float* normal,
                      float* opacity, float* t_final, uint32_t* n_last, const int32_t* gate,
                      cudaStream_t st) {
  const int v = validate_tile_cfg(cam, cfg);
  if (v) return v;
  if (!proj || !bins || !bins->vals || !bins->tile_ranges || !rgb || !depth || !normal ||
      !opacity || !t_final || !n_last)
    return GS2D_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(proj) & 15) return GS2D_ERR_INVALID_ARG;
  const int tx = gs2d_tiles_x(cam, cfg), ty = gs2d_tiles_y(cam, cfg);
  if (use_grouped(cfg->px_per_thread, tx * ty))
    render_fwd_kernel<false, 1, kGroup><<<tx * ty, kTileThreads, 0, st>>>(
        reinterpret_cast<const float4*>(proj), bins->vals, bins->tile_ranges, *cam, *cfg, tx, rgb,
        depth, normal, opacity, t_final, n_last, nullptr, gate);
  else
    GS2D_DISPATCH_P(cfg->px_per_thread, render_fwd_kernel<false, P><<<tx * ty, kTileThreads, 0, st>>>(
        reinterpret_cast<const float4*>(proj), bins->vals, bins->tile_ranges, *cam, *cfg, tx, rgb,
        depth, normal, opacity, t_final, n_last, nullptr, gate));
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int track_tile_launch(const float* proj, const gs2d_bins* bins, const gs2d_camera* cam,
                      const gs2d_config* cfg, const float* obs_rgb, const float* obs_depth,
                      const gs2d_track_params* prm, float* loss_part, float* pose_part,
                      const TrackStep& ts, int32_t* status, cudaStream_t st) {
  const int v = validate_tile_cfg(cam, cfg);
  if (v) return v;
  if (!proj || !bins || !bins->vals || !bins->tile_ranges || !obs_rgb || !obs_depth || !prm ||
      !loss_part || !pose_part || !ts.pose || !ts.adam || !ts.counter || !status)
    return GS2D_ERR_INVALID_ARG;
  const int tx = gs2d_tiles_x(cam, cfg), ty = gs2d_tiles_y(cam, cfg);
  if (use_grouped(cfg->px_per_thread, tx * ty))
    track_tile_kernel<1, kGroup><<<tx * ty, kTileThreads, 0, st>>>(
        reinterpret_cast<const float4*>(proj), bins->vals, bins->tile_ranges, *cam, *cfg, tx,
        obs_rgb, obs_depth, *prm, loss_part, pose_part, ts, status);
  else
    GS2D_DISPATCH_P(cfg->px_per_thread, track_tile_kernel<P><<<tx * ty, kTileThreads, 0, st>>>(
        reinterpret_cast<const float4*>(proj), bins->vals, bins->tile_ranges, *cam, *cfg, tx,
        obs_rgb, obs_depth, *prm, loss_part, pose_part, ts, status));
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int surfel_grad_launch(const gs2d_surfels* s, const int32_t* active, int m, int accumulate,
                       const float* pose, const int32_t* tiles, const uint32_t* surfel_off, int Q,
                       const float* proj, const float* partials, float* d_mu, float* d_quat,
                       float* d_scale, float* d_opac, float* d_rgb, float* pose_part,
                       const int32_t* gate, cudaStream_t st) {
  if (m <= 0) return GS2D_OK;
  surfel_grad_kernel<<<(m + 255) / 256, 256, 0, st>>>(s->mu, s->quat, s->scale, m, active,
                                                      accumulate, pose, tiles, surfel_off, Q, proj,
                                                      partials,
                                                      d_mu, d_quat, d_scale, d_opac, d_rgb,
                                                      pose_part, s->n, gate);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int pose_reduce_launch(const float* part, int n_part, float* out, const int32_t* gate,
                       cudaStream_t st) {
  pose_reduce_kernel<<<1, 256, 0, st>>>(part, n_part, out, gate);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

size_t render_bwd_ws_bytes(int n, size_t cap, int n_tiles, bool full, int Q) {
  return carve_bwd_ws(nullptr, n, cap, n_tiles, full, Q).bytes;
}

int render_bwd_launch(const float* proj, const gs2d_bins* bins, const int32_t* tiles_per_surfel,
                      const gs2d_surfels* s, const float* pose, const gs2d_camera* cam,
                      const gs2d_config* cfg, const float* t_final, const uint32_t* n_last,
                      const float* d_rgb, const float* d_depth, const float* d_normal,
                      const float* d_opacity, float* d_mu, float* d_quat, float* d_scale,
                      float* d_opac, float* d_rgb_out, float* d_pose6, void* workspace,
                      size_t ws_bytes, size_t* ws_needed, const int32_t* gate, cudaStream_t st) {
  const int v = validate_tile_cfg(cam, cfg);
  if (v) return v;
  if (!proj || !bins || !bins->vals || !bins->tile_ranges || !t_final || !n_last || !d_rgb ||
      !d_depth || !s)
    return GS2D_ERR_INVALID_ARG;
  const bool any = d_mu || d_quat || d_scale || d_opac || d_rgb_out;
  const bool full = any;
  if (full && !(d_mu && d_quat && d_scale && d_opac && d_rgb_out)) return GS2D_ERR_INVALID_ARG;
  if (full && (!bins->isect_emit || !bins->surfel_off || !tiles_per_surfel || !s->mu ||
               !s->quat || !s->scale || !pose))
    return GS2D_ERR_INVALID_ARG;
  if (!full && !d_pose6) return GS2D_ERR_INVALID_ARG;
  const int tx = gs2d_tiles_x(cam, cfg), ty = gs2d_tiles_y(cam, cfg);
  const int n_tiles = tx * ty;
  // partials sized for the largest tile shape, so the size follows from
  // (n, capacity, n_tiles) alone
  const size_t need = render_bwd_ws_bytes(s->n, bins->capacity, n_tiles, full, kBwdMaxRegions);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  const BwdWs w = carve_bwd_ws(workspace, s->n, bins->capacity, n_tiles, full, kBwdMaxRegions);
  const float4* p4 = reinterpret_cast<const float4*>(proj);
  if (full) {
    // a view of few tiles (fewer than two per SM) replays half tiles
    const bool small = n_tiles < 2 * 152;
    const int Q = bwd_regions(*cfg, small ? kBwdRegionSmall : kBwdRegion);
    const int units = n_tiles * Q;
    const int blocks = (units + kBwdWarps - 1) / kBwdWarps;
    if (small)
      render_bwd_warp_kernel<kBwdRegionSmall><<<blocks, kBwdWarps * 32, 0, st>>>(
          p4, bins->vals, bins->isect_emit, bins->tile_ranges, *cam, *cfg, tx, Q, units, t_final,
          n_last, d_rgb, d_depth, d_normal, d_opacity, w.partials, gate);
    else
      render_bwd_warp_kernel<kBwdRegion><<<blocks, kBwdWarps * 32, 0, st>>>(
          p4, bins->vals, bins->isect_emit, bins->tile_ranges, *cam, *cfg, tx, Q, units, t_final,
          n_last, d_rgb, d_depth, d_normal, d_opacity, w.partials, gate);
    GS2D_LAUNCH_CHECK();
    if (s->n > 0) {
      const int nb = (s->n + 255) / 256;
      surfel_grad_kernel<<<nb, 256, 0, st>>>(s->mu, s->quat, s->scale, s->n, nullptr, 0, pose,
                                             tiles_per_surfel, bins->surfel_off, Q, proj,
                                             w.partials, d_mu,
                                             d_quat, d_scale, d_opac, d_rgb_out, w.pose_part, s->n,
                                             gate);
      GS2D_LAUNCH_CHECK();
      if (d_pose6) {
        pose_reduce_kernel<<<1, 256, 0, st>>>(w.pose_part, nb, d_pose6, gate);
        GS2D_LAUNCH_CHECK();
      }
    } else if (d_pose6) {
      GS2D_CUDA_TRY(cudaMemsetAsync(d_pose6, 0, 6 * sizeof(float), st));
    }
  } else {
    GS2D_DISPATCH_P(cfg->px_per_thread, render_bwd_kernel<P><<<n_tiles, kTileThreads, 0, st>>>(
        p4, bins->vals, bins->tile_ranges, *cam, *cfg, tx, t_final, n_last, d_rgb, d_depth,
        d_normal, d_opacity, w.pose_part, gate));
    GS2D_LAUNCH_CHECK();
    pose_reduce_kernel<<<1, 256, 0, st>>>(w.pose_part, n_tiles, d_pose6, gate);
    GS2D_LAUNCH_CHECK();
  }
  return GS2D_OK;
}

}  // namespace gs2d

using namespace gs2d;

extern "C" {

int gs2d_render_fwd(const float* proj, const gs2d_bins* bins, const gs2d_camera* cam,
                    const gs2d_config* cfg, float* rgb, float* depth, float* normal,
                    float* opacity, float* t_final, uint32_t* n_last, gs2d_stream stream) {
  if (!bins) return GS2D_ERR_INVALID_ARG;
  return render_fwd_launch(proj, bins, cam, cfg, rgb, depth, normal, opacity, t_final, n_last,
                           bins->status, (cudaStream_t)stream);
}

int gs2d_render_count(const float* proj, const gs2d_bins* bins, const gs2d_camera* cam,
                      const gs2d_config* cfg, unsigned long long* counts, gs2d_stream stream) {
  const int v = validate_tile_cfg(cam, cfg);
  if (v) return v;
  if (!proj || !bins || !bins->vals || !bins->tile_ranges || !counts) return GS2D_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  GS2D_CUDA_TRY(cudaMemsetAsync(counts, 0, 5 * sizeof(unsigned long long), st));
  const int tx = gs2d_tiles_x(cam, cfg), ty = gs2d_tiles_y(cam, cfg);
  GS2D_DISPATCH_P(cfg->px_per_thread, render_fwd_kernel<true, P><<<tx * ty, kTileThreads, 0, st>>>(
      reinterpret_cast<const float4*>(proj), bins->vals, bins->tile_ranges, *cam, *cfg, tx, nullptr,
      nullptr, nullptr, nullptr, nullptr, nullptr, counts, bins->status));
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

void gs2d_set_grouped_tiles(int max_tiles) { g_grouped_max_tiles = max_tiles < -1 ? -1 : max_tiles; }

size_t gs2d_render_bwd_workspace(int n, size_t capacity, int n_tiles) {
  return render_bwd_ws_bytes(n, capacity, n_tiles, true, kBwdMaxRegions);
}

int gs2d_render_bwd(const float* proj, const gs2d_bins* bins, const int32_t* tiles_per_surfel,
                    const gs2d_surfels* s, const float* pose, const gs2d_camera* cam,
                    const gs2d_config* cfg, const float* t_final, const uint32_t* n_last,
                    const float* d_rgb, const float* d_depth, const float* d_normal,
                    const float* d_opacity, float* d_mu, float* d_quat, float* d_scale,
                    float* d_opac, float* d_rgb_out, float* d_pose6, void* workspace,
                    size_t ws_bytes, size_t* ws_needed, gs2d_stream stream) {
  if (!bins) return GS2D_ERR_INVALID_ARG;
  return render_bwd_launch(proj, bins, tiles_per_surfel, s, pose, cam, cfg, t_final, n_last, d_rgb,
                           d_depth, d_normal, d_opacity, d_mu, d_quat, d_scale, d_opac, d_rgb_out,
                           d_pose6, workspace, ws_bytes, ws_needed, bins->status,
                           (cudaStream_t)stream);
}

}  // extern "C"
