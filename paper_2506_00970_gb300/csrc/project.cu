// gs2d_project: per-surfel camera-space splat, homography set-up and tile
// footprint (Sec. III-A, Eq. Puv, hc, homo, wth).
//
// For surfel g with camera-space columns m_u = s_u t_uc, m_v = s_v t_vc and
// centre mu_c (Eq. hc), the image of (u, v, 1) is (x'z, y'z, z) = A (u, v, 1)
// with A = diag(fx, fy, 1) [m_u m_v mu_c] and rows a1, a2, a3 (Eq. homo), in
// image coordinates relative to the principal point, x' = x - cx.  A pixel
// ray (x', y') fixes the planes h_x = a1 - x' a3 and h_y = a2 - y' a3 through
// the camera centre, and (u, v, 1) ~ h_x x h_y.  Expanding the cross product
// the x'y' term vanishes (a3 x a3 = 0), so the intersection is *linear* in
// the pixel coordinates: with c1 = a2 x a3, c2 = a3 x a1,
//     p(x', y') = (x' - x0) c1 + (y' - y0) c2 + (0, 0, det(A) / mu_c.z),
//     u = p0 / p2,  v = p1 / p2,  z = a3 . (u, v, 1) = det(A) / p2,
// where (x0, y0) = (a1.z, a2.z) / a3.z is the projected centre (u = v = 0
// there, and z = mu_c.z).  Writing p about the projected centre instead of
// the image origin avoids the cancellation of a large constant term in FP32.
// The compositing kernels re-base p on their tile's first pixel once per
// staged surfel and then evaluate it with six FMAs per (pixel, surfel) pair,
// without inverting the homography (Sec. III-A).
//
// Footprint: pixels can only pass the cutoff and alpha tests inside the disc
// u^2 + v^2 <= rho^2, rho^2 = 1.01 min(cutoff_r2, 2 ln(alpha / alpha_min)),
// and only where the hit depth exceeds the near plane.  The bounding box of
// the image of that clipped disc is exact (footprint_bounds), so a surfel
// that reaches past the camera plane -- a wall beside the camera -- covers
// only the pixels it can actually reach instead of the whole image.
#include <math.h>

#include "gs2d_common.cuh"
#include "tile_scan.cuh"
#include "tile_walk.cuh"
#include "gs2d_internal.h"

namespace gs2d {

// Image-plane bounding box (principal-point relative) of the disc
// u^2 + v^2 <= rho^2 of the splat with homography rows a1, a2, a3, clipped to
// camera depth z >= zmin.  x' = (a1 . U) / (a3 . U), U = (u, v, 1), is
// linear-fractional, so over the convex clipped disc its extremes lie on the
// boundary: at a point of the circle where x' is stationary, i.e.
// (a1 x a3) . (U' x U) = 0 <=> w_x cos t + w_y sin t = rho w_z with
// w = a1 x a3, if that point has z >= zmin; or at an end of the chord where
// the circle meets z = zmin (along the chord z is constant and x' linear).
// Same for y' with a2.  Returns false if no part of the disc has z >= zmin.
// Unit vectors (c, s) with (wx, wy) . (c, s) = t |(wx, wy)|; t is clamped to
// [-1, 1] (the points stay on the circle, so an extra candidate can only
// widen the box).  ok: R > 0 and, if exact, |t| <= 1.
__device__ __forceinline__ void circle_line(float wx, float wy, float t, bool exact, float& c0,
                                            float& s0, float& c1, float& s1, bool& ok) {
  const float R = sqrtf(fmaf(wx, wx, wy * wy));
  ok = R > 0.f && (!exact || fabsf(t) <= 1.f);
  if (!(R > 0.f)) {
    c0 = s0 = c1 = s1 = 0.f;
    return;
  }
  const float hx = wx / R, hy = wy / R;
  const float tc = fminf(fmaxf(t, -1.f), 1.f);
  const float q = sqrtf(fmaxf(1.f - tc * tc, 0.f));
  c0 = tc * hx - q * hy;
  s0 = tc * hy + q * hx;
  c1 = tc * hx + q * hy;
  s1 = tc * hy - q * hx;
}

__device__ bool footprint_bounds(F3 a1, F3 a2, F3 a3, float rho, float zmin, float& x0, float& x1,
                                 float& y0, float& y1) {
  float cu[6], sv[6];
  bool ok[6];
  const F3 wx = cross3(a1, a3), wy = cross3(a2, a3);
  const float Rx = sqrtf(fmaf(wx.x, wx.x, wx.y * wx.y));
  const float Ry = sqrtf(fmaf(wy.x, wy.x, wy.y * wy.y));
  // stationary points of x' and y' on the circle (tangents of the image);
  // where none exists the disc reaches past the camera plane and the extreme
  // lies on the chord below
  circle_line(wx.x, wx.y, Rx > 0.f ? rho * wx.z / Rx : 0.f, false, cu[0], sv[0], cu[1], sv[1], ok[0]);
  ok[1] = ok[0];
  circle_line(wy.x, wy.y, Ry > 0.f ? rho * wy.z / Ry : 0.f, false, cu[2], sv[2], cu[3], sv[3], ok[2]);
  ok[3] = ok[2];
  const float R3 = sqrtf(fmaf(a3.x, a3.x, a3.y * a3.y));
  circle_line(a3.x, a3.y, R3 > 0.f ? (zmin - a3.z) / (rho * R3) : 2.f, true, cu[4], sv[4], cu[5],
              sv[5], ok[4]);
  ok[5] = ok[4];
  // a stationary direction that degenerates (R == 0) leaves the extent open
  const bool open_x = !(Rx > 0.f), open_y = !(Ry > 0.f);
  x0 = y0 = 3.0e38f;
  x1 = y1 = -3.0e38f;
  bool any = false;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    if (!ok[k]) continue;
    const float u = rho * cu[k], v = rho * sv[k];
    const float z = fmaf(a3.x, u, fmaf(a3.y, v, a3.z));
    if (!(z >= zmin * (1.f - 1e-5f))) continue;
    const float zi = 1.f / z;
    const float x = fmaf(a1.x, u, fmaf(a1.y, v, a1.z)) * zi;
    const float y = fmaf(a2.x, u, fmaf(a2.y, v, a2.z)) * zi;
    x0 = fminf(x0, x);
    x1 = fmaxf(x1, x);
    y0 = fminf(y0, y);
    y1 = fmaxf(y1, y);
    any = true;
  }
  if (!any) return false;
  if (open_x) {
    x0 = -3.0e38f;
    x1 = 3.0e38f;
  }
  if (open_y) {
    y0 = -3.0e38f;
    y1 = 3.0e38f;
  }
  return true;
}

__device__ __forceinline__ void project_one(int i, const float* __restrict__ mu,
                                            const float* __restrict__ quat,
                                            const float* __restrict__ scale,
                                            const float* __restrict__ opacity,
                                            const float* __restrict__ rgb, const float* sp,
                                            const gs2d_camera& cam, const gs2d_config& cfg,
                                            float4* o, int32_t* __restrict__ k_out) {
  const float* Rcw = sp;

  // quaternion -> rotation columns t_u, t_v, t_n
  float4 q = reinterpret_cast<const float4*>(quat)[i];
  const float qinv = rsqrtf(fmaf(q.x, q.x, fmaf(q.y, q.y, fmaf(q.z, q.z, q.w * q.w))));
  const float w = q.x * qinv, x = q.y * qinv, y = q.z * qinv, z = q.w * qinv;
  const F3 tu = f3(1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y));
  const F3 tv = f3(2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x));
  const F3 tn = f3(2.f * (x * z + w * y), 2.f * (y * z - w * x), 1.f - 2.f * (x * x + y * y));

  const F3 muw = f3(mu[3 * i], mu[3 * i + 1], mu[3 * i + 2]);
  const F3 mu_c = mat_mul(Rcw, muw) + f3(sp[9], sp[10], sp[11]);
  const float su = scale[2 * i], sv = scale[2 * i + 1];
  const F3 m_u = su * mat_mul(Rcw, tu);
  const F3 m_v = sv * mat_mul(Rcw, tv);
  const F3 tn_c = mat_mul(Rcw, tn);
  const float alpha = opacity[i];

  // rows of A = diag(fx, fy, 1) [m_u m_v mu_c] (principal point at the origin)
  const F3 a3 = f3(m_u.z, m_v.z, mu_c.z);
  const F3 a1 = f3(cam.fx * m_u.x, cam.fx * m_v.x, cam.fx * mu_c.x);
  const F3 a2 = f3(cam.fy * m_u.y, cam.fy * m_v.y, cam.fy * mu_c.y);
  const F3 c1 = cross3(a2, a3), c2 = cross3(a3, a1);
  const float det = dot3(a1, c1);
  const float xc = a1.z / a3.z, yc = a2.z / a3.z;
  const float p2c = det / a3.z;
  const F3 nrm = cross3(m_u, m_v);
  const float nn = dot3(nrm, nrm);
  const float inn = nn > 0.f ? 1.f / nn : 0.f;
  const F3 du = inn * cross3(m_v, nrm), dv = inn * cross3(nrm, m_u);

  // tile footprint: the disc u^2 + v^2 <= rho^2 clipped to z >= near
  int tx0 = 1, ty0 = 1, tx1 = 0, ty1 = 0;
  int pi0 = 1, pj0 = 1, pi1 = 0, pj1 = 0;
  if (mu_c.z > cam.near_z && alpha >= cfg.alpha_min) {
    const float rho2 = 1.01f * fminf(cfg.cutoff_r2, 2.f * logf(alpha / cfg.alpha_min));
    if (rho2 > 0.f) {
      float x0, x1, y0, y1;
      if (footprint_bounds(a1, a2, a3, sqrtf(rho2), 0.99f * cam.near_z, x0, x1, y0, y1)) {
        x0 += cam.cx;
        x1 += cam.cx;
        y0 += cam.cy;
        y1 += cam.cy;
        const float i0 = fmaxf(ceilf(x0 - 0.5f), 0.f);
        const float i1 = fminf(floorf(x1 - 0.5f), (float)(cam.width - 1));
        const float j0 = fmaxf(ceilf(y0 - 0.5f), 0.f);
        const float j1 = fminf(floorf(y1 - 0.5f), (float)(cam.height - 1));
        if (i0 <= i1 && j0 <= j1) {
          pi0 = (int)i0;
          pi1 = (int)i1;
          pj0 = (int)j0;
          pj1 = (int)j1;
          tx0 = (int)i0 / cfg.tile_w;
          tx1 = (int)i1 / cfg.tile_w;
          ty0 = (int)j0 / cfg.tile_h;
          ty1 = (int)j1 / cfg.tile_h;
        }
      }
    }
  }
  const int k = (tx0 <= tx1 && ty0 <= ty1) ? (tx1 - tx0 + 1) * (ty1 - ty0 + 1) : 0;
  *k_out = k;

  const float rgb0 = rgb[3 * i], rgb1 = rgb[3 * i + 1], rgb2 = rgb[3 * i + 2];
  const uint32_t r01 = (uint32_t)tx0 | ((uint32_t)ty0 << 16);
  const uint32_t r23 = (uint32_t)tx1 | ((uint32_t)ty1 << 16);
  const uint32_t b01 = (uint32_t)pi0 | ((uint32_t)pi1 << 16);
  const uint32_t b23 = (uint32_t)pj0 | ((uint32_t)pj1 << 16);
  o[0] = make_float4(xc, yc, p2c, c1.x);
  o[1] = make_float4(c1.y, c1.z, c2.x, c2.y);
  o[2] = make_float4(c2.z, det, alpha, rgb0);
  o[3] = make_float4(rgb1, rgb2, tn_c.x, tn_c.y);
  o[4] = make_float4(tn_c.z, nrm.x, nrm.y, nrm.z);
  o[5] = make_float4(du.x, du.y, du.z, dv.x);
  o[6] = make_float4(dv.y, dv.z, mu_c.z, 0.f);
  o[7] = make_float4(__uint_as_float(r01), __uint_as_float(r23), __uint_as_float(b01),
                     __uint_as_float(b23));
}

// One surfel per thread.  The same per-surfel code as the batched projection
// (project_one), so single views and batches write bit-identical records.
__global__ void __launch_bounds__(256) project_kernel(
    const float* __restrict__ mu, const float* __restrict__ quat, const float* __restrict__ scale,
    const float* __restrict__ opacity, const float* __restrict__ rgb, int n,
    const float* __restrict__ pose, gs2d_camera cam, gs2d_config cfg,
    float4* __restrict__ proj, int32_t* __restrict__ tiles_out, const int32_t* __restrict__ gate) {
  // records are assembled in shared memory (9 float4 per thread: padded so
  // both the per-thread writes and the block's coalesced copy-out are free
  // of bank conflicts) and written as one contiguous 32 KB run per block
  __shared__ float4 s_out[256 * 9];
  __shared__ float sp[12];
  if (gate && *gate) return;
  if (threadIdx.x < 12) sp[threadIdx.x] = pose[threadIdx.x];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n)
    project_one(i, mu, quat, scale, opacity, rgb, sp, cam, cfg, s_out + threadIdx.x * 9,
                tiles_out + i);
  __syncthreads();
  const int base = blockIdx.x * blockDim.x;
  const int valid = min((int)blockDim.x, n - base);
  float4* dst = proj + (size_t)base * (kProjFloats / 4);
  for (int v = threadIdx.x; v < valid * 8; v += blockDim.x) dst[v] = s_out[(v >> 3) * 9 + (v & 7)];
}

// Tile counters a fused projection keeps in shared memory (larger tile grids
// count with global atomics).
constexpr int kHistTiles = 2048;
constexpr int kGridSpins = 1 << 22;  // polls of the grid barrier before it reports a timeout

// Grid-wide barrier of a cooperative launch (every block resident): block
// arrivals counted on *bar (zeroed before the launch), thread 0 polls with a
// bounded wait; past the limit it records GS2D_ERR_TIMEOUT in *status and
// the block returns false (all later kernels skip on the status).
__device__ __forceinline__ bool grid_sync(uint32_t* bar, uint32_t blocks, int32_t* status,
                                          int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    for (int i = 0;; ++i) {
      uint32_t v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= blocks) break;
      if (i >= kGridSpins) {
        atomicExch(status, (int32_t)GS2D_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__global__ void __launch_bounds__(256) project_fused_kernel(
    const float* __restrict__ mu, const float* __restrict__ quat, const float* __restrict__ scale,
    const float* __restrict__ opacity, const float* __restrict__ rgb, int n,
    const float* __restrict__ pose, gs2d_camera cam, gs2d_config cfg, int tiles_x, int tiles_y,
    float4* __restrict__ proj, int32_t* __restrict__ tiles_out, const int32_t* __restrict__ gate,
    SortFuse fz, int32_t* __restrict__ status) {
  // records are assembled in shared memory (9 float4 per thread: padded so
  // both the per-thread writes and the block's coalesced copy-out are free
  // of bank conflicts) and written as one contiguous 32 KB run per chunk of
  // 256 surfels; the grid is resident (a block per slot) and strides over
  // the chunks, so there is no partial last wave
  __shared__ float4 s_out[256 * 9];
  __shared__ uint32_t s_hist[kHistTiles];
  __shared__ float sp[12];
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_carry;
  __shared__ bool s_last;
  __shared__ bool s_emit[256];  // does the chunk's surfel touch a tile?
  __shared__ WalkScratch s_walk[8];
  if (gate && *gate) return;
  if (threadIdx.x < 12) sp[threadIdx.x] = pose[threadIdx.x];
  const bool local = fz.n_tiles <= kHistTiles;
  if (local)
    for (int t = threadIdx.x; t < fz.n_tiles; t += blockDim.x) s_hist[t] = 0u;
  __syncthreads();
  // every block takes an equal contiguous share of the surfels (passes of
  // blockDim.x), so no block trails the others by a whole extra chunk
  const int share = (n + (int)gridDim.x - 1) / (int)gridDim.x;
  const int my0 = min(n, (int)blockIdx.x * share), my1 = min(n, my0 + share);
  for (int base = my0; base < my1; base += blockDim.x) {
    const int i = base + (int)threadIdx.x;
    s_emit[threadIdx.x] = false;
    int k = 0, tx0 = 1, ty0 = 1, tx1 = 0;
    if (i < my1) {
      project_one(i, mu, quat, scale, opacity, rgb, sp, cam, cfg, s_out + threadIdx.x * 9,
                  tiles_out + i);
      const float4 rc = s_out[threadIdx.x * 9 + 7];
      const uint32_t r01 = __float_as_uint(rc.x), r23 = __float_as_uint(rc.y);
      tx0 = (int)(r01 & 0xFFFF);
      ty0 = (int)(r01 >> 16);
      tx1 = (int)(r23 & 0xFFFF);
      const int ty1 = (int)(r23 >> 16);
      if (tx0 <= tx1 && ty0 <= ty1) {
        s_emit[threadIdx.x] = true;
        k = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
      }
    }
    // tile counts of the warp's rectangles, walked cooperatively
    warp_tile_walk(k, tx0, ty0, tx1, fz.tiles_x, fz.n_tiles, s_walk[threadIdx.x >> 5],
                   [&](int, int t) { atomicAdd(local ? s_hist + t : fz.tile_count + t, 1u); });
    __syncthreads();
    const int valid = min((int)blockDim.x, my1 - base);
    float4* dst = proj + (size_t)base * (kProjFloats / 4);
    // only the records of surfels that touch a tile are ever read (the
    // scatter and the tile kernel reach records through the tile lists), so
    // culled surfels' records are not written
    for (int v = threadIdx.x; v < valid * 8; v += blockDim.x)
      if (s_emit[v >> 3]) dst[v] = s_out[(v >> 3) * 9 + (v & 7)];
    __syncthreads();
  }
  // the block's counts, one global atomic per touched tile
  if (local)
    for (int t = threadIdx.x; t < fz.n_tiles; t += blockDim.x)
      if (s_hist[t]) atomicAdd(fz.tile_count + t, s_hist[t]);
  if (fz.seg_keys && local) {
    // fused scatter (a cooperative launch): once every block's counts are
    // in, each block scans them itself, claims its slots in the tiles it
    // touches and writes its pairs' keys (depth bits << 32 | id), exactly as
    // the binning's scatter kernel would; block 0 also writes the tile
    // ranges, K, the capacity check and the launch order
    __shared__ int s_ok;
    if (!grid_sync(fz.bar, gridDim.x, status, &s_ok)) return;
    uint32_t* s_start = reinterpret_cast<uint32_t*>(s_out);             // [kHistTiles]
    uint32_t* s_n = s_start + kHistTiles;                               // [257]
    unsigned long long* s_key = reinterpret_cast<unsigned long long*>(s_n + 264);  // [256]
    constexpr int kPer = kHistTiles / 256;
    const int per = (fz.n_tiles + 255) / 256;
    const int t0 = (int)threadIdx.x * per;
    uint32_t c[kPer];
    uint32_t sum = 0u;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      c[k] = (k < per && t0 + k < fz.n_tiles) ? __ldcg(fz.tile_count + t0 + k) : 0u;
      sum += c[k];
    }
    uint32_t K;
    uint32_t run = block_exscan256<uint32_t>(sum, s_w, &K);
#pragma unroll
    for (int k = 0; k < kPer; ++k)
      if (k < per && t0 + k < fz.n_tiles) {
        s_start[t0 + k] = run;
        run += c[k];
      }
    if (blockIdx.x == 0)
      tile_scan_order_small<kPer>(fz.tile_count, fz.n_tiles, fz.ranges, fz.n_isect, fz.capacity,
                                  fz.long_list, fz.n_long, fz.long_len, status, fz.order, s_n,
                                  s_w);
    __syncthreads();
    if ((unsigned long long)K > (unsigned long long)fz.capacity) return;  // block 0 flagged it
    for (int t = threadIdx.x; t < fz.n_tiles; t += blockDim.x) {
      const uint32_t cb = s_hist[t];
      if (cb) s_hist[t] = s_start[t] + atomicAdd(fz.cursor + t, cb);
    }
    __syncthreads();
    const unsigned long long* wkey = s_key + (threadIdx.x & ~31);
    for (int base = my0; base < my1; base += blockDim.x) {
      const int i = base + (int)threadIdx.x;
      int k = 0, tx0 = 1, ty0 = 1, tx1 = 0;
      unsigned long long key = 0ull;
      if (i < my1) {
        k = max(tiles_out[i], 0);
        if (k > 0) {
          // this block wrote the record: read it back past L1
          const float4* rec = proj + (size_t)i * (kProjFloats / 4);
          const float4 rc = __ldcg(rec + 7);
          const uint32_t r01 = __float_as_uint(rc.x), r23 = __float_as_uint(rc.y);
          tx0 = (int)(r01 & 0xFFFF);
          ty0 = (int)(r01 >> 16);
          tx1 = (int)(r23 & 0xFFFF);
          key = ((unsigned long long)__float_as_uint(__ldcg(rec + 6).z) << 32) | (uint32_t)i;
        }
      }
      s_key[threadIdx.x] = key;
      __syncwarp();
      warp_tile_walk(k, tx0, ty0, tx1, fz.tiles_x, fz.n_tiles, s_walk[threadIdx.x >> 5],
                     [&](int owner, int t) {
                       const uint32_t pos = atomicAdd(s_hist + t, 1u);
                       if ((long long)pos < fz.capacity) fz.seg_keys[pos] = wkey[owner];
                     });
      __syncwarp();
    }
    return;
  }
  // the last block to finish turns the counts into tile ranges
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(fz.done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (local) {
    tile_scan_order_small<kHistTiles / 256>(fz.tile_count, fz.n_tiles, fz.ranges, fz.n_isect,
                                            fz.capacity, fz.long_list, fz.n_long, fz.long_len,
                                            status, fz.order, s_hist, s_w);
    return;
  }
  tile_scan_block(fz.tile_count, fz.n_tiles, fz.ranges, fz.n_isect, fz.capacity, fz.long_list,
                  fz.n_long, fz.long_len, status, s_w, &s_carry);
  if (fz.order) {
    __syncthreads();
    tile_order_block(fz.tile_count, fz.n_tiles, fz.order, s_hist, s_w);
  }
}

// All views of a batch in one launch (blockIdx.y = view): record j of a view
// is surfel active[j] (or j), written to that view's record array.
struct ProjView {
  const float* pose;
  const int32_t* active;
  int m;
  float4* proj;
  int32_t* tiles;
  const int32_t* status;
  gs2d_camera cam;
  gs2d_config cfg;
};
struct ProjTable {
  ProjView v[GS2D_MAX_VIEWS];
};

__global__ void __launch_bounds__(256) project_batch_kernel(
    const float* __restrict__ mu, const float* __restrict__ quat, const float* __restrict__ scale,
    const float* __restrict__ opacity, const float* __restrict__ rgb, int n, ProjTable tab) {
  __shared__ float4 s_out[256 * 9];
  __shared__ float sp[12];
  const ProjView& pv = tab.v[blockIdx.y];
  const int base = blockIdx.x * blockDim.x;
  if (base >= pv.m || (pv.status && *pv.status)) return;
  if (threadIdx.x < 12) sp[threadIdx.x] = pv.pose[threadIdx.x];
  __syncthreads();
  const int j = base + threadIdx.x;
  if (j < pv.m) {
    const int sid = pv.active ? min(max(pv.active[j], 0), n - 1) : j;
    project_one(sid, mu, quat, scale, opacity, rgb, sp, pv.cam, pv.cfg, s_out + threadIdx.x * 9,
                pv.tiles + j);
  }
  __syncthreads();
  const int valid = min((int)blockDim.x, pv.m - base);
  float4* dst = pv.proj + (size_t)base * (kProjFloats / 4);
  for (int v = threadIdx.x; v < valid * 8; v += blockDim.x) dst[v] = s_out[(v >> 3) * 9 + (v & 7)];
}

bool project_can_fuse_scatter(int n_tiles) { return n_tiles > 0 && n_tiles <= kHistTiles; }

int project_launch(const gs2d_surfels* s, const gs2d_camera* cam, const float* pose,
                   const gs2d_config* cfg, float* proj_out, int32_t* tiles_per_surfel_out,
                   const int32_t* gate, cudaStream_t st, const SortFuse* fuse) {
  if (!s || !cam || !pose || !cfg || !proj_out || !tiles_per_surfel_out) return GS2D_ERR_INVALID_ARG;
  if (s->n < 0 || (s->n > 0 && (!s->mu || !s->quat || !s->scale || !s->opacity || !s->rgb)))
    return GS2D_ERR_INVALID_ARG;
  if (cam->width <= 0 || cam->height <= 0 || cfg->tile_w <= 0 || cfg->tile_h <= 0)
    return GS2D_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(s->quat) | reinterpret_cast<uintptr_t>(proj_out)) & 15)
    return GS2D_ERR_INVALID_ARG;
  const int tx = tiles_along(cam->width, cfg->tile_w), ty = tiles_along(cam->height, cfg->tile_h);
  if (tx > 65535 || ty > 65535) return GS2D_ERR_INVALID_ARG;
  const int threads = 256;
  const int chunks = (s->n + threads - 1) / threads;
  if (fuse) {
    // a resident grid (with no surfel one block still runs the empty scan)
    static int resident = 0;
    if (!resident) {
      int per_sm = 0, dev = 0, sms = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, project_fused_kernel, threads,
                                                        0) != cudaSuccess ||
          cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GS2D_ERR_CUDA;
      resident = max(per_sm, 1) * max(sms, 1);
    }
    const int blocks = max(min(chunks, resident), 1);
    if (fuse->seg_keys) {
      if (!project_can_fuse_scatter(fuse->n_tiles)) return GS2D_ERR_INVALID_ARG;
      // blocks wait on one another at the grid barrier: a cooperative launch
      cudaLaunchConfig_t lc = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeCooperative;
      at[0].val.cooperative = 1;
      lc.gridDim = dim3(blocks);
      lc.blockDim = dim3(threads);
      lc.dynamicSmemBytes = 0;
      lc.stream = st;
      lc.attrs = at;
      lc.numAttrs = 1;
      GS2D_CUDA_TRY(cudaLaunchKernelEx(&lc, project_fused_kernel, s->mu, s->quat, s->scale,
                                       s->opacity, s->rgb, s->n, pose, *cam, *cfg, tx, ty,
                                       reinterpret_cast<float4*>(proj_out), tiles_per_surfel_out,
                                       gate, *fuse, const_cast<int32_t*>(gate)));
    } else {
      project_fused_kernel<<<blocks, threads, 0, st>>>(
          s->mu, s->quat, s->scale, s->opacity, s->rgb, s->n, pose, *cam, *cfg, tx, ty,
          reinterpret_cast<float4*>(proj_out), tiles_per_surfel_out, gate, *fuse,
          const_cast<int32_t*>(gate));
    }
  } else {
    if (s->n == 0) return GS2D_OK;
    project_kernel<<<chunks, threads, 0, st>>>(s->mu, s->quat, s->scale, s->opacity, s->rgb, s->n,
                                               pose, *cam, *cfg,
                                               reinterpret_cast<float4*>(proj_out),
                                               tiles_per_surfel_out, gate);
  }
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

}  // namespace gs2d

using namespace gs2d;

extern "C" {

gs2d_config gs2d_default_config(void) {
  gs2d_config c;
  c.tile_w = 16;
  c.tile_h = 16;
  c.px_per_thread = 1;
  c.alpha_min = 1.0f / 255.0f;
  c.alpha_max = 0.99f;
  c.t_min = 1e-4f;
  c.cutoff_r2 = 9.0f;
  return c;
}

gs2d_track_params gs2d_default_track_params(void) {
  gs2d_track_params p;
  p.lambda_d = 1.0f;
  p.lr = 1e-3f;
  p.beta1 = 0.9f;
  p.beta2 = 0.999f;
  p.eps = 1e-8f;
  p.weight_decay = 0.0f;
  p.stop_tol = 1e-5f;
  p.opacity_thresh = 0.95f;
  p.depth_mode = 1;
  return p;
}

const char* gs2d_status_string(int s) {
  switch (s) {
    case GS2D_OK: return "ok";
    case GS2D_ERR_INVALID_ARG: return "invalid argument";
    case GS2D_ERR_WORKSPACE: return "workspace missing or too small";
    case GS2D_ERR_CAPACITY: return "intersection capacity exceeded";
    case GS2D_ERR_CUDA: return "CUDA launch error";
    case GS2D_ERR_TIMEOUT: return "device wait timed out";
    case GS2D_ERR_NONFINITE: return "non-finite value";
    default: return "unknown status";
  }
}

int gs2d_tiles_x(const gs2d_camera* cam, const gs2d_config* cfg) {
  return tiles_along(cam->width, cfg->tile_w);
}
int gs2d_tiles_y(const gs2d_camera* cam, const gs2d_config* cfg) {
  return tiles_along(cam->height, cfg->tile_h);
}

int gs2d_project(const gs2d_surfels* s, const gs2d_camera* cam, const float* pose,
                 const gs2d_config* cfg, float* proj_out, int32_t* tiles_per_surfel_out,
                 gs2d_stream stream) {
  return project_launch(s, cam, pose, cfg, proj_out, tiles_per_surfel_out, nullptr,
                        (cudaStream_t)stream);
}

int gs2d_project_batch(const gs2d_surfels* s, const gs2d_view* views, int n_views,
                       gs2d_stream stream) {
  if (!s || !views || n_views <= 0 || n_views > GS2D_MAX_VIEWS) return GS2D_ERR_INVALID_ARG;
  if (s->n <= 0 || !s->mu || !s->quat || !s->scale || !s->opacity || !s->rgb)
    return GS2D_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(s->quat) & 15) return GS2D_ERR_INVALID_ARG;
  ProjTable tab;
  int max_m = 0;
  for (int v = 0; v < n_views; ++v) {
    const gs2d_view& w = views[v];
    if (!w.pose || !w.proj || !w.tiles_per_surfel || (reinterpret_cast<uintptr_t>(w.proj) & 15))
      return GS2D_ERR_INVALID_ARG;
    if (w.cam.width <= 0 || w.cam.height <= 0 || w.cfg.tile_w <= 0 || w.cfg.tile_h <= 0)
      return GS2D_ERR_INVALID_ARG;
    const int m = w.active ? w.n_active : s->n;
    if (m < 0 || (w.active && m > s->n)) return GS2D_ERR_INVALID_ARG;
    tab.v[v] = ProjView{w.pose, w.active, m, reinterpret_cast<float4*>(w.proj), w.tiles_per_surfel,
                        w.bins.status, w.cam, w.cfg};
    max_m = max(max_m, m);
  }
  if (max_m == 0) return GS2D_OK;
  const dim3 grid((max_m + 255) / 256, n_views);
  project_batch_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(s->mu, s->quat, s->scale,
                                                               s->opacity, s->rgb, s->n, tab);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

}  // extern "C"
