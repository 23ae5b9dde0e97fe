// Full backward replay with one warp per tile region (Sec. III-B reverse
// mode of the compositing, Eqs. of the splat intersection).
//
// A tile of tile_w x tile_h pixels is cut into 8 x 4 pixel blocks (block b
// at x offset 8 (b % (tile_w / 8)), y offset 4 (b / (tile_w / 8))); a region
// is R consecutive blocks, and one warp replays one region: lane l owns pixel
// (l & 7, l >> 3) of each of the region's R blocks.  The warp walks the
// tile's list back to front, 32 staged records at a time, and for each entry
// whose footprint touches the region evaluates only the touched blocks (a
// warp-uniform branch per block), sums the entry's 16 gradient terms over
// the lane's R pixels in registers and then over the warp through shared
// memory.  Nothing is shared between warps, so there is no block
// barrier: a region's partial sums go straight to its own slot,
//   partials[(emit * Q + region) * 16 + c],   Q = regions per tile,
// the pair sums of (beta, u beta, v beta, g, u g, v g, u^2 g, u v g, v^2 g,
// w dC, w dN, 0), g the pair's opacity gradient (the splat gradient
// Gv = beta n + o g (u d_u + v d_v) is linear in them, so the per-surfel
// reduction forms sum Gv, sum u Gv, sum v Gv from the surfel's n, d_u, d_v),
// and every (entry, region) slot is written exactly once (zeros where the
// footprint misses the region, no pixel of it blends the entry, or the entry
// lies past the region's last blended entry).  The per-surfel reduction
// adds a surfel's Q slots per tile in emission order: deterministic, no
// atomics.
#pragma once

#include "tile_loops.cuh"

namespace gs2d {

// 8 x 4 blocks per region (pixels per lane): a whole 256-pixel tile per warp
// when the view has tiles enough to fill the GPU (one partial per (tile,
// surfel)), half a tile for small views (twice the work units).
constexpr int kBwdRegion = 8;
constexpr int kBwdRegionSmall = 4;
constexpr int kBwdWarps = 4;       // warps (independent work items) per block
constexpr int kBwdWarpBlocks = 4;  // resident blocks per SM the registers are sized for
// Regions per tile of a tile shape with R blocks per region, and the most
// any shape (up to 1024 pixels) and region size can have.
__host__ __device__ inline int bwd_regions(const gs2d_config& c, int R = kBwdRegion) {
  return c.tile_w * c.tile_h / (32 * R);
}
constexpr int kBwdMaxRegions = 1024 / (32 * kBwdRegionSmall);

// Per-warp shared memory: the staged records of 32 list entries and the
// region's per-pixel upstream gradients, [k][0] = (dC, dD), [k][1] = (dN,
// dO T_final) for the lane's pixel of block k (dO T_final enters the opacity
// image's term of every pair's alpha gradient).
template <int R>
struct WarpBwdSmem {
  float4 rec[32][kBwdVec4];
  float4 up[R][2][32];
  float red[32][20];  // one entry's 16 per-lane sums, rows padded to 20 floats
};

// Bit k set if the footprint (packed absolute pixel ranges) touches block k
// of the region.
template <int R>
__device__ __forceinline__ uint32_t region_mask(float bi, float bj, int tile_x0, int tile_y0,
                                                int wpr, int b0) {
  const uint32_t I = __float_as_uint(bi), J = __float_as_uint(bj);
  const int i0 = (int)(I & 0xFFFF) - tile_x0, i1 = (int)(I >> 16) - tile_x0;
  const int j0 = (int)(J & 0xFFFF) - tile_y0, j1 = (int)(J >> 16) - tile_y0;
  uint32_t m = 0u;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int b = b0 + k;
    const int ox = (b % wpr) * 8, oy = (b / wpr) * 4;
    if (!(i1 < ox || i0 > ox + 7 || j1 < oy || j0 > oy + 3)) m |= 1u << k;
  }
  return m;
}

// Replays one region.  region in [0, Q); b0 = region * R is its first block.
template <int R>
__device__ __forceinline__ void bwd_region(
    const float4* __restrict__ proj, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ emit, int start, int end, int tile_x0, int tile_y0, int region,
    int Q, const gs2d_camera& cam, const gs2d_config& cfg, const float* __restrict__ T_final,
    const uint32_t* __restrict__ n_last, const float* __restrict__ g_rgb,
    const float* __restrict__ g_depth, const float* __restrict__ g_normal,
    const float* __restrict__ g_opac, float* __restrict__ partials, WarpBwdSmem<R>& sm) {
  const int lane = threadIdx.x & 31;
  const int wpr = cfg.tile_w >> 3;
  const int b0 = region * R;
  const float xt = (float)tile_x0 + 0.5f - cam.cx, yt = (float)tile_y0 + 0.5f - cam.cy;
  const float fxfy = cam.fx * cam.fy;
  // pixel ray r = (rx, ry, 1): rx = (x + 0.5 - cx) / fx from the tile-relative
  // pixel centre lx as rx0 + lx / fx
  const float ifx = 1.f / cam.fx, ify = 1.f / cam.fy;
  const float rx0 = xt * ifx, ry0 = yt * ify;
  float T[R], acc[R], lx[R], ly[R];
  uint32_t nl[R];
  uint32_t my_nl = 0u;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int b = b0 + k;
    const int ox = (b % wpr) * 8 + (lane & 7), oy = (b / wpr) * 4 + (lane >> 3);
    const int px = tile_x0 + ox, py = tile_y0 + oy;
    lx[k] = (float)ox;
    ly[k] = (float)oy;
    T[k] = 1.f;
    acc[k] = 0.f;
    nl[k] = 0u;
    float4 u0 = make_float4(0.f, 0.f, 0.f, 0.f), u1 = u0;
    if (px < cam.width && py < cam.height) {
      const size_t p = (size_t)py * cam.width + px;
      T[k] = T_final[p];
      nl[k] = n_last[p];
      u0 = make_float4(g_rgb[3 * p], g_rgb[3 * p + 1], g_rgb[3 * p + 2], g_depth[p]);
      if (g_normal) u1 = make_float4(g_normal[3 * p], g_normal[3 * p + 1], g_normal[3 * p + 2], 0.f);
      if (g_opac) u1.w = g_opac[p] * T[k];
    }
    sm.up[k][0][lane] = u0;
    sm.up[k][1][lane] = u1;
    my_nl = max(my_nl, nl[k]);
  }
  const int hi = start + (int)__reduce_max_sync(0xffffffffu, my_nl);
  const size_t slot_base = (size_t)region;
  for (int bend = hi; bend > start; bend -= 32) {
    const int bstart = max(start, bend - 32);
    const int cnt = bend - bstart;
    __syncwarp();
    uint32_t my_emit = 0u, my_mask = 0u;
    if (lane < cnt) {
      const int idx = bstart + lane;
      stage_record_to<kBwdVec4>(proj, vals[idx], xt, yt, sm.rec[lane]);
      my_emit = emit[idx];
      const float4 r6 = sm.rec[lane][6];
      my_mask = region_mask<R>(r6.z, r6.w, tile_x0, tile_y0, wpr, b0);
      if (!my_mask) {
        float4* z = reinterpret_cast<float4*>(partials + ((size_t)my_emit * Q + slot_base) * kRedVals);
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < kRedVals / 4; ++q) z[q] = zero;
      }
    }
    __syncwarp();
    uint32_t hits = __ballot_sync(0xffffffffu, my_mask != 0u);
    while (hits) {
      const int j = 31 - __clz(hits);
      hits &= ~(1u << j);
      const uint32_t m = __shfl_sync(0xffffffffu, my_mask, j);
      const uint32_t e_j = __shfl_sync(0xffffffffu, my_emit, j);
      const int jrel = bstart + j - start;
      const float4 r0 = sm.rec[j][0], r1 = sm.rec[j][1], r2 = sm.rec[j][2];
      float val[kRedVals];
#pragma unroll
      for (int i = 0; i < kRedVals; ++i) val[i] = 0.f;
      bool contrib = false;
#pragma unroll
      for (int k = 0; k < R; ++k) {
        if (!((m >> k) & 1u)) continue;  // warp-uniform
        if (jrel >= (int)nl[k]) continue;
        Eval e;
        if (!eval_pair(r0, r1, r2, lx[k], ly[k], cam.near_z, cfg.cutoff_r2, cfg.alpha_min,
                       cfg.alpha_max, e))
          continue;
        const float4 r3 = sm.rec[j][3], r4 = sm.rec[j][4], r5 = sm.rec[j][5];
        const float4 r6 = sm.rec[j][6];
        const float4 u0 = sm.up[k][0][lane], u1 = sm.up[k][1][lane];
        const F3 col = f3(r2.w, r3.x, r3.y);
        const F3 tn = f3(r3.z, r3.w, r4.x);
        const F3 gC = f3(u0.x, u0.y, u0.z), gN = f3(u1.x, u1.y, u1.z);
        const float gD = u0.w;
        const float om = 1.f - e.a;
        const float iom = __fdividef(1.f, om);
        const float Tb = T[k] * iom;
        const float w = e.a * Tb;
        const float vj = dot3(col, gC) + e.z * gD + dot3(tn, gN);
        const float ga = Tb * vj - (acc[k] - u1.w) * iom;
        acc[k] = fmaf(w, vj, acc[k]);
        T[k] = Tb;
        // g = dL/d(opacity) of the pair; the splat gradient is
        // Gv = beta n + o g (u d_u + v d_v) with
        // beta = (w dD - o g (u d_u + v d_v) . r) / (n . r), 1 / (n . r) = fx fy rinv
        const float g = e.araw <= cfg.alpha_max ? e.G * ga : 0.f;
        const float rx = fmaf(lx[k], ifx, rx0), ry = fmaf(ly[k], ify, ry0);
        const float dur = fmaf(r5.x, rx, fmaf(r5.y, ry, r5.z));
        const float dvr = fmaf(r5.w, rx, fmaf(r6.x, ry, r6.y));
        const float Pr = fmaf(e.u, dur, e.v * dvr);
        const float beta = fmaf(-r2.z * g, Pr, w * gD) * fxfy * e.rinv;
        const float ug = e.u * g, vg = e.v * g;
        val[0] += beta;
        val[1] = fmaf(e.u, beta, val[1]);
        val[2] = fmaf(e.v, beta, val[2]);
        val[3] += g;
        val[4] += ug;
        val[5] += vg;
        val[6] = fmaf(e.u, ug, val[6]);
        val[7] = fmaf(e.u, vg, val[7]);
        val[8] = fmaf(e.v, vg, val[8]);
        val[9] = fmaf(w, gC.x, val[9]);
        val[10] = fmaf(w, gC.y, val[10]);
        val[11] = fmaf(w, gC.z, val[11]);
        val[12] = fmaf(w, gN.x, val[12]);
        val[13] = fmaf(w, gN.y, val[13]);
        val[14] = fmaf(w, gN.z, val[14]);
        contrib = true;
      }
      float* dst = partials + ((size_t)e_j * Q + slot_base) * kRedVals;
      if (__any_sync(0xffffffffu, contrib)) {
        // sum over the warp through shared memory: lane l writes its 16
        // sums as row l, then lane l adds up column l & 15 over the rows of
        // its half-warp (the upper half four rows on, so the halves read
        // disjoint banks; 80-byte rows keep the row stores conflict-free)
        float4* row = reinterpret_cast<float4*>(&sm.red[lane][0]);
#pragma unroll
        for (int q = 0; q < kRedVals / 4; ++q)
          row[q] = make_float4(val[4 * q], val[4 * q + 1], val[4 * q + 2], val[4 * q + 3]);
        __syncwarp();
        const int c = lane & 15, upper = lane >> 4;
        float part[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) part[i] = sm.red[upper ? 16 + ((i + 4) & 15) : i][c];
#pragma unroll
        for (int h = 8; h > 0; h >>= 1)
#pragma unroll
          for (int i = 0; i < h; ++i) part[i] += part[i + h];
        const float sum = part[0] + __shfl_xor_sync(0xffffffffu, part[0], 16);
        if (lane < kRedVals) dst[lane] = sum;
        __syncwarp();  // the next entry rewrites red
      } else if (lane < kRedVals) {
        dst[lane] = 0.f;
      }
    }
  }
  // entries past the region's last blended entry contribute nothing
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int idx = max(hi, start) + lane; idx < end; idx += 32) {
    float4* z = reinterpret_cast<float4*>(partials + ((size_t)emit[idx] * Q + slot_base) * kRedVals);
#pragma unroll
    for (int q = 0; q < kRedVals / 4; ++q) z[q] = zero;
  }
}

}  // namespace gs2d
