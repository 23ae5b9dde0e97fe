// Device code of the per-tile compositing loops, shared by the single-view
// kernels (render.cu) and the batched persistent kernels (batch.cu): the
// pixel layout of a tile, record staging, the (pixel, surfel) evaluation, the
// front-to-back forward loop and the back-to-front backward loops (full and
// pose-only).  The method and its derivation are described in render.cu.
#pragma once

#include "gs2d_common.cuh"
#include "loss_pixel.cuh"

namespace gs2d {

constexpr int kTileThreads = 256;
constexpr int kRedVals = 16;

// Thread -> pixel map of a tile with P pixels per thread: each warp owns an
// 8 x 4P block of pixels (lane l: column l & 7, rows (l >> 3) + 4k for
// k < P), so a warp can skip a surfel whose footprint misses its block.  A
// tile holds 256 P pixels: tile_w a multiple of 8, tile_h of 4P, and
// (tile_w / 8) x (tile_h / 4P) = 8 warps.
template <int P>
struct TilePix {
  int px, py;      // the thread's first pixel; pixel k is (px, py + 4k)
  int bx0, by0;    // first pixel of the warp's 8 x 4P block
  float lx, ly;    // first pixel's centre relative to the tile's first pixel centre
};
template <int P>
__device__ __forceinline__ TilePix<P> tile_pixel(int tile, int tiles_x, int tile_w, int tile_h) {
  TilePix<P> t;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpr = tile_w >> 3;
  const int ox = (w % wpr) * 8, oy = (w / wpr) * 4 * P;
  t.bx0 = tx * tile_w + ox;
  t.by0 = ty * tile_h + oy;
  t.px = t.bx0 + (lane & 7);
  t.py = t.by0 + (lane >> 3);
  t.lx = (float)(ox + (lane & 7));
  t.ly = (float)(oy + (lane >> 3));
  (void)tile_h;
  return t;
}

// A tile shape for P pixels per thread: 256 P pixels, widths a multiple of
// 8, heights of 4P (eight 8 x 4P warp blocks), P in {1, 2, 3, 4}.
__host__ __device__ inline bool tile_cfg_ok(const gs2d_config& c) {
  const int P = c.px_per_thread;
  if (P < 1 || P > 4) return false;
  return c.tile_w > 0 && c.tile_h > 0 && c.tile_w * c.tile_h == kTileThreads * P &&
         c.tile_w % 8 == 0 && c.tile_h % (4 * P) == 0;
}

// Runs the statement given after p (which names P) with P = p in {1, 2, 3, 4}.
#define GS2D_DISPATCH_P(p, ...)           \
  do {                                    \
    switch (p) {                          \
      case 2: {                           \
        constexpr int P = 2;              \
        __VA_ARGS__;                      \
      } break;                            \
      case 3: {                           \
        constexpr int P = 3;              \
        __VA_ARGS__;                      \
      } break;                            \
      case 4: {                           \
        constexpr int P = 4;              \
        __VA_ARGS__;                      \
      } break;                            \
      default: {                          \
        constexpr int P = 1;              \
        __VA_ARGS__;                      \
      } break;                            \
    }                                     \
  } while (0)

// Stages one projected record for a tile: p is re-based on the tile's first
// pixel centre (xt, yt) (principal-point relative): c0t = p(xt, yt).  Every
// pass stages through this function, so they evaluate identical numbers.
__device__ __forceinline__ float4 stage_c0(const float4 r0, const float4 r1, const float4 r2,
                                           float xt, float yt) {
  // r0 = (x0, y0, p2c, c1x), r1 = (c1y, c1z, c2x, c2y), r2 = (c2z, det, alpha, rgb0)
  const float dx = xt - r0.x, dy = yt - r0.y;
  return make_float4(fmaf(dy, r1.z, dx * r0.w), fmaf(dy, r1.w, dx * r1.x),
                     fmaf(dy, r2.x, fmaf(dx, r1.y, r0.z)), r0.w);
}

// Does the footprint (packed pixel ranges) touch the warp's 8 x 4P block?
template <int P>
__device__ __forceinline__ bool warp_hits(float bi, float bj, int bx0, int by0) {
  const uint32_t I = __float_as_uint(bi), J = __float_as_uint(bj);
  const int i0 = I & 0xFFFF, i1 = I >> 16, j0 = J & 0xFFFF, j1 = J >> 16;
  return !(i1 < bx0 || i0 > bx0 + 7 || j1 < by0 || j0 > by0 + 4 * P - 1);
}

// Mask of the tile's 8 warp blocks (8 x 4P pixels each) that a footprint
// (packed pixel ranges) touches; bit w for warp w.
template <int P>
__device__ __forceinline__ uint32_t footprint_mask(float bi, float bj, int tile_x0, int tile_y0,
                                                   int tile_w) {
  const uint32_t I = __float_as_uint(bi), J = __float_as_uint(bj);
  const int i0 = (int)(I & 0xFFFF) - tile_x0, i1 = (int)(I >> 16) - tile_x0;
  const int j0 = (int)(J & 0xFFFF) - tile_y0, j1 = (int)(J >> 16) - tile_y0;
  const int wpr = tile_w >> 3;
  uint32_t m = 0u;
#pragma unroll
  for (int w = 0; w < kTileThreads / 32; ++w) {
    const int ox = (w % wpr) * 8, oy = (w / wpr) * 4 * P;
    if (!(i1 < ox || i0 > ox + 7 || j1 < oy || j0 > oy + 4 * P - 1)) m |= 1u << w;
  }
  return m;
}

// Per-warp compaction of a staged batch: the indices (in staging order) of
// the surfels whose footprint touches this warp's block.  Returns the count.
__device__ __forceinline__ int warp_hit_list(const uint32_t* s_mask, uint8_t* my_list, int cnt,
                                             int warp, int lane) {
  int n = 0;
#pragma unroll 2
  for (int c = 0; c < cnt; c += 32) {
    const int j = c + lane;
    const bool hit = j < cnt && ((s_mask[j] >> warp) & 1u);
    const uint32_t b = __ballot_sync(0xffffffffu, hit);
    if (hit) my_list[n + __popc(b & ((1u << lane) - 1u))] = (uint8_t)j;
    n += __popc(b);
  }
  __syncwarp();
  return n;
}

// Evaluation of one (pixel, surfel) pair shared by every pass, so all take
// bit-identical skip decisions.  Returns false if skipped.
struct Eval {
  float rinv, u, v, z, G, araw, a;
};
__device__ __forceinline__ bool eval_pair(const float4 r0, const float4 r1, const float4 r2, float lx,
                                          float ly, float near_z, float cutoff_r2, float alpha_min,
                                          float alpha_max, Eval& e) {
  // r0 = c0t.xyz c1.x, r1 = c1.yz c2.xy, r2 = c2.z det alpha rgb0
  const float p0 = fmaf(ly, r1.z, fmaf(lx, r0.w, r0.x));
  const float p1 = fmaf(ly, r1.w, fmaf(lx, r1.x, r0.y));
  const float p2 = fmaf(ly, r2.x, fmaf(lx, r1.y, r0.z));
  e.rinv = __fdividef(1.0f, p2);
  e.u = __fmul_rn(p0, e.rinv);
  e.v = __fmul_rn(p1, e.rinv);
  const float rr = fmaf(e.u, e.u, __fmul_rn(e.v, e.v));
  if (!(rr <= cutoff_r2)) return false;
  e.z = __fmul_rn(r2.y, e.rinv);
  if (!(e.z > near_z)) return false;
  e.G = __expf(-0.5f * rr);
  e.araw = __fmul_rn(r2.z, e.G);
  e.a = fminf(e.araw, alpha_max);
  return e.a >= alpha_min;
}

// Stages the record of surfel id at dst (stage_record: row threadIdx.x of
// s_rec): the forward layout (5 float4) or the backward layout (7 float4);
// slot 4.y/z (forward) or 6.z/w (backward) carries the packed pixel
// footprint.
template <int kStride>
__device__ __forceinline__ void stage_record_to(const float4* __restrict__ proj, uint32_t id,
                                                float xt, float yt, float4* dst) {
  const float4* src = proj + (size_t)id * (kProjFloats / 4);
  const float4 r0 = src[0], r1 = src[1], r2 = src[2], r7 = src[7];
  dst[0] = stage_c0(r0, r1, r2, xt, yt);
  dst[1] = r1;
  dst[2] = r2;
  dst[3] = src[3];
  if (kStride == kFwdVec4) {
    dst[4] = make_float4(src[4].x, r7.z, r7.w, 0.f);
  } else {
    const float4 r6 = src[6];
    dst[4] = src[4];
    dst[5] = src[5];
    dst[6] = make_float4(r6.x, r6.y, r7.z, r7.w);
  }
}
template <int kStride>
__device__ __forceinline__ void stage_record(const float4* __restrict__ proj, uint32_t id, float xt,
                                             float yt, float4 (*s_rec)[kStride]) {
  stage_record_to<kStride>(proj, id, xt, yt, s_rec[threadIdx.x]);
}

struct FwdState {
  float T, D;
  F3 C, N;
  uint32_t last;
};

// Front-to-back compositing of the thread's P pixels over its tile's list
// (ids[0, end - start): the surfel ids of entries start .. end - 1, in
// global or shared memory).  Each warp visits only the staged surfels whose footprint touches its
// block; a surfel's staged record is read once for all P pixels.  With
// kCount it counts (cnt[0..4]) evaluated pairs, pairs inside the cutoff,
// blended pairs, and the evaluated pairs and those inside the cutoff up to
// each pixel's last blended pair (the pairs a backward replay evaluates).
struct HitLists {
  uint32_t mask[kTileThreads];
  uint8_t list[kTileThreads / 32][kTileThreads];
  int count[kTileThreads / 32];  // each warp's hit count of the last staged batch
};

// kG > 1 (one pixel per thread, no counting): the warp's hits are taken kG at
// a time -- their records loaded and their (pixel, surfel) pairs evaluated
// independently, then blended in list order -- so a pixel's walk keeps kG
// evaluations in flight instead of one.  Same evaluations, same order, same
// results; pairs after a pixel's stop are evaluated and dropped.
template <int kStride, bool kCount, int P, int kG = 1>
__device__ __forceinline__ void fwd_tile(const float4* __restrict__ proj,
                                         const uint32_t* ids, int start, int end,
                                         float xt, float yt, int tile_x0, int tile_y0,
                                         const TilePix<P>& tp, const bool (&inside)[P],
                                         const gs2d_camera& cam, const gs2d_config& cfg,
                                         float4 (*s_rec)[kStride], HitLists& hl, uint32_t* cnt,
                                         FwdState (&st)[P]) {
  bool done[P];
  bool all_done = true;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    st[k].T = 1.f;
    st[k].D = 0.f;
    st[k].C = f3(0.f, 0.f, 0.f);
    st[k].N = f3(0.f, 0.f, 0.f);
    st[k].last = 0;
    done[k] = !inside[k];
    all_done = all_done && done[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kFp = kStride == kFwdVec4 ? 4 : 6;  // slot holding the footprint
  // kCount: per pixel, evaluations (inside the cutoff) so far and at its
  // last blended pair
  uint32_t ev_k[P], in_k[P], last_ev[P], last_in[P];
#pragma unroll
  for (int k = 0; k < P; ++k) ev_k[k] = in_k[k] = last_ev[k] = last_in[k] = 0u;
  float lyk[P];
#pragma unroll
  for (int k = 0; k < P; ++k) lyk[k] = k ? tp.ly + 4.f * k : tp.ly;
  for (int b = start; b < end; b += kTileThreads) {
    if (__syncthreads_count(!all_done) == 0) break;
    const int idx = b + (int)threadIdx.x;
    if (idx < end) {
      stage_record<kStride>(proj, ids[idx - start], xt, yt, s_rec);
      const float4 rf = s_rec[threadIdx.x][kFp];
      hl.mask[threadIdx.x] = kStride == kFwdVec4
                                 ? footprint_mask<P>(rf.y, rf.z, tile_x0, tile_y0, cfg.tile_w)
                                 : footprint_mask<P>(rf.z, rf.w, tile_x0, tile_y0, cfg.tile_w);
    }
    __syncthreads();
    const int cnt_b = min(kTileThreads, end - b);
    const int nh = warp_hit_list(hl.mask, hl.list[warp], cnt_b, warp, lane);
    if (lane == 0) hl.count[warp] = nh;
    if (P == 1 && kG > 1 && !kCount && !all_done) {
      FwdState& q = st[0];
      for (int h0 = 0; h0 < nh && !all_done; h0 += kG) {
        int jg[kG];
        float ag[kG], zg[kG], cg[kG];
        bool hg[kG];
#pragma unroll
        for (int g = 0; g < kG; ++g) {
          // past the end: re-evaluate the last hit, never blended
          jg[g] = hl.list[warp][min(h0 + g, nh - 1)];
          const float4 r0 = s_rec[jg[g]][0], r1 = s_rec[jg[g]][1], r2 = s_rec[jg[g]][2];
          Eval e;
          hg[g] = eval_pair(r0, r1, r2, tp.lx, tp.ly, cam.near_z, cfg.cutoff_r2, cfg.alpha_min,
                            cfg.alpha_max, e) &&
                  h0 + g < nh;
          ag[g] = e.a;
          zg[g] = e.z;
          cg[g] = r2.w;
        }
#pragma unroll
        for (int g = 0; g < kG; ++g) {
          if (!hg[g]) continue;
          const float Tn = q.T * (1.f - ag[g]);
          if (Tn < cfg.t_min) {
            all_done = true;
            break;
          }
          const float4 r3 = s_rec[jg[g]][3];
          const float tnz = s_rec[jg[g]][4].x;
          const float w = ag[g] * q.T;
          q.C.x = fmaf(w, cg[g], q.C.x);
          q.C.y = fmaf(w, r3.x, q.C.y);
          q.C.z = fmaf(w, r3.y, q.C.z);
          q.D = fmaf(w, zg[g], q.D);
          q.N.x = fmaf(w, r3.z, q.N.x);
          q.N.y = fmaf(w, r3.w, q.N.y);
          q.N.z = fmaf(w, tnz, q.N.z);
          q.T = Tn;
          q.last = (uint32_t)(b + jg[g] + 1 - start);
        }
      }
    } else if (P == 1 && !all_done) {
      // one pixel: stop at its saturation
      FwdState& q = st[0];
      for (int h = 0; h < nh; ++h) {
        const int j = hl.list[warp][h];
        const float4 r0 = s_rec[j][0], r1 = s_rec[j][1], r2 = s_rec[j][2];
        Eval e;
        const bool hit = eval_pair(r0, r1, r2, tp.lx, tp.ly, cam.near_z, cfg.cutoff_r2,
                                   cfg.alpha_min, cfg.alpha_max, e);
        if (kCount) {
          ++cnt[0];
          if (fmaf(e.u, e.u, __fmul_rn(e.v, e.v)) <= cfg.cutoff_r2) ++cnt[1];
        }
        if (!hit) continue;
        const float Tn = q.T * (1.f - e.a);
        if (Tn < cfg.t_min) {
          all_done = true;
          break;
        }
        if (kCount) {
          last_ev[0] = cnt[0];
          last_in[0] = cnt[1];
        }
        const float4 r3 = s_rec[j][3];
        const float tnz = s_rec[j][4].x;
        const float w = e.a * q.T;
        q.C.x = fmaf(w, r2.w, q.C.x);
        q.C.y = fmaf(w, r3.x, q.C.y);
        q.C.z = fmaf(w, r3.y, q.C.z);
        q.D = fmaf(w, e.z, q.D);
        q.N.x = fmaf(w, r3.z, q.N.x);
        q.N.y = fmaf(w, r3.w, q.N.y);
        q.N.z = fmaf(w, tnz, q.N.z);
        q.T = Tn;
        q.last = (uint32_t)(b + j + 1 - start);
        if (kCount) ++cnt[2];
      }
    } else if (!all_done) {
      for (int h = 0; h < nh; ++h) {
        const int j = hl.list[warp][h];
        const float4 r0 = s_rec[j][0], r1 = s_rec[j][1], r2 = s_rec[j][2];
#pragma unroll
        for (int k = 0; k < P; ++k) {
          if (done[k]) continue;
          Eval e;
          const bool hit = eval_pair(r0, r1, r2, tp.lx, lyk[k], cam.near_z, cfg.cutoff_r2,
                                     cfg.alpha_min, cfg.alpha_max, e);
          if (kCount) {
            ++cnt[0];
            ++ev_k[k];
            if (fmaf(e.u, e.u, __fmul_rn(e.v, e.v)) <= cfg.cutoff_r2) {
              ++cnt[1];
              ++in_k[k];
            }
          }
          if (!hit) continue;
          const float Tn = st[k].T * (1.f - e.a);
          if (Tn < cfg.t_min) {
            done[k] = true;
            continue;
          }
          if (kCount) {
            last_ev[k] = ev_k[k];
            last_in[k] = in_k[k];
          }
          const float4 r3 = s_rec[j][3];
          const float tnz = s_rec[j][4].x;
          const float w = e.a * st[k].T;
          st[k].C.x = fmaf(w, r2.w, st[k].C.x);
          st[k].C.y = fmaf(w, r3.x, st[k].C.y);
          st[k].C.z = fmaf(w, r3.y, st[k].C.z);
          st[k].D = fmaf(w, e.z, st[k].D);
          st[k].N.x = fmaf(w, r3.z, st[k].N.x);
          st[k].N.y = fmaf(w, r3.w, st[k].N.y);
          st[k].N.z = fmaf(w, tnz, st[k].N.z);
          st[k].T = Tn;
          st[k].last = (uint32_t)(b + j + 1 - start);
          if (kCount) ++cnt[2];
        }
        all_done = true;
#pragma unroll
        for (int k = 0; k < P; ++k) all_done = all_done && done[k];
        if (all_done) break;
      }
    }
  }
  if (kCount) {
#pragma unroll
    for (int k = 0; k < P; ++k) {
      cnt[3] += last_ev[k];
      cnt[4] += last_in[k];
    }
  }
}

// Shared-memory scratch of the pose-only backward loops: the staged
// records and the tile's largest blended-entry count.
struct BwdSmem {
  float4 rec[kTileThreads][kBwdVec4];
  uint32_t max_nl;
};

// Per-pixel inputs of a backward replay: final transmittance, number of
// blended list entries, upstream gradients of colour, depth, normal, opacity.
struct PixGrad {
  float Tf;
  uint32_t nl;
  F3 gC, gN;
  float gD, gO;
};

// One replayed (pixel, surfel) pair of the pose-only backward: the blending
// gradient from the running state (T, acc) and the pair's rank-one splat
// gradient Gv, accumulated as sum Gv and sum z Gv (and the blended normals
// for the normal image's term).  rec: the staged record; r2 its third float4.
template <bool kNormal>
__device__ __forceinline__ void pose_pair(const Eval& e, const float4 r2, const float4* rec,
                                          const PixGrad& pgk, float rx, float ryk, float fxfy,
                                          float alpha_max, float gOT, float& T, float& acc, F3& sG,
                                          F3& szG, F3& sN) {
  const F3 gC = pgk.gC, gN = pgk.gN;
  const float gD = pgk.gD;
  const float4 r3 = rec[3], r4 = rec[4], r5 = rec[5], r6 = rec[6];
  const float iom = __fdividef(1.f, 1.f - e.a);
  const float Tb = T * iom;
  const float w = e.a * Tb;
  float vj = fmaf(r2.w, gC.x, fmaf(r3.x, gC.y, fmaf(r3.y, gC.z, e.z * gD)));
  if (kNormal) vj = fmaf(r3.z, gN.x, fmaf(r3.w, gN.y, fmaf(r4.x, gN.z, vj)));
  const float ga = Tb * vj - (acc - gOT) * iom;
  acc = fmaf(w, vj, acc);
  T = Tb;
  const float s = e.araw <= alpha_max ? -e.G * r2.z * ga : 0.f;
  // P = u d_u + v d_v; q = s P
  const float Px = fmaf(e.u, r5.x, e.v * r5.w);
  const float Py = fmaf(e.u, r5.y, e.v * r6.x);
  const float Pz = fmaf(e.u, r5.z, e.v * r6.y);
  const float Pr = fmaf(Px, rx, fmaf(Py, ryk, Pz));
  const float beta = fmaf(s, Pr, w * gD) * fxfy * e.rinv;
  const float Gx = fmaf(beta, r4.y, -s * Px);
  const float Gy = fmaf(beta, r4.z, -s * Py);
  const float Gz = fmaf(beta, r4.w, -s * Pz);
  sG.x += Gx;
  sG.y += Gy;
  sG.z += Gz;
  szG.x = fmaf(e.z, Gx, szG.x);
  szG.y = fmaf(e.z, Gy, szG.y);
  szG.z = fmaf(e.z, Gz, szG.z);
  if (kNormal) sN = sN + w * f3(r3.z, r3.w, r4.x);
}

// Pose-only back-to-front replay (tracking): the thread's P pixels walk the
// tile's list from each pixel's last blended entry to the front, undoing the
// compositing (T / (1 - a)) and accumulating the pose gradient per pixel;
// each warp visits only the surfels whose footprint touches its block.  With the hit point X = z r and r fixed
// per pixel, sum_pairs X x Gv = r x sum_pairs z Gv, so a pair only adds Gv
// and z Gv; with q = s (u d_u + v d_v), s = -G dL/dG, the pair's
// Gv = beta n - q, beta = (q . r + gz) / (n . r).  kNormal adds the normal
// image's term t_nc x w gN per pair (tracking has no normal gradient).
// kG > 1 (one pixel per thread): hits are taken kG at a time, their pairs
// evaluated independently and then replayed in back-to-front order (as in
// fwd_tile).  staged: the tile's whole list (at most one batch) is still
// staged in sm.rec with the per-warp hit lists of fwd_tile<kBwdVec4> in hl
// (the fused tracking kernel), so neither is rebuilt; entries past a
// pixel's last blended one are skipped per pixel as always.
template <bool kNormal, int P, int kG = 1>
__device__ __forceinline__ void bwd_tile_pose(const float4* __restrict__ proj,
                                              const uint32_t* ids, int start, int end,
                                              float xt, float yt, int tile_x0, int tile_y0,
                                              const TilePix<P>& tp, const bool (&inside)[P],
                                              float rx, float ry, const gs2d_camera& cam,
                                              const gs2d_config& cfg, const PixGrad (&pg)[P],
                                              BwdSmem& sm, HitLists& hl, float (&pr)[6],
                                              bool staged = false) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float fxfy = cam.fx * cam.fy;
  if (threadIdx.x == 0) sm.max_nl = 0u;
  __syncthreads();
  uint32_t my_nl = 0;
  bool any_inside = false;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    my_nl = max(my_nl, pg[k].nl);
    any_inside = any_inside || inside[k];
  }
  if (my_nl) atomicMax(&sm.max_nl, my_nl);
  __syncthreads();
  const int hi = start + (int)sm.max_nl;
  float T[P], acc[P], gOT[P];
  F3 szG[P];
  F3 sG = f3(0.f, 0.f, 0.f), sNg = f3(0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < P; ++k) {
    T[k] = pg[k].Tf;
    acc[k] = 0.f;
    gOT[k] = pg[k].gO * pg[k].Tf;
    szG[k] = f3(0.f, 0.f, 0.f);
  }
  F3 sN[P];
  float lyk[P], ryk[P];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    sN[k] = f3(0.f, 0.f, 0.f);
    lyk[k] = k ? tp.ly + 4.f * k : tp.ly;
    ryk[k] = k ? ry + (4.f * k) / cam.fy : ry;
  }
  for (int bend = hi; bend > start; bend -= kTileThreads) {
    const int bstart = max(start, bend - kTileThreads);
    const int cnt = bend - bstart;
    int nh;
    if (staged) {
      // one batch: bstart == start, records and hit lists as fwd_tile left them
      nh = hl.count[warp];
    } else {
      __syncthreads();
      if ((int)threadIdx.x < cnt) {
        stage_record<kBwdVec4>(proj, ids[bstart - start + (int)threadIdx.x], xt, yt, sm.rec);
        const float4 rf = sm.rec[threadIdx.x][6];
        hl.mask[threadIdx.x] = footprint_mask<P>(rf.z, rf.w, tile_x0, tile_y0, cfg.tile_w);
      }
      __syncthreads();
      nh = warp_hit_list(hl.mask, hl.list[warp], cnt, warp, lane);
    }
    if (!any_inside) continue;
    if (P == 1 && kG > 1) {
      for (int h0 = nh - 1; h0 >= 0; h0 -= kG) {
        int jg[kG];
        bool vg[kG];
        Eval eg[kG];
        float4 r2g[kG];
#pragma unroll
        for (int g = 0; g < kG; ++g) {
          // before the start: re-evaluate the first hit, never replayed
          jg[g] = hl.list[warp][max(h0 - g, 0)];
          const float4 r0 = sm.rec[jg[g]][0], r1 = sm.rec[jg[g]][1];
          r2g[g] = sm.rec[jg[g]][2];
          vg[g] = eval_pair(r0, r1, r2g[g], tp.lx, lyk[0], cam.near_z, cfg.cutoff_r2,
                            cfg.alpha_min, cfg.alpha_max, eg[g]) &&
                  h0 - g >= 0 && bstart + jg[g] - start < (int)pg[0].nl;
        }
#pragma unroll
        for (int g = 0; g < kG; ++g)
          if (vg[g])
            pose_pair<kNormal>(eg[g], r2g[g], sm.rec[jg[g]], pg[0], rx, ryk[0], fxfy,
                               cfg.alpha_max, gOT[0], T[0], acc[0], sG, szG[0], sN[0]);
      }
      continue;
    }
    for (int h = nh - 1; h >= 0; --h) {
      const int jj = hl.list[warp][h];
      const int jrel = bstart + jj - start;
      const float4 r0 = sm.rec[jj][0], r1 = sm.rec[jj][1], r2 = sm.rec[jj][2];
#pragma unroll
      for (int k = 0; k < P; ++k) {
        if (!inside[k] || jrel >= (int)pg[k].nl) continue;
        Eval e;
        if (!eval_pair(r0, r1, r2, tp.lx, lyk[k], cam.near_z, cfg.cutoff_r2, cfg.alpha_min,
                       cfg.alpha_max, e))
          continue;
        pose_pair<kNormal>(e, r2, sm.rec[jj], pg[k], rx, ryk[k], fxfy, cfg.alpha_max, gOT[k], T[k],
                           acc[k], sG, szG[k], sN[k]);
      }
    }
  }
  // theta: r x sum z Gv (+ sum_pairs t_nc x w gN = N x gN over the pairs)
  F3 th = f3(0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < P; ++k)
    th = th + cross3(f3(rx, ryk[k], 1.f), szG[k]) + cross3(sN[k], pg[k].gN);
  (void)sNg;
  pr[0] += sG.x;
  pr[1] += sG.y;
  pr[2] += sG.z;
  pr[3] += th.x;
  pr[4] += th.y;
  pr[5] += th.z;
}

// Block sum of a per-thread 6-vector, written by threads 0..5.
__device__ __forceinline__ void block_sum6(const float (&pr)[6], float (*s_pose)[6],
                                           float* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float v = pr[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) s_pose[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    float v = 0.f;
    for (int ww = 0; ww < kTileThreads / 32; ++ww) v += s_pose[ww][threadIdx.x];
    out[threadIdx.x] = v;
  }
}

}  // namespace gs2d
