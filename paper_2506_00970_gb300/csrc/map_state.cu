// Map state of 2DGS-SLAM (Eq. map): the per-keyframe state update of
// Sec. III-F, the map correction of Sec. IV-C, the occlusion pruning of
// Sec. III-F and a stable compaction of the surfel arrays.  All of them are
// one pass over the map's structure-of-arrays: HBM-bound, grid-stride loops
// over at most 152 x 32 blocks, loads and stores coalesced per array.
#include "gs2d_common.cuh"
#include "gs2d_internal.h"
#include "gs2d_map.h"
#include "scan.cuh"

namespace gs2d {

constexpr int kMapThreads = 256;
constexpr int kMapMaxBlocks = 152 * 32;
constexpr int kCompactPer = 4;                         // items per thread
constexpr int kCompactBlock = kMapThreads * kCompactPer;

__host__ __device__ inline int map_blocks(int n) {
  const int b = (n + kMapThreads - 1) / kMapThreads;
  return b < 1 ? 1 : (b > kMapMaxBlocks ? kMapMaxBlocks : b);
}

// Warp-aggregated increment of a device counter.
__device__ __forceinline__ void count_add(uint32_t* c, bool flag) {
  const uint32_t b = __ballot_sync(0xffffffffu, flag);
  if (c && (threadIdx.x & 31) == 0 && b) atomicAdd(c, (uint32_t)__popc(b));
}

__global__ void __launch_bounds__(kMapThreads) map_observe_kernel(
    const float* __restrict__ contrib, const float* __restrict__ mu, int n,
    const float* __restrict__ pose, int kf, gs2d_state_params prm, gs2d_map_state st,
    uint32_t* __restrict__ counts) {
  // camera centre c = -R^T t of the keyframe
  const float cx = -(pose[0] * pose[9] + pose[3] * pose[10] + pose[6] * pose[11]);
  const float cy = -(pose[1] * pose[9] + pose[4] * pose[10] + pose[7] * pose[11]);
  const float cz = -(pose[2] * pose[9] + pose[5] * pose[10] + pose[8] * pose[11]);
  const int stride = gridDim.x * blockDim.x;
  // every lane of a warp runs the same number of iterations (ballots)
  const int n_up = (n + 31) & ~31;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_up; i += stride) {
    bool vis_act = false, closer = false, deact = false, react = false;
    if (i < n) {
      const bool vis = contrib[i] > prm.vis_threshold;
      if (st.delta[i]) {
        int tl = st.t_l[i];
        if (vis) {
          vis_act = true;
          tl = kf;
          st.t_l[i] = kf;
          const float dx = mu[3 * i] - cx, dy = mu[3 * i + 1] - cy, dz = mu[3 * i + 2] - cz;
          const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
          if (d < st.d_c[i]) {
            st.d_c[i] = d;
            st.t_c[i] = kf;
            closer = true;
          }
        }
        if ((long long)kf - tl > prm.inactive_after) {
          st.delta[i] = 0;
          deact = true;
        }
      } else if (prm.reactivate && vis && st.t_c[i] > prm.loop_h) {
        st.delta[i] = 1;
        st.t_l[i] = kf;
        react = true;
      }
    }
    if (counts) {
      count_add(counts, vis_act);
      count_add(counts + 1, closer);
      count_add(counts + 2, deact);
      count_add(counts + 3, react);
    }
  }
}

// Pose increments dT_j = (T^o_cw)^-1 T_cw: dR = R_o^T R, dt = R_o^T (t - t_o),
// and the unit quaternion of dR.
// Record layout: dR [9], dt [3], q [4] (w, x, y, z).
__global__ void map_delta_kernel(const float* __restrict__ old_p, const float* __restrict__ new_p,
                                 int n_kf, float* __restrict__ delta) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_kf) return;
  const float* A = old_p + 12 * j;
  const float* B = new_p + 12 * j;
  float D[9], t[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      D[3 * r + c] = B[r] * A[c] + B[3 + r] * A[3 + c] + B[6 + r] * A[6 + c];
    t[r] = B[r] * (A[9] - B[9]) + B[3 + r] * (A[10] - B[10]) + B[6 + r] * (A[11] - B[11]);
  }
  const float4 q = quat_from_matrix(D);
  float* o = delta + 16 * j;
#pragma unroll
  for (int k = 0; k < 9; ++k) o[k] = D[k];
  o[9] = t[0];
  o[10] = t[1];
  o[11] = t[2];
  o[12] = q.x;
  o[13] = q.y;
  o[14] = q.z;
  o[15] = q.w;
}

__global__ void __launch_bounds__(kMapThreads) map_correct_kernel(
    float* __restrict__ mu, float4* __restrict__ quat, const int32_t* __restrict__ t_c, int n,
    const float* __restrict__ delta, int n_kf, int32_t* __restrict__ n_skipped) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int j = t_c[i];
    if (j < 0 || j >= n_kf) {
      if (n_skipped) atomicAdd(n_skipped, 1);
      continue;
    }
    const float* d = delta + 16 * j;
    const float x = mu[3 * i], y = mu[3 * i + 1], z = mu[3 * i + 2];
    mu[3 * i] = fmaf(d[0], x, fmaf(d[1], y, fmaf(d[2], z, d[9])));
    mu[3 * i + 1] = fmaf(d[3], x, fmaf(d[4], y, fmaf(d[5], z, d[10])));
    mu[3 * i + 2] = fmaf(d[6], x, fmaf(d[7], y, fmaf(d[8], z, d[11])));
    const float4 q = quat[i];                   // (w, x, y, z)
    const float aw = d[12], ax = d[13], ay = d[14], az = d[15];
    // Hamilton product q(dR) q: R(q(dR) q) = dR R(q)
    quat[i] = make_float4(aw * q.x - ax * q.y - ay * q.z - az * q.w,
                          aw * q.y + ax * q.x + ay * q.w - az * q.z,
                          aw * q.z - ax * q.w + ay * q.x + az * q.y,
                          aw * q.w + ax * q.z - ay * q.y + az * q.x);
  }
}

__global__ void __launch_bounds__(kMapThreads) map_prune_kernel(const float* __restrict__ contrib,
                                                                const int32_t* __restrict__ t_c,
                                                                int n, int r, float thr,
                                                                uint8_t* __restrict__ keep) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    keep[i] = (t_c[i] == r && contrib[i] < thr) ? 0 : 1;
}

// Compaction, pass 1: kept items per block of kCompactBlock (item
// base + k * 256 + thread for k < 4: each warp access is 32 consecutive items).
__global__ void __launch_bounds__(kMapThreads) compact_count_kernel(const uint8_t* __restrict__ keep,
                                                                    int n,
                                                                    int32_t* __restrict__ blk) {
  __shared__ int s_w[kMapThreads / 32];
  const int base = blockIdx.x * kCompactBlock + threadIdx.x;
  int c = 0;
#pragma unroll
  for (int k = 0; k < kCompactPer; ++k) {
    const int i = base + k * kMapThreads;
    c += (i < n && keep[i]) ? 1 : 0;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kMapThreads / 32; ++w) s += s_w[w];
    blk[blockIdx.x] = s;
  }
}

// Pass 2 (one block): exclusive scan of the block counts, in place; n_out.
__global__ void __launch_bounds__(kMapThreads) compact_scan_kernel(int32_t* __restrict__ blk,
                                                                   int nb,
                                                                   int32_t* __restrict__ n_out) {
  __shared__ int s_w[kMapThreads / 32];
  int carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kMapThreads) {
    const int b = b0 + (int)threadIdx.x;
    const int v = b < nb ? blk[b] : 0;
    int total;
    const int pre = block_exscan256(v, s_w, &total);
    if (b < nb) blk[b] = carry + pre;
    carry += total;
  }
  if (threadIdx.x == 0) *n_out = carry;
}

template <typename T>
__device__ __forceinline__ void copy_n(const T* __restrict__ in, T* __restrict__ out, int i, int o,
                                       int w) {
  for (int k = 0; k < w; ++k) out[(size_t)o * w + k] = in[(size_t)i * w + k];
}

// Pass 3: scatter every kept item to its slot.  The block's items are taken
// in four rounds of 256 consecutive items (coalesced loads and, for runs of
// kept items, coalesced stores), each round ranked by a block scan.
__global__ void __launch_bounds__(kMapThreads) compact_scatter_kernel(
    const uint8_t* __restrict__ keep, int n, const int32_t* __restrict__ blk, gs2d_surfels s,
    gs2d_map_state st, float* __restrict__ mu_o, float* __restrict__ quat_o,
    float* __restrict__ scale_o, float* __restrict__ opac_o, float* __restrict__ rgb_o,
    gs2d_map_state so, int32_t* __restrict__ new_index) {
  __shared__ int s_w[kMapThreads / 32];
  int carry = blk[blockIdx.x];
  for (int k = 0; k < kCompactPer; ++k) {
    const int i = blockIdx.x * kCompactBlock + k * kMapThreads + (int)threadIdx.x;
    const bool kf = i < n && keep[i];
    int total;
    const int o = carry + block_exscan256(kf ? 1 : 0, s_w, &total);
    carry += total;
    if (i < n && new_index) new_index[i] = kf ? o : -1;
    if (!kf) continue;
    copy_n(s.mu, mu_o, i, o, 3);
    reinterpret_cast<float4*>(quat_o)[o] = reinterpret_cast<const float4*>(s.quat)[i];
    copy_n(s.scale, scale_o, i, o, 2);
    opac_o[o] = s.opacity[i];
    copy_n(s.rgb, rgb_o, i, o, 3);
    if (st.delta) so.delta[o] = st.delta[i];
    if (st.t_c) so.t_c[o] = st.t_c[i];
    if (st.d_c) so.d_c[o] = st.d_c[i];
    if (st.t_l) so.t_l[o] = st.t_l[i];
  }
}

__global__ void __launch_bounds__(kMapThreads) map_expand_values_kernel(
    const float* __restrict__ vals, const int32_t* __restrict__ idx, int n, float fill,
    float* __restrict__ out) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int k = idx[i];
    out[i] = k >= 0 ? vals[k] : fill;
  }
}

}  // namespace gs2d

using namespace gs2d;

extern "C" {

int gs2d_map_observe(const float* contrib, const float* mu, int n, const float* pose_cw,
                     int kf_id, const gs2d_state_params* prm, const gs2d_map_state* st,
                     uint32_t* counts, gs2d_stream stream) {
  if (n < 0 || !prm || !st || !pose_cw) return GS2D_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (counts && cudaMemsetAsync(counts, 0, 4 * sizeof(uint32_t), s) != cudaSuccess)
    return GS2D_ERR_CUDA;
  if (n == 0) return GS2D_OK;
  if (!contrib || !mu || !st->delta || !st->t_c || !st->d_c || !st->t_l)
    return GS2D_ERR_INVALID_ARG;
  map_observe_kernel<<<map_blocks(n), kMapThreads, 0, s>>>(contrib, mu, n, pose_cw, kf_id, *prm,
                                                           *st, counts);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

size_t gs2d_map_correct_workspace(int n_kf) {
  return align_up((size_t)(n_kf > 0 ? n_kf : 1) * 16 * sizeof(float), 256);
}

int gs2d_map_correct(float* mu, float* quat, const int32_t* t_c, int n, const float* poses_old,
                     const float* poses_new, int n_kf, void* workspace, size_t ws_bytes,
                     size_t* ws_needed, int32_t* n_skipped, gs2d_stream stream) {
  if (n < 0 || n_kf < 0) return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_map_correct_workspace(n_kf);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_skipped && cudaMemsetAsync(n_skipped, 0, sizeof(int32_t), s) != cudaSuccess)
    return GS2D_ERR_CUDA;
  if (n == 0) return GS2D_OK;
  if (!mu || !quat || !t_c || (n_kf > 0 && (!poses_old || !poses_new)))
    return GS2D_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(quat) & 15) return GS2D_ERR_INVALID_ARG;
  float* delta = static_cast<float*>(workspace);
  if (n_kf > 0) {
    map_delta_kernel<<<(n_kf + 127) / 128, 128, 0, s>>>(poses_old, poses_new, n_kf, delta);
    GS2D_LAUNCH_CHECK();
  }
  map_correct_kernel<<<map_blocks(n), kMapThreads, 0, s>>>(mu, reinterpret_cast<float4*>(quat),
                                                           t_c, n, delta, n_kf, n_skipped);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int gs2d_map_prune(const float* contrib, const int32_t* t_c, int n, int r, float vis_threshold,
                   uint8_t* keep, gs2d_stream stream) {
  if (n < 0) return GS2D_ERR_INVALID_ARG;
  if (n == 0) return GS2D_OK;
  if (!contrib || !t_c || !keep) return GS2D_ERR_INVALID_ARG;
  map_prune_kernel<<<map_blocks(n), kMapThreads, 0, (cudaStream_t)stream>>>(contrib, t_c, n, r,
                                                                           vis_threshold, keep);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int gs2d_map_expand_values(const float* vals, const int32_t* new_index, int n, float fill,
                           float* out, gs2d_stream stream) {
  if (n < 0) return GS2D_ERR_INVALID_ARG;
  if (n == 0) return GS2D_OK;
  if (!vals || !new_index || !out) return GS2D_ERR_INVALID_ARG;
  map_expand_values_kernel<<<map_blocks(n), kMapThreads, 0, (cudaStream_t)stream>>>(
      vals, new_index, n, fill, out);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

size_t gs2d_map_compact_workspace(int n) {
  const size_t nb = (size_t)((n > 0 ? n : 1) + kCompactBlock - 1) / kCompactBlock;
  return align_up(nb * sizeof(int32_t), 256);
}

int gs2d_map_compact(const uint8_t* keep, int n, const gs2d_surfels* s, const gs2d_map_state* st,
                     float* mu_out, float* quat_out, float* scale_out, float* opacity_out,
                     float* rgb_out, const gs2d_map_state* st_out, int32_t* new_index,
                     int32_t* n_out, void* workspace, size_t ws_bytes, size_t* ws_needed,
                     gs2d_stream stream) {
  if (n < 0 || !s || !n_out) return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_map_compact_workspace(n);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  cudaStream_t cs = (cudaStream_t)stream;
  if (n == 0) {
    if (cudaMemsetAsync(n_out, 0, sizeof(int32_t), cs) != cudaSuccess) return GS2D_ERR_CUDA;
    return GS2D_OK;
  }
  if (!keep || !s->mu || !s->quat || !s->scale || !s->opacity || !s->rgb || !mu_out ||
      !quat_out || !scale_out || !opacity_out || !rgb_out)
    return GS2D_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(s->quat) | reinterpret_cast<uintptr_t>(quat_out)) & 15)
    return GS2D_ERR_INVALID_ARG;
  gs2d_map_state si = st ? *st : gs2d_map_state{nullptr, nullptr, nullptr, nullptr};
  gs2d_map_state so = st_out ? *st_out : gs2d_map_state{nullptr, nullptr, nullptr, nullptr};
  // a state array is copied only when both sides give it
  if (!so.delta) si.delta = nullptr;
  if (!so.t_c) si.t_c = nullptr;
  if (!so.d_c) si.d_c = nullptr;
  if (!so.t_l) si.t_l = nullptr;
  const int nb = (n + kCompactBlock - 1) / kCompactBlock;
  int32_t* blk = static_cast<int32_t*>(workspace);
  compact_count_kernel<<<nb, kMapThreads, 0, cs>>>(keep, n, blk);
  GS2D_LAUNCH_CHECK();
  compact_scan_kernel<<<1, kMapThreads, 0, cs>>>(blk, nb, n_out);
  GS2D_LAUNCH_CHECK();
  compact_scatter_kernel<<<nb, kMapThreads, 0, cs>>>(keep, n, blk, *s, si, mu_out, quat_out,
                                                     scale_out, opacity_out, rgb_out, so,
                                                     new_index);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

}  // extern "C"
