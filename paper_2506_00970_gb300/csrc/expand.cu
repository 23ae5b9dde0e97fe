// Map expansion (Sec. III-E): new surfels from a keyframe's RGB-D image,
// gated by a voxel hash table of the active map's occupied space.
//
// Passes (all on the caller's stream, no host round trip):
//   select P_s     count + scan + scatter of the pixels with a valid depth
//                  and u_keep < ratio (stable: pixel order);
//   points         per point of P_s: world position, the normal of Eq.
//                  normal_fromD from the observed depth, and the create test
//                  (normal valid, voxel free);
//   nearest        per point of P_s: the distance to its nearest other point
//                  of P_s, by an exhaustive search in tiles of 256 points
//                  staged in shared memory, two queries per thread, the
//                  candidates split over 16 blocks per query block and
//                  min-combined (exact;
//                  O(|P_s|^2) flops, a fraction of a millisecond at the
//                  paper's sparse downsampling);
//   emit           count + scan + scatter of the created points into the
//                  map arrays at n_map + rank, with the tangent frame, the
//                  quaternion and the state; optionally their voxels are
//                  inserted into the table.
// Voxel table: open addressing with linear probing over 64-bit keys, every
// probe loop bounded by the capacity.
#include "gs2d_common.cuh"
#include "gs2d_expand.h"
#include "gs2d_internal.h"
#include "scan.cuh"

namespace gs2d {

constexpr int kExThreads = 256;
constexpr int kExPer = 4;                          // items per thread in selections
constexpr int kExBlock = kExThreads * kExPer;
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kVoxBits = 21;
constexpr int kVoxHalf = 1 << (kVoxBits - 1);

__device__ __forceinline__ unsigned long long voxel_key(float x, float y, float z, float vox) {
  const float inv = 1.f / vox;
  int c[3] = {(int)floorf(x * inv), (int)floorf(y * inv), (int)floorf(z * inv)};
  unsigned long long k = 0ull;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int v = min(max(c[a], -kVoxHalf), kVoxHalf - 1) + kVoxHalf;
    k |= (unsigned long long)v << (kVoxBits * a);
  }
  return k;
}

// 64-bit finaliser of SplitMix64 (Steele, Lea, Flood 2014).
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ void voxel_put(const gs2d_voxel_table& t, unsigned long long key) {
  const uint32_t mask = t.capacity - 1u;
  uint32_t s = (uint32_t)mix64(key) & mask;
  for (uint32_t probe = 0; probe < t.capacity; ++probe, s = (s + 1u) & mask) {
    const unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(t.keys) + s,
                                              kEmptyKey, key);
    if (prev == kEmptyKey || prev == key) return;
  }
  atomicExch(t.status, (int)GS2D_ERR_CAPACITY);
}

__device__ __forceinline__ bool voxel_has(const gs2d_voxel_table& t, unsigned long long key) {
  const uint32_t mask = t.capacity - 1u;
  uint32_t s = (uint32_t)mix64(key) & mask;
  for (uint32_t probe = 0; probe < t.capacity; ++probe, s = (s + 1u) & mask) {
    const unsigned long long k = t.keys[s];
    if (k == key) return true;
    if (k == kEmptyKey) return false;
  }
  return false;
}

__global__ void __launch_bounds__(kExThreads) voxel_clear_kernel(gs2d_voxel_table t) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < t.capacity;
       i += gridDim.x * blockDim.x)
    t.keys[i] = kEmptyKey;
  if (blockIdx.x == 0 && threadIdx.x == 0) *t.status = 0;
}

__global__ void __launch_bounds__(kExThreads) voxel_insert_kernel(gs2d_voxel_table t,
                                                                 const float* __restrict__ pts,
                                                                 const uint8_t* __restrict__ mask,
                                                                 int m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    if (mask && !mask[i]) continue;
    voxel_put(t, voxel_key(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], t.voxel));
  }
}

__global__ void __launch_bounds__(kExThreads) voxel_query_kernel(gs2d_voxel_table t,
                                                                const float* __restrict__ pts,
                                                                int m, uint8_t* __restrict__ occ) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    occ[i] = voxel_has(t, voxel_key(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], t.voxel)) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// selections (stable): count per block of kExBlock items, scan, scatter
// ---------------------------------------------------------------------------
struct PsPred {   // pixel p enters P_s
  const float* depth;
  const float* u_keep;
  float ratio;
  __device__ bool operator()(int p) const {
    const float d = depth[p];
    return d > 0.f && d < INFINITY && u_keep[p] < ratio;
  }
};
struct FlagPred {  // item k is flagged
  const uint8_t* flag;
  __device__ bool operator()(int k) const { return flag[k] != 0; }
};

template <class Pred>
__global__ void __launch_bounds__(kExThreads) select_count_kernel(Pred pred, int n,
                                                                 const int32_t* __restrict__ n_dev,
                                                                 int32_t* __restrict__ blk) {
  __shared__ int s_w[kExThreads / 32];
  if (n_dev) n = min(n, *n_dev);
  const int base = blockIdx.x * kExBlock + threadIdx.x * kExPer;
  int c = 0;
#pragma unroll
  for (int k = 0; k < kExPer; ++k) c += (base + k < n && pred(base + k)) ? 1 : 0;
  int total;
  block_exscan256(c, s_w, &total);
  if (threadIdx.x == 0) blk[blockIdx.x] = total;
}

// exclusive scan of nb block counts in place; *total = the sum
__global__ void __launch_bounds__(kExThreads) select_scan_kernel(int32_t* __restrict__ blk, int nb,
                                                                int32_t* __restrict__ total) {
  __shared__ int s_w[kExThreads / 32];
  int carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kExThreads) {
    const int b = b0 + (int)threadIdx.x;
    const int v = b < nb ? blk[b] : 0;
    int t;
    const int pre = block_exscan256(v, s_w, &t);
    if (b < nb) blk[b] = carry + pre;
    carry += t;
  }
  if (threadIdx.x == 0) *total = carry;
}

template <class Pred>
__global__ void __launch_bounds__(kExThreads) select_scatter_kernel(
    Pred pred, int n, const int32_t* __restrict__ n_dev, const int32_t* __restrict__ blk,
    int32_t* __restrict__ out) {
  __shared__ int s_w[kExThreads / 32];
  if (n_dev) n = min(n, *n_dev);
  const int base = blockIdx.x * kExBlock + threadIdx.x * kExPer;
  bool f[kExPer];
  int c = 0;
#pragma unroll
  for (int k = 0; k < kExPer; ++k) {
    f[k] = base + k < n && pred(base + k);
    c += f[k] ? 1 : 0;
  }
  int total;
  int o = blk[blockIdx.x] + block_exscan256(c, s_w, &total);
#pragma unroll
  for (int k = 0; k < kExPer; ++k)
    if (f[k]) out[o++] = base + k;
}

// ---------------------------------------------------------------------------
// points of P_s
// ---------------------------------------------------------------------------
__device__ __forceinline__ F3 back_project(const gs2d_camera& cam, int px, int py, float d) {
  return f3(d * ((px + 0.5f - cam.cx) / cam.fx), d * ((py + 0.5f - cam.cy) / cam.fy), d);
}

__device__ __forceinline__ F3 rot_t(const float* R, F3 v) {   // R^T v, R row-major
  return f3(R[0] * v.x + R[3] * v.y + R[6] * v.z, R[1] * v.x + R[4] * v.y + R[7] * v.z,
            R[2] * v.x + R[5] * v.y + R[8] * v.z);
}

__device__ __forceinline__ bool depth_ok(float d) { return d > 0.f && d < INFINITY; }

__global__ void __launch_bounds__(kExThreads) ps_point_kernel(
    const float* __restrict__ depth, gs2d_camera cam, const float* __restrict__ pose,
    const int32_t* __restrict__ idx,
    const int32_t* __restrict__ m_dev, gs2d_voxel_table table, int use_table,
    float4* __restrict__ pts, float4* __restrict__ nrm, uint8_t* __restrict__ create,
    unsigned* __restrict__ nnd2) {
  __shared__ float T[12];   // T_cw: R row-major, t
  const int m = *m_dev;
  if ((int)(blockIdx.x * blockDim.x) >= m) return;
  if (threadIdx.x < 12) T[threadIdx.x] = pose[threadIdx.x];
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int W = cam.width, H = cam.height;
  const int p = idx[k];
  const int px = p % W, py = p / W;
  const F3 Xc = back_project(cam, px, py, depth[p]);
  const F3 Xw = rot_t(T, f3(Xc.x - T[9], Xc.y - T[10], Xc.z - T[11]));
  pts[k] = make_float4(Xw.x, Xw.y, Xw.z, 0.f);
  nnd2[k] = __float_as_uint(INFINITY);
  // Eq. normal_fromD: central differences of the back-projected points
  bool ok = px >= 1 && py >= 1 && px < W - 1 && py < H - 1;
  F3 n = f3(0.f, 0.f, 0.f);
  if (ok) {
    const float dl = depth[p - 1], dr = depth[p + 1], du = depth[p - W], dd = depth[p + W];
    ok = depth_ok(dl) && depth_ok(dr) && depth_ok(du) && depth_ok(dd);
    if (ok) {
      const F3 xl = back_project(cam, px - 1, py, dl), xr = back_project(cam, px + 1, py, dr);
      const F3 xu = back_project(cam, px, py - 1, du), xd = back_project(cam, px, py + 1, dd);
      const F3 gx = 0.5f * (xr - xl), gy = 0.5f * (xd - xu);
      const F3 c = cross3(gx, gy);
      const float l2 = dot3(c, c);
      ok = l2 > 0.f;
      if (ok) n = rot_t(T, rsqrtf(l2) * c);
    }
  }
  bool free_vox = true;
  if (ok && use_table) free_vox = !voxel_has(table, voxel_key(Xw.x, Xw.y, Xw.z, table.voxel));
  nrm[k] = make_float4(n.x, n.y, n.z, sqrtf(dot3(Xc, Xc)));   // w: distance to the viewpoint
  create[k] = (ok && free_vox) ? 1 : 0;
}

// Squared distance from each point of P_s to its nearest other point, as
// the bits of a non-negative float (ordered like the values) min-combined
// with atomicMin: each thread takes two queries (every staged candidate is
// read once for both), blockIdx.y splits the candidates so that small P_s
// still fill the GPU; the result does not depend on the order of the atomics.
constexpr int kNnSplit = 16;
constexpr int kNnQ = 2 * kExThreads;   // queries per block
__global__ void __launch_bounds__(kExThreads) nearest_kernel(const float4* __restrict__ pts,
                                                            const int32_t* __restrict__ m_dev,
                                                            unsigned* __restrict__ nnd2) {
  __shared__ float4 s_p[kExThreads];
  const int m = *m_dev;
  const int k0 = blockIdx.x * kNnQ;
  if (k0 >= m) return;
  const int per = (m + kNnSplit - 1) / kNnSplit;
  const int c_lo = blockIdx.y * per, c_hi = min(m, c_lo + per);
  if (c_lo >= c_hi) return;
  const int ka = k0 + (int)threadIdx.x, kb = ka + kExThreads;
  const float4 qa = ka < m ? pts[ka] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 qb = kb < m ? pts[kb] : make_float4(0.f, 0.f, 0.f, 0.f);
  float ba = INFINITY, bb = INFINITY;
  for (int j0 = c_lo; j0 < c_hi; j0 += kExThreads) {
    __syncthreads();
    if (j0 + (int)threadIdx.x < c_hi) s_p[threadIdx.x] = pts[j0 + threadIdx.x];
    __syncthreads();
    const int cnt = min(kExThreads, c_hi - j0);
    if (j0 + cnt <= k0 || j0 >= k0 + kNnQ) {
      // no query of this block among these candidates: no self test
#pragma unroll 4
      for (int j = 0; j < cnt; ++j) {
        const float4 c = s_p[j];
        const float ax = c.x - qa.x, ay = c.y - qa.y, az = c.z - qa.z;
        const float bx = c.x - qb.x, by = c.y - qb.y, bz = c.z - qb.z;
        ba = fminf(ba, fmaf(ax, ax, fmaf(ay, ay, az * az)));
        bb = fminf(bb, fmaf(bx, bx, fmaf(by, by, bz * bz)));
      }
    } else {
      for (int j = 0; j < cnt; ++j) {
        const float4 c = s_p[j];
        const float ax = c.x - qa.x, ay = c.y - qa.y, az = c.z - qa.z;
        const float bx = c.x - qb.x, by = c.y - qb.y, bz = c.z - qb.z;
        const float da = fmaf(ax, ax, fmaf(ay, ay, az * az));
        const float db = fmaf(bx, bx, fmaf(by, by, bz * bz));
        if (j0 + j != ka) ba = fminf(ba, da);
        if (j0 + j != kb) bb = fminf(bb, db);
      }
    }
  }
  if (ka < m && ba < INFINITY) atomicMin(nnd2 + ka, __float_as_uint(ba));
  if (kb < m && bb < INFINITY) atomicMin(nnd2 + kb, __float_as_uint(bb));
}

struct EmitArgs {
  const float* rgb;
  const float* u_angle;
  const int32_t* idx;      // pixel of each P_s point
  const float4* pts;
  const float4* nrm;
  const unsigned* nnd2;   // squared nearest distance (float bits)
  float max_scale;
  const int32_t* sel;      // P_s point of each created surfel
  const int32_t* k_dev;    // number created
  float* mu;
  float* quat;
  float* scale;
  float* opacity;
  float* rgb_out;
  gs2d_map_state st;
  int n_map, capacity;
  float opac0;
  int kf_id;
  gs2d_voxel_table table;
  int insert;
  int32_t* n_new;
};

__global__ void __launch_bounds__(kExThreads) emit_kernel(EmitArgs a) {
  const int k = *a.k_dev;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r == 0) {
    *a.n_new = k;
    if ((long long)a.n_map + k > a.capacity && a.table.status)
      atomicExch(a.table.status, (int)GS2D_ERR_CAPACITY);
  }
  if (r >= k || (long long)a.n_map + k > a.capacity) return;
  const int j = a.sel[r];
  const int p = a.idx[j];
  const float4 X = a.pts[j];
  const float4 N = a.nrm[j];
  // orthonormal basis of the normal's plane (Duff et al. 2017)
  const float sg = copysignf(1.f, N.z);
  const float aa = -1.f / (sg + N.z);
  const float bb = N.x * N.y * aa;
  const F3 b1 = f3(1.f + sg * N.x * N.x * aa, sg * bb, -sg * N.x);
  const F3 b2 = f3(bb, sg + N.y * N.y * aa, -N.y);
  float sp, cp;
  sincospif(2.f * a.u_angle[p], &sp, &cp);
  const F3 tn = f3(N.x, N.y, N.z);
  const F3 tu = cp * b1 + sp * b2;
  const F3 tv = cross3(tn, tu);
  const float D[9] = {tu.x, tv.x, tn.x, tu.y, tv.y, tn.y, tu.z, tv.z, tn.z};
  const int o = a.n_map + r;
  a.mu[3 * o] = X.x;
  a.mu[3 * o + 1] = X.y;
  a.mu[3 * o + 2] = X.z;
  reinterpret_cast<float4*>(a.quat)[o] = quat_from_matrix(D);
  const float d2 = __uint_as_float(a.nnd2[j]);
  const float s = d2 < INFINITY ? sqrtf(d2) : a.max_scale;
  a.scale[2 * o] = s;
  a.scale[2 * o + 1] = s;
  a.opacity[o] = a.opac0;
  a.rgb_out[3 * o] = a.rgb[3 * p];
  a.rgb_out[3 * o + 1] = a.rgb[3 * p + 1];
  a.rgb_out[3 * o + 2] = a.rgb[3 * p + 2];
  if (a.st.delta) a.st.delta[o] = 1;
  if (a.st.t_c) a.st.t_c[o] = a.kf_id;
  if (a.st.t_l) a.st.t_l[o] = a.kf_id;
  if (a.st.d_c) a.st.d_c[o] = N.w;
  if (a.insert) voxel_put(a.table, voxel_key(X.x, X.y, X.z, a.table.voxel));
}

struct ExWs {
  int32_t *blk, *blk2, *idx, *sel, *m, *k;
  float4 *pts, *nrm;
  unsigned* nnd2;
  uint8_t* create;
  size_t bytes;
};

ExWs carve_expand(void* base, int P) {
  Carver c(base);
  ExWs w;
  const int nb = (P + kExBlock - 1) / kExBlock;
  w.blk = c.take<int32_t>(nb);
  w.blk2 = c.take<int32_t>(nb);
  w.m = c.take<int32_t>(1);
  w.k = c.take<int32_t>(1);
  w.idx = c.take<int32_t>(P);
  w.sel = c.take<int32_t>(P);
  w.pts = c.take<float4>(P);
  w.nrm = c.take<float4>(P);
  w.nnd2 = c.take<unsigned>(P);
  w.create = c.take<uint8_t>(P);
  w.bytes = align_up(c.off, 256);
  return w;
}

bool table_ok(const gs2d_voxel_table* t) {
  return t && t->keys && t->status && t->capacity > 0 && (t->capacity & (t->capacity - 1)) == 0 &&
         t->voxel > 0.f;
}

int blocks_for(long long n) { return (int)max(1ll, min((n + kExThreads - 1) / kExThreads, 152ll * 32)); }

}  // namespace gs2d

using namespace gs2d;

extern "C" {

int gs2d_voxel_clear(const gs2d_voxel_table* t, gs2d_stream stream) {
  if (!table_ok(t)) return GS2D_ERR_INVALID_ARG;
  voxel_clear_kernel<<<blocks_for(t->capacity), kExThreads, 0, (cudaStream_t)stream>>>(*t);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int gs2d_voxel_insert(const gs2d_voxel_table* t, const float* points, const uint8_t* mask, int m,
                      gs2d_stream stream) {
  if (!table_ok(t) || m < 0 || (m > 0 && !points)) return GS2D_ERR_INVALID_ARG;
  if (m == 0) return GS2D_OK;
  voxel_insert_kernel<<<blocks_for(m), kExThreads, 0, (cudaStream_t)stream>>>(*t, points, mask, m);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int gs2d_voxel_query(const gs2d_voxel_table* t, const float* points, int m, uint8_t* occupied,
                     gs2d_stream stream) {
  if (!table_ok(t) || m < 0 || (m > 0 && (!points || !occupied))) return GS2D_ERR_INVALID_ARG;
  if (m == 0) return GS2D_OK;
  voxel_query_kernel<<<blocks_for(m), kExThreads, 0, (cudaStream_t)stream>>>(*t, points, m,
                                                                           occupied);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

size_t gs2d_expand_workspace(const gs2d_camera* cam) {
  if (!cam || cam->width <= 0 || cam->height <= 0) return 0;
  return carve_expand(nullptr, cam->width * cam->height).bytes;
}

int gs2d_expand(const float* rgb, const float* depth, const gs2d_camera* cam, const float* pose_cw,
                const float* u_keep, const float* u_angle, const gs2d_voxel_table* table,
                const gs2d_expand_params* prm, int n_map, int capacity, float* mu, float* quat,
                float* scale, float* opacity, float* rgb_out, const gs2d_map_state* st,
                int32_t* n_new, void* workspace, size_t ws_bytes, size_t* ws_needed,
                gs2d_stream stream) {
  if (!cam || cam->width <= 0 || cam->height <= 0 || !prm || !n_new) return GS2D_ERR_INVALID_ARG;
  if ((long long)cam->width * cam->height > (1ll << 30)) return GS2D_ERR_INVALID_ARG;
  const int P = cam->width * cam->height;
  const ExWs sz = carve_expand(nullptr, P);
  if (ws_needed) *ws_needed = sz.bytes;
  if (!workspace || ws_bytes < sz.bytes) return GS2D_ERR_WORKSPACE;
  if (!rgb || !depth || !pose_cw || !u_keep || !u_angle || !mu || !quat || !scale || !opacity ||
      !rgb_out || n_map < 0 || capacity < n_map || !(prm->ratio > 0.f && prm->ratio <= 1.f))
    return GS2D_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(quat) & 15) return GS2D_ERR_INVALID_ARG;
  if (table && !table_ok(table)) return GS2D_ERR_INVALID_ARG;
  if (prm->insert_new && !table) return GS2D_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const ExWs w = carve_expand(workspace, P);
  const int nb = (P + kExBlock - 1) / kExBlock;
  const PsPred ps{depth, u_keep, prm->ratio};
  select_count_kernel<PsPred><<<nb, kExThreads, 0, s>>>(ps, P, nullptr, w.blk);
  GS2D_LAUNCH_CHECK();
  select_scan_kernel<<<1, kExThreads, 0, s>>>(w.blk, nb, w.m);
  GS2D_LAUNCH_CHECK();
  select_scatter_kernel<PsPred><<<nb, kExThreads, 0, s>>>(ps, P, nullptr, w.blk, w.idx);
  GS2D_LAUNCH_CHECK();
  const gs2d_voxel_table tb = table ? *table : gs2d_voxel_table{nullptr, 0u, 1.f, nullptr};
  const int pb = (P + kExThreads - 1) / kExThreads;
  ps_point_kernel<<<pb, kExThreads, 0, s>>>(depth, *cam, pose_cw, w.idx, w.m, tb, table ? 1 : 0, w.pts,
                                            w.nrm, w.create, w.nnd2);
  GS2D_LAUNCH_CHECK();
  nearest_kernel<<<dim3((P + kNnQ - 1) / kNnQ, kNnSplit), kExThreads, 0, s>>>(w.pts, w.m, w.nnd2);
  GS2D_LAUNCH_CHECK();
  const FlagPred fp{w.create};
  select_count_kernel<FlagPred><<<nb, kExThreads, 0, s>>>(fp, P, w.m, w.blk2);
  GS2D_LAUNCH_CHECK();
  select_scan_kernel<<<1, kExThreads, 0, s>>>(w.blk2, nb, w.k);
  GS2D_LAUNCH_CHECK();
  select_scatter_kernel<FlagPred><<<nb, kExThreads, 0, s>>>(fp, P, w.m, w.blk2, w.sel);
  GS2D_LAUNCH_CHECK();
  EmitArgs a;
  a.rgb = rgb;
  a.u_angle = u_angle;
  a.idx = w.idx;
  a.pts = w.pts;
  a.nrm = w.nrm;
  a.nnd2 = w.nnd2;
  a.max_scale = prm->max_scale;
  a.sel = w.sel;
  a.k_dev = w.k;
  a.mu = mu;
  a.quat = quat;
  a.scale = scale;
  a.opacity = opacity;
  a.rgb_out = rgb_out;
  a.st = st ? *st : gs2d_map_state{nullptr, nullptr, nullptr, nullptr};
  a.n_map = n_map;
  a.capacity = capacity;
  a.opac0 = prm->opacity;
  a.kf_id = prm->kf_id;
  a.table = tb;
  a.insert = prm->insert_new;
  a.n_new = n_new;
  emit_kernel<<<pb, kExThreads, 0, s>>>(a);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

}  // extern "C"
