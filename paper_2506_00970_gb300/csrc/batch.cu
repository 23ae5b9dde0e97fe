// Batched views: one persistent launch per render pass over every
// (view, tile) work item of up to GS2D_MAX_VIEWS views -- the keyframes of a
// mapping window (Sec. III-E) or frames of uneven resolution, each over its
// own active surfel subset (Sec. III-C).  Blocks take items from an atomic
// counter (no spinning), so large and small views balance across the SMs.
// The view table is a by-value kernel parameter: a launch is fully described
// by its arguments and can be captured in a CUDA graph.  The per-tile work is
// the single-view code of tile_loops.cuh, so every view's images and partial
// gradients equal those of the single-view entry points.
#include <mutex>

#include "bwd_warp.cuh"
#include "gs2d_common.cuh"
#include "gs2d_internal.h"
#include "tile_loops.cuh"

namespace gs2d {

struct ViewDev {
  gs2d_camera cam;
  gs2d_config cfg;
  int tiles_x, n_tiles, item0;      // first work item of this view
  const float4* proj;
  const uint32_t* vals;
  const uint32_t* emit;
  const int32_t* ranges;
  const int32_t* status;
  float *rgb, *depth, *normal, *opac, *T;
  uint32_t* nlast;
  const float *d_rgb, *d_depth, *d_normal, *d_opac;
  float* partials;                  // this view's (tile, region, surfel) partials
};
struct ViewTable {
  int n_views, n_items;
  ViewDev v[GS2D_MAX_VIEWS];
};

__device__ __forceinline__ int view_of(const ViewTable& tab, int item) {
  int v = 0;
  while (v + 1 < tab.n_views && item >= tab.v[v + 1].item0) ++v;
  return v;
}

// Work order of the persistent passes: every (view, tile) item sorted by
// decreasing list length (a counting sort on the length's octave and its
// next three bits), so the heaviest tiles start first and the launch ends on
// short items instead of idling SMs behind a late long one.  Items of a view
// with a failed status sort last.  Results do not depend on the order (each
// item writes only its own pixels and partial slots).
constexpr int kOrderBuckets = 256;
constexpr int kOrderThreads = 1024;
__device__ __forceinline__ int length_bucket(uint32_t len) {
  if (len < 16u) return (int)len;
  const int oct = 31 - __clz(len);  // >= 4
  return 16 + (oct - 4) * 8 + (int)((len >> (oct - 3)) & 7u);  // <= 239
}
__global__ void __launch_bounds__(kOrderThreads) order_items_kernel(ViewTable tab,
                                                                  int32_t* __restrict__ order) {
  __shared__ uint32_t hist[kOrderBuckets];
  for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) hist[b] = 0u;
  __syncthreads();
  for (int v = 0; v < tab.n_views; ++v) {
    const ViewDev& V = tab.v[v];
    const bool dead = V.status && *V.status;
    for (int t = threadIdx.x; t < V.n_tiles; t += blockDim.x) {
      const uint32_t len = dead ? 0u : (uint32_t)max(V.ranges[2 * t + 1] - V.ranges[2 * t], 0);
      atomicAdd(&hist[length_bucket(len)], 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive scan, longest bucket first
    uint32_t run = 0u;
    for (int b = kOrderBuckets - 1; b >= 0; --b) {
      const uint32_t c = hist[b];
      hist[b] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int v = 0; v < tab.n_views; ++v) {
    const ViewDev& V = tab.v[v];
    const bool dead = V.status && *V.status;
    for (int t = threadIdx.x; t < V.n_tiles; t += blockDim.x) {
      const uint32_t len = dead ? 0u : (uint32_t)max(V.ranges[2 * t + 1] - V.ranges[2 * t], 0);
      order[atomicAdd(&hist[length_bucket(len)], 1u)] = V.item0 + t;
    }
  }
}

template <int P>
__global__ void __launch_bounds__(kTileThreads, P == 1 ? 4 : (P == 2 ? 4 : 2)) fwd_batch_kernel(ViewTable tab,
                                                                 uint32_t* __restrict__ queue,
                                                                 const int32_t* __restrict__ order) {
  __shared__ float4 s_rec[kTileThreads][kFwdVec4];
  __shared__ HitLists hl;
  __shared__ int s_item;
  while (true) {
    if (threadIdx.x == 0) {
      const int k = (int)atomicAdd(queue, 1u);
      s_item = k < tab.n_items ? order[k] : tab.n_items;
    }
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= tab.n_items) return;
    const ViewDev& V = tab.v[view_of(tab, item)];
    if (V.status && *V.status) continue;
    const int tile = item - V.item0;
    const TilePix<P> tp = tile_pixel<P>(tile, V.tiles_x, V.cfg.tile_w, V.cfg.tile_h);
    bool inside[P];
#pragma unroll
    for (int k = 0; k < P; ++k) inside[k] = tp.px < V.cam.width && tp.py + 4 * k < V.cam.height;
    const int tile_x0 = (tile % V.tiles_x) * V.cfg.tile_w;
    const int tile_y0 = (tile / V.tiles_x) * V.cfg.tile_h;
    const float xt = (float)tile_x0 + 0.5f - V.cam.cx, yt = (float)tile_y0 + 0.5f - V.cam.cy;
    FwdState st[P];
    const int start = V.ranges[2 * tile];
    fwd_tile<kFwdVec4, false, P>(V.proj, V.vals + start, start, V.ranges[2 * tile + 1], xt, yt,
                                 tile_x0, tile_y0, tp, inside, V.cam, V.cfg, s_rec, hl, nullptr,
                                 st);
#pragma unroll
    for (int k = 0; k < P; ++k) {
      if (!inside[k]) continue;
      const size_t p = (size_t)(tp.py + 4 * k) * V.cam.width + tp.px;
      V.rgb[3 * p] = st[k].C.x;
      V.rgb[3 * p + 1] = st[k].C.y;
      V.rgb[3 * p + 2] = st[k].C.z;
      V.depth[p] = st[k].D;
      V.normal[3 * p] = st[k].N.x;
      V.normal[3 * p + 1] = st[k].N.y;
      V.normal[3 * p + 2] = st[k].N.z;
      V.opac[p] = 1.f - st[k].T;
      V.T[p] = st[k].T;
      V.nlast[p] = st[k].last;
    }
  }
}

// Full backward of every view: persistent warps take (tile, region) work
// units (Q regions per tile, the same for every view of a launch) from an
// atomic counter, items in the heavy-first order; each unit is the
// single-view replay of bwd_warp.cuh.
__global__ void __launch_bounds__(kBwdWarps * 32, kBwdWarpBlocks) bwd_batch_kernel(
    ViewTable tab, int Q, uint32_t* __restrict__ queue, const int32_t* __restrict__ order) {
  __shared__ WarpBwdSmem<kBwdRegion> sm[kBwdWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_units = tab.n_items * Q;
  while (true) {
    uint32_t u = 0u;
    if (lane == 0) u = atomicAdd(queue, 1u);
    const int unit = (int)__shfl_sync(0xffffffffu, u, 0);
    if (unit >= n_units) return;
    const int slot = unit / Q, region = unit - slot * Q;
    const int item = order[slot];
    const ViewDev& V = tab.v[view_of(tab, item)];
    if (V.status && *V.status) continue;
    const int tile = item - V.item0;
    bwd_region<kBwdRegion>(V.proj, V.vals, V.emit, V.ranges[2 * tile], V.ranges[2 * tile + 1],
                           (tile % V.tiles_x) * V.cfg.tile_w, (tile / V.tiles_x) * V.cfg.tile_h,
                           region, Q, V.cam, V.cfg, V.T, V.nlast, V.d_rgb, V.d_depth, V.d_normal,
                           V.d_opac, V.partials, sm[warp]);
  }
}

__global__ void zero_words_kernel(uint32_t* p, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    p[i] = 0u;
}

namespace {

int view_tiles(const gs2d_view& w, int* tx) {
  *tx = gs2d_tiles_x(&w.cam, &w.cfg);
  return *tx * gs2d_tiles_y(&w.cam, &w.cfg);
}

int check_view(const gs2d_view& w) {
  if (w.cam.width <= 0 || w.cam.height <= 0) return GS2D_ERR_INVALID_ARG;
  if (!tile_cfg_ok(w.cfg)) return GS2D_ERR_INVALID_ARG;
  int tx;
  const long long nt = view_tiles(w, &tx);
  if (nt <= 0 || nt > 65535) return GS2D_ERR_INVALID_ARG;
  if (!w.proj || !w.bins.vals || !w.bins.tile_ranges || !w.bins.status) return GS2D_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(w.proj) & 15) return GS2D_ERR_INVALID_ARG;
  return GS2D_OK;
}

struct BatchWs {
  uint32_t* queue;        // [2] fwd, bwd work counters
  int32_t* order;         // [items] heavy-first work order
  float* partials[GS2D_MAX_VIEWS];
  float* pose_part;       // [max parts * 6]
  size_t bytes;
};

BatchWs carve_batch_ws(void* base, const gs2d_view* views, int n_views, int n) {
  Carver c(base);
  BatchWs w{};
  w.queue = c.take<uint32_t>(64);
  size_t items = 0;
  for (int v = 0; v < n_views; ++v) {
    int tx;
    items += (size_t)max(view_tiles(views[v], &tx), 0);
  }
  w.order = c.take<int32_t>(items > 0 ? items : 1);
  int max_parts = 1;
  for (int v = 0; v < n_views; ++v) {
    const size_t cap = views[v].bins.capacity > 0 ? views[v].bins.capacity : 1;
    w.partials[v] = c.take<float>(cap * bwd_regions(views[v].cfg) * 16);
    const int m = views[v].active ? views[v].n_active : n;
    max_parts = max(max_parts, (m + 255) / 256);
  }
  w.pose_part = c.take<float>((size_t)max_parts * 6);
  w.bytes = align_up(c.off, 256);
  return w;
}

int persistent_grid(const void* kernel, int threads = kTileThreads) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess)
    return 0;
  return sms * max(per_sm, 1);
}

int build_table(const gs2d_view* views, int n_views, const BatchWs* w, ViewTable* tab) {
  if (!views || n_views <= 0 || n_views > GS2D_MAX_VIEWS) return GS2D_ERR_INVALID_ARG;
  tab->n_views = n_views;
  int items = 0;
  for (int v = 0; v < n_views; ++v) {
    const gs2d_view& s = views[v];
    const int r = check_view(s);
    if (r) return r;
    // one persistent launch runs one pixels-per-thread variant
    if (s.cfg.px_per_thread != views[0].cfg.px_per_thread) return GS2D_ERR_INVALID_ARG;
    ViewDev& d = tab->v[v];
    d.cam = s.cam;
    d.cfg = s.cfg;
    d.n_tiles = view_tiles(s, &d.tiles_x);
    d.item0 = items;
    items += d.n_tiles;
    d.proj = reinterpret_cast<const float4*>(s.proj);
    d.vals = s.bins.vals;
    d.emit = s.bins.isect_emit;
    d.ranges = s.bins.tile_ranges;
    d.status = s.bins.status;
    d.rgb = s.rgb;
    d.depth = s.depth;
    d.normal = s.normal;
    d.opac = s.opacity;
    d.T = s.t_final;
    d.nlast = s.n_last;
    d.d_rgb = s.d_rgb;
    d.d_depth = s.d_depth;
    d.d_normal = s.d_normal;
    d.d_opac = s.d_opacity;
    d.partials = w ? w->partials[v] : nullptr;
  }
  tab->n_items = items;
  return GS2D_OK;
}

// Side streams of one device for the binning of up to kSideStreams views:
// each view's kernels go to its own non-blocking stream, forked from and
// joined back to the caller's stream by events (parallel branches when
// captured into a CUDA graph), so the stages of different views overlap.
// More views bin in one launch per stage (bin_sort_batch_launch): sharing
// streams, views would queue behind each other.  Created on the first
// batched binning call with several views on the device.
constexpr int kSideStreams = 8;
struct SidePool {
  bool ready = false;
  cudaStream_t s[kSideStreams];
  cudaEvent_t fork;
  cudaEvent_t join[kSideStreams];
};
std::mutex g_side_mu;
SidePool g_side[64];

SidePool* side_pool(int dev) {
  if (dev < 0 || dev >= 64) return nullptr;
  SidePool& P = g_side[dev];
  if (P.ready) return &P;
  for (int k = 0; k < kSideStreams; ++k) {
    if (cudaStreamCreateWithFlags(&P.s[k], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&P.join[k], cudaEventDisableTiming) != cudaSuccess) return nullptr;
  }
  if (cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  P.ready = true;
  return &P;
}

}  // namespace
}  // namespace gs2d

using namespace gs2d;

extern "C" {

size_t gs2d_bin_sort_batch_workspace(const gs2d_view* views, int n_views, int n) {
  return bin_sort_batch_bytes(views, n_views, n);
}

int gs2d_bin_sort_batch(const gs2d_view* views, int n_views, int n, void* workspace,
                        size_t ws_bytes, size_t* ws_needed, gs2d_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (!views || n_views <= 0 || n_views > GS2D_MAX_VIEWS || n < 0) return GS2D_ERR_INVALID_ARG;
  if (n_views > kSideStreams)
    return bin_sort_batch_launch(views, n_views, n, workspace, ws_bytes, ws_needed, st);
  // one view per side stream; the workspace layout is the batched launch's
  const size_t need = bin_sort_batch_bytes(views, n_views, n);
  if (need == 0) return GS2D_ERR_INVALID_ARG;
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  int dev = 0;
  GS2D_CUDA_TRY(cudaGetDevice(&dev));
  // one host thread at a time enqueues on a device's side streams
  std::lock_guard<std::mutex> lock(g_side_mu);
  SidePool* P = n_views > 1 ? side_pool(dev) : nullptr;
  if (n_views > 1 && !P) return GS2D_ERR_CUDA;
  if (P) {
    GS2D_CUDA_TRY(cudaEventRecord(P->fork, st));
    for (int k = 0; k < n_views; ++k) GS2D_CUDA_TRY(cudaStreamWaitEvent(P->s[k], P->fork, 0));
  }
  char* base = static_cast<char*>(workspace) + bin_sort_batch_header();
  int r = GS2D_OK;
  for (int v = 0; v < n_views && r == GS2D_OK; ++v) {
    const gs2d_view& w = views[v];
    const int m = w.active ? w.n_active : n;
    const size_t bytes = bin_sort_batch_view_bytes(m, w.bins.capacity);
    r = gs2d_bin_sort(w.proj, w.tiles_per_surfel, m, &w.cam, &w.cfg, base, bytes, nullptr, &w.bins,
                      (gs2d_stream)(P ? P->s[v] : st));
    base += bytes;
  }
  if (P)  // join every branch back, also after an error
    for (int k = 0; k < n_views; ++k) {
      GS2D_CUDA_TRY(cudaEventRecord(P->join[k], P->s[k]));
      GS2D_CUDA_TRY(cudaStreamWaitEvent(st, P->join[k], 0));
    }
  return r;
}

size_t gs2d_render_batch_workspace(const gs2d_view* views, int n_views, int n) {
  if (!views || n_views <= 0 || n_views > GS2D_MAX_VIEWS) return 0;
  return carve_batch_ws(nullptr, views, n_views, n).bytes;
}

int gs2d_render_fwd_batch(const gs2d_view* views, int n_views, void* workspace, size_t ws_bytes,
                          size_t* ws_needed, gs2d_stream stream) {
  ViewTable tab;
  int r = build_table(views, n_views, nullptr, &tab);
  if (r) return r;
  for (int v = 0; v < n_views; ++v)
    if (!views[v].rgb || !views[v].depth || !views[v].normal || !views[v].opacity ||
        !views[v].t_final || !views[v].n_last)
      return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_render_batch_workspace(views, n_views, 0);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const BatchWs w = carve_batch_ws(workspace, views, n_views, 0);
  zero_words_kernel<<<1, 64, 0, st>>>(w.queue, 2);
  GS2D_LAUNCH_CHECK();
  order_items_kernel<<<1, kOrderThreads, 0, st>>>(tab, w.order);
  GS2D_LAUNCH_CHECK();
  GS2D_DISPATCH_P(views[0].cfg.px_per_thread, {
    const int grid = min(persistent_grid(reinterpret_cast<const void*>(fwd_batch_kernel<P>)),
                         tab.n_items);
    if (grid <= 0) return GS2D_ERR_CUDA;
    fwd_batch_kernel<P><<<grid, kTileThreads, 0, st>>>(tab, w.queue, w.order);
  });
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int gs2d_render_bwd_batch(const gs2d_view* views, int n_views, const gs2d_surfels* s, float* d_mu,
                          float* d_quat, float* d_scale, float* d_opac, float* d_rgb,
                          void* workspace, size_t ws_bytes, size_t* ws_needed, gs2d_stream stream) {
  if (!s || !s->mu || !s->quat || !s->scale || s->n <= 0) return GS2D_ERR_INVALID_ARG;
  if (!d_mu || !d_quat || !d_scale || !d_opac || !d_rgb) return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_render_batch_workspace(views, n_views, s->n);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  const BatchWs w = carve_batch_ws(workspace, views, n_views, s->n);
  ViewTable tab;
  int r = build_table(views, n_views, &w, &tab);
  if (r) return r;
  for (int v = 0; v < n_views; ++v) {
    const gs2d_view& x = views[v];
    if (!x.t_final || !x.n_last || !x.d_rgb || !x.d_depth || !x.bins.isect_emit ||
        !x.bins.surfel_off || !x.tiles_per_surfel || !x.pose)
      return GS2D_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  zero_words_kernel<<<1, 64, 0, st>>>(w.queue, 2);
  GS2D_LAUNCH_CHECK();
  order_items_kernel<<<1, kOrderThreads, 0, st>>>(tab, w.order);
  GS2D_LAUNCH_CHECK();
  const int Q = bwd_regions(views[0].cfg);
  const int grid = min(persistent_grid(reinterpret_cast<const void*>(bwd_batch_kernel),
                                       kBwdWarps * 32),
                       (tab.n_items * Q + kBwdWarps - 1) / kBwdWarps);
  if (grid <= 0) return GS2D_ERR_CUDA;
  bwd_batch_kernel<<<grid, kBwdWarps * 32, 0, st>>>(tab, Q, w.queue + 1, w.order);
  GS2D_LAUNCH_CHECK();
  // surfels outside every view's subset receive zero: clear, then add view by view
  GS2D_CUDA_TRY(cudaMemsetAsync(d_mu, 0, sizeof(float) * 3 * s->n, st));
  GS2D_CUDA_TRY(cudaMemsetAsync(d_quat, 0, sizeof(float) * 4 * s->n, st));
  GS2D_CUDA_TRY(cudaMemsetAsync(d_scale, 0, sizeof(float) * 2 * s->n, st));
  GS2D_CUDA_TRY(cudaMemsetAsync(d_opac, 0, sizeof(float) * s->n, st));
  GS2D_CUDA_TRY(cudaMemsetAsync(d_rgb, 0, sizeof(float) * 3 * s->n, st));
  for (int v = 0; v < n_views; ++v) {
    const gs2d_view& x = views[v];
    const int m = x.active ? x.n_active : s->n;
    r = surfel_grad_launch(s, x.active, m, 1, x.pose, x.tiles_per_surfel, x.bins.surfel_off, Q,
                           x.proj, w.partials[v], d_mu, d_quat, d_scale, d_opac, d_rgb, w.pose_part,
                           x.bins.status, st);
    if (r) return r;
    if (x.d_pose6) {
      r = pose_reduce_launch(w.pose_part, (m + 255) / 256, x.d_pose6, x.bins.status, st);
      if (r) return r;
    }
  }
  return GS2D_OK;
}

}  // extern "C"
