// gs2d_bin_sort: tile binning and depth ordering of (tile, surfel) pairs
// (the per-tile depth ordering of the splats, Sec. III-A).
//
// Output order: by tile, then by the FP32 bit pattern of the surfel's centre
// depth mu_c.z (positive floats order like their bits), then by surfel id.
// A tile's list is short (hundreds of entries), so instead of a global depth
// sort the pairs are binned first and every tile sorts its own segment:
//   1. scan: per surfel (id order) its tile count k_i -> emission offset
//      (exclusive scan with decoupled look-back) and the total K; every
//      covered tile's counter is incremented;
//   2. tile scan: one block turns the tile counts into tile ranges;
//   3. scatter: every pair writes the 64-bit key (depth bits << 32 | id)
//      into its tile's segment at an atomically claimed slot (the order
//      inside a segment is arbitrary at this point);
//   4. tile sort: one block per tile sorts its segment by that key in shared
//      memory (bitonic network in its "flip" form, in which every comparator
//      puts the smaller key at the lower index, so a segment of any length
//      behaves as if padded with +inf), then writes the surfel ids, the
//      64-bit (tile, depth) keys and each pair's emission index.  Segments
//      longer than 2048 keys (dense views of large maps) go to a 1024-thread
//      block that sorts 16384-key chunks in shared memory and merges the
//      sorted runs in global memory.
// Because the key carries the id, the final order is unique and
// deterministic whatever order the atomics gave.  Emission index of the pair
// (surfel i, tile t) = surfel_off[i] + the row-major position of t in i's
// rectangle, so each surfel's pairs are contiguous in emission order (the
// backward pass stores its per-pair partials there).
#include <algorithm>
#include <mutex>

#include "gs2d_common.cuh"
#include "gs2d_internal.h"
#include "tile_scan.cuh"
#include "tile_sort.cuh"
#include "tile_walk.cuh"

namespace gs2d {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kChunk = kScanThreads * kScanItems;  // 4096 surfels per scan block
constexpr int kWarps = kScanThreads / 32;
constexpr int kSpinLimit = 1 << 22;                // default polls of a look-back wait
constexpr int kSortThreads = 256;
constexpr int kLongThreads = 1024;                 // long segments: one 1024-thread block
constexpr int kLongChunk = 16384;                  // keys per shared-memory chunk (128 KB)
constexpr size_t kSortBatchHeader = 256;           // batched binning: the scan's ticket

__device__ __forceinline__ unsigned long long ld_vol64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void st_vol64(unsigned long long* p, unsigned long long v) {
  *reinterpret_cast<volatile unsigned long long*>(p) = v;
}

// Exclusive scan over a 256-thread block; returns the exclusive prefix and
// writes the block total to *total (all threads).
__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t v, uint32_t* s_tmp, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_tmp[w] = inc;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t x = threadIdx.x < kWarps ? s_tmp[threadIdx.x] : 0u;
    uint32_t xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, xi, o);
      if (threadIdx.x >= o) xi += t;
    }
    if (threadIdx.x < kWarps) s_tmp[kWarps + threadIdx.x] = xi - x;
    if (threadIdx.x == kWarps - 1) s_tmp[2 * kWarps] = xi;
  }
  __syncthreads();
  const uint32_t r = s_tmp[kWarps + w] + inc - v;
  *total = s_tmp[2 * kWarps];
  __syncthreads();
  return r;
}

// Zeroes the per-call counters (tile counts and cursors, scan words, K).
__global__ void bin_init_kernel(uint32_t* __restrict__ zero_a, size_t n_a,
                                int32_t* __restrict__ n_isect, const int32_t* __restrict__ gate) {
  if (*gate) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_a; i += stride) zero_a[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_isect = 0;
}

// Per-block tile histograms live in shared memory when the tile grid fits.
constexpr int kSmemTiles = 6144;  // 2 x 24 KB: the scatter's histogram + bases
// dynamic shared memory the scatter kernel may take without raising its
// limit: 48 KB less its static arrays (s_walk, s_key: 6 KB)
constexpr size_t kScatterDefaultSmem = 48 * 1024 - 6 * 1024;

// 1a. Tile counts: every covered tile's counter is incremented, through a
// per-block shared-memory histogram (one global atomic per block and tile).
// Block vblock of vgrid (a view's share of a batched launch, or the grid).
__device__ __forceinline__ void count_body(const float4* __restrict__ proj,
                                           const int32_t* __restrict__ tiles, int n, int tiles_x,
                                           int n_tiles, uint32_t* __restrict__ tile_count,
                                           int vblock, int vgrid, uint32_t* s_hist,
                                           WalkScratch* s_walk) {
  const bool local = n_tiles <= kSmemTiles;
  if (local)
    for (int t = threadIdx.x; t < n_tiles; t += kScanThreads) s_hist[t] = 0u;
  __syncthreads();
  const int stride = vgrid * kScanThreads;
  // block-uniform trip count: every lane takes part in each warp walk
  for (int base = vblock * kScanThreads; base < n; base += stride) {
    const int i = base + (int)threadIdx.x;
    const int k = i < n ? max(tiles[i], 0) : 0;
    Rect r{1, 1, 0, 0};
    if (k > 0) r = load_rect(proj, (uint32_t)i);
    warp_tile_walk(k, r.tx0, r.ty0, r.tx1, tiles_x, n_tiles, s_walk[threadIdx.x >> 5],
                   [&](int, int t) { atomicAdd(local ? s_hist + t : tile_count + t, 1u); });
  }
  if (!local) return;
  __syncthreads();
  for (int t = threadIdx.x; t < n_tiles; t += kScanThreads)
    if (s_hist[t]) atomicAdd(tile_count + t, s_hist[t]);
}

__global__ void __launch_bounds__(kScanThreads) count_kernel(
    const float4* __restrict__ proj, const int32_t* __restrict__ tiles, int n, int tiles_x,
    int n_tiles, uint32_t* __restrict__ tile_count, const int32_t* __restrict__ gate) {
  extern __shared__ uint32_t s_hist[];
  __shared__ WalkScratch s_walk[kScanThreads / 32];
  if (*gate) return;
  count_body(proj, tiles, n, tiles_x, n_tiles, tile_count, blockIdx.x, gridDim.x, s_hist, s_walk);
}

// 1b. Exclusive scan of k_i over surfel ids with decoupled look-back (64-bit
// chunk words: flag in bits 62-63; a warp examines 32 predecessors at a
// time; the spin is bounded by spin_limit polls and past it records
// GS2D_ERR_TIMEOUT, takes the missing sums as zero and finishes, so every
// write stays in bounds and later kernels skip): the emission offsets
// surfel_off[i].  The chunk numbered `withheld` (a test of that path; -1 =
// none) never publishes its word, so its successor's wait runs out.
constexpr unsigned long long kF64Agg = 1ull << 62, kF64Inc = 2ull << 62,
                             kV64Mask = (1ull << 62) - 1;
struct ScanSmem {
  uint32_t k[kChunk];
  uint32_t tmp[2 * kWarps + 1];
  unsigned long long prefix;
};

// Chunk `chunk` of one view's scan; every chunk before it in that view was
// handed to a block that started earlier (tickets in chunk order).
__device__ __forceinline__ void emit_scan_body(const int32_t* __restrict__ tiles, int n,
                                               uint32_t* __restrict__ surfel_off,
                                               unsigned long long* __restrict__ chunk_status,
                                               int chunk, int32_t* __restrict__ gate,
                                               int spin_limit, int withheld, ScanSmem& sm) {
  uint32_t* s_k = sm.k;
  uint32_t* s_tmp = sm.tmp;
  const long long base = (long long)chunk * kChunk;
  if (base >= n) return;
  const int count = (int)min((long long)kChunk, (long long)n - base);
  for (int i = threadIdx.x; i < count; i += kScanThreads) s_k[i] = (uint32_t)max(tiles[base + i], 0);
  __syncthreads();
  // blocked: thread t owns items t*16 .. t*16+15
  uint32_t sum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int i = threadIdx.x * kScanItems + j;
    sum += i < count ? s_k[i] : 0u;
  }
  uint32_t btotal;
  const uint32_t excl = block_excl_scan256(sum, s_tmp, &btotal);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    unsigned long long* my = chunk_status + chunk;
    const bool publish = chunk != withheld;
    unsigned long long prefix = 0;
    if (chunk == 0) {
      if (lane == 0 && publish) st_vol64(my, kF64Inc | (unsigned long long)btotal);
    } else {
      if (lane == 0 && publish) st_vol64(my, kF64Agg | (unsigned long long)btotal);
      int hi = chunk - 1;
      int spins = 0;
      while (true) {
        const int p = hi - lane;
        unsigned long long sv = p >= 0 ? ld_vol64(chunk_status + p) : kF64Inc;
        uint32_t inc_mask, need_mask;
        while (true) {
          inc_mask = __ballot_sync(0xffffffffu, (sv & ~kV64Mask) == kF64Inc);
          // lanes up to and including the nearest inclusive predecessor
          need_mask = inc_mask ? (0xffffffffu >> (31 - (__ffs(inc_mask) - 1))) : 0xffffffffu;
          const uint32_t missing = __ballot_sync(0xffffffffu, (sv & ~kV64Mask) == 0ull) & need_mask;
          if (!missing) break;
          if (++spins > spin_limit) {
            if (lane == 0) atomicExch(gate, (int32_t)GS2D_ERR_TIMEOUT);
            if ((sv & ~kV64Mask) == 0ull) sv = kF64Inc;
            inc_mask = __ballot_sync(0xffffffffu, (sv & ~kV64Mask) == kF64Inc);
            need_mask = 0xffffffffu >> (31 - (__ffs(inc_mask) - 1));
            break;
          }
          __nanosleep(32);
          if ((sv & ~kV64Mask) == 0ull && p >= 0) sv = ld_vol64(chunk_status + p);
        }
        unsigned long long v = ((need_mask >> lane) & 1u) ? (sv & kV64Mask) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        prefix += v;
        if (inc_mask) break;
        hi -= 32;
      }
      if (lane == 0 && publish) st_vol64(my, kF64Inc | ((prefix + btotal) & kV64Mask));
    }
    if (lane == 0) sm.prefix = prefix;
  }
  __syncthreads();
  unsigned long long off = sm.prefix + excl;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int i = threadIdx.x * kScanItems + j;
    if (i < count) {
      surfel_off[base + i] = (uint32_t)min(off, 0xFFFFFFFFull);
      off += s_k[i];
    }
  }
}

__global__ void __launch_bounds__(kScanThreads) emit_scan_kernel(
    const int32_t* __restrict__ tiles, int n, uint32_t* __restrict__ surfel_off,
    unsigned long long* __restrict__ chunk_status, uint32_t* __restrict__ ticket,
    int32_t* __restrict__ gate, int spin_limit, int withheld) {
  __shared__ ScanSmem sm;
  __shared__ int s_chunk;
  if (*gate) return;
  if (threadIdx.x == 0) s_chunk = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  emit_scan_body(tiles, n, surfel_off, chunk_status, s_chunk, gate, spin_limit, withheld, sm);
}

// 2. Tile ranges from the tile counts (one block), K and the capacity check.
__global__ void __launch_bounds__(1024) tile_scan_kernel(const uint32_t* __restrict__ tile_count,
                                                        int n_tiles, int32_t* __restrict__ ranges,
                                                        int32_t* __restrict__ n_isect,
                                                        long long capacity,
                                                        uint32_t* __restrict__ long_list,
                                                        uint32_t* __restrict__ n_long,
                                                        int32_t* __restrict__ gate) {
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_carry;
  if (*gate) return;
  tile_scan_block(tile_count, n_tiles, ranges, n_isect, capacity, long_list, n_long, kSegSmem, gate,
                  s_w, &s_carry);
}

// 3. Scatter of the (depth bits << 32 | id) keys into the tile segments.
// A block counts its own pairs per tile in shared memory, claims one run of
// slots per tile with a single global atomic, and hands the slots out with
// shared-memory atomics; both passes walk the warp's pairs cooperatively
// (warp_tile_walk).
// Block vblock of a view (surfels 256 vblock .. + 255).
__device__ __forceinline__ void scatter_body(
    const float4* __restrict__ proj, const int32_t* __restrict__ tiles, int n, int tiles_x,
    int n_tiles, const int32_t* __restrict__ ranges, uint32_t* __restrict__ cursor,
    unsigned long long* __restrict__ seg_keys, long long capacity, int vblock, uint32_t* s_cnt,
    WalkScratch* s_walk, unsigned long long* s_key) {
  const bool local = n_tiles <= kSmemTiles;
  uint32_t* s_base = s_cnt + (local ? n_tiles : 0);
  if (local)
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) s_cnt[t] = 0u;
  __syncthreads();
  const int i = vblock * blockDim.x + threadIdx.x;
  const int k = i < n ? tiles[i] : 0;
  Rect r{1, 1, 0, 0};
  unsigned long long key = 0ull;
  if (k > 0) {
    r = load_rect(proj, (uint32_t)i);
    const uint32_t db = __float_as_uint(proj[(size_t)i * (kProjFloats / 4) + 6].z);
    key = ((unsigned long long)db << 32) | (uint32_t)i;
  }
  s_key[threadIdx.x] = key;
  WalkScratch& ws = s_walk[threadIdx.x >> 5];
  const unsigned long long* wkey = s_key + (threadIdx.x & ~31);
  const int kk = max(k, 0);
  if (local) {
    warp_tile_walk(kk, r.tx0, r.ty0, r.tx1, tiles_x, n_tiles, ws,
                   [&](int, int t) { atomicAdd(s_cnt + t, 1u); });
    __syncthreads();
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) {
      const uint32_t c = s_cnt[t];
      s_base[t] = c ? (uint32_t)ranges[2 * t] + atomicAdd(cursor + t, c) : 0u;
    }
    __syncthreads();
  } else {
    __syncwarp();
  }
  warp_tile_walk(kk, r.tx0, r.ty0, r.tx1, tiles_x, n_tiles, ws, [&](int owner, int t) {
    const long long pos = local ? (long long)atomicAdd(s_base + t, 1u)
                                : (long long)ranges[2 * t] + atomicAdd(cursor + t, 1u);
    if (pos < min((long long)ranges[2 * t + 1], capacity)) seg_keys[pos] = wkey[owner];
  });
}

__global__ void __launch_bounds__(256) scatter_kernel(
    const float4* __restrict__ proj, const int32_t* __restrict__ tiles, int n, int tiles_x,
    int n_tiles, const int32_t* __restrict__ ranges, uint32_t* __restrict__ cursor,
    unsigned long long* __restrict__ seg_keys, long long capacity,
    const int32_t* __restrict__ gate) {
  extern __shared__ uint32_t s_cnt[];  // [n_tiles] counts, then [n_tiles] bases
  __shared__ WalkScratch s_walk[8];
  __shared__ unsigned long long s_key[256];
  if (*gate) return;
  scatter_body(proj, tiles, n, tiles_x, n_tiles, ranges, cursor, seg_keys, capacity, blockIdx.x,
               s_cnt, s_walk, s_key);
}

// Tile t's segment (sorted here when at most kSegSmem keys, or with
// long_here any length).
__device__ __forceinline__ void tile_sort_body(
    int t, const float4* __restrict__ proj, int n, int tiles_x, const int32_t* __restrict__ ranges,
    unsigned long long* __restrict__ seg_keys, unsigned long long* __restrict__ seg_tmp,
    const uint32_t* __restrict__ surfel_off, uint32_t* __restrict__ vals,
    uint32_t* __restrict__ emit, unsigned long long* __restrict__ keys64, long long capacity,
    int long_here, unsigned long long* s_keys) {
  const int start = ranges[2 * t];
  const int end = (int)min((long long)ranges[2 * t + 1], capacity);
  const int len = end - start;
  if (len <= 0) return;
  if (len > kSegSmem) {
    // a long segment in this block (2048-key chunks + merges) when no
    // separate long-segment launch follows
    if (long_here)
      sort_long_segment<kSegSmem>(t, proj, n, tiles_x, ranges, seg_keys, seg_tmp, surfel_off, vals,
                                  emit, keys64, capacity, s_keys);
    return;
  }
  for (int i = threadIdx.x; i < len; i += blockDim.x) s_keys[i] = seg_keys[start + i];
  __syncthreads();
  bitonic_sort(s_keys, len);
  write_outputs(s_keys, len, start, t, tiles_x, n, proj, surfel_off, vals, emit, keys64);
}

// Segments of at most kSegSmem keys: sorted in shared memory by 256 threads (and,
// with long_here, longer ones too).
__global__ void __launch_bounds__(kSortThreads) tile_sort_kernel(
    const float4* __restrict__ proj, int n, int tiles_x, const int32_t* __restrict__ ranges,
    unsigned long long* __restrict__ seg_keys, unsigned long long* __restrict__ seg_tmp,
    const uint32_t* __restrict__ surfel_off, uint32_t* __restrict__ vals,
    uint32_t* __restrict__ emit, unsigned long long* __restrict__ keys64, long long capacity,
    int long_here, const int32_t* __restrict__ gate) {
  extern __shared__ unsigned long long s_keys[];
  if (*gate) return;
  tile_sort_body(blockIdx.x, proj, n, tiles_x, ranges, seg_keys, seg_tmp, surfel_off, vals, emit,
                 keys64, capacity, long_here, s_keys);
}

// Segments longer than kSegSmem, listed by the tile scan: a small persistent
// grid takes them one per block.
__global__ void __launch_bounds__(kLongThreads) tile_sort_long_kernel(
    const float4* __restrict__ proj, int n, int tiles_x, const int32_t* __restrict__ ranges,
    const uint32_t* __restrict__ long_list, const uint32_t* __restrict__ n_long,
    unsigned long long* __restrict__ seg_keys, unsigned long long* __restrict__ seg_tmp,
    const uint32_t* __restrict__ surfel_off, uint32_t* __restrict__ vals, uint32_t* __restrict__ emit,
    unsigned long long* __restrict__ keys64, long long capacity, const int32_t* __restrict__ gate) {
  extern __shared__ unsigned long long s_keys[];
  if (*gate) return;
  const int cnt = (int)*n_long;
  for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
    sort_long_segment<kLongChunk>((int)long_list[i], proj, n, tiles_x, ranges, seg_keys, seg_tmp,
                                  surfel_off, vals, emit, keys64, capacity, s_keys);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Several views in one launch per stage (gs2d_bin_sort_batch): each view keeps
// its own workspace region, counters and status word; a stage's blocks are
// split over the views by the offsets in the table, and the emission scan's
// chunks take tickets from one counter in view-major order, so every chunk's
// predecessors in its view started earlier (the look-back's condition).
struct SortViewDev {
  const float4* proj;
  const int32_t* tiles;
  int n, tiles_x, n_tiles;
  uint32_t* zero_begin;
  size_t zero_words;
  uint32_t *tile_count, *cursor, *n_long, *long_list;
  unsigned long long *estatus, *seg_keys, *seg_tmp;
  int32_t *ranges, *n_isect;
  uint32_t *surfel_off, *vals, *emit;
  unsigned long long* keys64;
  long long capacity;
  int32_t* gate;
  int count0, count_blocks, chunk0, scatter0, tile0;
};
struct SortTable {
  int n_views, count_total, chunk_total, scatter_total, tile_total;
  SortViewDev v[GS2D_MAX_VIEWS];
};

// The view whose share of a stage's blocks holds block b.
__device__ __forceinline__ int sort_view_of(const SortTable& T, int b, int SortViewDev::*first) {
  int v = 0;
  while (v + 1 < T.n_views && b >= T.v[v + 1].*first) ++v;
  return v;
}

__global__ void bin_init_batch_kernel(const SortTable T, uint32_t* __restrict__ batch_ticket) {
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *batch_ticket = 0u;
  const SortViewDev& V = T.v[blockIdx.y];
  if (*V.gate) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < V.zero_words; i += stride)
    V.zero_begin[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) *V.n_isect = 0;
}

__global__ void __launch_bounds__(kScanThreads) count_batch_kernel(const SortTable T) {
  extern __shared__ uint32_t s_hist[];
  __shared__ WalkScratch s_walk[kScanThreads / 32];
  const SortViewDev& V = T.v[sort_view_of(T, blockIdx.x, &SortViewDev::count0)];
  if (*V.gate) return;
  count_body(V.proj, V.tiles, V.n, V.tiles_x, V.n_tiles, V.tile_count, blockIdx.x - V.count0,
             V.count_blocks, s_hist, s_walk);
}

__global__ void __launch_bounds__(kScanThreads) emit_scan_batch_kernel(
    const SortTable T, uint32_t* __restrict__ batch_ticket, int spin_limit, int withheld) {
  __shared__ ScanSmem sm;
  __shared__ int s_t;
  if (threadIdx.x == 0) s_t = (int)atomicAdd(batch_ticket, 1u);
  __syncthreads();
  const int t = s_t;
  if (t >= T.chunk_total) return;
  const SortViewDev& V = T.v[sort_view_of(T, t, &SortViewDev::chunk0)];
  if (*V.gate) return;
  emit_scan_body(V.tiles, V.n, V.surfel_off, V.estatus, t - V.chunk0, V.gate, spin_limit,
                 withheld, sm);
}

__global__ void __launch_bounds__(1024) tile_scan_batch_kernel(const SortTable T) {
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_carry;
  const SortViewDev& V = T.v[blockIdx.x];
  if (*V.gate) return;
  tile_scan_block(V.tile_count, V.n_tiles, V.ranges, V.n_isect, V.capacity, V.long_list,
                  V.n_long, kSegSmem, V.gate, s_w, &s_carry);
}

__global__ void __launch_bounds__(256) scatter_batch_kernel(const SortTable T) {
  extern __shared__ uint32_t s_cnt[];
  __shared__ WalkScratch s_walk[8];
  __shared__ unsigned long long s_key[256];
  const SortViewDev& V = T.v[sort_view_of(T, blockIdx.x, &SortViewDev::scatter0)];
  if (*V.gate) return;
  scatter_body(V.proj, V.tiles, V.n, V.tiles_x, V.n_tiles, V.ranges, V.cursor, V.seg_keys,
               V.capacity, blockIdx.x - V.scatter0, s_cnt, s_walk, s_key);
}

__global__ void __launch_bounds__(kSortThreads) tile_sort_batch_kernel(const SortTable T) {
  extern __shared__ unsigned long long s_keys[];
  const SortViewDev& V = T.v[sort_view_of(T, blockIdx.x, &SortViewDev::tile0)];
  if (*V.gate) return;
  tile_sort_body(blockIdx.x - V.tile0, V.proj, V.n, V.tiles_x, V.ranges, V.seg_keys, V.seg_tmp,
                 V.surfel_off, V.vals, V.emit, V.keys64, V.capacity, 0, s_keys);
}

// Every view's segments longer than kSegSmem, numbered across the views
// (view-major) and taken one per block of a small grid in that numbering.
__global__ void __launch_bounds__(kLongThreads) tile_sort_long_batch_kernel(const SortTable T) {
  extern __shared__ unsigned long long s_keys[];
  __shared__ int s_first[GS2D_MAX_VIEWS + 1];
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int v = 0; v < T.n_views; ++v) {
      s_first[v] = acc;
      acc += *T.v[v].gate ? 0 : (int)*T.v[v].n_long;
    }
    s_first[T.n_views] = acc;
  }
  __syncthreads();
  const int total = s_first[T.n_views];
  int v = 0;
  for (int g = blockIdx.x; g < total; g += gridDim.x) {
    while (g >= s_first[v + 1]) ++v;
    const SortViewDev& V = T.v[v];
    sort_long_segment<kLongChunk>((int)V.long_list[g - s_first[v]], V.proj, V.n, V.tiles_x,
                                  V.ranges, V.seg_keys, V.seg_tmp, V.surfel_off, V.vals, V.emit,
                                  V.keys64, V.capacity, s_keys);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// workspace layout
struct SortWs {
  unsigned long long* seg_keys;  // [cap]
  unsigned long long* seg_tmp;   // [cap] merge buffer of long segments
  uint32_t* long_list;           // [n_tiles] tiles with segments over kSegSmem
  uint32_t* n_long;              // [1] (zeroed per call)
  uint32_t* proj_done;           // [1] blocks of a fused projection finished (zeroed per call)
  uint32_t* grid_bar;            // [1] grid barrier of a projection with fused scatter (zeroed)
  uint32_t* zero_begin;          // start of the zeroed region
  uint32_t* tile_count;          // [n_tiles]
  uint32_t* cursor;              // [n_tiles]
  uint32_t* ticket;              // [8]
  unsigned long long* estatus;   // [chunks_n]
  size_t zero_words;
  size_t bytes;
  int chunks_n;
};

SortWs carve_sort_ws(void* base, int n, size_t cap, int n_tiles) {
  SortWs w{};
  Carver c(base);
  const size_t nn = (size_t)(n > 0 ? n : 1);
  w.chunks_n = (int)((nn + kChunk - 1) / kChunk);
  w.seg_keys = c.take<unsigned long long>(cap > 0 ? cap : 1);
  w.seg_tmp = c.take<unsigned long long>(cap > 0 ? cap : 1);
  w.long_list = c.take<uint32_t>((size_t)(n_tiles > 0 ? n_tiles : 1));
  c.off = align_up(c.off, 256);
  const size_t zstart = c.off;
  w.zero_begin = base ? reinterpret_cast<uint32_t*>(static_cast<char*>(base) + zstart) : nullptr;
  size_t words = 0;
  auto zt = [&](size_t cnt) {
    uint32_t* p = base ? w.zero_begin + words : nullptr;
    words += (cnt + 63) / 64 * 64;
    return p;
  };
  w.tile_count = zt((size_t)n_tiles);
  w.cursor = zt((size_t)n_tiles);
  w.ticket = zt(8);
  w.n_long = zt(1);
  w.proj_done = zt(1);
  w.grid_bar = zt(1);
  w.estatus = reinterpret_cast<unsigned long long*>(zt((size_t)2 * w.chunks_n + 2));
  w.zero_words = words;
  w.bytes = align_up(zstart + words * sizeof(uint32_t), 256);
  return w;
}

// Look-back wait settings (gs2d_set_lookback_wait).
int g_lookback_spins = 0;
int g_lookback_withheld = -1;

// The long-segment kernel's dynamic shared memory exceeds the 48 KB default:
// raise its limit once per device (before any stream capture that bins).
cudaError_t long_sort_smem_ready(size_t bytes) {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(tile_sort_long_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

SortFuse sort_fuse_args(void* workspace, int n, const gs2d_bins* bins, int tiles_x, int n_tiles) {
  const SortWs w = carve_sort_ws(workspace, n, bins->capacity, n_tiles);
  SortFuse f;
  f.tile_count = w.tile_count;
  f.ranges = bins->tile_ranges;
  f.n_isect = bins->n_isect;
  f.capacity = (long long)bins->capacity;
  f.long_list = w.long_list;
  f.n_long = w.n_long;
  f.done = w.proj_done;
  f.tiles_x = tiles_x;
  f.n_tiles = n_tiles;
  f.long_len = kSegSmem;
  f.order = nullptr;
  f.seg_keys = nullptr;  // the caller opts in to the fused scatter
  f.cursor = w.cursor;
  f.bar = w.grid_bar;
  return f;
}

void sort_seg_args(void* workspace, int n, size_t capacity, int n_tiles,
                   unsigned long long** seg_keys, unsigned long long** seg_tmp) {
  const SortWs w = carve_sort_ws(workspace, n, capacity, n_tiles);
  *seg_keys = w.seg_keys;
  *seg_tmp = w.seg_tmp;
}

void sort_zero_region(void* workspace, int n, size_t capacity, int n_tiles, uint32_t** begin,
                      size_t* words) {
  const SortWs w = carve_sort_ws(workspace, n, capacity, n_tiles);
  *begin = w.zero_begin;
  *words = w.zero_words;
}

// Raises a kernel's dynamic shared-memory limit once per device.
cudaError_t smem_limit_ready(const void* fn, int bytes, bool* done_per_dev) {
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && done_per_dev[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done_per_dev[dev] = true;
  return e;
}

int bin_sort_launch(const float* proj, const int32_t* tiles_per_surfel, int n,
                    const gs2d_camera* cam, const gs2d_config* cfg, void* workspace,
                    size_t ws_bytes, size_t* ws_needed, const gs2d_bins* bins, bool need_emit,
                    cudaStream_t st, unsigned flags) {
  if (!cam || !cfg || !bins || n < 0) return GS2D_ERR_INVALID_ARG;
  if (n > 0 && (!proj || !tiles_per_surfel)) return GS2D_ERR_INVALID_ARG;
  if (!bins->vals || !bins->tile_ranges || !bins->n_isect || !bins->status) return GS2D_ERR_INVALID_ARG;
  if (need_emit && (!bins->isect_emit || !bins->surfel_off)) return GS2D_ERR_INVALID_ARG;
  if (bins->capacity >= (size_t)0x7FFFFFFF) return GS2D_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(proj) & 15) return GS2D_ERR_INVALID_ARG;
  if (cfg->tile_w <= 0 || cfg->tile_h <= 0) return GS2D_ERR_INVALID_ARG;
  const int tx = gs2d_tiles_x(cam, cfg), ty = gs2d_tiles_y(cam, cfg);
  if (tx <= 0 || ty <= 0 || (long long)tx * ty > 65535) return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_bin_sort_workspace(n, bins->capacity);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  const int n_tiles = tx * ty;
  const SortWs w = carve_sort_ws(workspace, n, bins->capacity, n_tiles);
  int32_t* gate = bins->status;
  const long long cap = (long long)bins->capacity;
  const float4* p4 = reinterpret_cast<const float4*>(proj);
  const size_t hist_smem = n_tiles <= kSmemTiles ? (size_t)n_tiles * sizeof(uint32_t) : 0;

  if (!(flags & kSortPreZeroed)) {
    bin_init_kernel<<<32, 256, 0, st>>>(w.zero_begin, w.zero_words, bins->n_isect, gate);
    GS2D_LAUNCH_CHECK();
  }
  const bool scanned = (flags & kSortPreScanned) != 0;
  if (n > 0 && !scanned) {
    const int blocks = min((n + kScanThreads - 1) / kScanThreads, 152 * 4);
    count_kernel<<<blocks, kScanThreads, hist_smem, st>>>(p4, tiles_per_surfel, n, tx, n_tiles,
                                                          w.tile_count, gate);
    GS2D_LAUNCH_CHECK();
    if (need_emit) {
      emit_scan_kernel<<<w.chunks_n, kScanThreads, 0, st>>>(
          tiles_per_surfel, n, bins->surfel_off, w.estatus, w.ticket, gate,
          g_lookback_spins > 0 ? g_lookback_spins : kSpinLimit, g_lookback_withheld);
      GS2D_LAUNCH_CHECK();
    }
  }
  if (!scanned) {
    tile_scan_kernel<<<1, 1024, 0, st>>>(w.tile_count, n_tiles, bins->tile_ranges, bins->n_isect,
                                         cap, w.long_list, w.n_long, gate);
    GS2D_LAUNCH_CHECK();
  }
  if (n == 0) return GS2D_OK;
  // two shared-memory histograms of more than ~5.4k tiles and the kernel's
  // static arrays exceed the default 48 KB per block: raise the limit once
  // per device (grids that fit never make the call, so captures of them are
  // unaffected)
  static bool scatter_ready[64] = {};
  if (2 * hist_smem > kScatterDefaultSmem &&
      smem_limit_ready(reinterpret_cast<const void*>(scatter_kernel), 2 * kSmemTiles * 4,
                       scatter_ready) != cudaSuccess)
    return GS2D_ERR_CUDA;
  scatter_kernel<<<(n + 255) / 256, 256, 2 * hist_smem, st>>>(
      p4, tiles_per_surfel, n, tx, n_tiles, bins->tile_ranges, w.cursor, w.seg_keys, cap, gate);
  GS2D_LAUNCH_CHECK();
  if (flags & kSortInTileKernel) return GS2D_OK;
  const size_t smem = (size_t)kSegSmem * sizeof(unsigned long long);
  const bool long_here = (flags & kSortLongInBlock) != 0;
  tile_sort_kernel<<<n_tiles, kSortThreads, smem, st>>>(
      p4, n, tx, bins->tile_ranges, w.seg_keys, w.seg_tmp, need_emit ? bins->surfel_off : nullptr,
      bins->vals, need_emit ? bins->isect_emit : nullptr,
      reinterpret_cast<unsigned long long*>(bins->keys), cap, long_here ? 1 : 0, gate);
  GS2D_LAUNCH_CHECK();
  if (!long_here) {
    // segments longer than kSegSmem (blocks of shorter ones return at once)
    const size_t long_smem = (size_t)kLongChunk * sizeof(unsigned long long);
    if (long_sort_smem_ready(long_smem) != cudaSuccess) return GS2D_ERR_CUDA;
    tile_sort_long_kernel<<<min(n_tiles, 152), kLongThreads, long_smem, st>>>(
        p4, n, tx, bins->tile_ranges, w.long_list, w.n_long, w.seg_keys, w.seg_tmp,
        need_emit ? bins->surfel_off : nullptr, bins->vals, need_emit ? bins->isect_emit : nullptr,
        reinterpret_cast<unsigned long long*>(bins->keys), cap, gate);
    GS2D_LAUNCH_CHECK();
  }
  return GS2D_OK;
}

size_t bin_sort_batch_view_bytes(int m, size_t capacity) {
  return align_up(gs2d_bin_sort_workspace(m, capacity), 256);
}

size_t bin_sort_batch_header() { return kSortBatchHeader; }

size_t bin_sort_batch_bytes(const gs2d_view* views, int n_views, int n) {
  if (!views || n_views <= 0 || n_views > GS2D_MAX_VIEWS || n < 0) return 0;
  size_t total = kSortBatchHeader;
  for (int v = 0; v < n_views; ++v) {
    const int m = views[v].active ? views[v].n_active : n;
    if (m < 0) return 0;
    total += bin_sort_batch_view_bytes(m, views[v].bins.capacity);
  }
  return total;
}

int bin_sort_batch_launch(const gs2d_view* views, int n_views, int n, void* workspace,
                          size_t ws_bytes, size_t* ws_needed, cudaStream_t st) {
  if (!views || n_views <= 0 || n_views > GS2D_MAX_VIEWS || n < 0) return GS2D_ERR_INVALID_ARG;
  const size_t need = bin_sort_batch_bytes(views, n_views, n);
  if (need == 0) return GS2D_ERR_INVALID_ARG;
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  SortTable T;
  T.n_views = n_views;
  T.count_total = T.chunk_total = T.scatter_total = T.tile_total = 0;
  size_t count_smem = 0, scatter_smem = 0;
  char* base = static_cast<char*>(workspace) + kSortBatchHeader;
  for (int v = 0; v < n_views; ++v) {
    const gs2d_view& x = views[v];
    const gs2d_bins* bins = &x.bins;
    const int m = x.active ? x.n_active : n;
    // the checks of bin_sort_launch, per view
    if (m > 0 && (!x.proj || !x.tiles_per_surfel)) return GS2D_ERR_INVALID_ARG;
    if (!bins->vals || !bins->tile_ranges || !bins->n_isect || !bins->status)
      return GS2D_ERR_INVALID_ARG;
    const bool emit = bins->isect_emit || bins->surfel_off;
    if (emit && (!bins->isect_emit || !bins->surfel_off)) return GS2D_ERR_INVALID_ARG;
    if (bins->capacity >= (size_t)0x7FFFFFFF) return GS2D_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(x.proj) & 15) return GS2D_ERR_INVALID_ARG;
    if (x.cfg.tile_w <= 0 || x.cfg.tile_h <= 0) return GS2D_ERR_INVALID_ARG;
    const int tx = gs2d_tiles_x(&x.cam, &x.cfg), ty = gs2d_tiles_y(&x.cam, &x.cfg);
    if (tx <= 0 || ty <= 0 || (long long)tx * ty > 65535) return GS2D_ERR_INVALID_ARG;
    const int n_tiles = tx * ty;
    const size_t bytes = bin_sort_batch_view_bytes(m, bins->capacity);
    const SortWs w = carve_sort_ws(base, m, bins->capacity, n_tiles);
    base += bytes;
    SortViewDev& d = T.v[v];
    d.proj = reinterpret_cast<const float4*>(x.proj);
    d.tiles = x.tiles_per_surfel;
    d.n = m;
    d.tiles_x = tx;
    d.n_tiles = n_tiles;
    d.zero_begin = w.zero_begin;
    d.zero_words = w.zero_words;
    d.tile_count = w.tile_count;
    d.cursor = w.cursor;
    d.n_long = w.n_long;
    d.long_list = w.long_list;
    d.estatus = w.estatus;
    d.seg_keys = w.seg_keys;
    d.seg_tmp = w.seg_tmp;
    d.ranges = bins->tile_ranges;
    d.n_isect = bins->n_isect;
    d.surfel_off = emit ? bins->surfel_off : nullptr;
    d.vals = bins->vals;
    d.emit = emit ? bins->isect_emit : nullptr;
    d.keys64 = reinterpret_cast<unsigned long long*>(bins->keys);
    d.capacity = (long long)bins->capacity;
    d.gate = bins->status;
    // the single-view launch shapes but for the counts (at most 152 blocks
    // per view, fewer per-block histograms to flush): a scan block per 4096
    // surfels, a scatter block per 256, a sort block per tile
    d.count0 = T.count_total;
    d.count_blocks = m > 0 ? min((m + kScanThreads - 1) / kScanThreads, 152) : 0;
    T.count_total += d.count_blocks;
    d.chunk0 = T.chunk_total;
    T.chunk_total += (m > 0 && emit) ? w.chunks_n : 0;
    d.scatter0 = T.scatter_total;
    T.scatter_total += m > 0 ? (m + 255) / 256 : 0;
    d.tile0 = T.tile_total;
    T.tile_total += m > 0 ? n_tiles : 0;
    if (n_tiles <= kSmemTiles) {
      count_smem = std::max(count_smem, (size_t)n_tiles * sizeof(uint32_t));
      scatter_smem = std::max(scatter_smem, (size_t)2 * n_tiles * sizeof(uint32_t));
    }
  }
  static bool ready_scatter[64] = {}, ready_long[64] = {};
  const size_t sort_smem = (size_t)kSegSmem * sizeof(unsigned long long);
  const size_t long_smem = (size_t)kLongChunk * sizeof(unsigned long long);
  if (smem_limit_ready(reinterpret_cast<const void*>(scatter_batch_kernel), (int)(2 * kSmemTiles * 4),
                       ready_scatter) != cudaSuccess ||
      smem_limit_ready(reinterpret_cast<const void*>(tile_sort_long_batch_kernel), (int)long_smem,
                       ready_long) != cudaSuccess)
    return GS2D_ERR_CUDA;
  uint32_t* batch_ticket = static_cast<uint32_t*>(workspace);
  bin_init_batch_kernel<<<dim3(32, n_views), 256, 0, st>>>(T, batch_ticket);
  GS2D_LAUNCH_CHECK();
  if (T.count_total > 0) {
    count_batch_kernel<<<T.count_total, kScanThreads, count_smem, st>>>(T);
    GS2D_LAUNCH_CHECK();
  }
  if (T.chunk_total > 0) {
    emit_scan_batch_kernel<<<T.chunk_total, kScanThreads, 0, st>>>(
        T, batch_ticket, g_lookback_spins > 0 ? g_lookback_spins : kSpinLimit, g_lookback_withheld);
    GS2D_LAUNCH_CHECK();
  }
  tile_scan_batch_kernel<<<n_views, 1024, 0, st>>>(T);
  GS2D_LAUNCH_CHECK();
  if (T.scatter_total > 0) {
    scatter_batch_kernel<<<T.scatter_total, 256, scatter_smem, st>>>(T);
    GS2D_LAUNCH_CHECK();
  }
  if (T.tile_total > 0) {
    tile_sort_batch_kernel<<<T.tile_total, kSortThreads, sort_smem, st>>>(T);
    GS2D_LAUNCH_CHECK();
    tile_sort_long_batch_kernel<<<min(T.tile_total, 152), kLongThreads, long_smem, st>>>(T);
    GS2D_LAUNCH_CHECK();
  }
  return GS2D_OK;
}

}  // namespace gs2d

using namespace gs2d;

extern "C" {

void gs2d_set_lookback_wait(int spin_limit, int withheld_chunk) {
  g_lookback_spins = spin_limit > 0 ? spin_limit : 0;
  g_lookback_withheld = withheld_chunk >= 0 ? withheld_chunk : -1;
}

size_t gs2d_bin_sort_workspace(int n, size_t capacity) {
  // sized for the largest tile grid the ABI accepts
  return carve_sort_ws(nullptr, n, capacity, 65535).bytes;
}

int gs2d_bin_sort(const float* proj, const int32_t* tiles_per_surfel, int n,
                  const gs2d_camera* cam, const gs2d_config* cfg, void* workspace,
                  size_t ws_bytes, size_t* ws_needed, const gs2d_bins* bins, gs2d_stream stream) {
  // without emission arrays the binning serves the forward pass only
  const bool emit = bins && (bins->isect_emit || bins->surfel_off);
  return bin_sort_launch(proj, tiles_per_surfel, n, cam, cfg, workspace, ws_bytes, ws_needed, bins,
                         emit, (cudaStream_t)stream);
}

}  // extern "C"
