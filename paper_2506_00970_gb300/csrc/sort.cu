// gs2d_bin_sort: tile binning and depth ordering of (tile, surfel) pairs
// ("2DGS ... sorts them by depth", Sec. III-A).
//
// Output order: by tile, then by the FP32 bit pattern of the surfel's centre
// depth mu_c.z (positive floats order like their bits), then by surfel id.
// Instead of one 48-bit key sort over all K intersections this runs
//   1. a stable LSD radix sort of the N surfels by depth bits (4 x 8-bit
//      passes over N items, culled surfels keyed 0xFFFFFFFF sort last),
//   2. an exclusive scan of the per-surfel tile counts in depth order and
//      the emission of every surfel's tiles at its offset (so emission order
//      is depth order and each surfel owns a contiguous emission range),
//   3. a stable LSD radix sort of the K emitted pairs by tile id (one or two
//      8-bit passes),
// which yields the same order with 4 passes over N and <= 2 over K.
// Every radix pass is a single kernel: blocks take chunks in launch order
// from an atomic ticket, rank their keys stably with warp match-any, publish
// per-digit chunk counts, and look back over earlier chunks' published
// counts (decoupled look-back) to find their global offsets.  The look-back
// spin is bounded: past the limit the kernel records GS2D_ERR_TIMEOUT and
// continues with a partial prefix that still keeps every write in bounds.
#include "gs2d_common.cuh"

namespace gs2d {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kChunk = kSortThreads * kSortItems;  // 4096 keys per block
constexpr int kWarps = kSortThreads / 32;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 22;
constexpr int kLookback = 16;

__device__ __forceinline__ uint32_t ld_vol(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ void st_vol(uint32_t* p, uint32_t v) {
  *reinterpret_cast<volatile uint32_t*>(p) = v;
}
__device__ __forceinline__ unsigned long long ld_vol64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void st_vol64(unsigned long long* p, unsigned long long v) {
  *reinterpret_cast<volatile unsigned long long*>(p) = v;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
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

// Zeroes the per-call counters and outputs that are accumulated or that
// must read zero where nothing is written (ranges of empty tiles).
__global__ void bin_init_kernel(uint32_t* __restrict__ zero_a, size_t n_a,
                                int32_t* __restrict__ ranges, int n_ranges,
                                int32_t* __restrict__ n_isect, const int32_t* __restrict__ gate) {
  if (*gate) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_a; i += stride) zero_a[i] = 0u;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)n_ranges; i += stride)
    ranges[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_isect = 0;
}

// Depth keys of all surfels (culled -> 0xFFFFFFFF), identity values, and the
// four 8-bit digit histograms of the depth sort.
__global__ void __launch_bounds__(256) depth_keys_kernel(
    const float4* __restrict__ proj, const int32_t* __restrict__ tiles, int n,
    uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, uint32_t* __restrict__ hist,
    const int32_t* __restrict__ gate) {
  if (*gate) return;
  __shared__ uint32_t h[4][256];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) (&h[0][0])[i] = 0u;
  __syncthreads();
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const int i = base + threadIdx.x;
    const bool ok = i < n;
    uint32_t k = 0xFFFFFFFFu;
    if (ok) {
      if (tiles[i] > 0) k = __float_as_uint(proj[(size_t)i * (kProjFloats / 4) + 6].z);
      keys[i] = k;
      vals[i] = (uint32_t)i;
    }
    const uint32_t active = __ballot_sync(0xffffffffu, ok);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint32_t d = (k >> (8 * p)) & 255u;
      const uint32_t peers = __match_any_sync(0xffffffffu, ok ? d : 256u) & active;
      if (ok && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&h[p][d], __popc(peers));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(hist + i, c);
  }
}

// One stable 8-bit LSD radix pass (key u32, value u32).  vals_in == nullptr
// means value = input index.  n comes from *n_dev when n_dev is non-null.
// hist: this pass's 256-bin histogram of all n keys.  chunk_status: zeroed
// [max_chunks * 256]; ticket: zeroed counter.
__global__ void __launch_bounds__(kSortThreads) radix_pass_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, const int32_t* __restrict__ n_dev,
    int n_static, int max_items, int shift, const uint32_t* __restrict__ hist,
    uint32_t* __restrict__ chunk_status, uint32_t* __restrict__ ticket, int32_t* __restrict__ gate) {
  __shared__ uint32_t s_keys[kChunk];
  __shared__ uint32_t s_vals[kChunk];
  __shared__ uint32_t s_wcnt[kWarps][256];
  __shared__ uint32_t s_gbase[256];
  __shared__ uint32_t s_bstart[256];
  __shared__ uint32_t s_tmp[2 * kWarps + 1];
  __shared__ int s_chunk;
  if (*gate) return;
  int n = n_dev ? *n_dev : n_static;
  n = min(n, max_items);
  if (threadIdx.x == 0) s_chunk = (int)atomicAdd(ticket, 1u);
  for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&s_wcnt[0][0])[i] = 0u;
  __syncthreads();
  const int chunk = s_chunk;
  const long long base = (long long)chunk * kChunk;
  if (base >= n) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();

  uint32_t key[kSortItems], val[kSortItems], local[kSortItems];
  // all global loads first (independent, coalesced per round), then rank
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const long long idx = base + w * (32 * kSortItems) + r * 32 + lane;
    const bool ok = idx < n;
    key[r] = ok ? keys_in[idx] : 0xFFFFFFFFu;
    val[r] = ok ? (vals_in ? vals_in[idx] : (uint32_t)idx) : 0u;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const long long idx = base + w * (32 * kSortItems) + r * 32 + lane;
    const bool ok = idx < n;
    const uint32_t d = ok ? (key[r] >> shift) & 255u : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t cnt = 0;
    if (ok) cnt = s_wcnt[w][d];
    __syncwarp();
    if (ok && (__ffs(peers) - 1) == lane) s_wcnt[w][d] = cnt + __popc(peers);
    __syncwarp();
    local[r] = cnt + __popc(peers & lt);
  }
  __syncthreads();
  // per-digit block counts and warp prefixes (thread = digit)
  const int d = threadIdx.x;
  uint32_t run = 0;
#pragma unroll
  for (int ww = 0; ww < kWarps; ++ww) {
    const uint32_t c = s_wcnt[ww][d];
    s_wcnt[ww][d] = run;
    run += c;
  }
  const uint32_t cnt_d = run;
  uint32_t btotal;
  const uint32_t bstart = block_excl_scan256(cnt_d, s_tmp, &btotal);
  s_bstart[d] = bstart;
  uint32_t gtotal;
  const uint32_t gexcl = block_excl_scan256(hist[d], s_tmp, &gtotal);

  // publish this chunk's digit count, then look back for the prefix over a
  // window of kLookback predecessors at a time (loads issued together)
  uint32_t* my = chunk_status + (size_t)chunk * 256 + d;
  uint32_t excl = 0;
  if (chunk == 0) {
    st_vol(my, kFlagInc | cnt_d);
  } else {
    st_vol(my, kFlagAgg | cnt_d);
    int hi = chunk - 1;
    int spins = 0;
    bool found = false;
    while (!found && hi >= 0) {
      uint32_t wv[kLookback];
#pragma unroll
      for (int k = 0; k < kLookback; ++k)
        wv[k] = (hi - k >= 0) ? ld_vol(chunk_status + (size_t)(hi - k) * 256 + d) : kFlagInc;
#pragma unroll
      for (int k = 0; k < kLookback; ++k) {
        if (found) break;
        uint32_t sv = wv[k];
        while ((sv & ~kValMask) == 0u) {
          if (++spins > kSpinLimit) {
            atomicExch(gate, (int32_t)GS2D_ERR_TIMEOUT);
            sv = kFlagInc;  // give up with a partial prefix: writes stay in bounds
            break;
          }
          __nanosleep(32);
          sv = ld_vol(chunk_status + (size_t)(hi - k) * 256 + d);
        }
        excl += sv & kValMask;
        if ((sv & ~kValMask) == kFlagInc) found = true;
      }
      hi -= kLookback;
    }
    st_vol(my, kFlagInc | ((excl + cnt_d) & kValMask));
  }
  s_gbase[d] = gexcl + excl - bstart;
  __syncthreads();

  // reorder the chunk by digit in shared memory, then write runs
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const long long idx = base + w * (32 * kSortItems) + r * 32 + lane;
    if (idx < n) {
      const uint32_t dd = (key[r] >> shift) & 255u;
      const uint32_t pos = s_bstart[dd] + s_wcnt[w][dd] + local[r];
      s_keys[pos] = key[r];
      s_vals[pos] = val[r];
    }
  }
  __syncthreads();
  const int count = (int)min((long long)kChunk, (long long)n - base);
  for (int i = threadIdx.x; i < count; i += kSortThreads) {
    const uint32_t k = s_keys[i];
    const uint32_t o = s_gbase[(k >> shift) & 255u] + (uint32_t)i;
    keys_out[o] = k;
    vals_out[o] = s_vals[i];
  }
}

// Exclusive scan of tiles[sorted_id[r]] over the depth order r with
// decoupled look-back (64-bit chunk words: flag in bits 62-63).  Writes
// surfel_off[id] and, from the chunk holding the last surfel, the total K.
constexpr unsigned long long kF64Agg = 1ull << 62, kF64Inc = 2ull << 62,
                             kV64Mask = (1ull << 62) - 1;
__global__ void __launch_bounds__(kSortThreads) emit_scan_kernel(
    const uint32_t* __restrict__ sorted_ids, const int32_t* __restrict__ tiles, int n,
    uint32_t* __restrict__ surfel_off, unsigned long long* __restrict__ chunk_status,
    uint32_t* __restrict__ ticket, int32_t* __restrict__ n_isect, long long capacity,
    int32_t* __restrict__ gate) {
  __shared__ uint32_t s_ids[kChunk];
  __shared__ uint32_t s_tmp[2 * kWarps + 1];
  __shared__ int s_chunk;
  __shared__ unsigned long long s_prefix;
  if (*gate) return;
  if (threadIdx.x == 0) s_chunk = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  const int chunk = s_chunk;
  const long long base = (long long)chunk * kChunk;
  if (base >= n) return;
  const int count = (int)min((long long)kChunk, (long long)n - base);
  for (int i = threadIdx.x; i < count; i += kSortThreads)
    s_ids[i] = min(sorted_ids[base + i], (uint32_t)(n - 1));
  __syncthreads();
  // blocked: thread t owns items t*16 .. t*16+15
  uint32_t k[kSortItems];
  uint32_t sum = 0;
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const int i = threadIdx.x * kSortItems + j;
    k[j] = i < count ? (uint32_t)tiles[s_ids[i]] : 0u;
    sum += k[j];
  }
  uint32_t btotal;
  uint32_t excl = block_excl_scan256(sum, s_tmp, &btotal);
  if (threadIdx.x < 32) {
    // warp look-back: lane l examines predecessor chunk - 1 - l (+32 per round)
    const int lane = threadIdx.x;
    unsigned long long* my = chunk_status + chunk;
    unsigned long long prefix = 0;
    if (chunk == 0) {
      if (lane == 0) st_vol64(my, kF64Inc | (unsigned long long)btotal);
    } else {
      if (lane == 0) st_vol64(my, kF64Agg | (unsigned long long)btotal);
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
          if (++spins > kSpinLimit) {
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
      if (lane == 0) st_vol64(my, kF64Inc | ((prefix + btotal) & kV64Mask));
    }
    if (lane == 0) s_prefix = prefix;
  }
  __syncthreads();
  unsigned long long off = s_prefix + excl;
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const int i = threadIdx.x * kSortItems + j;
    if (i < count) {
      surfel_off[s_ids[i]] = (uint32_t)min(off, 0xFFFFFFFFull);
      if (base + i == n - 1) {
        const unsigned long long K = off + k[j];
        *n_isect = (int32_t)min(K, (unsigned long long)0x7FFFFFFF);
        if (K > (unsigned long long)capacity) atomicExch(gate, (int32_t)GS2D_ERR_CAPACITY);
      }
      off += k[j];
    }
  }
}

// Emission: the r-th surfel in depth order writes its tiles (row-major over
// its rectangle) at emission positions off .. off + k - 1, and counts the
// tile digits for the tile sort.
__global__ void __launch_bounds__(256) emit_kernel(
    const uint32_t* __restrict__ sorted_ids, const int32_t* __restrict__ tiles,
    const float4* __restrict__ proj, int n, const uint32_t* __restrict__ surfel_off, int tiles_x,
    int n_tiles, uint32_t* __restrict__ tile_key, uint32_t* __restrict__ emit_id,
    uint32_t* __restrict__ hist, const int32_t* __restrict__ gate) {
  if (*gate) return;
  __shared__ uint32_t h[2][256];
  for (int i = threadIdx.x; i < 512; i += blockDim.x) (&h[0][0])[i] = 0u;
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) {
    const uint32_t id = min(sorted_ids[r], (uint32_t)(n - 1));
    const int k = tiles[id];
    if (k > 0) {
      const uint32_t off = surfel_off[id];
      const float4 rc = proj[(size_t)id * (kProjFloats / 4) + 7];
      const uint32_t r01 = __float_as_uint(rc.x), r23 = __float_as_uint(rc.y);
      const int tx0 = r01 & 0xFFFF, ty0 = r01 >> 16, tx1 = r23 & 0xFFFF;
      const int rw = max(tx1 - tx0 + 1, 1);
      // exactly k pairs, row-major over the rectangle (k equals its area)
      for (int j = 0; j < k; ++j) {
        const int tx = tx0 + j % rw, ty = ty0 + j / rw;
        const uint32_t t = (uint32_t)min(ty * tiles_x + tx, n_tiles - 1);
        tile_key[off + j] = t;
        emit_id[off + j] = id;
        atomicAdd(&h[0][t & 255u], 1u);
        atomicAdd(&h[1][(t >> 8) & 255u], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 512; i += blockDim.x) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(hist + i, c);
  }
}

// Sorted (tile, emission index) -> per-position surfel id, emission index,
// optional 64-bit key, and tile ranges.
__global__ void __launch_bounds__(256) finalize_kernel(
    const uint32_t* __restrict__ tkeys, const uint32_t* __restrict__ tvals,
    const uint32_t* __restrict__ emit_id, const float4* __restrict__ proj,
    const int32_t* __restrict__ n_isect, int cap, int n_tiles, uint32_t* __restrict__ vals,
    uint32_t* __restrict__ emit, unsigned long long* __restrict__ keys64,
    int32_t* __restrict__ ranges, const int32_t* __restrict__ gate) {
  if (*gate) return;
  const int K = min(*n_isect, cap);
  const int stride = gridDim.x * blockDim.x;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += stride) {
    const uint32_t t = tkeys[k];
    const uint32_t e = min(tvals[k], (uint32_t)(K - 1));
    const uint32_t id = emit_id[e];
    vals[k] = id;
    emit[k] = e;
    if (keys64) {
      const uint32_t db = __float_as_uint(proj[(size_t)id * (kProjFloats / 4) + 6].z);
      keys64[k] = ((unsigned long long)t << 32) | db;
    }
    if (t < (uint32_t)n_tiles) {
      if (k == 0 || tkeys[k - 1] != t) ranges[2 * t] = k;
      if (k == K - 1 || tkeys[k + 1] != t) ranges[2 * t + 1] = k + 1;
    }
  }
}

// ---------------------------------------------------------------------------
// workspace layout
struct SortWs {
  uint32_t *dk_a, *dk_b, *dv_a, *dv_b;      // depth keys / values [n]
  uint32_t *tk_a, *tk_b, *tv_a, *tv_b;      // tile keys / values [cap]
  uint32_t* emit_id;                        // [cap]
  uint32_t* zero_begin;                     // start of the zeroed region
  uint32_t* dhist;                          // [4*256]
  uint32_t* thist;                          // [2*256]
  uint32_t* tickets;                        // [8]
  uint32_t* dstatus;                        // [4][chunks_n*256]
  uint32_t* tstatus;                        // [2][chunks_cap*256]
  unsigned long long* estatus;              // [chunks_n]
  size_t zero_words;
  size_t bytes;
  int chunks_n, chunks_cap;
};

SortWs carve_sort_ws(void* base, int n, size_t cap) {
  SortWs w{};
  Carver c(base);
  const size_t nn = (size_t)(n > 0 ? n : 1);
  w.chunks_n = (int)((nn + kChunk - 1) / kChunk);
  w.chunks_cap = (int)((cap + kChunk - 1) / kChunk);
  if (w.chunks_cap < 1) w.chunks_cap = 1;
  w.dk_a = c.take<uint32_t>(nn);
  w.dk_b = c.take<uint32_t>(nn);
  w.dv_a = c.take<uint32_t>(nn);
  w.dv_b = c.take<uint32_t>(nn);
  const size_t cc = cap > 0 ? cap : 1;
  w.tk_a = c.take<uint32_t>(cc);
  w.tk_b = c.take<uint32_t>(cc);
  w.tv_a = c.take<uint32_t>(cc);
  w.tv_b = c.take<uint32_t>(cc);
  w.emit_id = c.take<uint32_t>(cc);
  // zeroed region: contiguous words
  c.off = align_up(c.off, 256);
  const size_t zstart = c.off;
  w.zero_begin = base ? reinterpret_cast<uint32_t*>(static_cast<char*>(base) + zstart) : nullptr;
  size_t words = 0;
  auto zt = [&](size_t cnt) {
    uint32_t* p = base ? w.zero_begin + words : nullptr;
    words += (cnt + 63) / 64 * 64;
    return p;
  };
  w.dhist = zt(4 * 256);
  w.thist = zt(2 * 256);
  w.tickets = zt(8);
  w.dstatus = zt((size_t)4 * w.chunks_n * 256);
  w.tstatus = zt((size_t)2 * w.chunks_cap * 256);
  uint32_t* es = zt((size_t)2 * w.chunks_n + 2);
  w.estatus = reinterpret_cast<unsigned long long*>(
      base ? reinterpret_cast<uint32_t*>(align_up(reinterpret_cast<uintptr_t>(es), 8)) : nullptr);
  w.zero_words = words;
  c.off = zstart + words * sizeof(uint32_t) + 8;
  w.bytes = align_up(c.off, 256);
  return w;
}

}  // namespace gs2d

using namespace gs2d;

extern "C" {

size_t gs2d_bin_sort_workspace(int n, size_t capacity) {
  return carve_sort_ws(nullptr, n, capacity).bytes;
}

int gs2d_bin_sort(const float* proj, const int32_t* tiles_per_surfel, int n,
                  const gs2d_camera* cam, const gs2d_config* cfg, void* workspace,
                  size_t ws_bytes, size_t* ws_needed, const gs2d_bins* bins, gs2d_stream stream) {
  if (!cam || !cfg || !bins || n < 0) return GS2D_ERR_INVALID_ARG;
  if (n > 0 && (!proj || !tiles_per_surfel)) return GS2D_ERR_INVALID_ARG;
  if (!bins->vals || !bins->isect_emit || !bins->surfel_off || !bins->tile_ranges ||
      !bins->n_isect || !bins->status)
    return GS2D_ERR_INVALID_ARG;
  if (bins->capacity >= (size_t)kValMask) return GS2D_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(proj) & 15) return GS2D_ERR_INVALID_ARG;
  const int tx = gs2d_tiles_x(cam, cfg), ty = gs2d_tiles_y(cam, cfg);
  if (tx <= 0 || ty <= 0 || (long long)tx * ty > 65535) return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_bin_sort_workspace(n, bins->capacity);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const SortWs w = carve_sort_ws(workspace, n, bins->capacity);
  const int n_tiles = tx * ty;
  int32_t* gate = bins->status;

  bin_init_kernel<<<64, 256, 0, st>>>(w.zero_begin, w.zero_words, bins->tile_ranges, 2 * n_tiles,
                                      bins->n_isect, gate);
  GS2D_LAUNCH_CHECK();
  if (n == 0) return GS2D_OK;
  const float4* p4 = reinterpret_cast<const float4*>(proj);
  {
    const int blocks = min((n + 255) / 256, 152 * 8);
    depth_keys_kernel<<<blocks, 256, 0, st>>>(p4, tiles_per_surfel, n, w.dk_a, w.dv_a, w.dhist, gate);
    GS2D_LAUNCH_CHECK();
  }
  // depth sort: 4 passes, ping-pong a -> b -> a -> b -> a
  uint32_t *ki = w.dk_a, *vi = w.dv_a, *ko = w.dk_b, *vo = w.dv_b;
  for (int p = 0; p < 4; ++p) {
    radix_pass_kernel<<<w.chunks_n, kSortThreads, 0, st>>>(
        ki, vi, ko, vo, nullptr, n, n, 8 * p, w.dhist + 256 * p,
        w.dstatus + (size_t)p * w.chunks_n * 256, w.tickets + p, gate);
    GS2D_LAUNCH_CHECK();
    uint32_t* t = ki;
    ki = ko;
    ko = t;
    t = vi;
    vi = vo;
    vo = t;
  }
  const uint32_t* sorted_ids = vi;
  emit_scan_kernel<<<w.chunks_n, kSortThreads, 0, st>>>(sorted_ids, tiles_per_surfel, n,
                                                        bins->surfel_off, w.estatus, w.tickets + 4,
                                                        bins->n_isect, (long long)bins->capacity, gate);
  GS2D_LAUNCH_CHECK();
  emit_kernel<<<(n + 255) / 256, 256, 0, st>>>(sorted_ids, tiles_per_surfel, p4, n, bins->surfel_off,
                                                tx, n_tiles, w.tk_a, w.emit_id, w.thist, gate);
  GS2D_LAUNCH_CHECK();
  // stable sort of the emission by tile: one pass if ids fit in 8 bits
  const int cap = (int)bins->capacity;
  const int grid_cap = w.chunks_cap;
  radix_pass_kernel<<<grid_cap, kSortThreads, 0, st>>>(w.tk_a, nullptr, w.tk_b, w.tv_b, bins->n_isect,
                                                       0, cap, 0, w.thist, w.tstatus, w.tickets + 5,
                                                       gate);
  GS2D_LAUNCH_CHECK();
  const uint32_t *tk = w.tk_b, *tv = w.tv_b;
  if (n_tiles > 256) {
    radix_pass_kernel<<<grid_cap, kSortThreads, 0, st>>>(
        w.tk_b, w.tv_b, w.tk_a, w.tv_a, bins->n_isect, 0, cap, 8, w.thist + 256,
        w.tstatus + (size_t)w.chunks_cap * 256, w.tickets + 6, gate);
    GS2D_LAUNCH_CHECK();
    tk = w.tk_a;
    tv = w.tv_a;
  }
  {
    const int blocks = max(1, min((cap + 255) / 256, 152 * 16));
    finalize_kernel<<<blocks, 256, 0, st>>>(tk, tv, w.emit_id, p4, bins->n_isect, cap, n_tiles,
                                            bins->vals,
                                            bins->isect_emit,
                                            reinterpret_cast<unsigned long long*>(bins->keys),
                                            bins->tile_ranges, gate);
    GS2D_LAUNCH_CHECK();
  }
  return GS2D_OK;
}

}  // extern "C"
