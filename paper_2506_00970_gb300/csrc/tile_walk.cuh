// Warp-cooperative enumeration of the (surfel, tile) pairs of the warp's 32
// surfel rectangles, used wherever every covered tile of every surfel is
// visited (the projection's tile histogram, the scatter's count and slot
// passes).
//
// Lane i brings the inclusive tile rectangle of its surfel with k_i tiles
// (k_i = 0: none).  The warp's T = sum k_i pairs -- in lane order, row-major
// inside a rectangle -- are cut into 32 contiguous runs of ceil(T / 32), one
// per lane.  A lane finds the rectangle that holds its run's first pair by a
// binary search over the warp's prefix sums and then walks row by row
// without a division.  The warp thus takes ceil(T / 32) steps however the
// k_i are spread; a loop of every lane over its own rectangle takes max k_i
// steps (and one integer division per tile), so a single large surfel close
// to the camera stalls its whole warp.
#pragma once

#include "gs2d_common.cuh"

namespace gs2d {

// Per-warp shared scratch of warp_tile_walk.
struct WalkScratch {
  int inc[32];  // inclusive prefix sums of k over the lanes
  int tx0[32], ty0[32], rw[32];
};

// Calls fn(owner_lane, tile) for every pair of the warp's rectangles (tile
// ids clamped to n_tiles - 1, as everywhere in the binning).  Every lane of
// the warp must call it, with k = 0 when its surfel covers no tile.
template <class F>
__device__ __forceinline__ void warp_tile_walk(int k, int tx0, int ty0, int tx1, int tiles_x,
                                               int n_tiles, WalkScratch& ws, F&& fn) {
  const int lane = threadIdx.x & 31;
  int inc = k;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  const int total = __shfl_sync(0xffffffffu, inc, 31);
  ws.inc[lane] = inc;
  ws.tx0[lane] = tx0;
  ws.ty0[lane] = ty0;
  ws.rw[lane] = max(tx1 - tx0 + 1, 1);
  __syncwarp();
  const int chunk = (total + 31) >> 5;
  int idx = lane * chunk;
  const int stop = min(idx + chunk, total);
  if (idx < stop) {
    // owner: the first lane whose inclusive prefix exceeds idx (the count
    // of lanes whose prefix does not; at most 31 since inc[31] = total > idx)
    int o = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1)
      if (ws.inc[o + step - 1] <= idx) o += step;
    int rw = ws.rw[o], x0 = ws.tx0[o], y0 = ws.ty0[o];
    int left = ws.inc[o] - idx;  // pairs of the owner's rectangle from idx on
    const int off = idx - (o ? ws.inc[o - 1] : 0);
    int row = off / rw, col = off - row * rw;
    for (; idx < stop; ++idx) {
      fn(o, min((y0 + row) * tiles_x + x0 + col, n_tiles - 1));
      if (--left == 0) {
        // next lane with a non-empty rectangle (exists while idx + 1 < total)
        if (idx + 1 >= stop) break;
        do {
          ++o;
        } while (ws.inc[o] == ws.inc[o - 1]);
        rw = ws.rw[o];
        x0 = ws.tx0[o];
        y0 = ws.ty0[o];
        left = ws.inc[o] - ws.inc[o - 1];
        row = 0;
        col = 0;
      } else if (++col == rw) {
        col = 0;
        ++row;
      }
    }
  }
  __syncwarp();
}

}  // namespace gs2d
