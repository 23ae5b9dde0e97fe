// Learned tracking-pose proposal network (not in the paper; it proposes the
// starting pose of the tracking loop of Sec. III-D): forward, loss,
// backward and AdamW on BF16 tensor cores with FP32 accumulation.
//
// Every contraction of the network but the first layer's forward (a direct
// convolution kernel, conv_s2_kernel below) -- each convolution's forward
// (implicit im2col GEMM), data gradient (stride-2 transposed gather) and
// weight gradient (split-K GEMM over the pixels), and each fully connected
// layer's three products -- runs through one tiled GEMM kernel
//     C[M, N] = sum_k A[m, k] B[n, k]
// whose operand tiles are gathered straight from the NHWC activations and
// the weights by an address mode (no im2col buffer is materialised):
//   K-major modes (8 consecutive k of one row are contiguous):
//     K_DENSE   row-major [rows][ld] matrix
//     K_IM2COL  conv forward: row = (b, oy, ox), k = tap * C + c
//     K_DGRADP  conv data gradient of one parity class (py, px) of the input
//               pixels: row = (b, cy, cx) -> pixel (2 cy + py, 2 cx + px),
//               k = t * C_out + co over the class's taps t, reading dZ at
//               ((iy + 1 - ky) / 2, (ix + 1 - kx) / 2)
//   row-major modes (8 consecutive rows of one k are contiguous):
//     R_DENSE   element (row, k) at p[k * ld + row]
//     R_IM2COL  conv weight gradient: row = tap * C + c, k = (b, oy, ox)
//     R_WTP     conv weights read transposed for a parity class:
//               row = c_in, k = t * C_out + co
// Pixel and tap indices come from shifts (channel counts are powers of two)
// and precomputed reciprocal multiplies (no integer division in the loop).
// Tiles of 128 x 64 x 32 move global -> shared memory with 16-byte cp.async
// (zero-filled where the gather falls outside), three stages deep; warps
// read fragments with ldmatrix (.trans for row-major tiles) and issue
// mma.m16n8k16 bf16 x bf16 -> f32.  Epilogues: bias + ReLU -> bf16, bias ->
// f32, ReLU mask of the stored activation -> bf16, or FP32 split-K partials
// that a second kernel sums in a fixed order.
#include <algorithm>

#include <cuda_bf16.h>
#include <math.h>

#include "conv_tma.h"
#include "gs2d_common.cuh"
#include "gs2d_net.h"
#include "track_update.cuh"

namespace gs2d {
namespace net {

typedef __nv_bfloat16 bf16;

enum Mode {
  K_DENSE = 0, K_IM2COL = 1, K_DGRADP = 3,  // K-major
  R_DENSE = 4, R_IM2COL = 5, R_WTP = 7      // row-major
};
enum Epi { E_BIAS_RELU = 0, E_BIAS_F32 = 1, E_MASK = 2, E_PARTIAL = 3 };

constexpr int BM = 128, BN = 64, BK = 32, STAGES = 3, THREADS = 256, PAD = 8;
constexpr int kLayers = GS2D_NET_LAYERS;
constexpr int kConv = 6;
constexpr int kCin[kConv] = {8, 32, 64, 128, 256, 256};
constexpr int kCout[kConv] = {32, 64, 128, 256, 256, 256};
constexpr int kHin[kConv + 1] = {120, 60, 30, 15, 8, 4, 2};
constexpr int kWin[kConv + 1] = {160, 80, 40, 20, 10, 5, 3};
constexpr int kFlat = 2 * 3 * 256;
constexpr int kHidden = 256;
constexpr int kOut = GS2D_NET_OUT;
constexpr int kOutPad = 8;  // FC2 rows padded to 8 in the bf16 weight copy

// Division by a runtime constant d for numerators below 2^31: with
// s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1,
// n / d = (umulhi(n, m) + n) >> s (the round-up reciprocal method).
struct FastDiv {
  uint32_t m, s;
};
inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t s = 0;
  while ((1ull << s) < d) ++s;
  const unsigned long long m = ((1ull << 32) * ((1ull << s) - d)) / d + 1;
  return FastDiv{(uint32_t)m, s};
}
__device__ __forceinline__ int fdiv(int n, FastDiv f) {
  return (int)(((unsigned long long)__umulhi((uint32_t)n, f.m) + (uint32_t)n) >> f.s);
}

struct Operand {
  const bf16* p;
  int ld;                // dense modes: leading dimension; R_WTP: C_out
  int rows;              // valid rows (M or N); multiple of 8 for row-major modes
  int H, W, C, Ho, Wo;   // conv geometry (input H x W x C, output Ho x Wo)
  int py, px, Hc, Wc;    // parity class of the data gradient (K_DGRADP, R_WTP)
  int c_shift;           // log2 C (channel counts are powers of two)
  int ld_shift;          // log2 ld (R_WTP)
  FastDiv f_hw, f_w;     // pixels per image and per row of the indexed pixel grid
};

// Taps of a parity class of the stride-2 data gradient: input row iy gets
// contributions from ky = 1 when iy is even and ky in {0, 2} when it is odd
// (iy + 1 - ky must be even); likewise for columns.  Tap t of the class is
// (t / nx, t % nx) over its ny x nx taps.
__device__ __forceinline__ void class_tap(int py, int px, int t, int& ky, int& kx) {
  const int nx = px ? 2 : 1;
  const int tyi = t / nx, txi = t - tyi * nx;
  ky = py ? 2 * tyi : 1;
  kx = px ? 2 * txi : 1;
}

struct Gemm {
  int M, N, K, k_split;
  Operand a, b;
  void* out;
  int ldc;
  const float* bias;
  const bf16* mask;
  int n_valid;
  void* part;            // split-K partials [S][M][N] (FP32)
  // output row remap of a parity-class data gradient: GEMM row (b, cy, cx)
  // -> pixel (b, 2 cy + py, 2 cx + px) of an H x W map
  int remap, rH, rW, rHc, rWc, rpy, rpx;
  int* err;              // set to 1 by a tensor-core kernel whose wait timed out
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int MODE>
__host__ __device__ constexpr bool is_kmajor() {
  return MODE < R_DENSE;
}
template <int MODE, int ROWS>
__host__ __device__ constexpr int tile_elems() {
  return is_kmajor<MODE>() ? ROWS * (BK + PAD) : BK * (ROWS + PAD);
}

// Per-thread gather state of one operand tile: a thread always loads the
// same rows (K-major) or row group (row-major) of the tile, so their pixel
// coordinates are found once; each K step only locates its tap and channel.
template <int MODE, int ROWS, int NT = THREADS, int KB = BK>
struct Loader {
  static constexpr int kVec = ROWS * KB / 8;
  static constexpr int kPer = kVec / NT;  // 16-byte vectors per thread and stage
  const bf16* base[kPer];  // K-major: row start (dense) or image start (gathers)
  int iy0[kPer], ix0[kPer];
  bool ok[kPer];
  int ky, kx, c;            // R_IM2COL: the row group's tap and channel

  __device__ __forceinline__ Loader(const Operand& o, int r0) {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int v = threadIdx.x + i * NT;
      if (is_kmajor<MODE>()) {
        const int row = r0 + v / (KB / 8);
        ok[i] = row < o.rows;
        iy0[i] = ix0[i] = 0;
        if (MODE == K_DENSE) {
          base[i] = o.p + (size_t)row * o.ld;
        } else if (MODE == K_IM2COL) {
          const int b = fdiv(row, o.f_hw), r = row - b * o.Ho * o.Wo;
          const int oy = fdiv(r, o.f_w), ox = r - oy * o.Wo;
          base[i] = o.p + (size_t)b * o.H * o.W * o.C;
          iy0[i] = 2 * oy - 1;
          ix0[i] = 2 * ox - 1;
        } else {  // K_DGRADP
          const int b = fdiv(row, o.f_hw), r = row - b * o.Hc * o.Wc;
          const int cy = fdiv(r, o.f_w), cx = r - cy * o.Wc;
          base[i] = o.p + (size_t)b * o.Ho * o.Wo * o.C;
          iy0[i] = 2 * cy + o.py;
          ix0[i] = 2 * cx + o.px;
        }
      } else {
        const int row0 = r0 + (v % (ROWS / 8)) * 8;
        ok[i] = row0 < o.rows;
        base[i] = o.p;
        iy0[i] = ix0[i] = 0;
      }
    }
    ky = kx = c = 0;
    if (MODE == R_IM2COL) {
      const int row0 = r0 + (threadIdx.x % (ROWS / 8)) * 8;
      const int tap = row0 >> o.c_shift;
      c = row0 & ((1 << o.c_shift) - 1);
      ky = tap / 3;
      kx = tap - ky * 3;
    }
  }

  __device__ __forceinline__ const bf16* kaddr(const Operand& o, int i, int k, int kend) const {
    if (!ok[i] || k >= kend) return nullptr;
    if (MODE == K_DENSE) return base[i] + k;
    const int tap = k >> o.c_shift, ch = k & ((1 << o.c_shift) - 1);
    if (MODE == K_IM2COL) {
      const int tky = tap / 3, tkx = tap - tky * 3;
      const int iy = iy0[i] + tky, ix = ix0[i] + tkx;
      if (iy < 0 || iy >= o.H || ix < 0 || ix >= o.W) return nullptr;
      return base[i] + ((size_t)iy * o.W + ix) * o.C + ch;
    }
    int tky, tkx;  // K_DGRADP
    class_tap(o.py, o.px, tap, tky, tkx);
    const int oy = (iy0[i] + 1 - tky) >> 1, ox = (ix0[i] + 1 - tkx) >> 1;
    if (oy < 0 || oy >= o.Ho || ox < 0 || ox >= o.Wo) return nullptr;
    return base[i] + ((size_t)oy * o.Wo + ox) * o.C + ch;
  }

  __device__ __forceinline__ const bf16* raddr(const Operand& o, int i, int row0, int k,
                                               int kend) const {
    if (!ok[i] || k >= kend) return nullptr;
    if (MODE == R_DENSE) return o.p + (size_t)k * o.ld + row0;
    if (MODE == R_IM2COL) {
      const int b = fdiv(k, o.f_hw), r = k - b * o.Ho * o.Wo;
      const int oy = fdiv(r, o.f_w), ox = r - oy * o.Wo;
      const int iy = 2 * oy - 1 + ky, ix = 2 * ox - 1 + kx;
      if (iy < 0 || iy >= o.H || ix < 0 || ix >= o.W) return nullptr;
      return o.p + (((size_t)b * o.H + iy) * o.W + ix) * o.C + c;
    }
    const int t = k >> o.ld_shift, co = k & ((1 << o.ld_shift) - 1);  // R_WTP
    int tky, tkx;
    class_tap(o.py, o.px, t, tky, tkx);
    return o.p + ((size_t)co * 9 + tky * 3 + tkx) * o.C + row0;
  }

  // One stage in the tcgen05 operand layout: 8 x 8 core matrices of 128
  // bytes (16 contiguous bytes along K for K-major tiles, along the rows for
  // row-major tiles).  K-major: core (row group g, k group q) at
  // g * 512 + q * 128 bytes; row-major: core (k group q, row group g) at
  // q * (ROWS / 8) * 128 + g * 128 bytes.
  __device__ __forceinline__ void load_core(unsigned char* s, const Operand& o, int r0, int k0,
                                            int kend) const {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int v = threadIdx.x + i * NT;
      if (is_kmajor<MODE>()) {
        const int r = v / (KB / 8), kq = (v % (KB / 8)) * 8;
        const bf16* src = kaddr(o, i, k0 + kq, kend);
        cp_async16(s + (r >> 3) * (KB / 8) * 128 + (kq >> 3) * 128 + (r & 7) * 16, src ? src : o.p,
                   src != nullptr);
      } else {
        const int kk = v / (ROWS / 8), rq = (v % (ROWS / 8)) * 8;
        const bf16* src = raddr(o, i, r0 + rq, k0 + kk, kend);
        cp_async16(s + (kk >> 3) * (ROWS / 8) * 128 + (rq >> 3) * 128 + (kk & 7) * 16,
                   src ? src : o.p, src != nullptr);
      }
    }
  }

  // One stage: the ROWS x BK tile at k0 into shared memory.
  __device__ __forceinline__ void load(bf16* s, const Operand& o, int r0, int k0, int kend) const {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int v = threadIdx.x + i * NT;
      if (is_kmajor<MODE>()) {
        const int r = v >> 2, kq = (v & 3) * 8;
        const bf16* src = kaddr(o, i, k0 + kq, kend);
        cp_async16(s + r * (BK + PAD) + kq, src ? src : o.p, src != nullptr);
      } else {
        const int kk = v / (ROWS / 8), rq = (v % (ROWS / 8)) * 8;
        const bf16* src = raddr(o, i, r0 + rq, k0 + kk, kend);
        cp_async16(s + kk * (ROWS + PAD) + rq, src ? src : o.p, src != nullptr);
      }
    }
  }
};

// A fragment of the m16 x k16 sub-tile at (r0, k0) of a stage.
template <int MODE, int ROWS>
__device__ __forceinline__ void frag_a(uint32_t a[4], const bf16* s, int r0, int k0) {
  const int l = threadIdx.x & 31, i = l >> 3, rr = l & 7;
  if (is_kmajor<MODE>())
    ldsm_x4(a, s + (r0 + rr + 8 * (i & 1)) * (BK + PAD) + k0 + 8 * (i >> 1));
  else
    ldsm_x4_t(a, s + (k0 + 8 * (i >> 1) + rr) * (ROWS + PAD) + r0 + 8 * (i & 1));
}
// B fragments of two n8 x k16 sub-tiles at (n0, k0), (n0 + 8, k0).
template <int MODE, int ROWS>
__device__ __forceinline__ void frag_b(uint32_t b[4], const bf16* s, int n0, int k0) {
  const int l = threadIdx.x & 31, i = l >> 3, rr = l & 7;
  if (is_kmajor<MODE>())
    ldsm_x4(b, s + (n0 + rr + 8 * (i >> 1)) * (BK + PAD) + k0 + 8 * (i & 1));
  else
    ldsm_x4_t(b, s + (k0 + 8 * (i & 1) + rr) * (ROWS + PAD) + n0 + 8 * (i >> 1));
}

// Output offset of GEMM row `row` (times the row stride ldc).
__device__ __forceinline__ size_t out_row(const Gemm& g, int row) {
  if (!g.remap) return (size_t)row;
  const int hw = g.rHc * g.rWc;
  const int b = row / hw, r = row - b * hw, cy = r / g.rWc, cx = r - cy * g.rWc;
  return ((size_t)b * g.rH + 2 * cy + g.rpy) * g.rW + 2 * cx + g.rpx;
}

template <int EPI>
__device__ __forceinline__ void apply_epi(const Gemm& g, int row, int col, float v0, float v1) {
  if (row >= g.M) return;
  if (EPI == E_BIAS_RELU) {
    if (col >= g.N) return;
    const float x0 = fmaxf(v0 + g.bias[col], 0.f), x1 = fmaxf(v1 + g.bias[col + 1], 0.f);
    *reinterpret_cast<__nv_bfloat162*>(static_cast<bf16*>(g.out) + out_row(g, row) * g.ldc + col) =
        __floats2bfloat162_rn(x0, x1);
  } else if (EPI == E_BIAS_F32) {
    float* o = static_cast<float*>(g.out) + out_row(g, row) * g.ldc;
    if (col < g.n_valid) o[col] = v0 + g.bias[col];
    if (col + 1 < g.n_valid) o[col + 1] = v1 + g.bias[col + 1];
  } else if (EPI == E_MASK) {
    if (col >= g.N) return;
    const size_t off = out_row(g, row) * g.ldc + col;
    const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(g.mask + off);
    const float x0 = __bfloat162float(m.x) > 0.f ? v0 : 0.f;
    const float x1 = __bfloat162float(m.y) > 0.f ? v1 : 0.f;
    *reinterpret_cast<__nv_bfloat162*>(static_cast<bf16*>(g.out) + off) = __floats2bfloat162_rn(x0, x1);
  } else {
    if (col >= g.N) return;
    float* o = static_cast<float*>(g.part) + ((size_t)blockIdx.z * g.M + row) * g.N + col;
    *reinterpret_cast<float2*>(o) = make_float2(v0, v1);
  }
}

// Sums the split-K partials of column pairs in split order and applies the
// epilogue.
template <int EPI>
__global__ void splitk_epilogue_kernel(const Gemm g, int S) {
  const size_t pairs = (size_t)g.M * (g.N / 2);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < pairs;
       e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / (g.N / 2)), col = 2 * (int)(e % (g.N / 2));
    float v0 = 0.f, v1 = 0.f;
    for (int z = 0; z < S; ++z) {
      const float2 p = *reinterpret_cast<const float2*>(
          static_cast<const float*>(g.part) + ((size_t)z * g.M + row) * g.N + col);
      v0 += p.x;
      v1 += p.y;
    }
    apply_epi<EPI>(g, row, col, v0, v1);
  }
}

// grid: (ceil(M / BM), ceil(N / BN), splits); 256 threads = 4 (M) x 2 (N)
// warps of 32 x 32 outputs each.
template <int AM, int BMODE, int EPI>
__global__ void __launch_bounds__(THREADS) gemm_kernel(const Gemm g) {
  constexpr int kA = tile_elems<AM, BM>(), kB = tile_elems<BMODE, BN>();
  __shared__ __align__(128) bf16 smem[STAGES * (kA + kB)];
  bf16* sA = smem;
  bf16* sB = smem + STAGES * kA;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * g.k_split;
  const int kend = min(g.K, kbeg + g.k_split);
  const int ntiles = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  const int warp = threadIdx.x >> 5, wm = (warp & 3) * 32, wn = (warp >> 2) * 32;
  const Loader<AM, BM> la(g.a, m0);
  const Loader<BMODE, BN> lb(g.b, n0);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < ntiles) {
      la.load(sA + s * kA, g.a, m0, kbeg + s * BK, kend);
      lb.load(sB + s * kB, g.b, n0, kbeg + s * BK, kend);
    }
    cp_async_commit();
  }
  for (int kt = 0; kt < ntiles; ++kt) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    const int nk = kt + STAGES - 1;
    if (nk < ntiles) {
      const int st = nk % STAGES;
      la.load(sA + st * kA, g.a, m0, kbeg + nk * BK, kend);
      lb.load(sB + st * kB, g.b, n0, kbeg + nk * BK, kend);
    }
    cp_async_commit();
    const bf16* a_s = sA + (kt % STAGES) * kA;
    const bf16* b_s = sB + (kt % STAGES) * kB;
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t af[2][4], bfr[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) frag_a<AM, BM>(af[i], a_s, wm + 16 * i, ks);
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) frag_b<BMODE, BN>(bfr[jj], b_s, wn + 16 * jj, ks);
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          mma_bf16(acc[i][j], af[i], bfr[j >> 1][2 * (j & 1)], bfr[j >> 1][2 * (j & 1) + 1]);
    }
  }
  cp_async_wait<0>();
  const int l = threadIdx.x & 31, gq = l >> 2, cq = l & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = m0 + wm + 16 * i + gq, col = n0 + wn + 8 * j + 2 * cq;
      apply_epi<EPI>(g, row, col, acc[i][j][0], acc[i][j][1]);
      apply_epi<EPI>(g, row + 8, col, acc[i][j][2], acc[i][j][3]);
    }
}

// ---------------------------------------------------------------------------
// The same GEMM on the 5th-generation tensor cores: one elected thread issues
// tcgen05.mma (M = 128, N = 64, K = 16, bf16 x bf16 -> f32) from shared-memory
// descriptors, the accumulator lives in tensor memory (128 lanes x 64
// columns), and each of the four warps reads its 32 lanes back with
// tcgen05.ld for the epilogue.  Operand tiles are gathered by the same
// loaders (cp.async) into the no-swizzle core-matrix layout; a stage is
// refilled after the tcgen05.commit of the MMAs that read it arrives on the
// stage's mbarrier.  Every wait is bounded: past the limit the kernel records
// an error in *err, stops issuing work, and still frees its tensor memory.
constexpr int TC_THREADS = 256, TC_STAGES = 3, TC_COLS = 64, TC_BK = 64;
constexpr int TC_A_BYTES = BM * TC_BK * 2, TC_B_BYTES = BN * TC_BK * 2;
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES;  // 72 KB
constexpr int kTcSpin = 1 << 24;

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// Shared-memory matrix descriptor, no swizzle: start address, the byte step
// between core matrices along K (leading) and along M / N (stride).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t k_step, uint32_t mn_step) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((k_step >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((mn_step >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: f32 accumulate, bf16 A and B, A / B
// K-major (0) or M/N-major (1), N = 64, M = 128.
__host__ __device__ constexpr uint32_t tc_idesc(bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (a_mn ? 1u << 15 : 0u) | (b_mn ? 1u << 16 : 0u) |
         ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int spins = 0; spins < kTcSpin; ++spins) {
    uint32_t ok;
    asm volatile(
        "{.reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}

template <int AM, int BMODE, int EPI>
__global__ void __launch_bounds__(TC_THREADS) gemm_tc_kernel(const Gemm g) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t s_bar[TC_STAGES + 1];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * g.k_split;
  const int kend = min(g.K, kbeg + g.k_split);
  const int ntiles = kend > kbeg ? (kend - kbeg + TC_BK - 1) / TC_BK : 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr bool a_mn = !is_kmajor<AM>(), b_mn = !is_kmajor<BMODE>();
  // descriptor steps: K-major core matrices 128 B apart along K and
  // TC_BK / 8 x 128 B along the rows; row-major ones 128 B apart along the
  // rows and ROWS / 8 x 128 B apart along K
  constexpr uint32_t a_k = a_mn ? (BM / 8) * 128 : 128, a_mn_step = a_mn ? 128 : (TC_BK / 8) * 128;
  constexpr uint32_t b_k = b_mn ? (BN / 8) * 128 : 128, b_mn_step = b_mn ? 128 : (TC_BK / 8) * 128;
  constexpr uint32_t idesc = tc_idesc(a_mn, b_mn);

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int i = 0; i <= TC_STAGES; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&s_bar[i])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(TC_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  const Loader<AM, BM, TC_THREADS, TC_BK> la(g.a, m0);
  const Loader<BMODE, BN, TC_THREADS, TC_BK> lb(g.b, n0);
  auto stage_a = [&](int s) { return tc_smem + s * TC_STAGE_BYTES; };
  auto stage_b = [&](int s) { return tc_smem + s * TC_STAGE_BYTES + TC_A_BYTES; };

#pragma unroll
  for (int s = 0; s < TC_STAGES - 1; ++s) {
    if (s < ntiles) {
      la.load_core(stage_a(s), g.a, m0, kbeg + s * TC_BK, kend);
      lb.load_core(stage_b(s), g.b, n0, kbeg + s * TC_BK, kend);
    }
    cp_async_commit();
  }
  // A wait that runs out in any thread is shared through s_fail: after the
  // next k-tile's barrier no thread issues MMAs or refills stages any more.
  bool fail = false;
  for (int kt = 0; kt < ntiles; ++kt) {
    const int st = kt % TC_STAGES;
    cp_async_wait<TC_STAGES - 2>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (*reinterpret_cast<volatile int*>(&s_fail)) fail = true;
    if (threadIdx.x == 0 && !fail) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = su32(stage_a(st)), sb = su32(stage_b(st));
#pragma unroll
      for (int j = 0; j < TC_BK / 16; ++j) {
        const uint64_t ad = smem_desc(sa + j * 2 * a_k, a_k, a_mn_step);
        const uint64_t bd = smem_desc(sb + j * 2 * b_k, b_k, b_mn_step);
        const uint32_t acc = (kt > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{.reg .pred p; setp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       su32(&s_bar[st])) : "memory");
    }
    // refill the stage read by the previous k-tile once its MMAs are done
    const int nk = kt + TC_STAGES - 1;
    if (nk < ntiles) {
      const int sl = nk % TC_STAGES;
      if (kt >= 1 && !fail && !mbar_wait(su32(&s_bar[sl]), (uint32_t)(((kt - 1) / TC_STAGES) & 1))) {
        fail = true;
        *reinterpret_cast<volatile int*>(&s_fail) = 1;
      }
      if (!fail) {
        la.load_core(stage_a(sl), g.a, m0, kbeg + nk * TC_BK, kend);
        lb.load_core(stage_b(sl), g.b, n0, kbeg + nk * TC_BK, kend);
      }
    }
    cp_async_commit();
  }
  cp_async_wait<0>();
  // Thread 0 issued MMAs at k-tile 0 at least (no wait precedes them); one
  // last commit tracks all it issued -- every one, or those before a
  // failure -- and every thread waits for it (bounded) before the tensor
  // memory is read or freed, so no MMA in flight outlives the allocation
  // unless that wait too runs out.
  if (threadIdx.x == 0 && ntiles > 0)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     su32(&s_bar[TC_STAGES])) : "memory");
  if (ntiles > 0 && !mbar_wait(su32(&s_bar[TC_STAGES]), 0u)) fail = true;
  if (fail) atomicExch(&s_fail, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (!s_fail) {
    // warp w reads the accumulator lanes of its quadrant (w % 4) and half the
    // columns (w / 4) into the (now idle) stage buffers as a row-major FP32
    // tile; then consecutive threads take consecutive column pairs of a row,
    // so the epilogue's loads and stores are coalesced
    constexpr int kLd = BN + 2;  // floats per staged row
    float* tile = reinterpret_cast<float*>(tc_smem);
    const int quad = warp & 3, half = warp >> 2;
    const int lrow = 32 * quad + lane;
#pragma unroll
    for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)c0;
      if (ntiles > 0) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
              "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = 0u;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) tile[lrow * kLd + c0 + j] = __uint_as_float(r[j]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BM * (BN / 2); e += TC_THREADS) {
      const int rr = e / (BN / 2), cc = 2 * (e % (BN / 2));
      const float2 v = *reinterpret_cast<const float2*>(&tile[rr * kLd + cc]);
      apply_epi<EPI>(g, m0 + rr, n0 + cc, v.x, v.y);
    }
  } else if (threadIdx.x == 0 && g.err) {
    atomicExch(g.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS));
}

// ---------------------------------------------------------------------------
// Direct convolution of the first layer (stride 2, 3 x 3 taps, zero padding
// 1, C_in = 8: one 16-byte chunk per pixel).  A tile is RB whole output rows of one image
// (RB Wo pixels) for all C_out channels.  The grid is resident (blocks per
// SM from the occupancy calculator) and each block walks the tiles
// t = blockIdx.x, + gridDim.x, ...: it copies the layer's weights into
// shared memory once, and for every tile the 2 RB + 1 input rows its pixels
// read (zero rows and columns where the padding lies), the next tile's rows
// in flight (cp.async, two buffers) while the current one computes.  Each
// warp gathers the A fragments of its 32 pixels -- their im2col rows, 8
// channels of one tap per 16-byte ldmatrix row -- straight from the staged
// rows and issues mma.m16n8k16.  Against the implicit-im2col GEMM, an input
// pixel leaves global memory once per tile instead of once per tap, the
// weights once per block, and no tile column is padding (C_out = 32 would
// fill half of a 64-wide tile).
// Staged rows: [row][column parity][column / 2][C_in] over the columns
// ix + 1 = 0 .. W + 1: pixels ox, ox + 1 read columns 2 ox + kx and
// 2 ox + 2 + kx under one tap, neighbours in one parity plane, so the eight
// pixels of an ldmatrix row group are eight consecutive 16-byte entries
// (distinct banks).  Layer 1 (input 79 MB, output 79 MB at batch 256) takes
// 51 us here against 124 us as an implicit-im2col GEMM.  The same scheme for
// layer 2 (C_in = 32; two 47 KB row buffers leave one block per SM) took
// 80-95 us against the GEMM's 62 us, so layer 2 stays a GEMM.
template <int CIN, int COUT, int H, int W, int RB>
struct ConvS2 {
  static constexpr int Ho = H / 2, Wo = W / 2;
  static constexpr int PIX = RB * Wo;               // output pixels per tile
  static constexpr int TPI = (Ho + RB - 1) / RB;    // tiles per image
  static constexpr int WARPS = (PIX + 31) / 32;     // 32 pixels per warp
  static constexpr int NTHREADS = WARPS * 32;
  static constexpr int RIN = 2 * RB + 1;            // staged input rows
  static constexpr int WP = (W + 2) / 2;            // entries per parity plane
  static constexpr int NCH = CIN / 8;               // 16-byte chunks per pixel
  static constexpr int K = 9 * CIN;
  static constexpr int KS = (K + 15) / 16;          // k16 steps
  static constexpr int KP = KS * 16 + 8;            // staged weight row, padded
  static constexpr int NT = COUT / 8;               // n8 tiles
  static constexpr int PATCH = RIN * 2 * WP * CIN;  // bf16 elements per buffer
  static constexpr int WSM = COUT * KP;
  static constexpr int SMEM = (2 * PATCH + WSM + 8) * 2;  // + one zero chunk
  static_assert(CIN == 8, "one 16-byte chunk per pixel");
  static_assert(H % 2 == 0 && W % 2 == 0 && COUT % 16 == 0, "shape");
  static_assert(PATCH % 8 == 0 && KP % 8 == 0, "16-byte rows");
};

// Issues the cp.async copies of tile t's input rows into patch.
template <class C, int CIN, int H, int W>
__device__ __forceinline__ void conv_stage_rows(bf16* patch, const bf16* __restrict__ x, int t) {
  const int b = t / C::TPI, iy0 = 2 * (t - b * C::TPI) * (C::PIX / C::Wo) - 1;
  const bf16* xb = x + (size_t)b * H * W * CIN;
  constexpr int ROWCH = (W + 2) * C::NCH;
  for (int e = threadIdx.x; e < C::RIN * ROWCH; e += C::NTHREADS) {
    const int r = e / ROWCH, rem = e - r * ROWCH;
    const int c = rem / C::NCH, q = rem - c * C::NCH;
    const int iy = iy0 + r, ix = c - 1;
    const bool ok = iy >= 0 && iy < H && ix >= 0 && ix < W;
    const int ent = c >> 1;
    bf16* dst = patch + ((r * 2 + (c & 1)) * C::WP + ent) * CIN + q * 8;
    cp_async16(dst, ok ? xb + ((size_t)iy * W + ix) * CIN + q * 8 : xb, ok);
  }
}

template <int CIN, int COUT, int H, int W, int RB>
__global__ void __launch_bounds__(ConvS2<CIN, COUT, H, W, RB>::NTHREADS) conv_s2_kernel(
    const bf16* __restrict__ x, const bf16* __restrict__ wt, const float* __restrict__ bias,
    bf16* __restrict__ out, int n_tiles) {
  using C = ConvS2<CIN, COUT, H, W, RB>;
  extern __shared__ __align__(128) unsigned char conv_smem[];
  bf16* patches = reinterpret_cast<bf16*>(conv_smem);
  bf16* wsm = patches + 2 * C::PATCH;
  bf16* zero = wsm + C::WSM;
  // weights [C_out][K] -> rows of KP, zero past K (copy group 0)
  constexpr int WCH = C::KP / 8;
  for (int e = threadIdx.x; e < COUT * WCH; e += C::NTHREADS) {
    const int n = e / WCH, q = e - n * WCH;
    const bool ok = q * 8 < C::K;
    cp_async16(wsm + n * C::KP + q * 8, ok ? wt + (size_t)n * C::K + q * 8 : wt, ok);
  }
  if (threadIdx.x == 0) *reinterpret_cast<uint4*>(zero) = make_uint4(0u, 0u, 0u, 0u);
  if ((int)blockIdx.x < n_tiles) conv_stage_rows<C, CIN, H, W>(patches, x, blockIdx.x);
  cp_async_commit();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mat = lane >> 3, rr = lane & 7;
  const int gq = lane >> 2, cq = lane & 3;
  // this lane's ldmatrix row in m16 tile i: pixel 32 warp + 16 i + rr + 8 (mat & 1)
  int prow[2], pcol[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int m = 32 * warp + 16 * i + rr + 8 * (mat & 1);
    const int dy = m / C::Wo;
    prow[i] = 2 * dy;
    pcol[i] = m - dy * C::Wo;
  }
  // the biases of this lane's output columns, loaded once
  float bv[C::NT][2];
#pragma unroll
  for (int n8 = 0; n8 < C::NT; ++n8) {
    bv[n8][0] = bias[8 * n8 + 2 * cq];
    bv[n8][1] = bias[8 * n8 + 2 * cq + 1];
  }
  int it = 0;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
    // the next tile's rows go to the other buffer, which the previous
    // iteration finished reading before its closing barrier
    const int tn = t + (int)gridDim.x;
    if (tn < n_tiles) conv_stage_rows<C, CIN, H, W>(patches + ((it + 1) & 1) * C::PATCH, x, tn);
    cp_async_commit();
    cp_async_wait<1>();  // the weights and this tile's rows have landed
    __syncthreads();
    const bf16* patch = patches + (it & 1) * C::PATCH;
    const int b = t / C::TPI, oy0 = (t - b * C::TPI) * RB;
    bool pok[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int m = 32 * warp + 16 * i + rr + 8 * (mat & 1);
      pok[i] = m < C::PIX && oy0 + prow[i] / 2 < C::Ho;
    }
    float acc[2][C::NT][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int n8 = 0; n8 < C::NT; ++n8)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[i][n8][v] = 0.f;
#pragma unroll 2
    for (int s = 0; s < C::KS; ++s) {
      const int k = 16 * s + 8 * (mat >> 1);  // this lane's k offset
      const int tap = k / CIN, q = (k % CIN) / 8;
      const int ky = tap / 3, kx = tap - 3 * ky;
      uint32_t af[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const bf16* src = zero;
        if (pok[i] && tap < 9) {
          const int r = prow[i] + ky, c = 2 * pcol[i] + kx, ent = c >> 1;
          src = patch + ((r * 2 + (c & 1)) * C::WP + ent) * CIN + q * 8;
        }
        ldsm_x4(af[i], src);
      }
#pragma unroll
      for (int jj = 0; jj < C::NT / 2; ++jj) {
        uint32_t bfr[4];
        ldsm_x4(bfr, wsm + (16 * jj + rr + 8 * (mat >> 1)) * C::KP + 16 * s + 8 * (mat & 1));
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          mma_bf16(acc[i][2 * jj], af[i], bfr[0], bfr[1]);
          mma_bf16(acc[i][2 * jj + 1], af[i], bfr[2], bfr[3]);
        }
      }
    }
    // bias + ReLU -> bf16, NHWC rows of C_out
    bf16* ob = out + ((size_t)b * C::Ho + oy0) * C::Wo * COUT;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = 32 * warp + 16 * i + gq + 8 * h;
        if (m >= C::PIX || oy0 + m / C::Wo >= C::Ho) continue;
#pragma unroll
        for (int n8 = 0; n8 < C::NT; ++n8) {
          const int col = 8 * n8 + 2 * cq;
          const float x0 = fmaxf(acc[i][n8][2 * h] + bv[n8][0], 0.f);
          const float x1 = fmaxf(acc[i][n8][2 * h + 1] + bv[n8][1], 0.f);
          *reinterpret_cast<__nv_bfloat162*>(ob + (size_t)m * COUT + col) =
              __floats2bfloat162_rn(x0, x1);
        }
      }
    __syncthreads();
  }
  cp_async_wait<0>();
}

static_assert(kCin[0] == 8 && kCout[0] == 32 && kHin[0] == 120 && kWin[0] == 160, "layer 1");

// Launches the direct kernel over the B images (a resident grid).
template <int CIN, int COUT, int H, int W, int RB>
int conv_s2(const bf16* x, int B, const bf16* wt, const float* bias, bf16* out, cudaStream_t st) {
  using C = ConvS2<CIN, COUT, H, W, RB>;
  auto kernel = conv_s2_kernel<CIN, COUT, H, W, RB>;
  static int slots[64] = {};  // resident blocks per device (0: not yet known)
  int dev = 0;
  GS2D_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return GS2D_ERR_CUDA;
  if (!slots[dev]) {
    GS2D_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    int per_sm = 0, sms = 0;
    GS2D_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, C::NTHREADS, C::SMEM));
    GS2D_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    slots[dev] = max(1, per_sm) * max(1, sms);
  }
  if (B <= 0) return GS2D_OK;
  const long long n_tiles = (long long)B * C::TPI;
  if (n_tiles > 0x7FFFFFFF) return GS2D_ERR_INVALID_ARG;
  const int grid = (int)(n_tiles < (long long)slots[dev] ? n_tiles : (long long)slots[dev]);
  kernel<<<grid, C::NTHREADS, C::SMEM, st>>>(x, wt, bias, out, (int)n_tiles);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

// Layer 1's weight gradient dW[c_out][k] = sum over output pixels p of
// dY[p][c_out] im2col(x)[p][k] (k = tap x 8 + c_in) as a direct kernel on
// the forward's staging: a tile is two output rows of one image, its five
// input rows staged in column-parity planes and its 160 x 32 output
// gradients beside them (the next tile's in flight); warp w contracts the
// tile's pixels 32 w .. 32 w + 31 with mma.m16n8k16 (A = dY^T by ldmatrix
// .trans from the staged gradients, B = each tap's 8 input channels by
// ldmatrix .trans from the staged rows), accumulating the 32 x 72 product
// over all its tiles in registers; lane c of warp w also adds channel c of
// the bias gradient db[c] = sum_p dY[p][c] over the same pixels.  The
// block's warps are summed in a fixed order into one partial per block
// ([32 x 72 weights | 32 bias] floats; reduce_partials_wide_kernel adds the
// blocks in a fixed order), so the result does not depend on timing.
// Reads the input map and the output gradients once (2 x 78.6 MB at batch
// 256).
constexpr int kW1Grid = 3 * 152;  // fixed grid: the partials' count and order
using W1 = ConvS2<8, 32, 120, 160, 2>;
constexpr int kW1Dy = W1::PIX * 32;  // bf16 per staged gradient tile
constexpr int kW1Smem = (2 * W1::PATCH + 2 * kW1Dy + 8) * 2;
constexpr int kW1Part = 32 * 72 + 32;  // floats per block partial
static_assert(W1::PIX == 160 && W1::NTHREADS == 160, "five warps of 32 pixels");

__device__ __forceinline__ void w1_stage_dy(bf16* dst, const bf16* __restrict__ dy, int t) {
  const int b = t / W1::TPI, oy0 = (t - b * W1::TPI) * 2;
  const bf16* src = dy + ((size_t)b * W1::Ho + oy0) * W1::Wo * 32;
  // pixel p's 16-byte chunk q lands at chunk q ^ ((p >> 1) & 3) of its row,
  // so that eight consecutive pixels' chunk q fall in distinct banks
  for (int e = threadIdx.x; e < kW1Dy / 8; e += W1::NTHREADS) {
    const int p = e >> 2, q = e & 3;
    cp_async16(dst + 32 * p + 8 * (q ^ ((p >> 1) & 3)), src + 8 * e, true);
  }
}

__global__ void __launch_bounds__(W1::NTHREADS) wgrad1_kernel(const bf16* __restrict__ x,
                                                              const bf16* __restrict__ dy,
                                                              float* __restrict__ part,
                                                              int n_tiles) {
  extern __shared__ __align__(128) unsigned char w1_smem[];
  bf16* patches = reinterpret_cast<bf16*>(w1_smem);
  bf16* dys = patches + 2 * W1::PATCH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mat = lane >> 3, rr = lane & 7, gq = lane >> 2, cq = lane & 3;
  if ((int)blockIdx.x < n_tiles) {
    conv_stage_rows<W1, 8, 120, 160>(patches, x, blockIdx.x);
    w1_stage_dy(dys, dy, blockIdx.x);
  }
  cp_async_commit();
  // this lane's B row in k16 step s: pixel 32 warp + 16 s + 8 (mat & 1) + rr
  int prow[2], pcol[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int m = 32 * warp + 16 * s + 8 * (mat & 1) + rr;
    const int dyr = m / W1::Wo;
    prow[s] = 2 * dyr;
    pcol[s] = m - dyr * W1::Wo;
  }
  float acc[2][9][4], bsum = 0.f;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int n8 = 0; n8 < 9; ++n8)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[i][n8][v] = 0.f;
  int it = 0;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
    const int tn = t + (int)gridDim.x;
    if (tn < n_tiles) {
      conv_stage_rows<W1, 8, 120, 160>(patches + ((it + 1) & 1) * W1::PATCH, x, tn);
      w1_stage_dy(dys + ((it + 1) & 1) * kW1Dy, dy, tn);
    }
    cp_async_commit();
    cp_async_wait<1>();  // this tile's rows and gradients have landed
    __syncthreads();
    const bf16* patch = patches + (it & 1) * W1::PATCH;
    const bf16* dyt = dys + (it & 1) * kW1Dy;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int p0 = 32 * warp + 16 * s;
      uint32_t af[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int p = p0 + 8 * (mat >> 1) + rr, q = 2 * i + (mat & 1);
        ldsm_x4_t(af[i], dyt + 32 * p + 8 * (q ^ ((p >> 1) & 3)));
      }
#pragma unroll
      for (int t0 = 0; t0 < 9; t0 += 2) {
        // matrices: tap t0 and t0 + 1 (the last pair's second is tap 8 again,
        // unused), pixels p0 .. p0 + 7 and p0 + 8 .. p0 + 15
        const int tap = min(t0 + (mat >> 1), 8);
        const int ky = tap / 3, kx = tap - 3 * ky;
        const int r = prow[s] + ky, c = 2 * pcol[s] + kx;
        uint32_t bf[4];
        ldsm_x4_t(bf, patch + ((r * 2 + (c & 1)) * W1::WP + (c >> 1)) * 8);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          mma_bf16(acc[i][t0], af[i], bf[0], bf[1]);
          if (t0 + 1 < 9) mma_bf16(acc[i][t0 + 1], af[i], bf[2], bf[3]);
        }
      }
    }
    // bias: channel `lane` over this warp's 32 pixels (chunk lane / 8 of
    // pixel p sits at chunk (lane / 8) ^ ((p >> 1) & 3))
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      const int p = 32 * warp + j;
      bsum += __bfloat162float(dyt[32 * p + 8 * ((lane >> 3) ^ ((p >> 1) & 3)) + (lane & 7)]);
    }
    __syncthreads();  // the buffers are refilled next iteration
  }
  cp_async_wait<0>();
  __syncthreads();
  // the warps' sums, added in warp order: warp w's 32 x 72 block staged,
  // then every thread adds its elements over the warps
  float* red = reinterpret_cast<float*>(w1_smem);  // 5 x 2304 floats fit the buffers
  static_assert(5 * 32 * 72 * 4 <= kW1Smem, "reduction area");
  __shared__ float bred[W1::WARPS][32];
  bred[warp][lane] = bsum;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int n8 = 0; n8 < 9; ++n8)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int m = 16 * i + gq + 8 * (v >> 1), n = 8 * n8 + 2 * cq + (v & 1);
        red[(warp * 32 + m) * 72 + n] = acc[i][n8][v];
      }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 72; e += W1::NTHREADS) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < W1::WARPS; ++w) v += red[w * 32 * 72 + e];
    part[(size_t)blockIdx.x * kW1Part + e] = v;
  }
  if (threadIdx.x < 32) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < W1::WARPS; ++w) v += bred[w][threadIdx.x];
    part[(size_t)blockIdx.x * kW1Part + 32 * 72 + threadIdx.x] = v;
  }
}

// Layer 2's data gradient dX[b][iy][ix][ci] = mask(b, iy, ix, ci) x
// sum over the taps (ky, kx) that reach (iy, ix) of sum_co dY[b][oy][ox][co]
// W[co][ky][kx][ci] with oy = (iy + 1 - ky) / 2, ox = (ix + 1 - kx) / 2 (the
// transpose of the stride-2 convolution; iy even is reached by ky = 1 only,
// iy odd by ky in {0, 2}, likewise for columns), mask = (layer-1 output > 0)
// (the ReLU).  A tile is four input rows 4a .. 4a + 3 of one image; it needs
// output-gradient rows 2a .. 2a + 2 (41 columns, the last and a missing row
// staged as zeros), staged with the next tile's in flight, and the weights
// stay in shared memory for the block's whole walk.  The 320 pixels fall in
// the four parity classes of 80 pixels (5 m16 row tiles each); warp w takes
// row tile w of every class (9 taps x 64 output channels of K in all), so
// the warps are balanced; A = the pixels' gradient rows (ldmatrix), B = the
// tap's weights (ldmatrix .trans).  Results go through shared memory so the
// masked bf16 gradient is written in whole rows; the tile's mask rows are
// copied in (cp.async) while it computes.
constexpr int kD2Ci = 32, kD2Co = 64, kD2H = 60, kD2W = 80, kD2Ho = 30, kD2Wo = 40;
constexpr int kD2Rows = 4;                          // input rows per tile
constexpr int kD2Tpi = kD2H / kD2Rows;              // tiles per image
constexpr int kD2Cols = kD2Wo + 1;                  // staged gradient columns
constexpr int kD2Dy = 3 * kD2Cols * kD2Co;          // bf16 per staged gradient tile
constexpr int kD2Wt = 9 * kD2Co * kD2Ci;            // bf16 of the weights
constexpr int kD2Out = kD2Rows * kD2W * kD2Ci;      // bf16 of a tile's result
constexpr int kD2Threads = 160;
constexpr int kD2Smem = (2 * kD2Dy + kD2Wt + 2 * kD2Out) * 2;
static_assert(kD2Rows * kD2W == 4 * 5 * 16 && kD2H % kD2Rows == 0, "5 row tiles per class");
static_assert(kCin[1] == kD2Ci && kCout[1] == kD2Co && kHin[1] == kD2H && kWin[1] == kD2W &&
                  kHin[2] == kD2Ho && kWin[2] == kD2Wo,
              "layer 2");

__device__ __forceinline__ void d2_stage_dy(bf16* dst, const bf16* __restrict__ dy, int t) {
  const int b = t / kD2Tpi, oy0 = 2 * (t - b * kD2Tpi);
  // row lr, column ox, chunk q at chunk q ^ (ox & 7) of its 128-byte row
  for (int e = threadIdx.x; e < 3 * kD2Cols * 8; e += kD2Threads) {
    const int lr = e / (kD2Cols * 8), rem = e - lr * kD2Cols * 8;
    const int ox = rem >> 3, q = rem & 7, oy = oy0 + lr;
    const bool ok = oy < kD2Ho && ox < kD2Wo;
    cp_async16(dst + (lr * kD2Cols + ox) * kD2Co + 8 * (q ^ (ox & 7)),
               ok ? dy + (((size_t)b * kD2Ho + oy) * kD2Wo + ox) * kD2Co + 8 * q : dy, ok);
  }
}

__global__ void __launch_bounds__(kD2Threads, 2) dgrad2_kernel(const bf16* __restrict__ dy,
                                                              const bf16* __restrict__ wt,
                                                              const bf16* __restrict__ mask,
                                                              bf16* __restrict__ dx, int n_tiles) {
  extern __shared__ __align__(128) unsigned char d2_smem[];
  bf16* dys = reinterpret_cast<bf16*>(d2_smem);
  bf16* wts = dys + 2 * kD2Dy;
  bf16* outs = wts + kD2Wt;
  bf16* masks = outs + kD2Out;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mat = lane >> 3, rr = lane & 7, gq = lane >> 2, cq = lane & 3;
  // weights [tap][co][ci], chunk q of row co at q ^ ((co >> 1) & 3)
  for (int e = threadIdx.x; e < kD2Wt / 8; e += kD2Threads) {
    const int co = e / 36, rem = e - co * 36, tap = rem >> 2, q = rem & 3;
    cp_async16(wts + (tap * kD2Co + co) * kD2Ci + 8 * (q ^ ((co >> 1) & 3)),
               wt + (size_t)co * 9 * kD2Ci + tap * kD2Ci + 8 * q, true);
  }
  if ((int)blockIdx.x < n_tiles) d2_stage_dy(dys, dy, blockIdx.x);
  cp_async_commit();
  int it = 0;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
    // this tile's gradient rows (and the weights) have landed, and the last
    // tile's write-out is done with the result and mask buffers
    cp_async_wait<0>();
    __syncthreads();
    const int b = t / kD2Tpi, iy0 = kD2Rows * (t - b * kD2Tpi);
    const size_t base = ((size_t)b * kD2H + iy0) * kD2W * kD2Ci;
    for (int e = threadIdx.x; e < kD2Out / 8; e += kD2Threads)
      cp_async16(masks + 8 * e, mask + base + 8 * (size_t)e, true);
    cp_async_commit();
    const int tn = t + (int)gridDim.x;
    if (tn < n_tiles) d2_stage_dy(dys + ((it + 1) & 1) * kD2Dy, dy, tn);
    cp_async_commit();
    const bf16* dyt = dys + (it & 1) * kD2Dy;
#pragma unroll 1
    for (int cls = 0; cls < 4; ++cls) {
      const int pr = cls >> 1, pc = cls & 1;
      // this lane's A row: class pixel u = 16 warp + 8 (mat & 1) + rr
      const int u = 16 * warp + 8 * (mat & 1) + rr;
      const int r = pr + 2 * (u / kD2Wo), ix = pc + 2 * (u % kD2Wo);
      float acc[4][4];
#pragma unroll
      for (int n8 = 0; n8 < 4; ++n8)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[n8][v] = 0.f;
      const int nky = pr ? 2 : 1, nkx = pc ? 2 : 1;
      for (int tyi = 0; tyi < nky; ++tyi)
        for (int txi = 0; txi < nkx; ++txi) {
          const int ky = pr ? 2 * tyi : 1, kx = pc ? 2 * txi : 1;
          const int lr = (r + 1 - ky) >> 1, ox = (ix + 1 - kx) >> 1;
          const bf16* arow = dyt + (lr * kD2Cols + ox) * kD2Co;
          const bf16* wtap = wts + (ky * 3 + kx) * kD2Co * kD2Ci;
#pragma unroll
          for (int kk = 0; kk < kD2Co / 16; ++kk) {
            uint32_t af[4];
            ldsm_x4(af, arow + 8 * ((2 * kk + (mat >> 1)) ^ (ox & 7)));
            const int co = 16 * kk + 8 * (mat & 1) + rr;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              uint32_t bf[4];
              ldsm_x4_t(bf, wtap + co * kD2Ci + 8 * ((2 * h + (mat >> 1)) ^ ((co >> 1) & 3)));
              mma_bf16(acc[2 * h], af, bf[0], bf[1]);
              mma_bf16(acc[2 * h + 1], af, bf[2], bf[3]);
            }
          }
        }
      // bf16 results into the tile's [row][column][ci] staging, chunk n8 of
      // pixel ix at n8 ^ ((ix >> 1) & 3)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int uo = 16 * warp + gq + 8 * hh;
        const int ro = pr + 2 * (uo / kD2Wo), xo = pc + 2 * (uo % kD2Wo);
        bf16* orow = outs + (ro * kD2W + xo) * kD2Ci;
#pragma unroll
        for (int n8 = 0; n8 < 4; ++n8)
          *reinterpret_cast<__nv_bfloat162*>(orow + 8 * (n8 ^ ((xo >> 1) & 3)) + 2 * cq) =
              __floats2bfloat162_rn(acc[n8][2 * hh], acc[n8][2 * hh + 1]);
      }
    }
    cp_async_wait<1>();  // the mask rows have landed (the next gradient rows may not)
    __syncthreads();
    // masked rows out: 16-byte chunks
    {
      for (int e = threadIdx.x; e < kD2Out / 8; e += kD2Threads) {
        const int px = e >> 2, q = e & 3, ix = px % kD2W;
        const uint4 v = *reinterpret_cast<const uint4*>(outs + px * kD2Ci + 8 * (q ^ ((ix >> 1) & 3)));
        const uint4 m = *reinterpret_cast<const uint4*>(masks + 8 * e);
        const uint32_t vv[4] = {v.x, v.y, v.z, v.w}, mm[4] = {m.x, m.y, m.z, m.w};
        uint32_t o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          // a bf16 is > 0 iff its bits lie in [0x0001, 0x7F80] (positive,
          // nonzero, not NaN)
          const uint32_t lo = (mm[k] & 0xFFFFu) - 1u < 0x7F80u ? 0xFFFFu : 0u;
          const uint32_t hi = (mm[k] >> 16) - 1u < 0x7F80u ? 0xFFFF0000u : 0u;
          o[k] = vv[k] & (lo | hi);
        }
        *reinterpret_cast<uint4*>(dx + base + 8 * (size_t)e) = make_uint4(o[0], o[1], o[2], o[3]);
      }
    }
  }
  cp_async_wait<0>();
}

// Layer 2's weight and bias gradients dW[co][tap x 32 + ci] = sum_p dY[p][co]
// x[p, tap][ci], db[co] = sum_p dY[p][co], on the staging of wgrad1_kernel
// widened to 32 input channels: a tile is two output rows (80 pixels) of one
// image with its five input rows in column-parity planes and its 80 x 64
// output gradients (the next tile's in flight).  Warp w owns output channels
// 32 (w & 1) .. + 31 and the nine n8 column tiles 9 (w >> 1) .. + 8 of the
// 288 (tap, ci) columns: per 16 pixels two A fragments (dY^T, ldmatrix
// .trans) and nine B fragments (x, ldmatrix .trans), 18 mma.m16n8k16.  Thread
// t also adds channel t % 64 of the bias over pixels t / 64, + 4, ...  One
// partial per block ([64 x 288 | 64] floats; fixed grid, warps and blocks
// summed in a fixed order).
constexpr int kW2Ci = 32, kW2Co = 64, kW2H = 60, kW2W = 80, kW2Ho = 30, kW2Wo = 40;
constexpr int kW2Pix = 2 * kW2Wo;                     // output pixels per tile
constexpr int kW2Tpi = kW2Ho / 2;                     // tiles per image
constexpr int kW2Wp = (kW2W + 2) / 2;                 // entries per parity plane
constexpr int kW2Patch = 5 * 2 * kW2Wp * kW2Ci;       // bf16 per staged input tile
constexpr int kW2Dy = kW2Pix * kW2Co;                 // bf16 per staged gradient tile
constexpr int kW2Threads = 256;
constexpr int kW2Smem = (2 * kW2Patch + 2 * kW2Dy) * 2;
constexpr int kW2Grid = 2 * 152;                      // fixed grid: the partials' count
constexpr int kW2N = 9 * kW2Ci;
constexpr int kW2Part = kW2Co * kW2N + kW2Co;         // floats per block partial
static_assert(kCin[1] == kW2Ci && kCout[1] == kW2Co && kHin[1] == kW2H && kWin[1] == kW2W &&
                  kHin[2] == kW2Ho && kWin[2] == kW2Wo,
              "layer 2");
static_assert(kW2Pix % 16 == 0 && 8 * 4 * 9 * 8 == kW2Co * kW2N / 8, "warp split");

__device__ __forceinline__ void w2_stage(bf16* patch, bf16* dys, const bf16* __restrict__ x,
                                         const bf16* __restrict__ dy, int t) {
  const int b = t / kW2Tpi, oy0 = 2 * (t - b * kW2Tpi), iy0 = 2 * oy0 - 1;
  const bf16* xb = x + (size_t)b * kW2H * kW2W * kW2Ci;
  // input row r, padded column c = ix + 1: plane c & 1, entry c >> 1, chunk
  // q at q ^ ((entry >> 1) & 3)
  constexpr int ROWCH = (kW2W + 2) * 4;
  for (int e = threadIdx.x; e < 5 * ROWCH; e += kW2Threads) {
    const int r = e / ROWCH, rem = e - r * ROWCH;
    const int c = rem >> 2, q = rem & 3;
    const int iy = iy0 + r, ix = c - 1;
    const bool ok = iy >= 0 && iy < kW2H && ix >= 0 && ix < kW2W;
    const int ent = c >> 1;
    cp_async16(patch + ((r * 2 + (c & 1)) * kW2Wp + ent) * kW2Ci + 8 * (q ^ ((ent >> 1) & 3)),
               ok ? xb + ((size_t)iy * kW2W + ix) * kW2Ci + 8 * q : xb, ok);
  }
  // gradient pixel p, chunk q at q ^ (p & 7)
  const bf16* src = dy + ((size_t)b * kW2Ho + oy0) * kW2Wo * kW2Co;
  for (int e = threadIdx.x; e < kW2Dy / 8; e += kW2Threads) {
    const int p = e >> 3, q = e & 7;
    cp_async16(dys + p * kW2Co + 8 * (q ^ (p & 7)), src + 8 * e, true);
  }
}

__global__ void __launch_bounds__(kW2Threads) wgrad2_kernel(const bf16* __restrict__ x,
                                                            const bf16* __restrict__ dy,
                                                            float* __restrict__ part,
                                                            int n_tiles) {
  extern __shared__ __align__(128) unsigned char w2_smem[];
  bf16* patches = reinterpret_cast<bf16*>(w2_smem);
  bf16* dys = patches + 2 * kW2Patch;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mat = lane >> 3, rr = lane & 7, gq = lane >> 2, cq = lane & 3;
  const int mh = warp & 1, j0 = 9 * (warp >> 1);
  if ((int)blockIdx.x < n_tiles) w2_stage(patches, dys, x, dy, blockIdx.x);
  cp_async_commit();
  float acc[2][9][4], bsum = 0.f;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int n8 = 0; n8 < 9; ++n8)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[i][n8][v] = 0.f;
  int it = 0;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
    const int tn = t + (int)gridDim.x;
    if (tn < n_tiles)
      w2_stage(patches + ((it + 1) & 1) * kW2Patch, dys + ((it + 1) & 1) * kW2Dy, x, dy, tn);
    cp_async_commit();
    cp_async_wait<1>();  // this tile's rows and gradients have landed
    __syncthreads();
    const bf16* patch = patches + (it & 1) * kW2Patch;
    const bf16* dyt = dys + (it & 1) * kW2Dy;
#pragma unroll 1
    for (int p0 = 0; p0 < kW2Pix; p0 += 16) {
      uint32_t af[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int p = p0 + 8 * (mat >> 1) + rr, q = 4 * mh + 2 * i + (mat & 1);
        ldsm_x4_t(af[i], dyt + p * kW2Co + 8 * (q ^ (p & 7)));
      }
      // this lane's B row: pixel p0 + 8 (mat & 1) + rr
      const int pb = p0 + 8 * (mat & 1) + rr;
      const int dyr = pb / kW2Wo, ox = pb - dyr * kW2Wo;
#pragma unroll
      for (int jj = 0; jj < 9; jj += 2) {
        // matrices: column tiles j0 + jj and j0 + jj + 1 (the last pair's
        // second repeats the first, unused)
        const int j = j0 + min(jj + (mat >> 1), 8);
        const int tap = j >> 2, q = j & 3;
        const int ky = tap / 3, kx = tap - 3 * ky;
        const int r = 2 * dyr + ky, c = 2 * ox + kx, ent = c >> 1;
        uint32_t bf[4];
        ldsm_x4_t(bf, patch + ((r * 2 + (c & 1)) * kW2Wp + ent) * kW2Ci + 8 * (q ^ ((ent >> 1) & 3)));
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          mma_bf16(acc[i][jj], af[i], bf[0], bf[1]);
          if (jj + 1 < 9) mma_bf16(acc[i][jj + 1], af[i], bf[2], bf[3]);
        }
      }
    }
    {  // bias: channel threadIdx.x % 64 over pixels threadIdx.x / 64 + 4 k
      const int c = threadIdx.x & 63;
#pragma unroll 4
      for (int p = threadIdx.x >> 6; p < kW2Pix; p += 4)
        bsum += __bfloat162float(dyt[p * kW2Co + 8 * ((c >> 3) ^ (p & 7)) + (c & 7)]);
    }
    __syncthreads();  // the buffers are refilled next iteration
  }
  cp_async_wait<0>();
  __syncthreads();
  // the warps' blocks are disjoint: every warp writes its 32 x 72 block; the
  // bias's four pixel groups are added in order
  float* out = part + (size_t)blockIdx.x * kW2Part;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int n8 = 0; n8 < 9; ++n8)
#pragma unroll
      for (int hv = 0; hv < 2; ++hv) {
        const int m = 32 * mh + 16 * i + gq + 8 * hv, n = 8 * (j0 + n8) + 2 * cq;
        *reinterpret_cast<float2*>(out + m * kW2N + n) =
            make_float2(acc[i][n8][2 * hv], acc[i][n8][2 * hv + 1]);
      }
  float* red = reinterpret_cast<float*>(w2_smem);
  red[threadIdx.x] = bsum;
  __syncthreads();
  if (threadIdx.x < kW2Co)
    out[kW2Co * kW2N + threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + 64] +
                                      red[threadIdx.x + 128] + red[threadIdx.x + 192];
}

// out[m * n_out + n] = sum_s part[(s * M + m) * N + n] for m < m_valid,
// n < n_valid, summed in split order.
__global__ void reduce_partials_kernel(const float* __restrict__ part, int S, int M, int N,
                                       int m_valid, int n_valid, float* __restrict__ out) {
  const size_t total = (size_t)m_valid * n_valid;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(e / n_valid), n = (int)(e % n_valid);
    float acc = 0.f;
    for (int s = 0; s < S; ++s) acc += part[((size_t)s * M + m) * N + n];
    out[e] = acc;
  }
}

// sum_s part[s * ld + e] for e < E with many partials, into out0[e] for
// e < E0 and out1[e - E0] beyond: block (32, 32) takes 32 consecutive e,
// thread (x, y) adds s = y, y + 32, ... in order, and the 32 row sums are
// added in y order (a fixed order, so the result does not depend on timing).
__global__ void __launch_bounds__(1024) reduce_partials_wide_kernel(
    const float* __restrict__ part, int S, int ld, int E, int E0, float* __restrict__ out0,
    float* __restrict__ out1) {
  __shared__ float rows[32][33];
  const int e = blockIdx.x * 32 + threadIdx.x;
  float acc = 0.f;
  if (e < E)
#pragma unroll 8
    for (int s = threadIdx.y; s < S; s += 32) acc += part[(size_t)s * ld + e];
  rows[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && e < E) {
    float v = 0.f;
#pragma unroll
    for (int y = 0; y < 32; ++y) v += rows[y][threadIdx.x];
    if (e < E0)
      out0[e] = v;
    else
      out1[e - E0] = v;
  }
}

// Column sums of a bf16 matrix [rows][C] (C a multiple of 8 dividing 2048)
// over chunks of rows: part[chunk * C + c].  Thread t sums columns
// 8 (t % (C/8)) .. +7 over rows sub, sub + nsub, ... of the chunk (16-byte
// loads, a warp reads whole rows); the subs are then added in order.
__global__ void __launch_bounds__(256) colsum_partial_kernel(const bf16* __restrict__ z, int rows,
                                                             int C, int rows_per_block,
                                                             float* __restrict__ part) {
  __shared__ float s[256 * 8];
  const int t = threadIdx.x, groups = C / 8, nsub = 256 / groups;
  const int g8 = t % groups, sub = t / groups;
  const int r0 = blockIdx.x * rows_per_block, r1 = min(rows, r0 + rows_per_block);
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (sub < nsub)
    for (int r = r0 + sub; r < r1; r += nsub) {
      const uint4 v = *reinterpret_cast<const uint4*>(z + (size_t)r * C + 8 * g8);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[2 * q] += __low2float(h[q]);
        acc[2 * q + 1] += __high2float(h[q]);
      }
    }
#pragma unroll
  for (int q = 0; q < 8; ++q) s[t * 8 + q] = acc[q];
  __syncthreads();
  for (int c = t; c < C; c += 256) {
    const int gc = c / 8, q = c % 8;
    float tot = 0.f;
    for (int k = 0; k < nsub; ++k) tot += s[(k * groups + gc) * 8 + q];
    part[(size_t)blockIdx.x * C + c] = tot;
  }
}

// bfloat16 copy of the weights; FC2 rows padded with zeros to 8.
struct CastArgs {
  const float* src[kLayers];
  bf16* dst[kLayers];
  int count[kLayers];      // floats copied
  int padded[kLayers];     // bf16 elements written (>= count; the rest zero)
};
__global__ void cast_weights_kernel(const CastArgs a) {
  const int L = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.padded[L]; i += gridDim.x * blockDim.x)
    a.dst[L][i] = __float2bfloat16_rn(i < a.count[L] ? a.src[L][i] : 0.f);
}

// Loss 1/(2B) sum |y - t|^2 (one block, fixed order) and dz2 = (y - t) / B
// in bf16, [B][8] with the two padding columns zero.
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ y,
                                                   const float* __restrict__ t, int B,
                                                   float* __restrict__ loss, bf16* __restrict__ dz) {
  __shared__ float s[256];
  float acc = 0.f;
  const float inv = 1.f / (float)B;
  for (int e = threadIdx.x; e < B * kOutPad; e += 256) {
    const int b = e / kOutPad, j = e % kOutPad;
    float d = 0.f;
    if (j < kOut) {
      d = y[b * kOut + j] - t[b * kOut + j];
      acc += d * d;
    }
    dz[e] = __float2bfloat16_rn(d * inv);
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = 0.5f * s[0] * inv;
}

// Box downsampling of an observed RGB-D frame by an integer factor: each
// output pixel is the mean colour of its factor x factor block and the mean
// of the block's valid (finite, positive) depths, 0 if it has none.  Sums in
// row-major order within the block.
__global__ void __launch_bounds__(256) downsample_kernel(const float* __restrict__ rgb,
                                                         const float* __restrict__ depth, int W,
                                                         int f, int wo, int n,
                                                         float* __restrict__ rgb_out,
                                                         float* __restrict__ depth_out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int oy = o / wo, ox = o % wo;
  float r = 0.f, g = 0.f, b = 0.f, d = 0.f;
  int nd = 0;
  for (int dy = 0; dy < f; ++dy) {
    const size_t row = (size_t)(oy * f + dy) * W + (size_t)ox * f;
    for (int dx = 0; dx < f; ++dx) {
      const size_t p = row + dx;
      r += rgb[3 * p];
      g += rgb[3 * p + 1];
      b += rgb[3 * p + 2];
      const float z = depth[p];
      if (z > 0.f && z < INFINITY) {
        d += z;
        ++nd;
      }
    }
  }
  const float inv = 1.f / (float)(f * f);
  rgb_out[3 * o] = r * inv;
  rgb_out[3 * o + 1] = g * inv;
  rgb_out[3 * o + 2] = b * inv;
  depth_out[o] = nd ? d / (float)nd : 0.f;
}

__global__ void pack_kernel(const float* __restrict__ r_rgb, const float* __restrict__ r_d,
                            const float* __restrict__ r_o, const float* __restrict__ o_rgb,
                            const float* __restrict__ o_d, size_t n_px, bf16* __restrict__ x) {
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_px;
       p += (size_t)gridDim.x * blockDim.x) {
    const float o = r_o[p];
    const float dr = o > 0.5f ? r_d[p] / o - GS2D_NET_DEPTH_OFFSET : 0.f;
    const float od = o_d[p];
    const float dd = od > 0.f ? od - GS2D_NET_DEPTH_OFFSET : 0.f;
    __nv_bfloat162 v[4];
    v[0] = __floats2bfloat162_rn(r_rgb[3 * p], r_rgb[3 * p + 1]);
    v[1] = __floats2bfloat162_rn(r_rgb[3 * p + 2], dr);
    v[2] = __floats2bfloat162_rn(o_rgb[3 * p], o_rgb[3 * p + 1]);
    v[3] = __floats2bfloat162_rn(o_rgb[3 * p + 2], dd);
    *reinterpret_cast<uint4*>(x + 8 * p) = *reinterpret_cast<const uint4*>(v);
  }
}

__global__ void adamw_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                             float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps,
                             float wd, float bc1, float bc2) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    float pi = p[i] * (1.f - lr * wd);
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    pi -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
  }
}

__global__ void apply_kernel(const float* __restrict__ y, int B, float* __restrict__ poses) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float tau[6], dR[9], dt[3], R[9], t[3];
  for (int k = 0; k < 6; ++k) tau[k] = y[6 * b + k] * GS2D_NET_TAU_SCALE;
  se3_exp_f(tau, dR, dt);
  float* P = poses + 12 * b;
  for (int k = 0; k < 9; ++k) R[k] = P[k];
  for (int k = 0; k < 3; ++k) t[k] = P[9 + k];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c)
      P[3 * r + c] = dR[3 * r] * R[c] + dR[3 * r + 1] * R[3 + c] + dR[3 * r + 2] * R[6 + c];
    P[9 + r] = dR[3 * r] * t[0] + dR[3 * r + 1] * t[1] + dR[3 * r + 2] * t[2] + dt[r];
  }
}

// SE(3) logarithm: rotation vector w with |w| = atan2(|v| / 2, (tr R - 1) / 2)
// along v = vee(R - R^T), rho = V(w)^-1 t with V^-1 = I - K/2 +
// (1 - A / (2B)) / th^2 K^2, A = sin th / th, B = (1 - cos th) / th^2.
__device__ __forceinline__ void se3_log_f(const float R[9], const float t[3], float tau[6]) {
  const float vx = R[7] - R[5], vy = R[2] - R[6], vz = R[3] - R[1];
  const float s2 = 0.5f * sqrtf(vx * vx + vy * vy + vz * vz);
  const float c = 0.5f * (R[0] + R[4] + R[8] - 1.f);
  const float th = atan2f(s2, c);
  const float f = s2 > 1e-7f ? th / (2.f * s2) : 0.5f;
  const float w[3] = {f * vx, f * vy, f * vz};
  const float th2 = th * th;
  float D;
  if (th < 1e-2f) {
    D = 1.f / 12.f + th2 / 720.f;
  } else {
    const float A = sinf(th) / th, B = (1.f - cosf(th)) / th2;
    D = (1.f - A / (2.f * B)) / th2;
  }
  const float K[9] = {0.f, -w[2], w[1], w[2], 0.f, -w[0], -w[1], w[0], 0.f};
  for (int r = 0; r < 3; ++r) {
    float acc = 0.f;
    for (int q = 0; q < 3; ++q) {
      const float K2 = K[3 * r] * K[q] + K[3 * r + 1] * K[3 + q] + K[3 * r + 2] * K[6 + q];
      const float Vi = ((r == q) ? 1.f : 0.f) - 0.5f * K[3 * r + q] + D * K2;
      acc += Vi * t[q];
    }
    tau[r] = acc;
  }
  tau[3] = w[0];
  tau[4] = w[1];
  tau[5] = w[2];
}

__global__ void target_kernel(const float* __restrict__ init, const float* __restrict__ gt, int B,
                              float* __restrict__ target) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float* Pi = init + 12 * b;
  const float* Pg = gt + 12 * b;
  float R[9], t[3], tau[6];
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q)
      R[3 * r + q] = Pg[3 * r] * Pi[3 * q] + Pg[3 * r + 1] * Pi[3 * q + 1] + Pg[3 * r + 2] * Pi[3 * q + 2];
  for (int r = 0; r < 3; ++r)
    t[r] = Pg[9 + r] - (R[3 * r] * Pi[9] + R[3 * r + 1] * Pi[10] + R[3 * r + 2] * Pi[11]);
  se3_log_f(R, t, tau);
  for (int k = 0; k < 6; ++k) target[6 * b + k] = tau[k] / GS2D_NET_TAU_SCALE;
}

__global__ void accept_kernel(const float* __restrict__ lp, const float* __restrict__ li,
                              const float* __restrict__ prop, int B, float* __restrict__ poses,
                              int32_t* __restrict__ accepted) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const bool take = lp[b] <= li[b];
  if (take)
    for (int k = 0; k < 12; ++k) poses[12 * b + k] = prop[12 * b + k];
  if (accepted) accepted[b] = take ? 1 : 0;
}

// Where the proposal of element b is taken (the same test as accept_kernel,
// evaluated before accept_kernel updates anything), its rendered images
// replace the kept ones: n_px pixels of colour (3 floats), accumulated depth
// and opacity per element.
__global__ void keep_images_kernel(const float* __restrict__ lp, const float* __restrict__ li,
                                   int B, size_t n_px, const float* __restrict__ p_rgb,
                                   const float* __restrict__ p_d, const float* __restrict__ p_o,
                                   float* __restrict__ k_rgb, float* __restrict__ k_d,
                                   float* __restrict__ k_o) {
  const size_t per = 5 * n_px;  // floats per element: rgb, depth, opacity
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)B * per;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t b = e / per, r = e - b * per;
    if (!(lp[b] <= li[b])) continue;
    if (r < 3 * n_px) {
      k_rgb[b * 3 * n_px + r] = p_rgb[b * 3 * n_px + r];
    } else if (r < 4 * n_px) {
      k_d[b * n_px + r - 3 * n_px] = p_d[b * n_px + r - 3 * n_px];
    } else {
      k_o[b * n_px + r - 4 * n_px] = p_o[b * n_px + r - 4 * n_px];
    }
  }
}

// accept_kernel, and the kept pose's loss: loss_init[b] <- loss_prop[b]
// where the proposal is taken.
__global__ void accept_loss_kernel(const float* __restrict__ lp, float* __restrict__ li,
                                   const float* __restrict__ prop, int B, float* __restrict__ poses,
                                   int32_t* __restrict__ accepted) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const bool take = lp[b] <= li[b];
  if (take) {
    for (int k = 0; k < 12; ++k) poses[12 * b + k] = prop[12 * b + k];
    li[b] = lp[b];
  }
  if (accepted) accepted[b] = take ? 1 : 0;
}

// ---------------------------------------------------------------------------
// host side
struct Layout {
  size_t w_off[kLayers], b_off[kLayers], total;
  int fan_in[kLayers], rows[kLayers], wcount[kLayers], wpadded[kLayers];
  size_t wbf_off[kLayers], wbf_total;  // bf16 weight copy (elements)
};

Layout layout() {
  Layout L{};
  size_t off = 0, boff = 0;
  for (int l = 0; l < kLayers; ++l) {
    int rows, fan;
    if (l < kConv) {
      rows = kCout[l];
      fan = 9 * kCin[l];
    } else if (l == kConv) {
      rows = kHidden;
      fan = kFlat;
    } else {
      rows = kOut;
      fan = kHidden;
    }
    L.rows[l] = rows;
    L.fan_in[l] = fan;
    L.w_off[l] = off;
    off += (size_t)rows * fan;
    L.b_off[l] = off;
    off += rows;
    L.wcount[l] = rows * fan;
    L.wpadded[l] = (l == kLayers - 1 ? kOutPad : rows) * fan;
    L.wbf_off[l] = boff;
    boff += align_up((size_t)L.wpadded[l], 64);
  }
  L.total = off;
  L.wbf_total = boff;
  return L;
}

struct Ws {
  bf16* wbf;
  bf16* act[kConv + 1];  // act[0] unused (the caller's x), act[1..6] conv outputs
  bf16* h;               // [B][256]
  float* y;              // [B][6]
  bf16* dz2;             // [B][8]
  bf16* dzA;
  bf16* dzB;
  float* part;
  size_t part_floats;
  float* loss;
  int* err;              // tensor-core wait timeouts (0 = none)
  size_t bytes;
};

int splits_for(int M, int N, int K) {
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  int s = (2 * 152 + tiles - 1) / tiles;
  s = max(1, min(s, (K + 255) / 256));
  return s;
}
int k_split_for(int K, int s) { return (int)align_up((size_t)((K + s - 1) / s), 64); }

// Split-K count of a forward or data-gradient GEMM from its shape per sample
// at a nominal batch of 256 -- never from the actual batch, so every output
// row sums the same K ranges in the same order whatever the batch size.
constexpr int kNominalBatch = 256;
int splits_nominal(int rows_per_sample, int N, int K) {
  const long long tiles = ((long long)rows_per_sample * kNominalBatch + BM - 1) / BM *
                          ((N + BN - 1) / BN);
  if (tiles >= 2 * 152) return 1;
  const int s = (int)((2 * 152 + tiles - 1) / tiles);
  return max(1, min(s, K / 128));
}
int splits_count(int K, int s) {
  const int ks = s > 1 ? k_split_for(K, s) : (int)align_up((size_t)K, 64);
  return max((K + ks - 1) / ks, 1);
}
int class_hc(int H, int py) { return (H + 1 - py) / 2; }

// Rows per block of the bias-gradient column sums: about 304 blocks, a
// multiple of the rows one pass of the block covers (256 / (C / 8)).
int colsum_rows_per_block(int rows, int C) {
  const int nsub = 256 / (C / 8);
  const int want = (rows + 303) / 304;
  return max(nsub, (want + nsub - 1) / nsub * nsub);
}

size_t max_partials(int B) {
  // layers 1 and 2's weight and bias gradients
  size_t mx = max((size_t)kW1Grid * kW1Part, (size_t)kW2Grid * kW2Part);
  auto upd = [&](int M, int N, int K) {
    const int s = splits_for(M, N, K);
    const int ks = k_split_for(K, s);
    const int S = (K + ks - 1) / ks;
    mx = max(mx, (size_t)S * M * N);
  };
  auto nom = [&](int rps, int N, int K) {
    mx = max(mx, (size_t)splits_count(K, splits_nominal(rps, N, K)) * B * rps * N);
  };
  for (int l = 0; l < kConv; ++l) {
    upd(kCout[l], 9 * kCin[l], B * kHin[l + 1] * kWin[l + 1]);
    const int rows = B * kHin[l + 1] * kWin[l + 1];
    const int rpb = colsum_rows_per_block(rows, kCout[l]);
    mx = max(mx, (size_t)((rows + rpb - 1) / rpb) * kCout[l]);
    nom(kHin[l + 1] * kWin[l + 1], kCout[l], 9 * kCin[l]);
    for (int py = 0; py < 2; ++py)
      for (int px = 0; px < 2; ++px)
        nom(class_hc(kHin[l], py) * class_hc(kWin[l], px), kCin[l],
            (py ? 2 : 1) * (px ? 2 : 1) * kCout[l]);
  }
  upd(kHidden, kFlat, B);
  upd(kOutPad, kHidden, B);
  nom(1, kHidden, kFlat);
  nom(1, kOutPad, kHidden);
  nom(1, kFlat, kHidden);
  nom(1, kHidden, kOutPad);
  for (const int C : {kHidden, kOutPad}) {
    const int rpb = colsum_rows_per_block(B, C);
    mx = max(mx, (size_t)((B + rpb - 1) / rpb) * C);
  }
  return mx;
}

Ws carve(void* base, int B) {
  const Layout L = layout();
  Ws w{};
  Carver c(base);
  w.wbf = c.take<bf16>(L.wbf_total);
  size_t dz_max = (size_t)B * kFlat;
  for (int l = 1; l <= kConv; ++l) {
    const size_t n = (size_t)B * kHin[l] * kWin[l] * kCout[l - 1];
    w.act[l] = c.take<bf16>(n);
    dz_max = max(dz_max, n);
  }
  w.h = c.take<bf16>((size_t)B * kHidden);
  w.y = c.take<float>((size_t)B * kOut);
  w.dz2 = c.take<bf16>((size_t)B * kOutPad);
  w.dzA = c.take<bf16>(dz_max);
  w.dzB = c.take<bf16>(dz_max);
  w.part_floats = max_partials(B);
  w.part = c.take<float>(w.part_floats);
  w.loss = c.take<float>(64);
  w.err = c.take<int>(64);
  w.bytes = align_up(c.off, 256);
  return w;
}

Operand op(const bf16* p, int ld, int rows) {
  Operand o{};
  o.p = p;
  o.ld = ld;
  o.rows = rows;
  return o;
}
int log2_exact(int v) {
  int s = 0;
  while ((1 << s) < v) ++s;
  return s;
}
// Gathers over the output grid of conv layer l (K_IM2COL, R_IM2COL) with C
// channels of the gathered tensor (a power of two).
Operand conv_op(const bf16* p, int rows, int l, int C) {
  Operand o{};
  o.p = p;
  o.rows = rows;
  o.H = kHin[l];
  o.W = kWin[l];
  o.Ho = kHin[l + 1];
  o.Wo = kWin[l + 1];
  o.C = C;
  o.c_shift = log2_exact(C);
  o.f_hw = make_fastdiv((uint32_t)(o.Ho * o.Wo));
  o.f_w = make_fastdiv((uint32_t)o.Wo);
  return o;
}

// Launches one GEMM.  Split-K partial products (the deep-K weight
// gradients and the split deep layers) run on the tcgen05 kernel; GEMMs with
// a direct epilogue (large M, the gather-bound convolutions) on the mma.sync
// kernel, whose smaller blocks keep more warps resident to hide the gathers
// (measured on the batch-256 training step: all mma.sync 2.38 ms, this split
// 2.46 ms, all tcgen05 3.19 ms).
template <int AM, int BMODE, int EPI>
int run(Gemm g, int splits, cudaStream_t st, int* n_splits = nullptr) {
  constexpr bool tc = EPI == E_PARTIAL;
  const int align = tc ? TC_BK : BK;
  g.k_split = splits > 1 ? k_split_for(g.K, splits) : (int)align_up((size_t)g.K, align);
  const int S = max((g.K + g.k_split - 1) / g.k_split, 1);
  const dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, S);
  if (grid.y > 65535 || grid.z > 65535) return GS2D_ERR_INVALID_ARG;
  if constexpr (tc) {
    static bool ready[64] = {};
    int dev = 0;
    GS2D_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GS2D_ERR_CUDA;
    if (!ready[dev]) {
      GS2D_CUDA_TRY(cudaFuncSetAttribute(gemm_tc_kernel<AM, BMODE, EPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
      ready[dev] = true;
    }
    gemm_tc_kernel<AM, BMODE, EPI><<<grid, TC_THREADS, TC_SMEM, st>>>(g);
  } else {
    gemm_kernel<AM, BMODE, EPI><<<grid, THREADS, 0, st>>>(g);
  }
  GS2D_LAUNCH_CHECK();
  if (n_splits) *n_splits = S;
  return GS2D_OK;
}

// A forward or data-gradient GEMM with its epilogue: split-K (at the
// nominal-batch count for rows_per_sample) through FP32 partials and a
// fixed-order reduction when the tile grid is small.
template <int AM, int BMODE, int EPI>
int fused(Gemm g, int rows_per_sample, float* part, cudaStream_t st) {
  const int s = splits_nominal(rows_per_sample, g.N, g.K);
  if (s <= 1) return run<AM, BMODE, EPI>(g, 1, st);
  g.part = part;
  int S = 0;
  int r = run<AM, BMODE, E_PARTIAL>(g, s, st, &S);
  if (r) return r;
  const size_t pairs = (size_t)g.M * (g.N / 2);
  const int blocks = (int)max((size_t)1, min((pairs + 255) / 256, (size_t)4096));
  splitk_epilogue_kernel<EPI><<<blocks, 256, 0, st>>>(g, S);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

// weight gradient by split-K partials, reduced into out (m_valid x N)
template <int AM, int BMODE>
int wgrad(Gemm g, int m_valid, float* part, float* out, cudaStream_t st) {
  g.part = part;
  int S = 0;
  const int r = run<AM, BMODE, E_PARTIAL>(g, splits_for(g.M, g.N, g.K), st, &S);
  if (r) return r;
  const size_t total = (size_t)m_valid * g.N;
  const int blocks = (int)min((total + 255) / 256, (size_t)4096);
  reduce_partials_kernel<<<blocks, 256, 0, st>>>(part, S, g.M, g.N, m_valid, g.N, out);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

// Layer 1's weight gradient (wgrad1_kernel) into out_w [32][72] and its
// bias gradient into out_b [32].
int wgrad1(const bf16* x, const bf16* dy, int B, float* part, float* out_w, float* out_b,
           cudaStream_t st) {
  static bool ready[64] = {};
  int dev = 0;
  GS2D_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return GS2D_ERR_CUDA;
  if (!ready[dev]) {
    GS2D_CUDA_TRY(cudaFuncSetAttribute(wgrad1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kW1Smem));
    ready[dev] = true;
  }
  const long long n_tiles = (long long)B * W1::TPI;
  if (n_tiles <= 0 || n_tiles > 0x7FFFFFFF) return n_tiles <= 0 ? GS2D_OK : GS2D_ERR_INVALID_ARG;
  // a fixed grid (the partials' count), idle blocks contributing zeros
  wgrad1_kernel<<<kW1Grid, W1::NTHREADS, kW1Smem, st>>>(x, dy, part, (int)n_tiles);
  GS2D_LAUNCH_CHECK();
  reduce_partials_wide_kernel<<<kW1Part / 32, dim3(32, 32), 0, st>>>(part, kW1Grid, kW1Part,
                                                                     kW1Part, 32 * 72, out_w, out_b);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

// Layer 2's data gradient (dgrad2_kernel): dy [B][30][40][64], the layer's
// bf16 weights, mask = the layer-1 output [B][60][80][32], dx like mask.
int dgrad2(const bf16* dy, int B, const bf16* wt, const bf16* mask, bf16* dx, cudaStream_t st) {
  static int slots[64] = {};  // resident blocks per device (0: not yet known)
  int dev = 0;
  GS2D_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return GS2D_ERR_CUDA;
  if (!slots[dev]) {
    GS2D_CUDA_TRY(
        cudaFuncSetAttribute(dgrad2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kD2Smem));
    int per_sm = 0, sms = 0;
    GS2D_CUDA_TRY(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dgrad2_kernel, kD2Threads, kD2Smem));
    GS2D_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    slots[dev] = max(1, per_sm) * max(1, sms);
  }
  if (B <= 0) return GS2D_OK;
  const long long n_tiles = (long long)B * kD2Tpi;
  if (n_tiles > 0x7FFFFFFF) return GS2D_ERR_INVALID_ARG;
  const int grid = (int)(n_tiles < (long long)slots[dev] ? n_tiles : (long long)slots[dev]);
  dgrad2_kernel<<<grid, kD2Threads, kD2Smem, st>>>(dy, wt, mask, dx, (int)n_tiles);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

// Layer 2's weight gradient (wgrad2_kernel) into out_w [64][288] and its
// bias gradient into out_b [64].
int wgrad2(const bf16* x, const bf16* dy, int B, float* part, float* out_w, float* out_b,
           cudaStream_t st) {
  static bool ready[64] = {};
  int dev = 0;
  GS2D_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return GS2D_ERR_CUDA;
  if (!ready[dev]) {
    GS2D_CUDA_TRY(cudaFuncSetAttribute(wgrad2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kW2Smem));
    ready[dev] = true;
  }
  const long long n_tiles = (long long)B * kW2Tpi;
  if (n_tiles <= 0 || n_tiles > 0x7FFFFFFF) return n_tiles <= 0 ? GS2D_OK : GS2D_ERR_INVALID_ARG;
  wgrad2_kernel<<<kW2Grid, kW2Threads, kW2Smem, st>>>(x, dy, part, (int)n_tiles);
  GS2D_LAUNCH_CHECK();
  reduce_partials_wide_kernel<<<kW2Part / 32, dim3(32, 32), 0, st>>>(part, kW2Grid, kW2Part, kW2Part,
                                                                     kW2Co * kW2N, out_w, out_b);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int bias_grad(const bf16* z, int rows, int C, int c_valid, float* part, float* out, cudaStream_t st) {
  const int rpb = colsum_rows_per_block(rows, C);
  const int chunks = (rows + rpb - 1) / rpb;
  colsum_partial_kernel<<<chunks, 256, 0, st>>>(z, rows, C, rpb, part);
  GS2D_LAUNCH_CHECK();
  reduce_partials_wide_kernel<<<(c_valid + 31) / 32, dim3(32, 32), 0, st>>>(part, chunks, C, c_valid,
                                                                           c_valid, out, nullptr);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int cast(const float* params, const Ws& w, cudaStream_t st) {
  const Layout L = layout();
  CastArgs a{};
  for (int l = 0; l < kLayers; ++l) {
    a.src[l] = params + L.w_off[l];
    a.dst[l] = w.wbf + L.wbf_off[l];
    a.count[l] = L.wcount[l];
    a.padded[l] = L.wpadded[l];
  }
  cast_weights_kernel<<<dim3(64, kLayers), 256, 0, st>>>(a);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int forward(const float* params, const bf16* x, int B, const Ws& w, float* y, cudaStream_t st,
            bool do_cast = true) {
  const Layout L = layout();
  GS2D_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  int r = do_cast ? cast(params, w, st) : GS2D_OK;
  if (r) return r;
  // layer 1: the direct kernel
  r = conv_s2<8, 32, 120, 160, 2>(x, B, w.wbf + L.wbf_off[0], params + L.b_off[0], w.act[1], st);
  if (r) return r;
  const bf16* in = w.act[1];
  for (int l = 1; l < kConv; ++l) {
    if (conv_tma_layer(l)) {
      // layers 2-4: tcgen05 with TMA-fed operands
      r = conv_tma_forward(l, in, B, w.wbf + L.wbf_off[l], params + L.b_off[l], w.act[l + 1],
                           w.err, st);
      if (r) return r;
      in = w.act[l + 1];
      continue;
    }
    Gemm g{};
    g.err = w.err;
    g.M = B * kHin[l + 1] * kWin[l + 1];
    g.N = kCout[l];
    g.K = 9 * kCin[l];
    g.a = conv_op(in, g.M, l, kCin[l]);
    g.b = op(w.wbf + L.wbf_off[l], g.K, g.N);
    g.out = w.act[l + 1];
    g.ldc = g.N;
    g.bias = params + L.b_off[l];
    r = fused<K_IM2COL, K_DENSE, E_BIAS_RELU>(g, kHin[l + 1] * kWin[l + 1], w.part, st);
    if (r) return r;
    in = w.act[l + 1];
  }
  {
    Gemm g{};
    g.err = w.err;
    g.M = B;
    g.N = kHidden;
    g.K = kFlat;
    g.a = op(in, kFlat, B);
    g.b = op(w.wbf + L.wbf_off[kConv], kFlat, kHidden);
    g.out = w.h;
    g.ldc = kHidden;
    g.bias = params + L.b_off[kConv];
    r = fused<K_DENSE, K_DENSE, E_BIAS_RELU>(g, 1, w.part, st);
    if (r) return r;
  }
  {
    Gemm g{};
    g.err = w.err;
    g.M = B;
    g.N = kOutPad;
    g.K = kHidden;
    g.a = op(w.h, kHidden, B);
    g.b = op(w.wbf + L.wbf_off[kConv + 1], kHidden, kOutPad);
    g.out = y;
    g.ldc = kOut;
    g.bias = params + L.b_off[kConv + 1];
    g.n_valid = kOut;
    r = fused<K_DENSE, K_DENSE, E_BIAS_F32>(g, 1, w.part, st);
    if (r) return r;
  }
  return GS2D_OK;
}

int backward(const float* params, const bf16* x, int B, const Ws& w, float* grad, cudaStream_t st) {
  const Layout L = layout();
  int r;
  // FC2: dz2 [B][8]
  {
    Gemm g{};
    g.err = w.err;
    g.M = kOutPad;
    g.N = kHidden;
    g.K = B;
    g.a = op(w.dz2, kOutPad, kOutPad);
    g.b = op(w.h, kHidden, kHidden);
    r = wgrad<R_DENSE, R_DENSE>(g, kOut, w.part, grad + L.w_off[kConv + 1], st);
    if (r) return r;
    r = bias_grad(w.dz2, B, kOutPad, kOut, w.part, grad + L.b_off[kConv + 1], st);
    if (r) return r;
    Gemm d{};
    d.err = w.err;
    d.M = B;
    d.N = kHidden;
    d.K = kOutPad;
    d.a = op(w.dz2, kOutPad, B);
    d.b = op(w.wbf + L.wbf_off[kConv + 1], kHidden, kHidden);
    d.out = w.dzA;
    d.ldc = kHidden;
    d.mask = w.h;
    r = fused<K_DENSE, R_DENSE, E_MASK>(d, 1, w.part, st);
    if (r) return r;
  }
  // FC1: dz1 = dzA [B][256]
  {
    Gemm g{};
    g.err = w.err;
    g.M = kHidden;
    g.N = kFlat;
    g.K = B;
    g.a = op(w.dzA, kHidden, kHidden);
    g.b = op(w.act[kConv], kFlat, kFlat);
    r = wgrad<R_DENSE, R_DENSE>(g, kHidden, w.part, grad + L.w_off[kConv], st);
    if (r) return r;
    r = bias_grad(w.dzA, B, kHidden, kHidden, w.part, grad + L.b_off[kConv], st);
    if (r) return r;
    Gemm d{};
    d.err = w.err;
    d.M = B;
    d.N = kFlat;
    d.K = kHidden;
    d.a = op(w.dzA, kHidden, B);
    d.b = op(w.wbf + L.wbf_off[kConv], kFlat, kFlat);
    d.out = w.dzB;
    d.ldc = kFlat;
    d.mask = w.act[kConv];
    r = fused<K_DENSE, R_DENSE, E_MASK>(d, 1, w.part, st);
    if (r) return r;
  }
  // conv layers, last to first: dz of layer l's output is in cur
  bf16* cur = w.dzB;
  bf16* nxt = w.dzA;
  for (int l = kConv - 1; l >= 0; --l) {
    const bf16* a_in = l == 0 ? x : w.act[l];
    const int P = B * kHin[l + 1] * kWin[l + 1];
    Gemm g{};
    g.err = w.err;
    g.M = kCout[l];
    g.N = 9 * kCin[l];
    g.K = P;
    g.a = op(cur, kCout[l], kCout[l]);
    g.b = conv_op(a_in, g.N, l, kCin[l]);
    if (l == 0) {
      r = wgrad1(x, cur, B, w.part, grad + L.w_off[0], grad + L.b_off[0], st);
      if (r) return r;
      break;
    }
    if (l == 1) {
      r = wgrad2(a_in, cur, B, w.part, grad + L.w_off[1], grad + L.b_off[1], st);
      if (r) return r;
    } else {
      r = wgrad<R_DENSE, R_IM2COL>(g, kCout[l], w.part, grad + L.w_off[l], st);
      if (r) return r;
      r = bias_grad(cur, P, kCout[l], kCout[l], w.part, grad + L.b_off[l], st);
      if (r) return r;
    }
    // data gradient: layer 2's by its direct kernel; the others by one GEMM
    // per parity class of the input pixels, each with only the taps that
    // reach it (9 taps over the 4 classes)
    if (l == 1) {
      r = dgrad2(cur, B, w.wbf + L.wbf_off[1], w.act[1], nxt, st);
      if (r) return r;
    }
    for (int py = 0; py < 2 && l != 1; ++py)
      for (int px = 0; px < 2; ++px) {
        const int Hc = class_hc(kHin[l], py), Wc = class_hc(kWin[l], px);
        Gemm d{};
        d.err = w.err;
        d.M = B * Hc * Wc;
        d.N = kCin[l];
        d.K = (py ? 2 : 1) * (px ? 2 : 1) * kCout[l];
        d.a = conv_op(cur, d.M, l, kCout[l]);
        d.a.py = py;
        d.a.px = px;
        d.a.Hc = Hc;
        d.a.Wc = Wc;
        d.a.f_hw = make_fastdiv((uint32_t)(Hc * Wc));
        d.a.f_w = make_fastdiv((uint32_t)Wc);
        Operand wt{};
        wt.p = w.wbf + L.wbf_off[l];
        wt.ld = kCout[l];
        wt.ld_shift = log2_exact(kCout[l]);
        wt.rows = kCin[l];
        wt.C = kCin[l];
        wt.py = py;
        wt.px = px;
        d.b = wt;
        d.out = nxt;
        d.ldc = kCin[l];
        d.mask = w.act[l];
        d.remap = 1;
        d.rH = kHin[l];
        d.rW = kWin[l];
        d.rHc = Hc;
        d.rWc = Wc;
        d.rpy = py;
        d.rpx = px;
        r = fused<K_DGRADP, R_WTP, E_MASK>(d, Hc * Wc, w.part, st);
        if (r) return r;
      }
    bf16* t = cur;
    cur = nxt;
    nxt = t;
  }
  return GS2D_OK;
}

bool aligned16(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace net
}  // namespace gs2d

using namespace gs2d;
using namespace gs2d::net;

extern "C" {

size_t gs2d_net_param_count(void) { return layout().total; }

int gs2d_net_layout(size_t* w_off, size_t* b_off, int* fan_in) {
  if (!w_off || !b_off || !fan_in) return GS2D_ERR_INVALID_ARG;
  const Layout L = layout();
  for (int l = 0; l < kLayers; ++l) {
    w_off[l] = L.w_off[l];
    b_off[l] = L.b_off[l];
    fan_in[l] = L.fan_in[l];
  }
  return GS2D_OK;
}

size_t gs2d_net_workspace(int batch) {
  if (batch <= 0) return 0;
  return carve(nullptr, batch).bytes;
}

int gs2d_net_downsample_rgbd(const float* rgb, const float* depth, int height, int width,
                             int factor, float* rgb_out, float* depth_out, gs2d_stream stream) {
  if (height <= 0 || width <= 0 || factor <= 0 || height % factor || width % factor || !rgb ||
      !depth || !rgb_out || !depth_out)
    return GS2D_ERR_INVALID_ARG;
  const int ho = height / factor, wo = width / factor;
  const int n = ho * wo;
  gs2d::net::downsample_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      rgb, depth, width, factor, wo, n, rgb_out, depth_out);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int gs2d_net_pack_input(const float* r_rgb, const float* r_depth, const float* r_opacity,
                        const float* o_rgb, const float* o_depth, int batch, int height,
                        int width, uint16_t* x, gs2d_stream stream) {
  if (batch <= 0 || height <= 0 || width <= 0) return GS2D_ERR_INVALID_ARG;
  if (!r_rgb || !r_depth || !r_opacity || !o_rgb || !o_depth || !aligned16(x))
    return GS2D_ERR_INVALID_ARG;
  const size_t n = (size_t)batch * height * width;
  const int blocks = (int)min((n + 255) / 256, (size_t)152 * 16);
  pack_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(r_rgb, r_depth, r_opacity, o_rgb, o_depth, n,
                                                       reinterpret_cast<bf16*>(x));
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int gs2d_net_forward(const float* params, const uint16_t* x, int batch, float* y, void* workspace,
                     size_t ws_bytes, size_t* ws_needed, gs2d_stream stream) {
  if (batch <= 0 || !params || !y || !aligned16(x)) return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_net_workspace(batch);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  const Ws w = carve(workspace, batch);
  return forward(params, reinterpret_cast<const bf16*>(x), batch, w, y, (cudaStream_t)stream);
}

int gs2d_net_prepare(const float* params, int batch, void* workspace, size_t ws_bytes,
                     size_t* ws_needed, gs2d_stream stream) {
  if (batch <= 0 || !params) return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_net_workspace(batch);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  return cast(params, carve(workspace, batch), (cudaStream_t)stream);
}

int gs2d_net_forward_prepared(const float* params, const uint16_t* x, int batch, float* y,
                              void* workspace, size_t ws_bytes, size_t* ws_needed,
                              gs2d_stream stream) {
  if (batch <= 0 || !params || !y || !aligned16(x)) return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_net_workspace(batch);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  const Ws w = carve(workspace, batch);
  return forward(params, reinterpret_cast<const bf16*>(x), batch, w, y, (cudaStream_t)stream,
                 false);
}

int gs2d_net_grad(const float* params, const uint16_t* x, const float* target, int batch,
                  float* loss, float* grad, float* y, void* workspace, size_t ws_bytes,
                  size_t* ws_needed, gs2d_stream stream) {
  if (batch <= 0 || !params || !target || !loss || !grad || !aligned16(x))
    return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_net_workspace(batch);
  if (ws_needed) *ws_needed = need;
  if (!workspace || ws_bytes < need) return GS2D_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const Ws w = carve(workspace, batch);
  const bf16* xb = reinterpret_cast<const bf16*>(x);
  int r = forward(params, xb, batch, w, w.y, st);
  if (r) return r;
  loss_kernel<<<1, 256, 0, st>>>(w.y, target, batch, loss, w.dz2);
  GS2D_LAUNCH_CHECK();
  r = backward(params, xb, batch, w, grad, st);
  if (r) return r;
  if (y) GS2D_CUDA_TRY(cudaMemcpyAsync(y, w.y, sizeof(float) * kOut * batch,
                                       cudaMemcpyDeviceToDevice, st));
  return GS2D_OK;
}

int gs2d_net_adamw(float* params, const float* grad, float* m, float* v, size_t n, int step,
                   float lr, float beta1, float beta2, float eps, float weight_decay,
                   gs2d_stream stream) {
  if (!params || !grad || !m || !v || n == 0 || step < 1) return GS2D_ERR_INVALID_ARG;
  const float bc1 = (float)(1.0 - pow((double)beta1, step));
  const float bc2 = (float)(1.0 - pow((double)beta2, step));
  const int blocks = (int)min((n + 255) / 256, (size_t)152 * 8);
  adamw_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, n, lr, beta1, beta2, eps,
                                                        weight_decay, bc1, bc2);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int gs2d_net_apply(const float* y, int batch, float* poses, gs2d_stream stream) {
  if (batch <= 0 || !y || !poses) return GS2D_ERR_INVALID_ARG;
  apply_kernel<<<(batch + 127) / 128, 128, 0, (cudaStream_t)stream>>>(y, batch, poses);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int gs2d_net_target(const float* poses_init, const float* poses_gt, int batch, float* target,
                    gs2d_stream stream) {
  if (batch <= 0 || !poses_init || !poses_gt || !target) return GS2D_ERR_INVALID_ARG;
  target_kernel<<<(batch + 127) / 128, 128, 0, (cudaStream_t)stream>>>(poses_init, poses_gt, batch,
                                                                      target);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int gs2d_net_accept(const float* loss_prop, const float* loss_init, const float* proposal,
                    int batch, float* poses, int32_t* accepted, gs2d_stream stream) {
  if (batch <= 0 || !loss_prop || !loss_init || !proposal || !poses) return GS2D_ERR_INVALID_ARG;
  accept_kernel<<<(batch + 127) / 128, 128, 0, (cudaStream_t)stream>>>(loss_prop, loss_init, proposal,
                                                                      batch, poses, accepted);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

int gs2d_net_accept_keep(const float* loss_prop, float* loss_init, const float* proposal, int batch,
                         float* poses, int32_t* accepted, size_t n_px, const float* prop_rgb,
                         const float* prop_depth, const float* prop_opacity, float* kept_rgb,
                         float* kept_depth, float* kept_opacity, gs2d_stream stream) {
  if (batch <= 0 || n_px == 0 || !loss_prop || !loss_init || !proposal || !poses || !prop_rgb ||
      !prop_depth || !prop_opacity || !kept_rgb || !kept_depth || !kept_opacity)
    return GS2D_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t total = (size_t)batch * 5 * n_px;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
  keep_images_kernel<<<blocks, 256, 0, st>>>(loss_prop, loss_init, batch, n_px, prop_rgb, prop_depth,
                                             prop_opacity, kept_rgb, kept_depth, kept_opacity);
  GS2D_LAUNCH_CHECK();
  accept_loss_kernel<<<(batch + 127) / 128, 128, 0, st>>>(loss_prop, loss_init, proposal, batch,
                                                         poses, accepted);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

}  // extern "C"
