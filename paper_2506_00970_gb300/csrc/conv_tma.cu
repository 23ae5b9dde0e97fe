// Forward 3x3 / stride 2 / padding 1 convolutions of the proposal network
// (layers 2-4: NHWC bfloat16 maps 60x80x32 -> 30x40x64 -> 15x20x128 ->
// 8x10x256) on the 5th-generation tensor cores with TMA-fed operands.
//
// One CTA computes an output tile of 128 pixels (TH rows x TW columns of one
// image) for all C_out channels as a 128 x C_out x (9 C_in) product: one
// tcgen05.mma (M = 128, N = C_out, K = 16, bf16 x bf16 -> f32 in tensor
// memory) per tap and 16 input channels.  Its operands come straight from
// tiled TMA loads, no gather in software:
//  * A (im2col rows): for tap (ky, kx) and KB channels (KB = 32 or 64, a
//    64- or 128-byte row per pixel), a box of the input map {KB channels,
//    2 TW columns, 2 TH rows} starting at input pixel (2 ox0 + kx - 1,
//    2 oy0 + ky - 1) with element stride 2 in both pixel dimensions loads
//    the TH x TW input pixels that tap reads -- zero-filled where the
//    padding lies (negative or past-the-edge coordinates).  In shared memory
//    output pixel m's KB channels are row m, written with the TMA's 64- or
//    128-byte swizzle: the K-major swizzled layout tcgen05 reads (8-row
//    atoms of 8 x KB x 2 bytes), the K steps of 16 channels 32 bytes apart
//    inside a row.
//  * B (weights [C_out][9 C_in], K = tap x C_in + channel): a box {KB k,
//    C_out rows} in the same swizzled K-major layout.
// One thread issues the loads S stages ahead (mbarrier transaction counts)
// and the MMAs; a stage is refilled once the tcgen05.commit of the MMAs that
// read it has arrived.  Four warps read the accumulator back (tcgen05.ld)
// and apply bias, ReLU and the bfloat16 rounding of the other kernels.
// Every wait is bounded: past the limit the kernel records an error in
// *err, stops issuing, waits (bounded) for what it issued and frees its
// tensor memory.  Layers 5 and 6 (4 x 5 and 2 x 3 outputs) put several whole
// images in one tile: a box's fourth dimension spans them.  Layers 3 and 4
// at large batches use a persistent, warp-specialised form with two TMEM
// accumulators (conv_tma_pers_kernel).
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "conv_tma.h"
#include "gs2d_common.cuh"

namespace gs2d {
namespace net {
namespace {

using bf16 = __nv_bfloat16;
constexpr int kConvThreads = 128;
constexpr int kWaitSpins = 1 << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kWaitSpins; ++i) {
    uint32_t ok;
    asm volatile(
        "{.reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}
// Shared-memory matrix descriptor of a K-major operand with rows of SW bytes
// (64 or 128) under the matching swizzle: start address, leading offset 16
// bytes (unused by the swizzled K-major layouts), stride 8 x SW bytes
// between the 8-row atoms, swizzle mode in bits 61-63 (2 = 128 B, 4 = 64 B).
template <int SW>
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
  constexpr uint64_t mode = SW == 128 ? 2ull : 4ull;
  return (uint64_t)((saddr >> 4) & 0x3FFF) | (1ull << 16) |
         ((uint64_t)(((8 * SW) >> 4) & 0x3FFF) << 32) | (1ull << 46) | (mode << 61);
}
// Instruction descriptor of kind::f16: f32 accumulate, bf16 A and B, both
// K-major, N = n, M = 128.
__host__ __device__ constexpr uint32_t mma_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// A tile is NI images' TW x TH output pixels (NI = 1: a 128-pixel part of one
// image; NI > 1: whole small images, TW x TH = the output map) times NB of the
// C_out channels.  One box per tap and channel block spans the NI images
// (its fourth dimension), so image g's pixels are rows [g TW TH, (g + 1) TW TH)
// of the 128-row MMA tile; rows past NI TW TH hold stale data whose results
// the epilogue drops.
template <int CIN, int COUT, int HI, int WI, int TW, int TH, int S, int NI = 1, int NB = COUT>
struct ConvTma {
  static constexpr int HO = (HI + 1) / 2, WO = (WI + 1) / 2;
  static constexpr int TX = (WO + TW - 1) / TW, TY = (HO + TH - 1) / TH;
  static constexpr int KB = CIN < 64 ? CIN : 64;  // channels per box row
  static constexpr int SW = KB * 2;               // row bytes = swizzle span
  static constexpr int CB = CIN / KB;             // boxes (stages) per tap
  static constexpr int KS = 9 * CB;               // stages per tile
  static constexpr int MMAS = KB / 16;            // MMAs per stage
  static constexpr int ROWS = NI * TW * TH;       // rows one input box lands
  static constexpr int BOX_BYTES = ROWS * SW;     // one input box (NI images)
  static constexpr int A_BYTES = 128 * SW;        // the 128-row A operand
  static constexpr int B_BYTES = NB * SW;         // one weight box
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int TX_BYTES = BOX_BYTES + B_BYTES;  // bytes a stage's loads bring
  static constexpr int SMEM = S * STAGE + 1024;   // + slack for 1024-byte alignment
  static constexpr int TMEM_COLS = NB;
  static constexpr int NSPLIT = COUT / NB;        // channel groups (grid.y)
  static_assert(NI == 1 ? TW * TH == 128 : (TX == 1 && TY == 1 && ROWS <= 128),
                "one 128-row MMA tile: a part of one image, or whole images");
  static_assert(KB == 32 || KB == 64, "64- or 128-byte swizzled rows");
  static_assert(CIN % KB == 0 && NB >= 32 && NB <= 256 && (NB & (NB - 1)) == 0 &&
                    COUT % NB == 0,
                "tensor-memory columns: a power of two in [32, 256]");
  static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "swizzle atoms stay aligned");
  static_assert(2 * TW <= 256 && 2 * TH <= 256, "TMA box dimensions");
};

template <int CIN, int COUT, int HI, int WI, int TW, int TH, int S, int NI, int NB>
__global__ void __launch_bounds__(kConvThreads) conv_tma_kernel(
    const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w,
    const float* __restrict__ bias, bf16* __restrict__ out, int B, int* __restrict__ err) {
  using C = ConvTma<CIN, COUT, HI, WI, TW, TH, S, NI, NB>;
  extern __shared__ unsigned char conv_raw[];
  __shared__ __align__(8) uint64_t s_full[S], s_empty[S], s_done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  unsigned char* stages = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(conv_raw) + 1023) & ~(uintptr_t)1023);
  const int tile = blockIdx.x;
  // NI == 1: tile -> (image, TH x TW part); NI > 1: images tile NI .. tile NI + NI - 1
  const int img = NI == 1 ? tile / (C::TX * C::TY) : tile * NI;
  const int r = NI == 1 ? tile % (C::TX * C::TY) : 0;
  const int oy0 = (r / C::TX) * TH, ox0 = (r % C::TX) * TW;
  const int nb0 = (int)blockIdx.y * NB;  // first output channel of the tile
  const int warp = threadIdx.x >> 5;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int i = 0; i < S; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_done)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(C::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  // warp 0's lane 0 issues every load and MMA; its other lanes wait for it
  // at the __syncwarp below rather than spinning beside it
  if (threadIdx.x == 0) {
    // stage s: the input box of tap s / CB, channels cb .. cb + KB, and the
    // matching weight box
    auto load = [&](int s) {
      const int st = s % S;
      const uint32_t base = smem_u32(stages + st * C::STAGE);
      const uint32_t bar = smem_u32(&s_full[st]);
      const int tap = s / C::CB, cb = (s % C::CB) * C::KB;
      const int ky = tap / 3, kx = tap - 3 * (tap / 3);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                   "r"(C::TX_BYTES)
                   : "memory");
      // images past the batch read as zeros (out-of-range coordinates)
      tma_load_4d(base, &map_x, cb, 2 * ox0 + kx - 1, 2 * oy0 + ky - 1, img, bar);
      tma_load_2d(base + C::A_BYTES, &map_w, tap * CIN + cb, nb0, bar);
    };
    bool fail = false;
    int issued = 0, consumed = 0;
    for (; issued < S && issued < C::KS; ++issued) load(issued);
    for (int s = 0; s < C::KS; ++s) {
      const int st = s % S;
      if (!bar_wait(smem_u32(&s_full[st]), (uint32_t)((s / S) & 1))) {
        fail = true;
        break;
      }
      consumed = s + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(stages + st * C::STAGE);
#pragma unroll
      for (int j = 0; j < C::MMAS; ++j) {
        // K step j of the stage: 16 channels, 32 bytes into every swizzled row
        const uint64_t ad = sw_desc<C::SW>(base + 32 * j);
        const uint64_t bd = sw_desc<C::SW>(base + C::A_BYTES + 32 * j);
        const uint32_t acc = (s > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{.reg .pred p; setp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(mma_idesc(NB)), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&s_empty[st]))
          : "memory");
      // refill the stage the previous step read once its MMA is done (the
      // MMA just issued keeps the tensor pipe busy meanwhile)
      if (s >= 1 && issued < C::KS) {
        const int ps = (s - 1) % S;
        if (!bar_wait(smem_u32(&s_empty[ps]), (uint32_t)(((s - 1) / S) & 1))) {
          fail = true;
          break;
        }
        load(issued++);
      }
    }
    // one last commit tracks every MMA issued (all, or those before a failure)
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&s_done))
        : "memory");
    if (fail) {
      s_fail = 1;
      // loads still in flight must land before the CTA exits (bounded)
      for (int s = consumed; s < issued; ++s)
        bar_wait(smem_u32(&s_full[s % S]), (uint32_t)((s / S) & 1));
    }
  }
  if (warp == 0) __syncwarp();
  if (!bar_wait(smem_u32(&s_done), 0u)) atomicExch(&s_fail, 1);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!*reinterpret_cast<volatile int*>(&s_fail)) {
    // TMEM lane = row m: image img + m / (TW TH), output pixel (oy0 + q / TW,
    // ox0 + q % TW) with q = m % (TW TH)
    const int m = threadIdx.x;
    const int g = m / (TW * TH), q = m % (TW * TH);
    const int oy = oy0 + q / TW, ox = ox0 + q % TW;
    const bool ok = g < NI && img + g < B && oy < C::HO && ox < C::WO;
    bf16* dst = out + (((size_t)(img + g) * C::HO + oy) * C::WO + ox) * COUT + nb0;
    const float* bs = bias + nb0;
#pragma unroll 1
    for (int c0 = 0; c0 < NB; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
          "%10, %11, %12, %13, %14, %15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (ok) {
        uint32_t packed[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float x0 = fmaxf(__uint_as_float(v[2 * j]) + bs[c0 + 2 * j], 0.f);
          const float x1 = fmaxf(__uint_as_float(v[2 * j + 1]) + bs[c0 + 2 * j + 1], 0.f);
          const __nv_bfloat162 b2 = __floats2bfloat162_rn(x0, x1);
          packed[j] = *reinterpret_cast<const uint32_t*>(&b2);
        }
        uint4* d = reinterpret_cast<uint4*>(dst + c0);
        d[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        d[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
      }
    }
  } else if (threadIdx.x == 0 && err) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS));
}

// Persistent form for grids of many tiles (layers 2-4 at large batches):
// each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ... with three
// roles -- warp 4 issues the TMA loads S stages ahead across tile boundaries,
// warp 5 issues the MMAs into one of two TMEM accumulators, warps 0-3 read
// the other accumulator back -- so a tile's epilogue overlaps the next
// tile's loads and MMAs, and barrier set-up and TMEM allocation happen once
// per CTA.  Barriers: full/empty per stage (loads <-> MMAs), tfull/tempty
// per accumulator (MMAs <-> epilogue; tempty takes one arrival per epilogue
// warp).  Every tile sums its K steps in the same order as conv_tma_kernel,
// so results do not depend on the form or the grid.  Waits are bounded; a
// role whose wait runs out records the failure and stops; the MMA issuer's
// last commit tracks every MMA issued and all threads wait for it before
// the tensor memory is freed, and the loader waits for its loads in flight.
constexpr int kPersThreads = 192;

template <int CIN, int COUT, int HI, int WI, int TW, int TH, int S>
__global__ void __launch_bounds__(kPersThreads) conv_tma_pers_kernel(
    const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w,
    const float* __restrict__ bias, bf16* __restrict__ out, int n_tiles, int* __restrict__ err) {
  using C = ConvTma<CIN, COUT, HI, WI, TW, TH, S>;
  extern __shared__ unsigned char conv_raw[];
  __shared__ __align__(8) uint64_t s_full[S], s_empty[S], s_tfull[2], s_tempty[2], s_done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail, s_issued, s_consumed;
  unsigned char* stages = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(conv_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int my_n = (int)blockIdx.x < n_tiles
                       ? (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                       : 0;
  if (threadIdx.x == 0) {
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
    for (int i = 0; i < S; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_empty[i])));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_tfull[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&s_tempty[b])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_done)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(2 * C::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp == 4) {
    if (lane == 0) {
      int g = 0;
      bool fail = false;
      for (int k = 0; k < my_n && !fail; ++k) {
        const int tile = (int)blockIdx.x + k * (int)gridDim.x;
        const int img = tile / (C::TX * C::TY), r = tile % (C::TX * C::TY);
        const int oy0 = (r / C::TX) * TH, ox0 = (r % C::TX) * TW;
        for (int s = 0; s < C::KS; ++s, ++g) {
          const int st = g % S;
          // the MMAs that read this stage's previous fill are done
          if (g >= S && !bar_wait(smem_u32(&s_empty[st]), (uint32_t)((g / S - 1) & 1))) {
            fail = true;
            break;
          }
          const uint32_t base = smem_u32(stages + st * C::STAGE);
          const uint32_t bar = smem_u32(&s_full[st]);
          const int tap = s / C::CB, cb = (s % C::CB) * C::KB;
          const int ky = tap / 3, kx = tap - 3 * (tap / 3);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                       "r"(C::TX_BYTES)
                       : "memory");
          tma_load_4d(base, &map_x, cb, 2 * ox0 + kx - 1, 2 * oy0 + ky - 1, img, bar);
          tma_load_2d(base + C::A_BYTES, &map_w, tap * CIN + cb, 0, bar);
          s_issued = g + 1;
        }
      }
      if (fail) atomicExch(&s_fail, 1);
    }
  } else if (warp == 5) {
    if (lane == 0) {
      int g = 0;
      bool fail = false;
      for (int k = 0; k < my_n && !fail; ++k) {
        const int buf = k & 1;
        // the epilogue has read this accumulator's previous tile
        if (k >= 2 && !bar_wait(smem_u32(&s_tempty[buf]), (uint32_t)(((k >> 1) - 1) & 1))) {
          fail = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_tmem = tmem + (uint32_t)(buf * C::TMEM_COLS);
        for (int s = 0; s < C::KS; ++s, ++g) {
          const int st = g % S;
          if (!bar_wait(smem_u32(&s_full[st]), (uint32_t)((g / S) & 1))) {
            fail = true;
            break;
          }
          s_consumed = g + 1;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t base = smem_u32(stages + st * C::STAGE);
#pragma unroll
          for (int j = 0; j < C::MMAS; ++j) {
            const uint64_t ad = sw_desc<C::SW>(base + 32 * j);
            const uint64_t bd = sw_desc<C::SW>(base + C::A_BYTES + 32 * j);
            const uint32_t acc = (s > 0 || j > 0) ? 1u : 0u;
            asm volatile(
                "{.reg .pred p; setp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}\n" ::"r"(acc_tmem),
                "l"(ad), "l"(bd), "r"(mma_idesc(COUT)), "r"(acc));
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  smem_u32(&s_empty[st]))
              : "memory");
        }
        if (fail) break;
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&s_tfull[buf]))
            : "memory");
      }
      // one last commit tracks every MMA issued
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&s_done))
          : "memory");
      if (fail) atomicExch(&s_fail, 1);
    }
  } else {
    // warps 0-3: TMEM lane = row m = threadIdx.x = output pixel (oy0 + m / TW, ox0 + m % TW)
    const int m = threadIdx.x;
    for (int k = 0; k < my_n; ++k) {
      const int buf = k & 1;
      if (!bar_wait(smem_u32(&s_tfull[buf]), (uint32_t)((k >> 1) & 1))) {
        atomicExch(&s_fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int tile = (int)blockIdx.x + k * (int)gridDim.x;
      const int img = tile / (C::TX * C::TY), r = tile % (C::TX * C::TY);
      const int oy = (r / C::TX) * TH + m / TW, ox = (r % C::TX) * TW + m % TW;
      const bool ok = oy < C::HO && ox < C::WO;
      bf16* dst = out + (((size_t)img * C::HO + oy) * C::WO + ox) * COUT;
#pragma unroll 1
      for (int c0 = 0; c0 < COUT; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr =
            tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(buf * C::TMEM_COLS + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15}, [%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (ok) {
          uint32_t packed[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float x0 = fmaxf(__uint_as_float(v[2 * j]) + bias[c0 + 2 * j], 0.f);
            const float x1 = fmaxf(__uint_as_float(v[2 * j + 1]) + bias[c0 + 2 * j + 1], 0.f);
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(x0, x1);
            packed[j] = *reinterpret_cast<const uint32_t*>(&b2);
          }
          uint4* d = reinterpret_cast<uint4*>(dst + c0);
          d[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
          d[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        }
      }
      // this accumulator may be overwritten once all four warps have read it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&s_tempty[buf]))
                     : "memory");
    }
  }
  __syncthreads();
  // every MMA issued has completed before the tensor memory is freed, and
  // loads issued but not consumed (after a failure) land before the CTA exits
  if (!bar_wait(smem_u32(&s_done), 0u)) atomicExch(&s_fail, 1);
  if (warp == 4 && lane == 0)
    for (int g = s_consumed; g < s_issued; ++g)
      bar_wait(smem_u32(&s_full[g % S]), (uint32_t)((g / S) & 1));
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && s_fail && err) atomicExch(err, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * C::TMEM_COLS));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (looked up once).
EncodeTiledFn encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Input map: NHWC bfloat16 {C, W, H, N}, box {KB, 2 TW, 2 TH, 1} with
// element stride 2 in W and H (TW x TH pixels land); weight map: [C_out]
// [9 C_in] as {9 C_in, C_out}, box {KB, C_out}; both with the swizzle of
// their KB x 2-byte rows.  Zero fill outside the tensors.
template <int CIN, int COUT, int HI, int WI, int TW, int TH, int S, int NI = 1, int NB = COUT>
int run(const bf16* x, int B, const bf16* w, const float* bias, bf16* out, int* err,
        cudaStream_t st) {
  using C = ConvTma<CIN, COUT, HI, WI, TW, TH, S, NI, NB>;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return GS2D_ERR_CUDA;
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(w) |
       reinterpret_cast<uintptr_t>(out)) & 15)
    return GS2D_ERR_INVALID_ARG;
  CUtensorMap mx, mw;
  const cuuint64_t xdim[4] = {(cuuint64_t)CIN, (cuuint64_t)WI, (cuuint64_t)HI, (cuuint64_t)B};
  const cuuint64_t xstr[3] = {(cuuint64_t)CIN * 2, (cuuint64_t)WI * CIN * 2,
                              (cuuint64_t)HI * WI * CIN * 2};
  const cuuint32_t xbox[4] = {(cuuint32_t)C::KB, 2 * TW, 2 * TH, (cuuint32_t)NI};
  const cuuint32_t xes[4] = {1, 2, 2, 1};
  if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(x), xdim, xstr, xbox, xes,
          CU_TENSOR_MAP_INTERLEAVE_NONE, C::SW == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return GS2D_ERR_CUDA;
  const cuuint64_t wdim[2] = {(cuuint64_t)9 * CIN, (cuuint64_t)COUT};
  const cuuint64_t wstr[1] = {(cuuint64_t)9 * CIN * 2};
  const cuuint32_t wbox[2] = {(cuuint32_t)C::KB, (cuuint32_t)NB};
  const cuuint32_t wes[2] = {1, 1};
  if (enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(w), wdim, wstr, wbox, wes,
          CU_TENSOR_MAP_INTERLEAVE_NONE, C::SW == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return GS2D_ERR_CUDA;
  // the dynamic shared memory exceeds the 48 KB default: raise the limit once
  // (before any stream capture that runs the network)
  static std::once_flag smem_once;
  static cudaError_t smem_err = cudaSuccess;
  std::call_once(smem_once, [] {
    smem_err = cudaFuncSetAttribute(conv_tma_kernel<CIN, COUT, HI, WI, TW, TH, S, NI, NB>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  });
  if (smem_err != cudaSuccess) return GS2D_ERR_CUDA;
  const int grid = NI == 1 ? B * C::TX * C::TY : (B + NI - 1) / NI;
  if (grid <= 0) return GS2D_OK;
  conv_tma_kernel<CIN, COUT, HI, WI, TW, TH, S, NI, NB>
      <<<dim3(grid, C::NSPLIT), kConvThreads, C::SMEM, st>>>(mx, mw, bias, out, B, err);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

// The persistent form on the GPU's resident CTAs (see conv_tma_pers_kernel).
template <int CIN, int COUT, int HI, int WI, int TW, int TH, int S>
int run_pers(const bf16* x, int B, const bf16* w, const float* bias, bf16* out, int* err,
             cudaStream_t st) {
  using C = ConvTma<CIN, COUT, HI, WI, TW, TH, S>;
  static_assert(2 * C::TMEM_COLS <= 512, "two accumulators fit the tensor memory");
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return GS2D_ERR_CUDA;
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(w) |
       reinterpret_cast<uintptr_t>(out)) & 15)
    return GS2D_ERR_INVALID_ARG;
  CUtensorMap mx, mw;
  const cuuint64_t xdim[4] = {(cuuint64_t)CIN, (cuuint64_t)WI, (cuuint64_t)HI, (cuuint64_t)B};
  const cuuint64_t xstr[3] = {(cuuint64_t)CIN * 2, (cuuint64_t)WI * CIN * 2,
                              (cuuint64_t)HI * WI * CIN * 2};
  const cuuint32_t xbox[4] = {(cuuint32_t)C::KB, 2 * TW, 2 * TH, 1};
  const cuuint32_t xes[4] = {1, 2, 2, 1};
  const CUtensorMapSwizzle sw =
      C::SW == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(x), xdim, xstr, xbox, xes,
          CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return GS2D_ERR_CUDA;
  const cuuint64_t wdim[2] = {(cuuint64_t)9 * CIN, (cuuint64_t)COUT};
  const cuuint64_t wstr[1] = {(cuuint64_t)9 * CIN * 2};
  const cuuint32_t wbox[2] = {(cuuint32_t)C::KB, COUT};
  const cuuint32_t wes[2] = {1, 1};
  if (enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(w), wdim, wstr, wbox, wes,
          CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return GS2D_ERR_CUDA;
  // the dynamic shared memory exceeds the 48 KB default: raise the limit
  // and size the resident grid once (before any stream capture)
  static std::once_flag once;
  static cudaError_t once_err = cudaSuccess;
  static int resident = 0;
  std::call_once(once, [] {
    auto kern = conv_tma_pers_kernel<CIN, COUT, HI, WI, TW, TH, S>;
    once_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    int per_sm = 0, dev = 0, sms = 0;
    if (once_err == cudaSuccess)
      once_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPersThreads, C::SMEM);
    if (once_err == cudaSuccess) once_err = cudaGetDevice(&dev);
    if (once_err == cudaSuccess)
      once_err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    resident = max(per_sm, 1) * max(sms, 1);
  });
  if (once_err != cudaSuccess) return GS2D_ERR_CUDA;
  const int n_tiles = B * C::TX * C::TY;
  if (n_tiles <= 0) return GS2D_OK;
  conv_tma_pers_kernel<CIN, COUT, HI, WI, TW, TH, S>
      <<<min(n_tiles, resident), kPersThreads, C::SMEM, st>>>(mx, mw, bias, out, n_tiles, err);
  GS2D_LAUNCH_CHECK();
  return GS2D_OK;
}

}  // namespace

bool conv_tma_layer(int layer) { return layer >= 1 && layer <= 5; }

// Stages in flight: with a grid that fills the GPU several CTAs share an SM
// (fewer stages each; the SM keeps as many loads in flight); a small batch's
// few CTAs each keep as many stages as shared memory holds.  The stage count
// changes no result (every tile sums its K steps in the same order).
int conv_tma_forward(int layer, const bf16* x, int B, const bf16* w, const float* bias, bf16* out,
                     int* err, cudaStream_t st) {
  constexpr int kFull = 2 * 152;  // CTAs that fill the GPU twice over
  switch (layer) {
    // layers 3 and 4 with more tiles than the GPU holds CTAs: the persistent
    // form (layer 2's grid is bound by its 64-byte strided input rows, not
    // by per-tile set-up: the persistent form measured the same there)
    case 1:
      return B * 10 >= kFull ? run<32, 64, 60, 80, 8, 16, 4>(x, B, w, bias, out, err, st)
                             : run<32, 64, 60, 80, 8, 16, 8>(x, B, w, bias, out, err, st);
    case 2:
      return B * 3 >= kFull ? run_pers<64, 128, 30, 40, 8, 16, 6>(x, B, w, bias, out, err, st)
                            : run<64, 128, 30, 40, 8, 16, 6>(x, B, w, bias, out, err, st);
    case 3:
      return B >= kFull / 2 ? run_pers<128, 256, 15, 20, 16, 8, 4>(x, B, w, bias, out, err, st)
                            : run<128, 256, 15, 20, 16, 8, 4>(x, B, w, bias, out, err, st);
    // layers 5 and 6 (4 x 5 and 2 x 3 outputs): whole images per tile (5 and
    // 21: 100 and 126 rows), the 256 output channels in halves or quarters so
    // the grid still spreads over the SMs
    case 4:
      return run<256, 256, 8, 10, 5, 4, 6, 5, 128>(x, B, w, bias, out, err, st);
    case 5:
      return run<256, 256, 4, 5, 3, 2, 8, 21, 32>(x, B, w, bias, out, err, st);
    default: return GS2D_ERR_INVALID_ARG;
  }
}

}  // namespace net
}  // namespace gs2d
