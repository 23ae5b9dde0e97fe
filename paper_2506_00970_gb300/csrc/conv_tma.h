// Forward convolutions of the proposal network's layers 2-6 on tcgen05 with
// TMA-fed operands (conv_tma.cu).  Internal to the library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gs2d {
namespace net {

// Whether conv layer `layer` (0-based: 1 .. 5 = the network's layers 2-6)
// runs on conv_tma_forward.
bool conv_tma_layer(int layer);

// out = bfloat16(ReLU(conv3x3_stride2_pad1(x, w) + bias)) for conv layer
// `layer`: x NHWC [B][H][W][C_in] bfloat16, w [C_out][9 C_in] bfloat16
// (k = (ky * 3 + kx) C_in + c), bias [C_out] FP32, out NHWC [B][Ho][Wo][C_out];
// device pointers, 16-byte aligned.  A wait that runs out sets *err to 1.
// GS2D_ERR_CUDA if the tensor maps cannot be made (nothing is launched).
int conv_tma_forward(int layer, const __nv_bfloat16* x, int B, const __nv_bfloat16* w,
                     const float* bias, __nv_bfloat16* out, int* err, cudaStream_t st);

}  // namespace net
}  // namespace gs2d
