// gs2d_bin_sort_static: tile binning and depth ordering without a caller
// workspace, for callers that cannot allocate device memory at the point
// where they bin -- e.g. code running inside a CUDA stream capture (where
// cudaMalloc is not allowed), a real-time loop with a no-allocation rule, or
// a host framework that owns every device allocation itself and only hands
// out input and output buffers.
//
// The scratch lives in a file-scope __device__ array of
// GS2D_SORT_STATIC_SCRATCH_BYTES (32 MiB), which every GPU that loads this
// library keeps until the process exits.  The arithmetic is exactly that of
// gs2d_bin_sort, which this entry point calls with the array as workspace.
#include <mutex>

#include "gs2d_common.cuh"

namespace gs2d {

static __device__ __align__(256) unsigned char g_sort_scratch[GS2D_SORT_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of this device's copy of g_sort_scratch.  In host code the
// symbol only names a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS2D_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GS2D_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return GS2D_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GS2D_OK;
}
}  // namespace

}  // namespace gs2d

extern "C" {

int gs2d_bin_sort_static(const float* proj, const int32_t* tiles_per_surfel, int n,
                         const gs2d_camera* cam, const gs2d_config* cfg, const gs2d_bins* bins,
                         gs2d_stream stream) {
  if (!bins || n < 0) return GS2D_ERR_INVALID_ARG;
  const size_t need = gs2d_bin_sort_workspace(n, bins->capacity);
  if (need > (size_t)GS2D_SORT_STATIC_SCRATCH_BYTES) return GS2D_ERR_WORKSPACE;
  void* scratch = nullptr;
  const int rc = gs2d::scratch_for_current_device(&scratch);
  if (rc != GS2D_OK) return rc;
  // gs2d_bin_sort's first kernel zeroes every counter, histogram and
  // look-back word it reads before writing them, so nothing left in the
  // array by an earlier call is ever read.
  return gs2d_bin_sort(proj, tiles_per_surfel, n, cam, cfg, scratch,
                       (size_t)GS2D_SORT_STATIC_SCRATCH_BYTES, nullptr, bins, stream);
}

}  // extern "C"
