// Right-hand-side evaluation whose receiver workspace lives in a fixed device array, for
// sbp_rhs_eval_noalloc: callers that must not have the library allocate device memory at call
// time (device memory reserved up front by another allocator, or loops that cannot afford the
// synchronisation of cudaMalloc / cudaFree) use it. The first call on a device looks the array's
// address up; it should come before any stream capture.
#include <cuda_runtime.h>

#include <mutex>

#include "sbp_device.h"

namespace sbp {

// Interpolated states (4 values per receiver) followed by interpolated viscous fluxes (6 per
// receiver), in the element type of the system. Every GPU that loads the library holds this
// array until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)SBP_NOALLOC_MAX_RECEIVERS * 10 * sizeof(double);
static __device__ __align__(256) unsigned char g_rhs_scratch[kStaticScratchBytes];

namespace {
std::mutex g_scratch_mu;
constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
}  // namespace

// Device address of g_rhs_scratch on the current device. The host-side name of the array is
// only a stand-in, so the address is looked up once per device (with that device current).
static cudaError_t static_scratch(void **ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_rhs_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *ptr = g_scratch_addr[dev];
  return cudaSuccess;
}

cudaError_t rhs_eval_static_scratch(InterpLaunch ia, RhsLaunch ra, int dtype, bool viscous, size_t elem,
                                    cudaStream_t s) {
  if ((size_t)ia.nrecv * 10 * elem > kStaticScratchBytes) return cudaErrorInvalidValue;
  void *base = nullptr;
  cudaError_t e = static_scratch(&base);
  if (e != cudaSuccess) return e;
  // the gather writes every entry that the right-hand side then reads, so no clearing is needed
  ia.qhat = base;
  ia.fvhat = viscous ? static_cast<char *>(base) + (size_t)4 * ia.nrecv * elem : nullptr;
  ra.qhat = ia.qhat;
  ra.fvhat = ia.fvhat;
  e = launch_interp(ia, dtype, viscous, s);
  if (e != cudaSuccess) return e;
  return launch_rhs(ra, dtype, viscous, s);
}

}  // namespace sbp
