// FP64 arithmetic-rate probe: the denominator of the FP64 roofline of the right-hand-side
// kernels. GB300 has no FP64 tensor path, so the FP64 rate is that of the SM's FP64 pipe; this
// kernel keeps it busy with independent fused multiply-adds and nothing else of weight.
#include <cuda_runtime.h>

#include "sbp_system.h"

namespace sbp {
namespace {

constexpr int kChains = 8;  // independent FMA chains per thread (hides the FP64 pipe latency)

__global__ void k_fp64_fma_probe(double *out, long iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3 * threadIdx.x + k;
  for (long it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace sbp

extern "C" sbp_status sbp_fp64_rate_probe(void *out, int grid, int block, long iters, double *flops, void *stream) {
  if (!out || grid <= 0 || block <= 0 || block > 1024 || (block & 31) || iters <= 0)
    return sbp::fail(SBP_ERR_ARG, "sbp_fp64_rate_probe: bad argument");
  // a = a * b + c converges to c / (1 - b): the values stay finite for any number of steps
  sbp::k_fp64_fma_probe<<<grid, block, 0, (cudaStream_t)stream>>>(static_cast<double *>(out), iters, 0.999999,
                                                                    1e-6);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return sbp::fail(SBP_ERR_CUDA, cudaGetErrorString(e));
  if (flops) *flops = 2.0 * sbp::kChains * (double)iters * (double)grid * (double)block;
  return SBP_OK;
}
