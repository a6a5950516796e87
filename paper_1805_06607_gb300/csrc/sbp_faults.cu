// Failure detection self-test of the batched form's grid barrier: a launch whose CTAs wait for
// more arrivals than the grid has, so that the bounded wait runs out, records SBP_ERR_TIMEOUT in
// an error word and returns. The CTAs are few and small, so they are all resident at once and
// every one of them reaches its own spin limit; no CTA waits without a bound.
#include <cuda_runtime.h>

#include "sbp_batch_impl.cuh"
#include "sbp_system.h"

namespace sbp {
namespace {

__global__ void k_barrier_selftest(unsigned *bar, int *err, unsigned arrivals, unsigned max_spins, int *passed) {
  const bool ok = grid_barrier(bar, bar + 1, arrivals, err, max_spins);
  if (threadIdx.x == 0 && ok) atomicAdd(passed, 1);
}

}  // namespace
}  // namespace sbp

extern "C" sbp_status sbp_barrier_selftest(int grid, int arrivals, unsigned max_spins, int *status, int *passed,
                                          void *stream) {
  if (grid < 1 || grid > 8 || arrivals < 1 || max_spins < 1 || max_spins > (1u << 16) || !status || !passed)
    return sbp::fail(SBP_ERR_ARG, "sbp_barrier_selftest: 1..8 CTAs, 1..65536 spins");
  cudaStream_t s = (cudaStream_t)stream;
  void *buf = nullptr;
  CUDA_TRY(cudaMalloc(&buf, 4 * sizeof(int)));
  unsigned *bar = static_cast<unsigned *>(buf);
  int *err = static_cast<int *>(buf) + 2, *np = static_cast<int *>(buf) + 3;
  cudaError_t e = cudaMemsetAsync(buf, 0, 4 * sizeof(int), s);
  if (e == cudaSuccess) {
    sbp::k_barrier_selftest<<<grid, 32, 0, s>>>(bar, err, (unsigned)arrivals, max_spins, np);
    e = cudaGetLastError();
  }
  int host[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e != cudaSuccess) return sbp::fail(SBP_ERR_CUDA, cudaGetErrorString(e));
  *status = host[0];
  *passed = host[1];
  return SBP_OK;
}
