// Batched persistent micro step instantiated for double.
#include "sbp_batch_impl.cuh"

namespace sbp {
cudaError_t launch_batch_f64(const BatchSubstep &b, int grid, bool viscous, bool curv_fine, int ty, cudaStream_t s) {
  return launch_batch_typed<double>(b, grid, viscous, curv_fine, ty, s);
}
cudaError_t batch_grid_f64(bool viscous, bool curv_fine, int ty, int *grid) {
  return batch_grid_typed<double>(viscous, curv_fine, ty, grid);
}
}  // namespace sbp
