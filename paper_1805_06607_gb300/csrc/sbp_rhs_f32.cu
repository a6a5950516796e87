// Right-hand-side kernels instantiated for float.
#include "sbp_rhs_impl.cuh"

namespace sbp {
cudaError_t launch_rhs_f32(const RhsLaunch &a, bool viscous, cudaStream_t s) {
  return launch_rhs_typed<float>(a, viscous, s);
}
}  // namespace sbp
