// Right-hand-side kernels instantiated for double.
#include "sbp_rhs_impl.cuh"

namespace sbp {
cudaError_t launch_rhs_f64(const RhsLaunch &a, bool viscous, cudaStream_t s) {
  return launch_rhs_typed<double>(a, viscous, s);
}
}  // namespace sbp
