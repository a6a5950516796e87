// Characteristic penalty matrix of the 3D SAT (Sec. 2.2 eq. (int)) applied to a state jump,
// shared by the Cartesian (sbp3_kernels.cu) and curvilinear (sbp3c_kernels.cu) operators.
#pragma once

#include <cuda_runtime.h>

namespace sbp {

// K^{side}_k dq through the eigen-decomposition of the 3D flux Jacobian along k: acoustic
// waves U +/- c|k| with strengths (dp +/- rho c dUn) / (2 c^2), entropy and shear waves at U.
template <typename T>
__device__ void penalty3(const T q[5], T gam, const T kv[3], int side, const T dq[5], T out[5]) {
  const T rho = q[0], ri = T(1) / rho;
  const T u[3] = {q[1] * ri, q[2] * ri, q[3] * ri};
  const T k2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T p = (gam - T(1)) * (q[4] - T(0.5) * rho * k2);
  const T c2 = gam * p * ri, c = sqrt(c2);
  const T H = (q[4] + p) * ri;
  const T kn = sqrt(kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]), kinv = T(1) / kn;
  const T nv[3] = {kv[0] * kinv, kv[1] * kinv, kv[2] * kinv};
  const T U = kv[0] * u[0] + kv[1] * u[1] + kv[2] * u[2], Un = U * kinv;
  T du[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) du[a] = (dq[1 + a] - u[a] * dq[0]) * ri;
  const T dp = (gam - T(1)) * (dq[4] - u[0] * dq[1] - u[1] * dq[2] - u[2] * dq[3] + T(0.5) * k2 * dq[0]);
  const T dUn = nv[0] * du[0] + nv[1] * du[1] + nv[2] * du[2];
  const T ap = (dp + rho * c * dUn) / (T(2) * c2), am = (dp - rho * c * dUn) / (T(2) * c2);
  const T a0 = dq[0] - dp / c2;
  T dut[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) dut[a] = du[a] - nv[a] * dUn;
  const T l0 = U, lp = U + c * kn, lm = U - c * kn;
  const T f0 = side > 0 ? fmax(l0, T(0)) : fmax(-l0, T(0));
  const T fp = side > 0 ? fmax(lp, T(0)) : fmax(-lp, T(0));
  const T fm = side > 0 ? fmax(lm, T(0)) : fmax(-lm, T(0));
  out[0] = f0 * a0 + fp * ap + fm * am;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    out[1 + a] = f0 * (a0 * u[a] + rho * dut[a]) + fp * ap * (u[a] + c * nv[a]) + fm * am * (u[a] - c * nv[a]);
  out[4] = f0 * (a0 * T(0.5) * k2 + rho * (u[0] * dut[0] + u[1] * dut[1] + u[2] * dut[2])) + fp * ap * (H + c * Un) +
           fm * am * (H - c * Un);
}

}  // namespace sbp
