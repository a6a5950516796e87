// Launch descriptors of the 3D curvilinear operator (sbp3c_kernels.cu): one structured mesh,
// non-periodic in every direction, arrays unpitched, point (i, j, k) at (k * nj + j) * ni + i.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace sbp {

struct Curv3Launch {
  int ni, nj, nk;
  size_t field;          // ni * nj * nk
  int visc;
  double gam, mu, lam, kap;
  const void *q;         // 5 planes
  void *out;             // 5 planes
  const void *met;       // 10 planes: M[m][j] = xi_m,x_j / J (m-major), then J
  void *prim;            // 4 planes (u, v, w, T); Navier-Stokes only
  void *flux;            // 15 planes: contravariant fluxes F^_m (5 variables each)
  int far;               // far-field SAT on every face towards qinf with sigma
  double sig, qinf[5];
};

// Interface SAT terms grouped by receiver point: point t (linear index pt[t]) owns terms
// off[t] .. off[t + 1] - 1, each (m, side, r) in term[3 e ..] with weight scale[e]; donor
// values qhat (5 x nrecv) and viscous fluxes fvhat (12 x nrecv, Navier-Stokes) of the element
// type. All device arrays.
struct Curv3Sat {
  int npt, nrecv;
  const long long *pt;
  const int *off, *term;
  const double *scale;
  const void *qhat, *fvhat;
  double sig;
};

// Metric terms of the mesh with coordinates xyz (3 device planes, FP64) into met (10 planes of
// the element type), using dx (9 device planes, FP64) as workspace.
cudaError_t launch3c_metrics(int ni, int nj, int nk, const double *xyz, double *dx, void *met, int dtype,
                             cudaStream_t s);
cudaError_t launch3c_rhs(const Curv3Launch &a, int dtype, cudaStream_t s);
// a.out += the interface SAT terms of s at state a.q (a.met, gas constants as for rhs).
cudaError_t launch3c_isat(const Curv3Launch &a, const Curv3Sat &s, int dtype, cudaStream_t st);
// out (5 planes of nrecv) = the 4 x 4 x 4 Lagrange gather of q's 5 planes at each receiver's
// stencil (base: 3 ints, w: 12 doubles per receiver; device).
cudaError_t launch3c_interp(int ni, int nj, size_t field, const void *q, int nrecv, const int *base, const double *w,
                            void *out, int dtype, cudaStream_t s);

}  // namespace sbp
