// Launch descriptors of the 3D curvilinear operator (sbp3c_kernels.cu): one structured mesh,
// non-periodic in every direction, arrays unpitched, point (i, j, k) at (k * nj + j) * ni + i.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "sbp_device.h"

namespace sbp {

struct Curv3Launch {
  int ni, nj, nk;
  size_t field;          // ni * nj * nk
  // stencil classes, 4 bits per direction (i, j, k), 0xFFF for a hole (the 3D Cartesian
  // systems' codes): every maximal active run along a line is one SBP segment; NULL: whole
  // lines (no holes)
  const uint16_t *cls;
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
// stencil (base: 3 ints, w: 12 doubles per receiver; device). The bases come from the caller:
// a stencil that does not lie inside the ni x nj x nk mesh records SBP_ERR_BOUNDS in *err and
// gives zeros, without reading out of range.
cudaError_t launch3c_interp(int ni, int nj, int nk, const void *q, int nrecv, const int *base, const double *w,
                            void *out, int *err, int dtype, cudaStream_t s);

// Donor values of a curvilinear mesh for another mesh's receivers (Sec. 2.2 interpolation with
// Sec. 3.3 Step 2's extrapolation in time): one thread per (extrapolation set, distinct donor
// point) writes the state q + sum_k beta[set][k] hist[k] (FP64 accumulation) and, for
// Navier-Stokes, the Cartesian viscous fluxes of that state by the mesh's own SBP derivatives
// and metric terms, point-major: dv[(set * npts + point) * kDvPitch + c] (c: 5 state values,
// then F^V_x, F^V_y, F^V_z, each momentum x, y, z and energy; kDvPitch elements per point so
// that a point's values are read by 16-byte loads).
constexpr int kDvPitch = 20;
struct Curv3Donor {
  Curv3Launch m;                       // the donor mesh (q, met, cls, gas constants)
  const void *hist[kMaxHist];
  double beta[kMaxSets][kMaxHist];
  int nb[kMaxSets];
  int nsets, npts;
  const long long *pts;                // linear indices (k nj + j) ni + i on the donor mesh
  void *dv;
  // Navier-Stokes: the distinct points the donor points' derivative stencils read (ntap linear
  // indices), 13 indices into them per donor point (the point, then the 4 taps along i, j and
  // k), and a workspace of 4 values (u, v, w, T of the extrapolated state) per set and tap point,
  // so that each tap's extrapolated primitives are formed once; NULL tpts: formed per use
  const long long *tpts;
  const int *tidx;
  int ntap;
  void *tv;
};
cudaError_t launch3c_donor(const Curv3Donor &a, int dtype, cudaStream_t s);

// Receiver values of one donor-value set: out_c[r] = sum over the 64 stencil points of
// wi wj wk dv[didx][c] (dv point-major as k3c_donor writes it; didx 64 and dwt 12 (element
// type) per receiver), c < 5 into qhat (5 x nrecv), c >= 5 into fvhat (12 x nrecv; nval = 17
// for Navier-Stokes, else 5). One thread per receiver.
struct Curv3Gather {
  const void *dv;
  const int *didx;
  const void *dwt;
  int nrecv, nval, ndv;
  void *qhat, *fvhat;
  int *err;   // SBP_BOUNDS_CHECK builds: where an out-of-range donor index is recorded
};
cudaError_t launch3c_gather(const Curv3Gather &a, int dtype, cudaStream_t s);

// Adams-Bashforth combine (Sec. 3.1-3.3) over the whole mesh: qn = q + sum_{h < nold} alpha[h]
// hold[h] + alpha[nold] rhs (FP64 accumulation); a non-finite or non-positive-density result at
// an active point raises SBP_ERR_NONFINITE in *err.
struct Curv3Ab {
  size_t field;
  const uint16_t *cls;                 // NULL: every point active
  const void *q, *rhs;
  const void *hold[kMaxHist];
  double alpha[kMaxHist];
  int nold;
  void *qn;
  int *err;
};
cudaError_t launch3c_ab(const Curv3Ab &a, int dtype, cudaStream_t s);

// Sponge layer (Sec. 5.1) of a mesh whose six faces are far field: a.out -= sigma (a.q - a.qinf)
// at the active points within d < depth index points of the nearest face, sigma = tab[d]
// (A ((depth - d) / depth)^2, computed on the host); after the SAT terms.
struct Curv3Sponge {
  int depth;        // 1..16
  double tab[16];
};
cudaError_t launch3c_sponge(const Curv3Launch &a, const Curv3Sponge &sp, int dtype, cudaStream_t s);

// Time step of the curvilinear mesh at state q (active points): min over points of
// 1 / (sum_m |u . k_m| + c |K| + 2 nu |K|^2), k_m = J M[m][:], |K|^2 = sum_m |k_m|^2,
// nu = max(mu, gamma mu / Pr) / rho, as the bits of a positive double min-reduced into *out.
cudaError_t launch3c_dt(const Curv3Launch &a, double pr, unsigned long long *out, cudaStream_t s, int dtype);

}  // namespace sbp
