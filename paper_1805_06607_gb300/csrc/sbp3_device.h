// Launch descriptors and launchers of the 3D Cartesian kernels (sbp3_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "sbp_device.h"
#include "sbp_internal.h"

namespace sbp {

// One 3D mesh as the kernels see it: point (i, j, k) at (k * nj + j) * pitch + i of each plane.
struct Dev3Mesh {
  int ni, nj, nk, pitch, per[3];
  size_t field;          // pitch * nj * nk
  const uint16_t *cls;   // 4 bits per direction, 0xFFF = hole
};

// Constants in the compute type (prepared on the host).
template <typename T>
struct K3 {
  T gam, mu, lam, kap;   // gamma, mu, -2/3 mu, mu / (Pr (gamma - 1))
  T sig_int, sig_phys;
  T qinf[5];
  T ih[3];               // 1 / h per direction
  // sponge layer: strength by index distance d < sponge_d to the nearest far-field face
  // (sponge_faces: bit f for a far-field face f = i-low, i-high, j-low, j-high, k-low, k-high)
  int sponge_d, sponge_faces;
  T sponge_tab[16];
};

constexpr int kRv3 = 17;  // receiver values: state (5), F^V_x, F^V_y, F^V_z (4 each)

struct Rhs3Launch {
  Dev3Mesh m;
  K3<float> cf;
  K3<double> cd;
  bool visc;
  const void *q;
  void *prim;   // 4 planes (u, v, w, T); Navier-Stokes only
  void *flux;   // 15 planes: F - F^V, G - G^V, H - H^V
  void *sat;    // 5 values per SAT point
  int nsat;
  const int64_t *sat_pt;     // (k * nj + j) * ni + i, sorted
  const uint32_t *sat_code;
  const int *sat_recv;
  const double *sat_scale;
  const int *row_sat;        // nj * nk + 1 offsets: SAT points of row (j, k)
  const void *dv;            // donor values: kRv3 planes of ndv (one extrapolation set)
  const int *didx;           // 64 per receiver
  const void *dwt;           // 12 per receiver, compute type
  int ndv, nrecv;
  int kchunk;                // > 0: the k-marching kernels with chunks of kchunk planes; 0: per-point kernels
  int mode;                  // 0: out = dq/dt; 1: also qnext = q + sum alpha hold + alpha dq/dt
  void *out;
  void *qnext;
  const void *hold[kMaxHist];
  double alpha[kMaxHist];
  int nold;
  int *err;
};

struct Donor3Launch {
  Dev3Mesh d;
  K3<float> cf;
  K3<double> cd;
  bool visc;
  const void *q;
  const void *hist[kMaxHist];
  double beta[kMaxSets][kMaxHist];
  int nb[kMaxSets];
  int nsets, npts;
  const int64_t *pts;   // linear index (k * nj + j) * ni + i on the donor mesh
  void *dv;             // dv[(set * kRv3 + c) * npts + d]
};

// Receiver values from one donor-value set: rv[c * nrecv + r] (qhat then fvhat layout).
struct Gather3Launch {
  const void *dv;
  const int *didx;
  const void *dwt;
  int ndv, nrecv, nval;
  void *qhat;
  void *fvhat;
  int *err;   // SBP_BOUNDS_CHECK builds: where an out-of-range donor index is recorded (may be null)
};

cudaError_t launch3_rhs(const Rhs3Launch &a, int dtype, cudaStream_t s);
cudaError_t launch3_donor(const Donor3Launch &a, int dtype, cudaStream_t s);
cudaError_t launch3_gather(const Gather3Launch &a, int dtype, cudaStream_t s);
cudaError_t launch3_dt(const Dev3Mesh &m, const K3<double> &k, double mu, double pr, const void *q, int dtype,
                       unsigned long long *out, cudaStream_t s);

}  // namespace sbp
