// Launch descriptors and launchers of the library's CUDA kernels (sbp_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "sbp_internal.h"

namespace sbp {

// One mesh as the kernels see it. Metrics are 5 planes (xi_x/J, xi_y/J, eta_x/J, eta_y/J, J)
// of the element type on curvilinear meshes; Cartesian meshes use the constants mc.
struct DevMesh {
  int ni, nj, pitch, per_i, per_j, cart;
  size_t field;
  const uint8_t *cls;
  const void *met;
  double mc[5];
};

struct Gas {
  double gamma, mu, pr, twall, sig_int, sig_phys;
  double qinf[4];
};

// Fused right-hand side (+ optional MRAB update) over all tiles of one mesh.
struct RhsLaunch {
  DevMesh m;
  Gas g;
  const void *q;
  // SAT points of this mesh, grouped by tile (tile_sat has one offset per tile + 1)
  const int *tile_sat;
  const uint32_t *sat_ij;   // i | j << 16
  const uint32_t *sat_code;
  const int *sat_recv;
  const double *sat_scale;
  const void *qhat;
  const void *fvhat;
  int nrecv;
  // epilogue: mode 0 writes dq/dt to out; mode 1 writes it to out (the newest history slot)
  // and qnext = q + sum_k alpha[k] hold[k] + alpha[nold] dq/dt (FP64 accumulation)
  int mode;
  void *out;
  void *qnext;
  const void *hold[kMaxHist];
  double alpha[kMaxHist];
  int nold;
  int *err;
};

// Interpolation of a (possibly extrapolated) donor state to the receivers of the other mesh.
struct InterpLaunch {
  DevMesh d;
  Gas g;
  const void *q;
  const void *hist[kMaxHist];
  double beta[kMaxHist];
  int nbeta;  // 0: plain state; else q + sum_k beta[k] hist[k]
  int nrecv;
  const int *base;
  const double *w;
  void *qhat;
  void *fvhat;  // NULL: skip the viscous fluxes
};

// Tile of the fused right-hand-side kernel.
constexpr int kTileX = 32, kTileY = 8;

cudaError_t launch_rhs(const RhsLaunch &a, int dtype, bool viscous, cudaStream_t s);
cudaError_t launch_interp(const InterpLaunch &a, int dtype, bool viscous, cudaStream_t s);
cudaError_t launch_dt(const DevMesh &m, const Gas &g, const void *q, int dtype, unsigned long long *out,
                      cudaStream_t s);
cudaError_t launch_metrics(const DevMesh &m, const double *x, const double *y, const double shift[4], void *met,
                           int dtype, cudaStream_t s);
// y_out = y + c1 k1 + c2 k2 (k2 may be NULL), FP64 accumulation, over n elements.
cudaError_t launch_axpy(const void *y, const void *k1, double c1, const void *k2, double c2, void *y_out, size_t n,
                        int dtype, cudaStream_t s);
size_t rhs_smem_bytes(int dtype, bool viscous, bool curvilinear);
// Interpolation + right-hand side with the receiver workspace in the library's fixed device
// array (sbp_noalloc.cu); the qhat/fvhat pointers of the descriptors are replaced.
cudaError_t rhs_eval_static_scratch(InterpLaunch ia, RhsLaunch ra, int dtype, bool viscous, size_t elem,
                                    cudaStream_t s);

}  // namespace sbp
