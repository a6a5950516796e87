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

// Constants of the right-hand side in the compute type, prepared on the host (converting
// double constants inside a float kernel would occupy GB300's narrow FP64 pipe).
template <typename T>
struct KConst {
  T gam, g1, mu, kap, mu43, mu23;  // gamma, gamma-1, mu, mu/(Pr(gamma-1)), 4/3 mu, 2/3 mu
  T sig_int, sig_phys, tw;          // penalties; wall energy factor Tw/(gamma(gamma-1))
  T qinf[4];
  T mc[5];                          // Cartesian metrics
  T jx, jy;                         // Cartesian J xi_x and J eta_y (1/hx, 1/hy)
  // Cartesian meshes: the derivative rows' weights times 1/hx (wx) and 1/hy (wy), so that a
  // row sum is the physical derivative d/dx or d/dy (rows as in the device table: closures
  // 0-3, interior 4, hole 5)
  T wx[6][4], wy[6][4];
  // sponge layer: strength by index distance d < sponge_d to the nearest far-field face
  // (sponge_faces: bit f set for a far-field face f = i-low, i-high, j-low, j-high)
  int sponge_d, sponge_faces;
  T sponge_tab[16];
};

// A rectangle of tiles [x0, x1) x [y0, y1) of the split kernels' grid (x in kTileX columns, y in
// the kernel's rows per CTA). mode 0: every tile; 1: the rectangle's tiles only (the grid is the
// rectangle); 2: every tile outside the rectangle.
struct TileBox {
  int mode, x0, x1, y0, y1;
};

// Right-hand side (+ optional MRAB update) of one mesh: k_flux then k_update.
struct RhsLaunch {
  DevMesh m;
  Gas g;
  // tiles of the flux and the update kernel this launch covers (split kernels only)
  TileBox fbox, ubox;
  KConst<float> cf;
  KConst<double> cd;
  const void *q;
  void *sat;  // per SAT point: its 4 penalty terms (written by k_flux, added by k_update)
  // SAT points of this mesh grouped by 32 x 8 tile (tile id = (i / 32) * ceil(nj / 8) + j / 8);
  // tile_sat has one offset per tile + 1
  const int *tile_sat;
  int rows_per_cta;  // 8, 16 or 32: rows per CTA of the split kernels' flux kernel
  int rows_upd;      // 4, 8, 16 or 32: rows per CTA of their update kernel (0: rows_per_cta)
  // strip = 0: split kernels (k_flux, k_update); kMarchW: the single-pass marching kernel
  // (k_march) with strips of kMarchW columns and chunks of `chunk` rows per CTA
  int strip, chunk;
  void *flux;        // 8 planes: F^_xi (4 variables), F^_eta (4 variables)
  // Navier-Stokes primitives (u, v, T: 3 planes of the state's layout). prim_in: the flux
  // kernel reads the primitives of q from here instead of computing them; prim_out: the
  // update (mode 1) writes the primitives of qnext here. Either may be null.
  const void *prim_in;
  void *prim_out;
  const uint32_t *sat_ij;   // i | j << 16
  const uint32_t *sat_code;
  const int *sat_recv;
  const double *sat_scale;
  const void *qhat;
  const void *fvhat;
  int nrecv;
  // When dv is set, the receiver values are gathered in the SAT stage instead of read from
  // qhat/fvhat: q^ = sum_16 w_a w_b dv[c][didx], with dv the per-donor-point values of
  // k_donor_vals (10 planes of ndv values: 4 state, 6 viscous fluxes).
  const void *dv;
  const int *didx;
  const void *dwt;  // donor weights in the compute type, 8 per receiver
  int ndv;
  int nsat;         // number of SAT points (length of the planes of `sat`)
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

// Values at the distinct donor points of one receiving mesh, for `nsets` extrapolation sets:
// set s holds q + sum_k beta[s][k] hist[k] (nb[s] terms) and, for Navier-Stokes, the Cartesian
// viscous fluxes of that state. Output dv[(s * 10 + c) * S + d], S = stride (npts when 0).
constexpr int kMaxSets = 16;
struct DonorLaunch {
  DevMesh d;
  Gas g;
  const void *q;
  const void *hist[kMaxHist];
  double beta[kMaxSets][kMaxHist];
  int nb[kMaxSets];
  int nsets;
  int npts;
  const uint32_t *pts;  // i | j << 16
  void *dv;
  // plane stride of dv in elements (0: npts), so that several launches can fill the segments
  // of one receiving mesh's donor values that come from different donor meshes
  int stride;
};

// Columns per CTA and threads per CTA of the right-hand-side kernels.
// Offsets of the four (offset, weight) pairs of each SBP 4-2 derivative row (rows 0..3 the
// boundary closures, 4 the interior row, 5 a hole), for the device table and host set-up.
#define SBP_ROW_OFFSETS {{0, 1, 2, 3}, {-1, 1, 0, 0}, {-2, -1, 1, 2}, {-3, -1, 1, 2}, {-2, -1, 1, 2}, {0, 0, 0, 0}}

constexpr int kTileX = 32;
// Columns of a single-pass (marching) strip: 256 threads cover 4 rows of its 64-column flux
// window (the strip plus a 3-point halo per side) in one pass.
constexpr int kMarchW = 58;
// Flag in the marching kernel's chunk (RhsLaunch::chunk; the rows of sbp_set_rhs_shape for strips
// of kMarchW columns): stage the state and metric rows by TMA tensor copies (k_march_tma)
// instead of per-thread cp.async (k_march); both give the same bits.
constexpr int kStageTma = 0x10000;
// Output columns of the column-marching kernel's strips (CTAs of 128 or 256 threads, one column
// per thread, 6 halo columns per side); it needs meshes at least as wide as its CTA.
constexpr int kColW128 = 128 - 12, kColW256 = 256 - 12;
constexpr int kNT = 256;

// One micro step of a batch of systems (a cooperative launch): donor values of the listed
// receiving meshes, then fluxes and updates of the listed tiles. items: (descriptor, tile x,
// tile y, 1 if the mesh is curvilinear).
struct BatchSubstep {
  const void *dl;     // DonorLaunch[n_dl] in device memory
  const int *dl_off;  // n_dl + 1 prefix sums of the (set, point) pairs per descriptor
  int n_dl;
  const void *rl;     // RhsLaunch[n_rl] in device memory
  int n_rl;
  const int *sat_off; // n_rl + 1 prefix sums of the SAT points per descriptor (single-pass items)
  const int *rl_curv; // per descriptor: curvilinear mesh
  const int4 *items;  // (descriptor, tile column, tile row, curvilinear)
  int n_items;
  int chunk;          // rows per item: 8, 16 = flux / derivative tile pair; >= 32 single-pass strips
  unsigned *bar_count;
  unsigned *bar_gen;
  int *err;
};
cudaError_t launch_batch_substep(const BatchSubstep &b, int grid, int dtype, bool viscous, bool curv_fine, int ty,
                                 cudaStream_t s);
cudaError_t batch_grid_size(int dtype, bool viscous, bool curv_fine, int ty, int *grid);

// Discrete adjoint of one mesh's right-hand side (FP64): given lam = adjoint of dq/dt at the
// state q, accumulate lq += (dR/dq)^T lam, write the adjoint of the receiver values
// (lrv, 10 per receiver: state then viscous fluxes) and of the far-field state (lqinf, 4 per
// SAT point). Scratch: mu (8 planes), ld (6 planes), lp (3 planes).
struct AdjLaunch {
  DevMesh m;
  KConst<double> k;
  bool viscous;
  const double *q, *lam;
  double *lq, *mu, *ld, *lp;
  int nsat;
  const uint32_t *sat_ij, *sat_code;
  const int *sat_recv;
  const double *sat_scale;
  const double *rv;  // receiver values used by the forward evaluation (10 x nrecv)
  int nrecv;
  double *lrv;
  double *lqinf;
  double *satlin;    // scratch: 24 per SAT point
};
// Adjoint of the receiver values back to the donor mesh: per distinct donor point d,
// ldv(d) = sum over (receiver, stencil slot) using d of w lrv (inverse lists inv_off/inv_re,
// entries r * 16 + slot), then through the donor values (state shat and its viscous fluxes)
// into lshat (4 planes on the donor mesh, accumulated). Scratch on the donor mesh: ld (6
// planes, cleared here), lp (3 planes).
struct AdjDonorLaunch {
  DevMesh d;
  KConst<double> k;
  bool viscous;
  const double *shat;  // donor state the receiver values were taken from
  int npts;
  const uint32_t *pts;
  const int *inv_off, *inv_re;
  const double *w;     // 8 per receiver
  const double *lrv;   // 10 x nrecv
  int nrecv;
  double *ldv;         // scratch 10 x npts
  double *lshat, *ld, *lp;
};
cudaError_t launch_rhs_adjoint(const AdjLaunch &a, cudaStream_t s);
cudaError_t launch_donor_adjoint(const AdjDonorLaunch &a, cudaStream_t s);
// Probe pressures p_p = sum_d w_d p(q_d) (8 weights per probe, base (i0, j0)) and the adjoint
// seed lq(d) += scale * 2 p_p w_d dp/dq(q_d); probes are applied one after another.
cudaError_t launch_probe(const DevMesh &m, const double *q, int nprobe, const int *base, const double *w,
                         double *pout, double *lq, double scale, double gamma, cudaStream_t s);

// Tangent (Jacobian-vector product) of one mesh's right-hand side (FP64): out = (dR/dq) qd +
// (dR/drv) rvd + (dR/dqinf) qinfd, with rvd the tangent of the receiver values from the donor
// state's tangent (TlDonorLaunch, run first). Scratch: pd (3 planes), fd (8 planes) on the mesh;
// the donor side's pd on the donor mesh.
struct TlLaunch {
  DevMesh m;
  KConst<double> k;
  bool viscous;
  const double *q, *qd;
  double *pd, *fd, *out;
  int nsat;
  const uint32_t *sat_ij, *sat_code;
  const int *sat_recv;
  const double *sat_scale;
  const double *rv, *rvd;
  int nrecv;
  double qinfd[4];
};
struct TlDonorLaunch {
  DevMesh d;
  KConst<double> k;
  bool viscous;
  const double *q, *qd;  // donor state and its tangent
  double *pd;            // scratch: 3 planes on the donor mesh
  int nrecv;
  const int *base;
  const double *w;
  double *rvd;           // 10 x nrecv
};
cudaError_t launch_rhs_tangent(const TlLaunch &a, const TlDonorLaunch &dn, cudaStream_t s);

// FP64 linear combinations and reductions used by the adjoint driver.
constexpr int kMaxLin = 8;
struct LinComb {
  double c[kMaxLin];
  const double *x[kMaxLin];
};
cudaError_t launch_lincomb(double *out, const double *base, const LinComb &lc, int nx, size_t n, cudaStream_t s);
cudaError_t launch_sum4(const double *x, int n, double *acc, cudaStream_t s);

cudaError_t launch_rhs(const RhsLaunch &a, int dtype, bool viscous, cudaStream_t s);
cudaError_t launch_interp(const InterpLaunch &a, int dtype, bool viscous, cudaStream_t s);
cudaError_t launch_donor_vals(const DonorLaunch &a, int dtype, bool viscous, cudaStream_t s);
cudaError_t launch_dt(const DevMesh &m, const Gas &g, const void *q, int dtype, unsigned long long *out,
                      cudaStream_t s);
cudaError_t launch_metrics(const DevMesh &m, const double *x, const double *y, const double shift[4], void *met,
                           int dtype, cudaStream_t s);
// out = q + sum_{k < nh} alpha[k] hist[k] (history order), FP64 accumulation, over n elements.
struct ABCombine {
  const void *hist[kMaxHist];
  double alpha[kMaxHist];
  int nh;
};
cudaError_t launch_ab_combine(const void *q, const ABCombine &c, void *out, size_t n, int dtype, cudaStream_t s);
// y_out = y + c1 k1 + c2 k2 (k2 may be NULL), FP64 accumulation, over n elements.
cudaError_t launch_axpy(const void *y, const void *k1, double c1, const void *k2, double c2, void *y_out, size_t n,
                        int dtype, cudaStream_t s);
// y = (double)x element by element through the integer widening of the FP32 forms.
cudaError_t launch_widen(const float *x, double *y, size_t n, cudaStream_t s);
// Interpolation + right-hand side with the receiver workspace in the library's fixed device
// array (sbp_noalloc.cu); the qhat/fvhat pointers of the descriptors are replaced.
cudaError_t rhs_eval_static_scratch(InterpLaunch ia, RhsLaunch ra, int dtype, bool viscous, size_t elem,
                                    cudaStream_t s);

}  // namespace sbp
