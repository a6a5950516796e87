/*
 * Plain FP64 CPU oracle for the SBP-SAT overset right-hand side (2D).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a small shared
 * library that the tests, the smoke check and the benchmark's CPU-baseline
 * leg load through ctypes.  The GPU library never links, includes or calls
 * it, and it shares no code, tables or helpers with the GPU library.
 *
 * Everything here is a direct restatement of the paper's definitions, one
 * full-array pass at a time, with no blocking or fusion:
 *   - SBP 4-2 diagonal-norm first derivative D (Sec. 2.1, App. C.1);
 *   - curvilinear metrics by D applied to the coordinates (Sec. 2.1, Sec. 4.1);
 *   - inviscid and viscous fluxes of the compressible Navier-Stokes
 *     equations (App. C.1), contravariant form dq/dt = -J sum_m D_m F^_m;
 *   - SAT interface penalty eq. (int) of Sec. 2.2, with the far-field and
 *     isothermal-wall penalties written in the same form (Sec. 5.1);
 *   - donor-cell tensor-product Lagrange interpolation (Sec. 2.2, Sec. 3.3);
 *   - hole cutting and donor search (Sec. 2.2);
 *   - the inviscid/viscous time-step estimate of Sec. 4.1 eqs. (ts_inv),
 *     (ts_visc), (ts_overall).
 * Where the paper is silent, the reading taken is stated next to the code
 * that takes it.
 *
 * The per-point loops run under OpenMP (orc_set_threads picks the thread
 * count): every point's arithmetic is independent of the others and of the
 * thread count, so the results are the same bits for any number of threads.
 * Accumulations into one point (the SAT terms) stay sequential.
 *
 * Array layout: every field is (nvar, nj, ni) with i fastest; a point index
 * is p = j*ni + i.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "orc_sbp.h"

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the per-point loops (n <= 0: the OpenMP default); returns the count in use. */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* iblank: in/out active mask (1 active, 0 hole).  ci/cj: class along i and along j.
 * Returns the number of hole-growing passes, or -1 if a whole line became inactive
 * although the mesh had points on it that another direction keeps active.              */
int orc_classes2d(int ni, int nj, int per_i, int per_j, signed char *iblank, signed char *ci,
                  signed char *cj) {
  int passes = 0;
  for (;;) {
    int too_short = 0;
    for (int j = 0; j < nj; ++j)
      classify_line(iblank + (long)j * ni, ni, 1, per_i, ci + (long)j * ni, 1, &too_short);
    for (int i = 0; i < ni; ++i)
      classify_line(iblank + i, nj, ni, per_j, cj + i, ni, &too_short);
    if (!too_short) break;
    ++passes;
    if (passes > 64) return -1;
  }
  /* a point inactive in one direction is a hole in both */
  for (long p = 0; p < (long)ni * nj; ++p)
    if (!iblank[p]) { ci[p] = CL_HOLE; cj[p] = CL_HOLE; }
  return passes;
}

/* ---------------------------------------------------------------------------------------- */
/* Metrics (reading of Sec. 2.1 / Sec. 4.1, which defer the form): x_xi, x_eta, y_xi, y_eta by
 * the same D used for the fluxes, J^-1 = x_xi y_eta - x_eta y_xi, and
 *   xi_x/J = y_eta, xi_y/J = -x_eta, eta_x/J = -y_xi, eta_y/J = x_xi, J = 1/J^-1.
 * met = [xi_x/J, xi_y/J, eta_x/J, eta_y/J, J] per point.  Inactive points get the finite
 * placeholder (1, 0, 0, 1, 1); nothing reads it.  shift = (sx_i, sy_i, sx_j, sy_j): the
 * coordinate jump across a periodic wrap in i and in j.                                    */
int orc_metrics2d(int ni, int nj, const double *shift, const double *x, const double *y,
                  const signed char *ci, const signed char *cj, double *met) {
  long N = (long)ni * nj;
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      long p = (long)j * ni + i;
      if (ci[p] == CL_HOLE) {
        met[p] = 1.0; met[N + p] = 0.0; met[2 * N + p] = 0.0; met[3 * N + p] = 1.0; met[4 * N + p] = 1.0;
        continue;
      }
      double x_xi = orc_d1(x + (long)j * ni, 1, ni, i, ci[p], shift[0]);
      double y_xi = orc_d1(y + (long)j * ni, 1, ni, i, ci[p], shift[1]);
      double x_eta = orc_d1(x + i, ni, nj, j, cj[p], shift[2]);
      double y_eta = orc_d1(y + i, ni, nj, j, cj[p], shift[3]);
      double jinv = x_xi * y_eta - x_eta * y_xi;
      if (!(jinv > 0.0)) return -1 - (int)p; /* zero or negative cell volume */
      met[p] = y_eta;
      met[N + p] = -x_eta;
      met[2 * N + p] = -y_xi;
      met[3 * N + p] = x_xi;
      met[4 * N + p] = 1.0 / jinv;
    }
  return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Physics.  q = (rho, rho u, rho v, rho E); p = (gamma-1)(rho E - rho |u|^2 / 2);
 * T = gamma p / rho (free stream rho = 1, c = 1, so T_inf = 1).                             */
typedef struct {
  double gamma, mu, pr;
} orc_gas;

/* Cartesian inviscid fluxes F (x) and G (y) of the Euler part of App. C.1. */
static void euler_flux(const double q[4], double gamma, double F[4], double G[4]) {
  double rho = q[0], u = q[1] / rho, v = q[2] / rho, E = q[3];
  double p = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
  F[0] = rho * u;      G[0] = rho * v;
  F[1] = rho * u * u + p; G[1] = rho * u * v;
  F[2] = rho * u * v;  G[2] = rho * v * v + p;
  F[3] = (E + p) * u;  G[3] = (E + p) * v;
}

/* Cartesian viscous fluxes at every active point (App. C.1): tau_ij = mu (du_i/dx_j +
 * du_j/dx_i) + lambda div(u) delta_ij with lambda = -2/3 mu (Stokes), heat flux
 * q_j = -mu/(Pr (gamma-1)) dT/dx_j; gradients by D and the chain rule
 * d/dx_j = sum_m J (xi_m,x_j / J) D_m.  fv = (Fx1, Fx2, Fx3, Fy1, Fy2, Fy3), the momentum and
 * energy components of F^V_x and F^V_y (the mass component is zero).                       */
int orc_viscflux2d(int ni, int nj, int per_i, int per_j, const signed char *ci, const signed char *cj,
                   const double *met, const double *q, double gamma, double mu, double pr, double *fv) {
  (void)per_j;
  long N = (long)ni * nj;
  double *prim = (double *)malloc(sizeof(double) * 3 * N); /* u, v, T */
  if (!prim) return -1;
#pragma omp parallel for schedule(static)
  for (long p = 0; p < N; ++p) {
    double rho = q[p], u = q[N + p] / rho, v = q[2 * N + p] / rho;
    double pr_ = (gamma - 1.0) * (q[3 * N + p] - 0.5 * rho * (u * u + v * v));
    prim[p] = u; prim[N + p] = v; prim[2 * N + p] = gamma * pr_ / rho;
  }
  (void)per_i;
  double lam = -2.0 / 3.0 * mu;
  double kap = mu / (pr * (gamma - 1.0));
#pragma omp parallel for schedule(static)
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      long p = (long)j * ni + i;
      if (ci[p] == CL_HOLE) { for (int c = 0; c < 6; ++c) fv[c * N + p] = 0.0; continue; }
      double g[3][2];
      for (int f = 0; f < 3; ++f) {
        const double *fl = prim + f * N;
        double dxi = orc_d1(fl + (long)j * ni, 1, ni, i, ci[p], 0.0);
        double deta = orc_d1(fl + i, ni, nj, j, cj[p], 0.0);
        double J = met[4 * N + p];
        g[f][0] = J * (met[p] * dxi + met[2 * N + p] * deta);
        g[f][1] = J * (met[N + p] * dxi + met[3 * N + p] * deta);
      }
      double ux = g[0][0], uy = g[0][1], vx = g[1][0], vy = g[1][1], Tx = g[2][0], Ty = g[2][1];
      double div = ux + vy;
      double txx = mu * (2.0 * ux) + lam * div;
      double txy = mu * (uy + vx);
      double tyy = mu * (2.0 * vy) + lam * div;
      double qx = -kap * Tx, qy = -kap * Ty;
      double u = prim[p], v = prim[N + p];
      fv[p] = txx; fv[N + p] = txy; fv[2 * N + p] = u * txx + v * txy - qx;
      fv[3 * N + p] = txy; fv[4 * N + p] = tyy; fv[5 * N + p] = u * txy + v * tyy - qy;
    }
  free(prim);
  return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Penalty matrix K^{+/-}_k = T ((|Lambda| +/- Lambda)/2) T^-1 of eq. (int) for the flux
 * Jacobian A_k = d(k_x F + k_y G)/dq at state q, with the full (unnormalised) metric gradient
 * k.  A_k has the three distinct eigenvalues U, U + c|k|, U - c|k| (U = k.u) and is
 * diagonalisable, so any function of it is given exactly by Sylvester's formula
 *   f(A) = sum_i f(l_i) prod_{j != i} (A - l_j I) / (l_i - l_j).
 * side = +1 gives K^+, side = -1 gives K^-.                                                 */
static void flux_jacobian(const double q[4], double gamma, double kx, double ky, double A[4][4]) {
  double rho = q[0], u = q[1] / rho, v = q[2] / rho, E = q[3];
  double p = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
  double U = kx * u + ky * v;
  double phi2 = 0.5 * (gamma - 1.0) * (u * u + v * v);
  double H = (E + p) / rho;
  double g1 = gamma - 1.0;
  A[0][0] = 0.0; A[0][1] = kx; A[0][2] = ky; A[0][3] = 0.0;
  A[1][0] = kx * phi2 - u * U; A[1][1] = U - (gamma - 2.0) * kx * u; A[1][2] = ky * u - g1 * kx * v; A[1][3] = g1 * kx;
  A[2][0] = ky * phi2 - v * U; A[2][1] = kx * v - g1 * ky * u; A[2][2] = U - (gamma - 2.0) * ky * v; A[2][3] = g1 * ky;
  A[3][0] = U * (phi2 - H); A[3][1] = kx * H - g1 * u * U; A[3][2] = ky * H - g1 * v * U; A[3][3] = gamma * U;
}

void orc_penalty_matrix2d(const double q[4], double gamma, double kx, double ky, int side, double K[4][4]) {
  double A[4][4];
  flux_jacobian(q, gamma, kx, ky, A);
  double rho = q[0], u = q[1] / rho, v = q[2] / rho;
  double p = (gamma - 1.0) * (q[3] - 0.5 * rho * (u * u + v * v));
  double c = sqrt(gamma * p / rho);
  double kn = sqrt(kx * kx + ky * ky);
  double lam[3] = {kx * u + ky * v, kx * u + ky * v + c * kn, kx * u + ky * v - c * kn};
  memset(K, 0, sizeof(double) * 16);
  for (int a = 0; a < 3; ++a) {
    double fl = 0.5 * (fabs(lam[a]) + side * lam[a]);
    /* P = prod_{b != a} (A - lam_b I)/(lam_a - lam_b) */
    double P[4][4], T[4][4];
    for (int r = 0; r < 4; ++r)
      for (int s = 0; s < 4; ++s) P[r][s] = (r == s) ? 1.0 : 0.0;
    for (int b = 0; b < 3; ++b) {
      if (b == a) continue;
      double den = lam[a] - lam[b];
      for (int r = 0; r < 4; ++r)
        for (int s = 0; s < 4; ++s) {
          double acc = 0.0;
          for (int t = 0; t < 4; ++t) acc += P[r][t] * (A[t][s] - (t == s ? lam[b] : 0.0));
          T[r][s] = acc / den;
        }
      memcpy(P, T, sizeof(P));
    }
    for (int r = 0; r < 4; ++r)
      for (int s = 0; s < 4; ++s) K[r][s] += fl * P[r][s];
  }
}

/* ---------------------------------------------------------------------------------------- */
/* Right-hand side on one mesh (Sec. 2.2 eq. (int)):
 *   dq/dt = -J sum_m D_m (F^I_m - F^V_m) + SAT
 * with contravariant fluxes F^_m = (xi_m,x/J) F + (xi_m,y/J) G.  Holes get dq/dt = 0.
 *
 * SAT terms are listed explicitly, one per (point, normal direction, side):
 *   kind 1 (interface): -p0^-1 [ (sigI K^side_k + sigma1 I)(q - qhat)
 *                                - side/2 (F^V_k - F^V_k hat) ] * scale
 *   kind 2 (far field): -p0^-1 sigP K^side_k (q - qinf)
 *   kind 3 (isothermal wall): -p0^-1 (sigP K^side_k + sigma1 I)(q - q_w),
 *        q_w = (rho, 0, 0, rho Tw / (gamma (gamma-1)))
 * where k = J (xi_m,x/J, xi_m,y/J) is the metric gradient of the normal direction m,
 * sigma1 = mu |k|^2 / 2, side = +1 at the low-index face ("+") and -1 at the high-index face.
 * qhat (4 x nrecv) and fvhat (6 x nrecv, Cartesian viscous fluxes) hold the interpolated
 * donor values for interface terms; fvhat may be NULL for Euler.                            */
int orc_rhs2d(int ni, int nj, int per_i, int per_j, const signed char *ci, const signed char *cj,
              const double *met, const double *q, int viscous, double gamma, double mu, double pr,
              int nterm, const int *t_pt, const int *t_dir, const int *t_side, const int *t_kind,
              const int *t_recv, const double *t_scale, int nrecv, const double *qhat,
              const double *fvhat, const double *qinf, double twall, double sig_int, double sig_phys,
              double *rhs) {
  (void)per_i; (void)per_j;
  long N = (long)ni * nj;
  double *fl = (double *)malloc(sizeof(double) * 8 * N); /* F^_xi (4), F^_eta (4) */
  double *fv = viscous ? (double *)malloc(sizeof(double) * 6 * N) : NULL;
  if (!fl || (viscous && !fv)) { free(fl); free(fv); return -1; }
  if (viscous) orc_viscflux2d(ni, nj, per_i, per_j, ci, cj, met, q, gamma, mu, pr, fv);

#pragma omp parallel for schedule(static)
  for (long p = 0; p < N; ++p) {
    double qp[4] = {q[p], q[N + p], q[2 * N + p], q[3 * N + p]};
    double F[4], G[4];
    euler_flux(qp, gamma, F, G);
    double Fv[4] = {0, 0, 0, 0}, Gv[4] = {0, 0, 0, 0};
    if (viscous) {
      Fv[1] = fv[p]; Fv[2] = fv[N + p]; Fv[3] = fv[2 * N + p];
      Gv[1] = fv[3 * N + p]; Gv[2] = fv[4 * N + p]; Gv[3] = fv[5 * N + p];
    }
    for (int v = 0; v < 4; ++v) {
      fl[v * N + p] = met[p] * (F[v] - Fv[v]) + met[N + p] * (G[v] - Gv[v]);
      fl[(4 + v) * N + p] = met[2 * N + p] * (F[v] - Fv[v]) + met[3 * N + p] * (G[v] - Gv[v]);
    }
  }
#pragma omp parallel for schedule(static)
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      long p = (long)j * ni + i;
      for (int v = 0; v < 4; ++v) {
        if (ci[p] == CL_HOLE) { rhs[v * N + p] = 0.0; continue; }
        double dxi = orc_d1(fl + v * N + (long)j * ni, 1, ni, i, ci[p], 0.0);
        double deta = orc_d1(fl + (4 + v) * N + i, ni, nj, j, cj[p], 0.0);
        rhs[v * N + p] = -met[4 * N + p] * (dxi + deta);
      }
    }

  for (int t = 0; t < nterm; ++t) {
    long p = t_pt[t];
    int m = t_dir[t], side = t_side[t], kind = t_kind[t];
    double J = met[4 * N + p];
    double kx = J * met[(2 * m) * N + p], ky = J * met[(2 * m + 1) * N + p];
    double qp[4] = {q[p], q[N + p], q[2 * N + p], q[3 * N + p]};
    double tgt[4];
    double sigI = (kind == 1) ? sig_int : sig_phys;
    double sig1 = 0.0;
    if (kind == 1) {
      int r = t_recv[t];
      if (r < 0 || r >= nrecv) { free(fl); free(fv); return -2; }
      for (int v = 0; v < 4; ++v) tgt[v] = qhat[(long)v * nrecv + r];
      if (viscous) sig1 = 0.5 * mu * (kx * kx + ky * ky);
    } else if (kind == 2) {
      for (int v = 0; v < 4; ++v) tgt[v] = qinf[v];
    } else {
      tgt[0] = qp[0]; tgt[1] = 0.0; tgt[2] = 0.0; tgt[3] = qp[0] * twall / (gamma * (gamma - 1.0));
      if (viscous) sig1 = 0.5 * mu * (kx * kx + ky * ky);
    }
    double K[4][4];
    orc_penalty_matrix2d(qp, gamma, kx, ky, side, K);
    double dq[4];
    for (int v = 0; v < 4; ++v) dq[v] = qp[v] - tgt[v];
    double sat[4];
    for (int v = 0; v < 4; ++v) {
      double acc = 0.0;
      for (int w = 0; w < 4; ++w) acc += K[v][w] * dq[w];
      sat[v] = -(sigI * acc + sig1 * dq[v]) / ORC_P0;
    }
    if (kind == 1 && viscous) {
      int r = t_recv[t];
      double own[4] = {0.0, kx * fv[p] + ky * fv[3 * N + p], kx * fv[N + p] + ky * fv[4 * N + p],
                       kx * fv[2 * N + p] + ky * fv[5 * N + p]};
      double hat[4] = {0.0, kx * fvhat[0L * nrecv + r] + ky * fvhat[3L * nrecv + r],
                       kx * fvhat[1L * nrecv + r] + ky * fvhat[4L * nrecv + r],
                       kx * fvhat[2L * nrecv + r] + ky * fvhat[5L * nrecv + r]};
      for (int v = 1; v < 4; ++v) sat[v] += 0.5 * side * (own[v] - hat[v]) / ORC_P0;
    }
    for (int v = 0; v < 4; ++v) rhs[v * N + p] += t_scale[t] * sat[v];
  }
  free(fl);
  free(fv);
  return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Donor-cell Lagrange interpolation (Sec. 2.2; shape functions of Sec. 3.3's P):
 * out[f][r] = sum_a sum_b wi[r][a] wj[r][b] field[f][j0+b][i0+a], indices wrapped on
 * periodic directions.  base = (i0, j0) per receiver; w = (wi[4], wj[4]) per receiver.   */
int orc_interp2d(int ni, int nj, int nf, const double *field, int nrecv, const int *base,
                 const double *w, double *out) {
  long N = (long)ni * nj;
#pragma omp parallel for schedule(static)
  for (int r = 0; r < nrecv; ++r) {
    for (int f = 0; f < nf; ++f) {
      double acc = 0.0;
      for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
          int ii = ((base[2 * r] + a) % ni + ni) % ni;
          int jj = ((base[2 * r + 1] + b) % nj + nj) % nj;
          acc += w[8 * r + a] * w[8 * r + 4 + b] * field[f * N + (long)jj * ni + ii];
        }
      out[(long)f * nrecv + r] = acc;
    }
  }
  return 0;
}

/* Lagrange basis on the nodes 0,1,2,3 and its derivative, at s. */
static void lagrange4(double s, double l[4], double dl[4]) {
  for (int a = 0; a < 4; ++a) {
    double v = 1.0, d = 0.0;
    for (int b = 0; b < 4; ++b) {
      if (b == a) continue;
      double prod = 1.0 / (a - b);
      for (int c = 0; c < 4; ++c) {
        if (c == a || c == b) continue;
        prod *= (s - c) / (a - c);
      }
      d += prod;
      v *= (s - b) / (a - b);
    }
    l[a] = v;
    dl[a] = d;
  }
}

/* Start of the 4-point donor stencil for a computational coordinate s on a line of n points:
 * i0 = floor(s) - 1, shifted inward at non-periodic ends.                                  */
static int stencil_start(double s, int n, int per) {
  int i0 = (int)floor(s) - 1;
  if (!per) {
    if (i0 < 0) i0 = 0;
    if (i0 > n - 4) i0 = n - 4;
  }
  return i0;
}

/* Donor search (Sec. 2.2): for each target point find computational coordinates (xi, eta) on
 * the donor mesh with X(xi, eta) = (px, py), X the mesh map interpolated by the same 4x4
 * Lagrange basis; Newton from the nearest mesh point, iterated to the rounding floor.
 * Outputs base (i0, j0), weights (wi[4], wj[4]) and (xi, eta).  Returns 0, or 1 + index of
 * the first target with no valid donor (outside the mesh, no convergence, or a stencil that
 * touches an inactive point).                                                             */
int orc_donors2d(int ni, int nj, int per_i, int per_j, const double *shift, const double *x,
                 const double *y, const signed char *iblank, int npts, const double *px,
                 const double *py, int *base, double *w, double *xe) {
  for (int t = 0; t < npts; ++t) {
    double best = INFINITY;
    int bi = 0, bj = 0;
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        long p = (long)j * ni + i;
        double d = (x[p] - px[t]) * (x[p] - px[t]) + (y[p] - py[t]) * (y[p] - py[t]);
        if (d < best) { best = d; bi = i; bj = j; }
      }
    double s = bi, r = bj;
    int ok = 0; /* consecutive small Newton steps */
    for (int it = 0; it < 100; ++it) {
      int i0 = stencil_start(s, ni, per_i), j0 = stencil_start(r, nj, per_j);
      double li[4], dli[4], lj[4], dlj[4];
      lagrange4(s - i0, li, dli);
      lagrange4(r - j0, lj, dlj);
      double X = 0, Y = 0, Xs = 0, Xr = 0, Ys = 0, Yr = 0;
      for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
          int ii = i0 + a, jj = j0 + b;
          int wi = 0, wj = 0;
          while (ii < 0) { ii += ni; wi -= 1; }
          while (ii >= ni) { ii -= ni; wi += 1; }
          while (jj < 0) { jj += nj; wj -= 1; }
          while (jj >= nj) { jj -= nj; wj += 1; }
          long p = (long)jj * ni + ii;
          double xv = x[p] + wi * shift[0] + wj * shift[2];
          double yv = y[p] + wi * shift[1] + wj * shift[3];
          X += li[a] * lj[b] * xv;  Y += li[a] * lj[b] * yv;
          Xs += dli[a] * lj[b] * xv; Xr += li[a] * dlj[b] * xv;
          Ys += dli[a] * lj[b] * yv; Yr += li[a] * dlj[b] * yv;
        }
      double fx = X - px[t], fy = Y - py[t];
      double det = Xs * Yr - Xr * Ys;
      if (det == 0.0) break;
      double ds = (Yr * fx - Xr * fy) / det;
      double dr = (-Ys * fx + Xs * fy) / det;
      s -= ds;
      r -= dr;
      /* quadratic convergence: once the step is below 1e-10 two more steps reach the
       * rounding floor of the coordinates (index coordinates can be ~10^3, so an absolute
       * 1e-14 is below one ulp there) */
      if (fabs(ds) < 1e-10 && fabs(dr) < 1e-10) {
        if (++ok == 3) break;
      }
    }
    if (ok < 3) return 1 + t;
    if (!per_i && (s < -1e-9 || s > ni - 1 + 1e-9)) return 1 + t;
    if (!per_j && (r < -1e-9 || r > nj - 1 + 1e-9)) return 1 + t;
    int i0 = stencil_start(s, ni, per_i), j0 = stencil_start(r, nj, per_j);
    double li[4], dli[4], lj[4], dlj[4];
    lagrange4(s - i0, li, dli);
    lagrange4(r - j0, lj, dlj);
    for (int b = 0; b < 4; ++b)
      for (int a = 0; a < 4; ++a) {
        int ii = ((i0 + a) % ni + ni) % ni, jj = ((j0 + b) % nj + nj) % nj;
        if (!iblank[(long)jj * ni + ii]) return 1 + t;
      }
    base[2 * t] = i0;
    base[2 * t + 1] = j0;
    for (int a = 0; a < 4; ++a) { w[8 * t + a] = li[a]; w[8 * t + 4 + a] = lj[a]; }
    xe[2 * t] = s;
    xe[2 * t + 1] = r;
  }
  return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Hole cutting (Sec. 2.2; reading: a background point is a hole when it lies inside the
 * closed outer-boundary polygon of the overlapping fine mesh and more than `margin` away from
 * that polygon).                                                                           */
int orc_holecut2d(long npts, const double *x, const double *y, int nb, const double *bx,
                  const double *by, double margin, signed char *iblank) {
  for (long p = 0; p < npts; ++p) {
    double X = x[p], Y = y[p];
    int inside = 0;
    double dmin = INFINITY;
    for (int e = 0; e < nb; ++e) {
      double ax = bx[e], ay = by[e];
      double cx = bx[(e + 1) % nb], cy = by[(e + 1) % nb];
      if (((ay > Y) != (cy > Y)) && (X < ax + (Y - ay) * (cx - ax) / (cy - ay))) inside = !inside;
      double ex = cx - ax, ey = cy - ay;
      double len2 = ex * ex + ey * ey;
      double tt = len2 > 0.0 ? ((X - ax) * ex + (Y - ay) * ey) / len2 : 0.0;
      if (tt < 0.0) tt = 0.0;
      if (tt > 1.0) tt = 1.0;
      double dx = X - (ax + tt * ex), dy = Y - (ay + tt * ey);
      double d = sqrt(dx * dx + dy * dy);
      if (d < dmin) dmin = d;
    }
    if (inside && dmin > margin) iblank[p] = 0;
  }
  return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Time-step estimate (Sec. 4.1; reading of the garbled eqs. (ts_inv)/(ts_visc)):
 *   dt_inv  = 1 / (sum_m |u . grad xi_m| + c sqrt(sum_m |grad xi_m|^2))
 *   dt_visc = 1 / (1/dt_inv + 2 nu* sum_m |grad xi_m|^2),  nu* = max(mu, gamma mu / Pr) / rho
 * and dt = min over active points of min(dt_inv, dt_visc) (viscous term only when mu > 0).
 * Returns the minimum (without the CFL factor).                                             */
double orc_dt2d(int ni, int nj, const signed char *ci, const double *met, const double *q, double gamma,
                double mu, double pr) {
  long N = (long)ni * nj;
  double best = INFINITY;
  for (long p = 0; p < N; ++p) {
    if (ci[p] == CL_HOLE) continue;
    double rho = q[p], u = q[N + p] / rho, v = q[2 * N + p] / rho;
    double pres = (gamma - 1.0) * (q[3 * N + p] - 0.5 * rho * (u * u + v * v));
    double c = sqrt(gamma * pres / rho);
    double J = met[4 * N + p];
    double conv = 0.0, g2 = 0.0;
    for (int m = 0; m < 2; ++m) {
      double kx = J * met[(2 * m) * N + p], ky = J * met[(2 * m + 1) * N + p];
      conv += fabs(u * kx + v * ky);
      g2 += kx * kx + ky * ky;
    }
    double inv = conv + c * sqrt(g2);
    double dt = 1.0 / inv;
    if (mu > 0.0) {
      double nu = fmax(mu, gamma * mu / pr) / rho;
      double dtv = 1.0 / (inv + 2.0 * nu * g2);
      if (dtv < dt) dt = dtv;
    }
    if (dt < best) best = dt;
  }
  return best;
}

/* ---------------------------------------------------------------------------------------- */
/* D applied along one line of n points with the classes in cls (for operator tests). */
int orc_apply_d1(int n, const signed char *cls, const double *f, double *out) {
  for (int i = 0; i < n; ++i) out[i] = (cls[i] == CL_HOLE) ? 0.0 : orc_d1(f, 1, n, i, cls[i], 0.0);
  return 0;
}
