/*
 * Plain FP64 CPU oracle for the SBP-SAT overset right-hand side, 3D Cartesian meshes.
 *
 * TEST INFRASTRUCTURE ONLY.  Compiled into the oracle's shared library next to orc2d.c; the
 * GPU library never links, includes or calls it, and shares nothing with it.
 *
 * The same definitions as orc2d.c written for three directions on uniform Cartesian meshes
 * (the paper's equations are the 3D compressible Navier-Stokes equations of App. C.1; its 3D
 * workloads are Cartesian):
 *   - SBP 4-2 first derivative D along each of i, j, k (Sec. 2.1);
 *   - dq/dt = -(D_x (F - F^V) + D_y (G - G^V) + D_z (H - H^V)) with D_x = D_xi / hx etc.;
 *   - viscous stresses with Stokes' hypothesis and Fourier heat flux (App. C.1);
 *   - SAT interface and far-field penalties of eq. (int) (Sec. 2.2, Sec. 5.1) with the
 *     characteristic matrices K^{+/-} of the 3D flux Jacobian (Sylvester's formula);
 *   - tensor-product Lagrange interpolation on 4 x 4 x 4 donor cells (Sec. 2.2);
 *   - the time-step estimate of Sec. 4.1 with three directions.
 *
 * Array layout: every field is (nvar, nk, nj, ni) with i fastest; p = (k*nj + j)*ni + i;
 * nvar = 5: q = (rho, rho u, rho v, rho w, rho E).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "orc_sbp.h"

/* Stencil classes along i, j and k from the active mask: every maximal active run along a
 * line is an SBP segment, runs shorter than 8 are made inactive (repeated), and a point
 * inactive along one direction is a hole in all three (the 2D reading, per direction). */
int orc_classes3d(int ni, int nj, int nk, int per_i, int per_j, int per_k, signed char *iblank,
                  signed char *ci, signed char *cj, signed char *ck) {
  int passes = 0;
  long nij = (long)ni * nj;
  for (;;) {
    int too_short = 0;
    for (int k = 0; k < nk; ++k)
      for (int j = 0; j < nj; ++j) {
        long o = (long)k * nij + (long)j * ni;
        classify_line(iblank + o, ni, 1, per_i, ci + o, 1, &too_short);
      }
    for (int k = 0; k < nk; ++k)
      for (int i = 0; i < ni; ++i) {
        long o = (long)k * nij + i;
        classify_line(iblank + o, nj, ni, per_j, cj + o, ni, &too_short);
      }
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        long o = (long)j * ni + i;
        classify_line(iblank + o, nk, nij, per_k, ck + o, nij, &too_short);
      }
    if (!too_short) break;
    ++passes;
    if (passes > 64) return -1;
  }
  for (long p = 0; p < nij * nk; ++p)
    if (!iblank[p]) { ci[p] = CL_HOLE; cj[p] = CL_HOLE; ck[p] = CL_HOLE; }
  return passes;
}

/* Derivative of a field along direction d at point (i, j, k), divided by the spacing. */
static double d3(const double *f, int ni, int nj, int nk, int i, int j, int k, int d, const signed char *cls,
                 double h) {
  long nij = (long)ni * nj, p = (long)k * nij + (long)j * ni + i;
  if (d == 0) return orc_d1(f + (long)k * nij + (long)j * ni, 1, ni, i, cls[p], 0.0) / h;
  if (d == 1) return orc_d1(f + (long)k * nij + i, ni, nj, j, cls[p], 0.0) / h;
  return orc_d1(f + (long)j * ni + i, nij, nk, k, cls[p], 0.0) / h;
}

/* Euler fluxes along x, y, z of App. C.1. */
static void euler_flux3(const double q[5], double gamma, double F[3][5]) {
  double rho = q[0], u[3] = {q[1] / rho, q[2] / rho, q[3] / rho}, E = q[4];
  double p = (gamma - 1.0) * (E - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  for (int d = 0; d < 3; ++d) {
    F[d][0] = rho * u[d];
    for (int c = 0; c < 3; ++c) F[d][1 + c] = rho * u[d] * u[c] + (c == d ? p : 0.0);
    F[d][4] = (E + p) * u[d];
  }
}

/* Viscous fluxes at every active point: fv = 12 planes, F^V_x (momentum x, y, z, energy),
 * then F^V_y, then F^V_z (the mass components are zero).  tau_ij = mu (du_i/dx_j +
 * du_j/dx_i) - 2/3 mu div(u) delta_ij, heat flux -mu/(Pr (gamma-1)) grad T, T = gamma p / rho. */
int orc_viscflux3d(int ni, int nj, int nk, const signed char *ci, const signed char *cj, const signed char *ck,
                   double hx, double hy, double hz, const double *q, double gamma, double mu, double pr,
                   double *fv) {
  long N = (long)ni * nj * nk;
  double *prim = (double *)malloc(sizeof(double) * 4 * N); /* u, v, w, T */
  if (!prim) return -1;
  for (long p = 0; p < N; ++p) {
    double rho = q[p], u = q[N + p] / rho, v = q[2 * N + p] / rho, w = q[3 * N + p] / rho;
    double pres = (gamma - 1.0) * (q[4 * N + p] - 0.5 * rho * (u * u + v * v + w * w));
    prim[p] = u; prim[N + p] = v; prim[2 * N + p] = w; prim[3 * N + p] = gamma * pres / rho;
  }
  const signed char *cl[3] = {ci, cj, ck};
  double h[3] = {hx, hy, hz};
  double lam = -2.0 / 3.0 * mu, kap = mu / (pr * (gamma - 1.0));
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        long p = ((long)k * nj + j) * ni + i;
        if (ci[p] == CL_HOLE) { for (int c = 0; c < 12; ++c) fv[c * N + p] = 0.0; continue; }
        double g[4][3]; /* g[f][d] = d prim_f / d x_d */
        for (int f = 0; f < 4; ++f)
          for (int d = 0; d < 3; ++d) g[f][d] = d3(prim + f * N, ni, nj, nk, i, j, k, d, cl[d], h[d]);
        double div = g[0][0] + g[1][1] + g[2][2];
        double tau[3][3];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) tau[a][b] = mu * (g[a][b] + g[b][a]) + (a == b ? lam * div : 0.0);
        double vel[3] = {prim[p], prim[N + p], prim[2 * N + p]};
        for (int d = 0; d < 3; ++d) {
          for (int c = 0; c < 3; ++c) fv[(4 * d + c) * N + p] = tau[d][c];
          double work = vel[0] * tau[d][0] + vel[1] * tau[d][1] + vel[2] * tau[d][2];
          fv[(4 * d + 3) * N + p] = work + kap * g[3][d];
        }
      }
  free(prim);
  return 0;
}

/* Flux Jacobian of k . (F, G, H) with respect to q (5 x 5). */
static void flux_jacobian3(const double q[5], double gamma, const double kv[3], double A[5][5]) {
  double rho = q[0], u[3] = {q[1] / rho, q[2] / rho, q[3] / rho}, E = q[4];
  double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double p = (gamma - 1.0) * (E - 0.5 * rho * q2);
  double U = kv[0] * u[0] + kv[1] * u[1] + kv[2] * u[2];
  double phi2 = 0.5 * (gamma - 1.0) * q2, H = (E + p) / rho, g1 = gamma - 1.0;
  A[0][0] = 0.0;
  for (int c = 0; c < 3; ++c) A[0][1 + c] = kv[c];
  A[0][4] = 0.0;
  for (int a = 0; a < 3; ++a) {
    A[1 + a][0] = kv[a] * phi2 - u[a] * U;
    for (int b = 0; b < 3; ++b)
      A[1 + a][1 + b] = kv[b] * u[a] - g1 * kv[a] * u[b] + (a == b ? U : 0.0);
    A[1 + a][4] = g1 * kv[a];
  }
  A[4][0] = U * (phi2 - H);
  for (int b = 0; b < 3; ++b) A[4][1 + b] = kv[b] * H - g1 * u[b] * U;
  A[4][4] = gamma * U;
}

/* K^{+/-}_k = T ((|Lambda| +/- Lambda)/2) T^-1 by Sylvester's formula over the three distinct
 * eigenvalues U, U + c|k|, U - c|k| of the (diagonalisable) flux Jacobian. */
void orc_penalty_matrix3d(const double q[5], double gamma, double kx, double ky, double kz, int side,
                          double K[5][5]) {
  double kv[3] = {kx, ky, kz};
  double A[5][5];
  flux_jacobian3(q, gamma, kv, A);
  double rho = q[0], u = q[1] / rho, v = q[2] / rho, w = q[3] / rho;
  double p = (gamma - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w));
  double c = sqrt(gamma * p / rho), kn = sqrt(kx * kx + ky * ky + kz * kz);
  double U = kx * u + ky * v + kz * w;
  double lam[3] = {U, U + c * kn, U - c * kn};
  memset(K, 0, sizeof(double) * 25);
  for (int a = 0; a < 3; ++a) {
    double fl = 0.5 * (fabs(lam[a]) + side * lam[a]);
    if (fl == 0.0) continue;
    double P[5][5], T[5][5];
    for (int r = 0; r < 5; ++r)
      for (int s = 0; s < 5; ++s) P[r][s] = (r == s) ? 1.0 : 0.0;
    for (int b = 0; b < 3; ++b) {
      if (b == a) continue;
      double den = lam[a] - lam[b];
      for (int r = 0; r < 5; ++r)
        for (int s = 0; s < 5; ++s) {
          double acc = 0.0;
          for (int t = 0; t < 5; ++t) acc += P[r][t] * (A[t][s] - (t == s ? lam[b] : 0.0));
          T[r][s] = acc / den;
        }
      memcpy(P, T, sizeof(P));
    }
    for (int r = 0; r < 5; ++r)
      for (int s = 0; s < 5; ++s) K[r][s] += fl * P[r][s];
  }
}

/* Right-hand side on one 3D Cartesian mesh with explicit SAT term lists:
 *   kind 1 (interface): -p0^-1 [(sigI K^side_k + sigma1 I)(q - qhat) - side/2 (F^V_k - F^V_k hat)]
 *                       * scale
 *   kind 2 (far field): -p0^-1 sigP K^side_k (q - qinf)
 * k = e_d / h_d for the normal direction d, sigma1 = mu |k|^2 / 2, side = +1 on the low-index
 * face, -1 on the high-index face.  qhat: 5 x nrecv; fvhat: 12 x nrecv (NULL for Euler). */
int orc_rhs3d(int ni, int nj, int nk, const signed char *ci, const signed char *cj, const signed char *ck,
              double hx, double hy, double hz, const double *q, int viscous, double gamma, double mu,
              double pr, int nterm, const long *t_pt, const int *t_dir, const int *t_side, const int *t_kind,
              const int *t_recv, const double *t_scale, int nrecv, const double *qhat, const double *fvhat,
              const double *qinf, double sig_int, double sig_phys, double *rhs) {
  long N = (long)ni * nj * nk;
  double *fl = (double *)malloc(sizeof(double) * 15 * N); /* (F - F^V), (G - G^V), (H - H^V) */
  double *fv = viscous ? (double *)malloc(sizeof(double) * 12 * N) : NULL;
  if (!fl || (viscous && !fv)) { free(fl); free(fv); return -1; }
  if (viscous) orc_viscflux3d(ni, nj, nk, ci, cj, ck, hx, hy, hz, q, gamma, mu, pr, fv);
  for (long p = 0; p < N; ++p) {
    double qp[5] = {q[p], q[N + p], q[2 * N + p], q[3 * N + p], q[4 * N + p]};
    double F[3][5];
    euler_flux3(qp, gamma, F);
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < 5; ++v) {
        double vis = (viscous && v > 0) ? fv[(4 * d + v - 1) * N + p] : 0.0;
        fl[(5 * d + v) * N + p] = F[d][v] - vis;
      }
  }
  const signed char *cl[3] = {ci, cj, ck};
  double h[3] = {hx, hy, hz};
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        long p = ((long)k * nj + j) * ni + i;
        for (int v = 0; v < 5; ++v) {
          if (ci[p] == CL_HOLE) { rhs[v * N + p] = 0.0; continue; }
          double s = 0.0;
          for (int d = 0; d < 3; ++d) s += d3(fl + (5 * d + v) * N, ni, nj, nk, i, j, k, d, cl[d], h[d]);
          rhs[v * N + p] = -s;
        }
      }
  for (int t = 0; t < nterm; ++t) {
    long p = t_pt[t];
    int d = t_dir[t], side = t_side[t], kind = t_kind[t];
    double kv[3] = {0.0, 0.0, 0.0};
    kv[d] = 1.0 / h[d];
    double qp[5] = {q[p], q[N + p], q[2 * N + p], q[3 * N + p], q[4 * N + p]};
    double tgt[5];
    double sigI = (kind == 1) ? sig_int : sig_phys, sig1 = 0.0;
    int r = t_recv[t];
    if (kind == 1) {
      if (r < 0 || r >= nrecv) { free(fl); free(fv); return -2; }
      for (int v = 0; v < 5; ++v) tgt[v] = qhat[(long)v * nrecv + r];
      if (viscous) sig1 = 0.5 * mu * kv[d] * kv[d];
    } else {
      for (int v = 0; v < 5; ++v) tgt[v] = qinf[v];
    }
    double K[5][5];
    orc_penalty_matrix3d(qp, gamma, kv[0], kv[1], kv[2], side, K);
    double dq[5], sat[5];
    for (int v = 0; v < 5; ++v) dq[v] = qp[v] - tgt[v];
    for (int v = 0; v < 5; ++v) {
      double acc = 0.0;
      for (int w = 0; w < 5; ++w) acc += K[v][w] * dq[w];
      sat[v] = -(sigI * acc + sig1 * dq[v]) / ORC_P0;
    }
    if (kind == 1 && viscous) {
      /* F^V_k = k_d F^V_d (only the normal direction's flux) */
      for (int c = 0; c < 4; ++c) {
        double own = kv[d] * fv[(4 * d + c) * N + p];
        double hat = kv[d] * fvhat[(long)(4 * d + c) * nrecv + r];
        sat[1 + c] += 0.5 * side * (own - hat) / ORC_P0;
      }
    }
    for (int v = 0; v < 5; ++v) rhs[v * N + p] += t_scale[t] * sat[v];
  }
  free(fl);
  free(fv);
  return 0;
}

/* out[f][r] = sum over the 4 x 4 x 4 donor cell of wi wj wk field[f] (indices wrapped on every
 * direction; non-periodic donors never reach past an edge).  base: 3 per receiver, w: 12 per
 * receiver (4 along i, 4 along j, 4 along k). */
int orc_interp3d(int ni, int nj, int nk, int nf, const double *field, int nrecv, const int *base, const double *w,
                 double *out) {
  long N = (long)ni * nj * nk;
  for (int r = 0; r < nrecv; ++r)
    for (int f = 0; f < nf; ++f) {
      double acc = 0.0;
      for (int c = 0; c < 4; ++c)
        for (int b = 0; b < 4; ++b)
          for (int a = 0; a < 4; ++a) {
            int ii = ((base[3 * r] + a) % ni + ni) % ni;
            int jj = ((base[3 * r + 1] + b) % nj + nj) % nj;
            int kk = ((base[3 * r + 2] + c) % nk + nk) % nk;
            acc += w[12 * r + a] * w[12 * r + 4 + b] * w[12 * r + 8 + c] * field[f * N + ((long)kk * nj + jj) * ni + ii];
          }
      out[(long)f * nrecv + r] = acc;
    }
  return 0;
}

/* Stable step of Sec. 4.1 on a Cartesian mesh: min over active points of
 * dt_visc = 1 / (1/dt_inv + 2 nu* sum_d 1/h_d^2), dt_inv = 1 / (sum_d |u_d|/h_d + c sqrt(sum_d 1/h_d^2)),
 * nu* = max(mu, gamma mu / Pr) / rho. */
double orc_dt3d(int ni, int nj, int nk, const signed char *ci, double hx, double hy, double hz, const double *q,
                double gamma, double mu, double pr) {
  long N = (long)ni * nj * nk;
  double ih[3] = {1.0 / hx, 1.0 / hy, 1.0 / hz};
  double s2 = ih[0] * ih[0] + ih[1] * ih[1] + ih[2] * ih[2];
  double best = INFINITY;
  for (long p = 0; p < N; ++p) {
    if (ci[p] == CL_HOLE) continue;
    double rho = q[p], u[3] = {q[N + p] / rho, q[2 * N + p] / rho, q[3 * N + p] / rho};
    double pres = (gamma - 1.0) * (q[4 * N + p] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
    double c = sqrt(gamma * pres / rho);
    double inv = fabs(u[0]) * ih[0] + fabs(u[1]) * ih[1] + fabs(u[2]) * ih[2] + c * sqrt(s2);
    double nu = fmax(mu, gamma * mu / pr) / rho;
    double dt = 1.0 / (inv + 2.0 * nu * s2);
    if (dt < best) best = dt;
  }
  return best;
}
