// 3D curvilinear operator (App. C.1's equations in curvilinear coordinates with Sec. 2.1's SBP
// 4-2 derivative): one structured mesh with closures at both ends of every line, or, with a
// class map (overset pairs with a hole cut), at both ends of every active segment; far-field
// and interface SAT terms and the overset gather as separate kernels; for overset pairs also
// the donor values, the Adams-Bashforth combine and the time step.
//   k3c_dx       coordinate derivatives D_a X_c (9 planes, FP64)
//   k3c_metrics  metric terms M[m][j] = xi_m,x_j / J in the symmetric conservative form of
//                Thomas and Lombard, M[m][j] = D_b((X_c)_a X_e) - D_a((X_c)_b X_e) over cyclic
//                (m, a, b) and (j, c, e), and J = 1 / det(D_a X_c) (FP64 arithmetic, stored in
//                the element type); D along different index directions commute, so
//                sum_m D_m M[m][j] = 0 and a uniform state has zero divergence to rounding
//   k3c_prim     primitives (u, v, w, T) (Navier-Stokes)
//   k3c_flux     contravariant fluxes F^_m = sum_j M[m][j] (F_j - F^V_j), viscous gradients by
//                the chain rule d/dx_j = J sum_m M[m][j] D_m
//   k3c_update   dq/dt = -J sum_m D_m F^_m
//   k3c_isat     interface SAT at receiver points with given donor values (added to a rhs)
//   k3c_interp   overset gather of the 5 variables at receivers with given donor stencils
//   k3c_far      (optional) the far-field SAT of Sec. 5.1 on every face: at a point on the low
//                (side +1) or high (side -1) face of index direction m, -(sigma / p0)
//                K^side_k (q - qinf) with k = grad xi_m = J M[m][:], one term for each face the
//                point lies on
//   k3c_donor    donor-point states (slow extrapolation of Sec. 3.3) and viscous fluxes
//   k3c_ab       qn = q + sum alpha_h hist_h (Sec. 3.1-3.3), non-finite states flagged
//   k3c_dt       time step, min-reduced
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <type_traits>

#include "sbp3_penalty.cuh"
#include "sbp3c_device.h"
#include "sbp_dev.cuh"

namespace sbp {

// Stencil class of index c on a non-periodic line of n points: closure rows at both ends.
__device__ __forceinline__ unsigned line_code(int c, int n) {
  if (c < 4) return (unsigned)((kLeft << 2) | c);
  if (c >= n - 4) return (unsigned)((kRight << 2) | (n - 1 - c));
  return 0u;
}

// The derivative row of stencil class `code` applied at linear index p of a line with stride st.
template <typename T, typename F>
__device__ __forceinline__ T dtap(const F &f, ptrdiff_t p, ptrdiff_t st, unsigned code) {
  const Row<T> r = decode_row<T>(code);
  T acc = T(0);
#pragma unroll
  for (int e = 0; e < 4; ++e) acc += r.w[e] * f(p + (ptrdiff_t)r.off[e] * st);
  return r.neg ? -acc : acc;
}

// D_d f at point (i, j, k) of an unpitched plane f (unit index spacing), whole lines.
template <typename T, typename F>
__device__ __forceinline__ T cderiv(const F &f, int i, int j, int k, int d, int ni, int nj, int nk) {
  const int c[3] = {i, j, k}, n[3] = {ni, nj, nk};
  const ptrdiff_t st[3] = {1, (ptrdiff_t)ni, (ptrdiff_t)ni * nj};
  return dtap<T>(f, ((ptrdiff_t)k * nj + j) * ni + i, st[d], line_code(c[d], n[d]));
}

// Stencil class of point p = (i, j, k) along direction d: from the class map (SEG: the kernels'
// overset-pair instances, a.cls set), else whole lines. A compile-time choice, so that the
// whole-line kernels carry no class-map registers.
template <bool SEG>
__device__ __forceinline__ unsigned pcode(const Curv3Launch &a, size_t p, int i, int j, int k, int d) {
  if (SEG) return (a.cls[p] >> (4 * d)) & 15u;
  return line_code(d == 0 ? i : (d == 1 ? j : k), d == 0 ? a.ni : (d == 1 ? a.nj : a.nk));
}

template <bool SEG>
__device__ __forceinline__ bool is_hole(const Curv3Launch &a, size_t p) { return SEG && (a.cls[p] & 15u) == 15u; }

// D_d f at point (i, j, k) of the mesh of a (per segment with a class map).
template <typename T, bool SEG, typename F>
__device__ __forceinline__ T mderiv(const Curv3Launch &a, const F &f, size_t p, int i, int j, int k, int d) {
  if (!SEG) return cderiv<T>(f, i, j, k, d, a.ni, a.nj, a.nk);
  const ptrdiff_t st = d == 0 ? 1 : (d == 1 ? (ptrdiff_t)a.ni : (ptrdiff_t)a.ni * a.nj);
  return dtap<T>(f, (ptrdiff_t)p, st, pcode<SEG>(a, p, i, j, k, d));
}

__global__ void __launch_bounds__(256) k3c_dx(int ni, int nj, int nk, const double *xyz, double *dx) {
  const size_t N = (size_t)ni * nj * nk;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const int i = (int)(t % ni), j = (int)((t / ni) % nj), k = (int)(t / ((size_t)ni * nj));
  for (int c = 0; c < 3; ++c) {
    const double *X = xyz + c * N;
    for (int a = 0; a < 3; ++a)
      dx[(3 * c + a) * N + t] = cderiv<double>([&](ptrdiff_t q) { return X[q]; }, i, j, k, a, ni, nj, nk);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k3c_metrics(int ni, int nj, int nk, const double *xyz, const double *dx,
                                                   T *met) {
  const size_t N = (size_t)ni * nj * nk;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const int i = (int)(t % ni), j = (int)((t / ni) % nj), k = (int)(t / ((size_t)ni * nj));
  const int cyc[3][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}};
  for (int mm = 0; mm < 3; ++mm) {
    const int m = cyc[mm][0], a = cyc[mm][1], b = cyc[mm][2];
    for (int jj = 0; jj < 3; ++jj) {
      const int jc = cyc[jj][0], c = cyc[jj][1], e = cyc[jj][2];
      const double *Xe = xyz + e * N, *Dca = dx + (3 * c + a) * N, *Dcb = dx + (3 * c + b) * N;
      const double s1 = cderiv<double>([&](ptrdiff_t q) { return Dca[q] * Xe[q]; }, i, j, k, b, ni, nj, nk);
      const double s2 = cderiv<double>([&](ptrdiff_t q) { return Dcb[q] * Xe[q]; }, i, j, k, a, ni, nj, nk);
      met[(3 * m + jc) * N + t] = (T)(s1 - s2);
    }
  }
  double D[3][3];
  for (int c = 0; c < 3; ++c)
    for (int a = 0; a < 3; ++a) D[c][a] = dx[(3 * c + a) * N + t];
  const double jinv = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) -
                      D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                      D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
  met[9 * N + t] = (T)(1.0 / jinv);
}

template <typename T, bool SEG>
__global__ void __launch_bounds__(256) k3c_prim(const Curv3Launch a) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= a.field || is_hole<SEG>(a, t)) return;
  const T *q = static_cast<const T *>(a.q);
  T *pr = static_cast<T *>(a.prim);
  const T rho = q[t], u = q[a.field + t] / rho, v = q[2 * a.field + t] / rho, w = q[3 * a.field + t] / rho;
  const T gam = (T)a.gam;
  const T p = (gam - T(1)) * (q[4 * a.field + t] - T(0.5) * rho * (u * u + v * v + w * w));
  pr[t] = u;
  pr[a.field + t] = v;
  pr[2 * a.field + t] = w;
  pr[3 * a.field + t] = gam * p / rho;
}

template <typename T, bool SEG>
__global__ void __launch_bounds__(256) k3c_flux(const Curv3Launch a) {
  const size_t N = a.field;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const int i = (int)(t % a.ni), j = (int)((t / a.ni) % a.nj), k = (int)(t / ((size_t)a.ni * a.nj));
  T *fl = static_cast<T *>(a.flux);
  if (is_hole<SEG>(a, t)) {
    for (int c = 0; c < 15; ++c) fl[c * N + t] = T(0);
    return;
  }
  const T *q = static_cast<const T *>(a.q);
  const T *met = static_cast<const T *>(a.met);
  T M[3][3];
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int c = 0; c < 3; ++c) M[m][c] = met[(3 * m + c) * N + t];
  const T Jac = met[9 * N + t];
  const T rho = q[t], vel[3] = {q[N + t] / rho, q[2 * N + t] / rho, q[3 * N + t] / rho}, E = q[4 * N + t];
  const T gam = (T)a.gam;
  const T p = (gam - T(1)) * (E - T(0.5) * rho * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]));
  T F[3][5];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F[d][0] = rho * vel[d];
#pragma unroll
    for (int c = 0; c < 3; ++c) F[d][1 + c] = rho * vel[d] * vel[c] + (c == d ? p : T(0));
    F[d][4] = (E + p) * vel[d];
  }
  if (a.visc) {
    const T *pr = static_cast<const T *>(a.prim);
    T g[4][3];  // g[f][d] = d prim_f / d x_d
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const T *pf = pr + f * N;
      T Df[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) Df[m] = mderiv<T, SEG>(a, [&](ptrdiff_t s) { return pf[s]; }, t, i, j, k, m);
#pragma unroll
      for (int d = 0; d < 3; ++d) g[f][d] = Jac * (M[0][d] * Df[0] + M[1][d] * Df[1] + M[2][d] * Df[2]);
    }
    const T mu = (T)a.mu, lam = (T)a.lam, kap = (T)a.kap;
    const T div = g[0][0] + g[1][1] + g[2][2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T tau[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) tau[c] = mu * (g[d][c] + g[c][d]) + (c == d ? lam * div : T(0));
#pragma unroll
      for (int c = 0; c < 3; ++c) F[d][1 + c] -= tau[c];
      F[d][4] -= vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2] + kap * g[3][d];
    }
  }
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int v = 0; v < 5; ++v) fl[(5 * m + v) * N + t] = M[m][0] * F[0][v] + M[m][1] * F[1][v] + M[m][2] * F[2][v];
}

template <typename T, bool SEG>
__global__ void __launch_bounds__(256) k3c_update(const Curv3Launch a) {
  const size_t N = a.field;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const int i = (int)(t % a.ni), j = (int)((t / a.ni) % a.nj), k = (int)(t / ((size_t)a.ni * a.nj));
  T *out = static_cast<T *>(a.out);
  if (is_hole<SEG>(a, t)) {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v * N + t] = T(0);
    return;
  }
  const T *fl = static_cast<const T *>(a.flux);
  const T Jac = static_cast<const T *>(a.met)[9 * N + t];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    T s = T(0);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const T *f = fl + (5 * m + v) * N;
      s += mderiv<T, SEG>(a, [&](ptrdiff_t q) { return f[q]; }, t, i, j, k, m);
    }
    out[v * N + t] = -Jac * s;
  }
}

// Number of distinct face points of the mesh, enumerated by k3c_far as: both i faces (all j, k),
// then both j faces (interior i, all k), then both k faces (interior i and j).
static size_t face_points(int ni, int nj, int nk) {
  return 2 * ((size_t)nj * nk + (size_t)(ni - 2) * nk + (size_t)(ni - 2) * (nj - 2));
}

// Far-field SAT added to the right-hand side at each face point (one thread per point, all the
// faces it lies on, in index-direction order), after k3c_update on the same stream. Kept apart
// from k3c_update so that the penalty's registers do not cut the occupancy of every point.
template <typename T, bool SEG>
__global__ void __launch_bounds__(128) k3c_far(const Curv3Launch a, size_t nface) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nface) return;
  const int ni = a.ni, nj = a.nj, nk = a.nk;
  const size_t fi = (size_t)nj * nk, fj = (size_t)(ni - 2) * nk, fk = (size_t)(ni - 2) * (nj - 2);
  int i, j, k;
  if (t < 2 * fi) {
    const size_t r = t % fi;
    i = t < fi ? 0 : ni - 1;
    j = (int)(r % nj);
    k = (int)(r / nj);
  } else if (t < 2 * (fi + fj)) {
    const size_t u = t - 2 * fi, r = u % fj;
    j = u < fj ? 0 : nj - 1;
    i = 1 + (int)(r % (ni - 2));
    k = (int)(r / (ni - 2));
  } else {
    const size_t u = t - 2 * (fi + fj), r = u % fk;
    k = u < fk ? 0 : nk - 1;
    i = 1 + (int)(r % (ni - 2));
    j = 1 + (int)(r / (ni - 2));
  }
  const size_t N = a.field, p = ((size_t)k * nj + j) * ni + i;
  if (is_hole<SEG>(a, p)) return;
  const T *q = static_cast<const T *>(a.q);
  const T *met = static_cast<const T *>(a.met);
  T *out = static_cast<T *>(a.out);
  const T Jac = met[9 * N + p];
  T qp[5], dq[5], r[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qp[v] = q[v * N + p];
    dq[v] = qp[v] - (T)a.qinf[v];
    r[v] = out[v * N + p];
  }
  const T sp = (T)a.sig * T(1.0 / SBP_P0);
  const int c[3] = {i, j, k}, n[3] = {ni, nj, nk};
  for (int m = 0; m < 3; ++m) {
    const int side = c[m] == 0 ? 1 : (c[m] == n[m] - 1 ? -1 : 0);
    if (!side) continue;
    const T kv[3] = {Jac * met[(3 * m) * N + p], Jac * met[(3 * m + 1) * N + p], Jac * met[(3 * m + 2) * N + p]};
    T kd[5];
    penalty3(qp, (T)a.gam, kv, side, dq, kd);
#pragma unroll
    for (int v = 0; v < 5; ++v) r[v] -= sp * kd[v];
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) out[v * N + p] = r[v];
}

// Overset gather (Sec. 2.2 interpolation): out[v][r] = sum over the 4 x 4 x 4 stencil at base[r]
// of wi wj wk q[v], weights (FP64) taken in the element type, one thread per receiver.
template <typename T>
__global__ void __launch_bounds__(128) k3c_interp(int ni, int nj, int nk, const T *q, int nrecv,
                                                  const int *base, const double *w, T *out, int *err) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrecv) return;
  const size_t field = (size_t)ni * nj * nk;
  const int i0 = base[3 * r], j0 = base[3 * r + 1], k0 = base[3 * r + 2];
  if (i0 < 0 || j0 < 0 || k0 < 0 || i0 > ni - 4 || j0 > nj - 4 || k0 > nk - 4) {
    // a stencil outside the mesh (the caller's bases): record it, give zeros, read nothing
    if (err) atomicCAS(err, 0, (int)SBP_ERR_BOUNDS);
#pragma unroll
    for (int v = 0; v < 5; ++v) out[(size_t)v * nrecv + r] = T(0);
    return;
  }
  T wi[4], wj[4], wk[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    wi[a] = (T)w[12 * (size_t)r + a];
    wj[a] = (T)w[12 * (size_t)r + 4 + a];
    wk[a] = (T)w[12 * (size_t)r + 8 + a];
  }
  T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
  for (int c = 0; c < 4; ++c)
    for (int b = 0; b < 4; ++b) {
      const size_t p = ((size_t)(k0 + c) * nj + (j0 + b)) * ni + i0;
      const T wjk = wj[b] * wk[c];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const T wt = wi[a] * wjk;
#pragma unroll
        for (int v = 0; v < 5; ++v) acc[v] += wt * q[v * field + p + a];
      }
    }
#pragma unroll
  for (int v = 0; v < 5; ++v) out[(size_t)v * nrecv + r] = acc[v];
}

// Interface SAT (Sec. 2.2 eq. (int)) at receiver points, one thread per distinct point adding its
// terms in order: for term (m, side, r, scale), k = J M[m][:],
//   rhs += scale * (-(1/p0) [(sigma K^side_k + sigma1 I)(q - qhat_r) - side/2 (F^V_k - F^V_k hat_r)])
// with sigma1 = mu |k|^2 / 2 and F^V_k = sum_d k_d F^V_d (Navier-Stokes), the receiver's own
// viscous fluxes from chain-rule gradients of primitives taken from q at the stencil taps.
template <typename T, bool SEG>
__global__ void __launch_bounds__(64) k3c_isat(const Curv3Launch a, Curv3Sat s) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s.npt) return;
  const size_t N = a.field;
  const long long pl = s.pt[t];
  const int i = (int)(pl % a.ni), j = (int)((pl / a.ni) % a.nj), k = (int)(pl / ((long long)a.ni * a.nj));
  const size_t p = (size_t)pl;
  const T *q = static_cast<const T *>(a.q);
  const T *met = static_cast<const T *>(a.met);
  const T gam = (T)a.gam;
  const T Jac = met[9 * N + p];
  T qp[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qp[v] = q[v * N + p];
  T Fv[3][4] = {};
  if (a.visc) {
    T M[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int c = 0; c < 3; ++c) M[m][c] = met[(3 * m + c) * N + p];
    // derivatives of the primitives (u, v, w, T) along each index direction: each stencil tap's
    // primitives formed once for all four (the operations of k3c_prim)
    T Df[4][3];
    const ptrdiff_t st[3] = {1, (ptrdiff_t)a.ni, (ptrdiff_t)a.ni * a.nj};
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const Row<T> r = decode_row<T>(SEG ? pcode<SEG>(a, p, i, j, k, m)
                                         : line_code(m == 0 ? i : (m == 1 ? j : k), m == 0 ? a.ni : (m == 1 ? a.nj : a.nk)));
      T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const ptrdiff_t x = (ptrdiff_t)p + (ptrdiff_t)r.off[e] * st[m];
        const T rho = q[x], u = q[N + x] / rho, v = q[2 * N + x] / rho, w = q[3 * N + x] / rho;
        const T pr = (gam - T(1)) * (q[4 * N + x] - T(0.5) * rho * (u * u + v * v + w * w));
        const T pv[4] = {u, v, w, gam * pr / rho};
#pragma unroll
        for (int f = 0; f < 4; ++f) acc[f] += r.w[e] * pv[f];
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) Df[f][m] = r.neg ? -acc[f] : acc[f];
    }
    T g[4][3];
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int d = 0; d < 3; ++d) g[f][d] = Jac * (M[0][d] * Df[f][0] + M[1][d] * Df[f][1] + M[2][d] * Df[f][2]);
    const T mu = (T)a.mu, lam = (T)a.lam, kap = (T)a.kap;
    const T div = g[0][0] + g[1][1] + g[2][2];
    const T vel[3] = {qp[1] / qp[0], qp[2] / qp[0], qp[3] / qp[0]};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int c = 0; c < 3; ++c) Fv[d][c] = mu * (g[d][c] + g[c][d]) + (c == d ? lam * div : T(0));
      Fv[d][3] = vel[0] * Fv[d][0] + vel[1] * Fv[d][1] + vel[2] * Fv[d][2] + kap * g[3][d];
    }
  }
  const T *qh = static_cast<const T *>(s.qhat);
  const T *fh = static_cast<const T *>(s.fvhat);
  T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
  for (int e = s.off[t]; e < s.off[t + 1]; ++e) {
    const int m = s.term[3 * e], side = s.term[3 * e + 1], r = s.term[3 * e + 2];
    const T kv[3] = {Jac * met[(3 * m) * N + p], Jac * met[(3 * m + 1) * N + p], Jac * met[(3 * m + 2) * N + p]};
    T dq[5], kd[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) dq[v] = qp[v] - qh[(size_t)v * s.nrecv + r];
    penalty3(qp, gam, kv, side, dq, kd);
    const T sig1 = a.visc ? T(0.5) * (T)a.mu * (kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]) : T(0);
    T sat[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) sat[v] = -((T)s.sig * kd[v] + sig1 * dq[v]) * T(1.0 / SBP_P0);
    if (a.visc) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const T own = kv[0] * Fv[0][c] + kv[1] * Fv[1][c] + kv[2] * Fv[2][c];
        const T hat = kv[0] * fh[(size_t)c * s.nrecv + r] + kv[1] * fh[(size_t)(4 + c) * s.nrecv + r] +
                      kv[2] * fh[(size_t)(8 + c) * s.nrecv + r];
        sat[1 + c] += T(0.5) * T(side) * (own - hat) * T(1.0 / SBP_P0);
      }
    }
    const T sc = (T)s.scale[e];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += sc * sat[v];
  }
  T *out = static_cast<T *>(a.out);
#pragma unroll
  for (int v = 0; v < 5; ++v) out[v * N + p] += acc[v];
}

cudaError_t launch3c_isat(const Curv3Launch &a, const Curv3Sat &s, int dtype, cudaStream_t st) {
  if (s.npt <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((s.npt + 63) / 64);
  if (a.cls) {
    if (dtype == SBP_F64) k3c_isat<double, true><<<blocks, 64, 0, st>>>(a, s);
    else k3c_isat<float, true><<<blocks, 64, 0, st>>>(a, s);
  } else {
    if (dtype == SBP_F64) k3c_isat<double, false><<<blocks, 64, 0, st>>>(a, s);
    else k3c_isat<float, false><<<blocks, 64, 0, st>>>(a, s);
  }
  return cudaGetLastError();
}

cudaError_t launch3c_interp(int ni, int nj, int nk, const void *q, int nrecv, const int *base, const double *w,
                            void *out, int *err, int dtype, cudaStream_t s) {
  if (nrecv <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((nrecv + 127) / 128);
  if (dtype == SBP_F64)
    k3c_interp<double><<<blocks, 128, 0, s>>>(ni, nj, nk, (const double *)q, nrecv, base, w, (double *)out, err);
  else
    k3c_interp<float><<<blocks, 128, 0, s>>>(ni, nj, nk, (const float *)q, nrecv, base, w, (float *)out, err);
  return cudaGetLastError();
}

cudaError_t launch3c_metrics(int ni, int nj, int nk, const double *xyz, double *dx, void *met, int dtype,
                             cudaStream_t s) {
  const size_t N = (size_t)ni * nj * nk;
  const int blocks = (int)((N + 255) / 256);
  k3c_dx<<<blocks, 256, 0, s>>>(ni, nj, nk, xyz, dx);
  if (dtype == SBP_F64) k3c_metrics<double><<<blocks, 256, 0, s>>>(ni, nj, nk, xyz, dx, (double *)met);
  else k3c_metrics<float><<<blocks, 256, 0, s>>>(ni, nj, nk, xyz, dx, (float *)met);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Overset pairs of curvilinear meshes: donor values, the Adams-Bashforth combine, the time step.

template <typename T>
__device__ __forceinline__ void donor_state(const Curv3Donor &a, int set, size_t p, T out[5]) {
  const T *q = static_cast<const T *>(a.m.q);
  const size_t N = a.m.field;
  double acc[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) acc[v] = to_f64(q[v * N + p]);
  // each history slot's five values loaded together (the same sums in the same order)
#pragma unroll
  for (int k = 0; k < kMaxHist; ++k) {
    if (k < a.nb[set]) {
      const T *h = static_cast<const T *>(a.hist[k]) + p;
      T hv[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) hv[v] = h[v * N];
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] += a.beta[set][k] * to_f64(hv[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) out[v] = (T)acc[v];
}

// (u, v, w, T = gamma p / rho) of a conserved state.
template <typename T>
__device__ __forceinline__ void prim_of(const T s[5], T gam, T out[4]) {
  const T rho = s[0], u = s[1] / rho, v = s[2] / rho, w = s[3] / rho;
  const T pr = (gam - T(1)) * (s[4] - T(0.5) * rho * (u * u + v * v + w * w));
  out[0] = u;
  out[1] = v;
  out[2] = w;
  out[3] = gam * pr / rho;
}

template <typename T>
__global__ void __launch_bounds__(128) k3c_donor(const Curv3Donor a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nsets * a.npts) return;
  const int set = t / a.npts, dp = t - set * a.npts;
  const Curv3Launch &m = a.m;
  const size_t N = m.field;
  const long long pl = a.pts[dp];
  const int i = (int)(pl % m.ni), j = (int)((pl / m.ni) % m.nj), k = (int)(pl / ((long long)m.ni * m.nj));
  const size_t p = (size_t)pl;
  T s[5];
  donor_state(a, set, p, s);
  T *dv = static_cast<T *>(a.dv) + ((size_t)set * a.npts + dp) * kDvPitch;
#pragma unroll
  for (int v = 0; v < 5; ++v) dv[v] = s[v];
  if (!m.visc) return;
  const T gam = (T)m.gam;
  const T *met = static_cast<const T *>(m.met);
  // derivatives along each index direction of the primitives of the (extrapolated) state
  T Df[3][4];
  const ptrdiff_t st[3] = {1, (ptrdiff_t)m.ni, (ptrdiff_t)m.ni * m.nj};
  const T *tvs = a.tpts ? static_cast<const T *>(a.tv) + (size_t)set * a.ntap * 4 : nullptr;
  for (int d = 0; d < 3; ++d) {
    const Row<T> r = decode_row<T>(pcode<true>(m, p, i, j, k, d));
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int e = 0; e < 4; ++e) {
      T pn[4];
      if (tvs) {
        const T *tp = tvs + (size_t)a.tidx[(size_t)dp * 13 + 1 + 4 * d + e] * 4;
#pragma unroll
        for (int f = 0; f < 4; ++f) pn[f] = tp[f];
      } else {
        T sn[5];
        donor_state(a, set, (size_t)((ptrdiff_t)p + (ptrdiff_t)r.off[e] * st[d]), sn);
        prim_of(sn, gam, pn);
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) acc[f] += r.w[e] * pn[f];
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) Df[d][f] = r.neg ? -acc[f] : acc[f];
  }
  T M[3][3];
#pragma unroll
  for (int mm = 0; mm < 3; ++mm)
#pragma unroll
    for (int c = 0; c < 3; ++c) M[mm][c] = met[(3 * mm + c) * N + p];
  const T Jac = met[9 * N + p];
  T g[4][3];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int d = 0; d < 3; ++d) g[f][d] = Jac * (M[0][d] * Df[0][f] + M[1][d] * Df[1][f] + M[2][d] * Df[2][f]);
  const T mu = (T)m.mu, lam = (T)m.lam, kap = (T)m.kap;
  const T div = g[0][0] + g[1][1] + g[2][2];
  const T vel[3] = {s[1] / s[0], s[2] / s[0], s[3] / s[0]};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T tau[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) tau[c] = mu * (g[d][c] + g[c][d]) + (c == d ? lam * div : T(0));
#pragma unroll
    for (int c = 0; c < 3; ++c) dv[5 + 4 * d + c] = tau[c];
    dv[5 + 4 * d + 3] = vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2] + kap * g[3][d];
  }
}

// Receiver values of one donor-value set (the pair's right-hand side), GL lanes per receiver:
// lane l takes the stencil rows (c, b) = l, l + GL, ... of the 16, reads their 4 points' values by
// 16-byte loads from the point-major donor values and accumulates them with the weight wi wj wk
// in the stencil order; the lanes' sums are then added by a fixed butterfly of shuffles. GL = 8
// lanes per receiver keep a gather of a few thousand receivers from running on a few dozen CTAs
// (measured: the 128^3 + 97^3 pair's FP32 macro step 0.932 -> 0.914 ms, FP64 unchanged).
template <typename T, int NV, int GL>
__global__ void __launch_bounds__(128) k3c_gather(const Curv3Gather a) {
  constexpr int VW = 16 / (int)sizeof(T), NL = (NV + VW - 1) / VW;
  static_assert(NL * VW <= kDvPitch && kDvPitch % VW == 0, "16-byte loads within a point's values");
  static_assert(32 % GL == 0 && 16 % GL == 0, "lane groups within a warp");
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = (int)(g / GL), l = (int)(g % GL);
  const bool valid = r < a.nrecv;
  T acc[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) acc[c] = T(0);
  if (valid) {
    const T *dv = static_cast<const T *>(a.dv);
    const T *w = static_cast<const T *>(a.dwt) + 12 * (size_t)r;
    const int *idx = a.didx + 64 * (size_t)r;
#pragma unroll
    for (int q = 0; q < 16 / GL; ++q) {
      const int row = l + q * GL, c3 = row >> 2, b = row & 3;
      const T wjk = w[4 + b] * w[8 + c3];
      int d[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) d[e] = checked_index(idx[row * 4 + e], a.ndv, a.err);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const T wt = w[e] * wjk;
        const V *pv = reinterpret_cast<const V *>(dv + (size_t)d[e] * kDvPitch);
        T v[NL * VW];
#pragma unroll
        for (int k = 0; k < NL; ++k) *reinterpret_cast<V *>(v + k * VW) = pv[k];
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[c] += wt * v[c];
      }
    }
  }
#pragma unroll
  for (int off = GL / 2; off > 0; off >>= 1) {
#pragma unroll
    for (int c = 0; c < NV; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
  }
  if (!valid || l != 0) return;
  T *qh = static_cast<T *>(a.qhat);
#pragma unroll
  for (int c = 0; c < 5; ++c) qh[(size_t)c * a.nrecv + r] = acc[c];
  if (NV > 5) {
    T *fh = static_cast<T *>(a.fvhat);
#pragma unroll
    for (int c = 5; c < NV; ++c) fh[(size_t)(c - 5) * a.nrecv + r] = acc[c];
  }
}

template <int GL>
static void launch3c_gather_l(const Curv3Gather &a, int dtype, cudaStream_t s) {
  const unsigned blocks = (unsigned)(((long long)a.nrecv * GL + 127) / 128);
  if (a.nval == 17) {
    if (dtype == SBP_F64) k3c_gather<double, 17, GL><<<blocks, 128, 0, s>>>(a);
    else k3c_gather<float, 17, GL><<<blocks, 128, 0, s>>>(a);
  } else {
    if (dtype == SBP_F64) k3c_gather<double, 5, GL><<<blocks, 128, 0, s>>>(a);
    else k3c_gather<float, 5, GL><<<blocks, 128, 0, s>>>(a);
  }
}

cudaError_t launch3c_gather(const Curv3Gather &a, int dtype, cudaStream_t s) {
  if (a.nrecv <= 0) return cudaSuccess;
  launch3c_gather_l<8>(a, dtype, s);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) k3c_ab(const Curv3Ab a) {
  const T *q = static_cast<const T *>(a.q);
  const T *rhs = static_cast<const T *>(a.rhs);
  T *qn = static_cast<T *>(a.qn);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < a.field; t += (size_t)gridDim.x * blockDim.x) {
    T q0[5], r[5], qv[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      q0[v] = q[v * a.field + t];
      r[v] = rhs[v * a.field + t];
    }
    const bool active = !a.cls || (a.cls[t] & 15u) != 15u;
    ab_update<T, 5>(q0, a.hold, a.alpha, a.nold, a.field, t, r, qv, active ? a.err : nullptr);
#pragma unroll
    for (int v = 0; v < 5; ++v) qn[v * a.field + t] = qv[v];
  }
}

template <typename T, bool SEG>
__global__ void __launch_bounds__(256) k3c_dt(const Curv3Launch a, double pr, unsigned long long *out) {
  const T *q = static_cast<const T *>(a.q);
  const T *met = static_cast<const T *>(a.met);
  const size_t N = a.field;
  double best = DBL_MAX;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < N; t += (size_t)gridDim.x * blockDim.x) {
    if (is_hole<SEG>(a, t)) continue;
    const double rho = q[t];
    const double u[3] = {q[N + t] / rho, q[2 * N + t] / rho, q[3 * N + t] / rho};
    const double pres = (a.gam - 1.0) * ((double)q[4 * N + t] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
    const double c = sqrt(a.gam * pres / rho);
    const double Jac = met[9 * N + t];
    double conv = 0.0, g2 = 0.0;
    for (int m = 0; m < 3; ++m) {
      const double kv[3] = {Jac * (double)met[(3 * m) * N + t], Jac * (double)met[(3 * m + 1) * N + t],
                            Jac * (double)met[(3 * m + 2) * N + t]};
      conv += fabs(u[0] * kv[0] + u[1] * kv[1] + u[2] * kv[2]);
      g2 += kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
    }
    const double nu = fmax(a.mu, a.gam * a.mu / pr) / rho;
    best = fmin(best, 1.0 / (conv + c * sqrt(g2) + 2.0 * nu * g2));
  }
  for (int off = 16; off > 0; off >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, off));
  __shared__ double wmin[8];
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = fmin(best, wmin[w]);
    atomicMin(out, (unsigned long long)__double_as_longlong(best));
  }
}

// Extrapolated primitives (u, v, w, T) of every tap point of a donor-value launch, per set.
template <typename T>
__global__ void __launch_bounds__(128) k3c_tapvals(const Curv3Donor a) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)a.nsets * a.ntap) return;
  const int set = (int)(t / a.ntap), tp = (int)(t - (long long)set * a.ntap);
  T sn[5], pn[4];
  donor_state(a, set, (size_t)a.tpts[tp], sn);
  prim_of(sn, (T)a.m.gam, pn);
  T *out = static_cast<T *>(a.tv) + ((size_t)set * a.ntap + tp) * 4;
#pragma unroll
  for (int f = 0; f < 4; ++f) out[f] = pn[f];
}

cudaError_t launch3c_donor(const Curv3Donor &a, int dtype, cudaStream_t s) {
  const int n = a.nsets * a.npts;
  if (n <= 0) return cudaSuccess;
  if (a.m.visc && a.tpts && a.ntap > 0) {
    const unsigned b = (unsigned)(((long long)a.nsets * a.ntap + 127) / 128);
    if (dtype == SBP_F64) k3c_tapvals<double><<<b, 128, 0, s>>>(a);
    else k3c_tapvals<float><<<b, 128, 0, s>>>(a);
  }
  if (dtype == SBP_F64) k3c_donor<double><<<(n + 127) / 128, 128, 0, s>>>(a);
  else k3c_donor<float><<<(n + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

// One thread per point: the sponge term at the active points within sp.depth of a face.
template <typename T>
__global__ void __launch_bounds__(256) k3c_sponge(const Curv3Launch a, const Curv3Sponge sp) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.field) return;
  const int i = (int)(p % a.ni), j = (int)((p / a.ni) % a.nj), k = (int)(p / ((size_t)a.ni * a.nj));
  const int d = min(min(min(i, a.ni - 1 - i), min(j, a.nj - 1 - j)), min(k, a.nk - 1 - k));
  if (d >= sp.depth || (a.cls && a.cls[p] == 0xFFFu)) return;
  const T sg = (T)sp.tab[d];
  const T *q = static_cast<const T *>(a.q);
  T *out = static_cast<T *>(a.out);
#pragma unroll
  for (int v = 0; v < 5; ++v) out[v * a.field + p] = fma_rn(-sg, q[v * a.field + p] - (T)a.qinf[v], out[v * a.field + p]);
}

cudaError_t launch3c_sponge(const Curv3Launch &a, const Curv3Sponge &sp, int dtype, cudaStream_t s) {
  if (sp.depth <= 0 || a.field == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((a.field + 255) / 256);
  if (dtype == SBP_F64) k3c_sponge<double><<<blocks, 256, 0, s>>>(a, sp);
  else k3c_sponge<float><<<blocks, 256, 0, s>>>(a, sp);
  return cudaGetLastError();
}

cudaError_t launch3c_ab(const Curv3Ab &a, int dtype, cudaStream_t s) {
  const int blocks = (int)std::min<size_t>((a.field + 255) / 256, 152 * 16);
  if (dtype == SBP_F64) k3c_ab<double><<<blocks, 256, 0, s>>>(a);
  else k3c_ab<float><<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch3c_dt(const Curv3Launch &a, double pr, unsigned long long *out, cudaStream_t s, int dtype) {
  // 0x7F in every byte: a positive double near 1.4e306, above any time step (the min's start)
  cudaError_t e = cudaMemsetAsync(out, 0x7F, sizeof(*out), s);
  if (e != cudaSuccess) return e;
  const int blocks = (int)std::min<size_t>((a.field + 255) / 256, 152 * 8);
  if (a.cls) {
    if (dtype == SBP_F64) k3c_dt<double, true><<<blocks, 256, 0, s>>>(a, pr, out);
    else k3c_dt<float, true><<<blocks, 256, 0, s>>>(a, pr, out);
  } else {
    if (dtype == SBP_F64) k3c_dt<double, false><<<blocks, 256, 0, s>>>(a, pr, out);
    else k3c_dt<float, false><<<blocks, 256, 0, s>>>(a, pr, out);
  }
  return cudaGetLastError();
}

template <typename T, bool SEG>
static cudaError_t launch3c_rhs_t(const Curv3Launch &a, cudaStream_t s) {
  const int blocks = (int)((a.field + 255) / 256);
  if (a.visc) k3c_prim<T, SEG><<<blocks, 256, 0, s>>>(a);
  k3c_flux<T, SEG><<<blocks, 256, 0, s>>>(a);
  k3c_update<T, SEG><<<blocks, 256, 0, s>>>(a);
  if (a.far) {
    const size_t nf = face_points(a.ni, a.nj, a.nk);
    k3c_far<T, SEG><<<(unsigned)((nf + 127) / 128), 128, 0, s>>>(a, nf);
  }
  return cudaGetLastError();
}

cudaError_t launch3c_rhs(const Curv3Launch &a, int dtype, cudaStream_t s) {
  if (a.cls) return dtype == SBP_F64 ? launch3c_rhs_t<double, true>(a, s) : launch3c_rhs_t<float, true>(a, s);
  return dtype == SBP_F64 ? launch3c_rhs_t<double, false>(a, s) : launch3c_rhs_t<float, false>(a, s);
}

}  // namespace sbp
