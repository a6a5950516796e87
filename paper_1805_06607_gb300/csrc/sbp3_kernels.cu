// 3D Cartesian right-hand side (App. C.1 equations in three directions, Sec. 2.1 SBP 4-2,
// Sec. 2.2 SAT and interpolation) and the donor-value / gather / time-step kernels:
//   k3_prim    primitives (u, v, w, T) of every point (Navier-Stokes)
//   k3_flux    F - F^V, G - G^V, H - H^V at every active point (gradients by D along i, j, k)
//   k3_sat     SAT terms of the boundary and receiver points (receiver values gathered from the
//              donor values over the 4 x 4 x 4 cell)
//   k3_update  -(D_x F^ + D_y G^ + D_z H^) + SAT and the MRAB epilogue (mode 1)
//   k3_donor   state (with the slow extrapolation of Sec. 3.3) and viscous fluxes at the
//              distinct donor points, per extrapolation set
//   k3_gather  receiver values of one set (sbp3_overset_interp)
//   k3_dt      time step of Sec. 4.1, min-reduced
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <cstring>

#include "sbp3_device.h"
#include "sbp_dev.cuh"

namespace sbp {

template <typename T>
__device__ __forceinline__ const K3<T> &kc3(const Rhs3Launch &a);
template <>
__device__ __forceinline__ const K3<float> &kc3<float>(const Rhs3Launch &a) {
  return a.cf;
}
template <>
__device__ __forceinline__ const K3<double> &kc3<double>(const Rhs3Launch &a) {
  return a.cd;
}
template <typename T>
__device__ __forceinline__ const K3<T> &kd3(const Donor3Launch &a);
template <>
__device__ __forceinline__ const K3<float> &kd3<float>(const Donor3Launch &a) {
  return a.cf;
}
template <>
__device__ __forceinline__ const K3<double> &kd3<double>(const Donor3Launch &a) {
  return a.cd;
}

__device__ __forceinline__ size_t pidx3(const Dev3Mesh &m, int i, int j, int k) {
  return ((size_t)k * m.nj + j) * m.pitch + i;
}

template <typename T>
__device__ __forceinline__ void prim5(const T q[5], T gam, T pr[4]) {
  T ri = T(1) / q[0];
  T u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
  T pres = (gam - T(1)) * (q[4] - T(0.5) * (q[1] * u + q[2] * v + q[3] * w));
  pr[0] = u;
  pr[1] = v;
  pr[2] = w;
  pr[3] = gam * pres * ri;
}

// Indices of the 4 taps of direction d's derivative row at (i, j, k).
template <typename T>
__device__ __forceinline__ void taps3(const Dev3Mesh &m, int i, int j, int k, int d, const Row<T> &r, size_t idx[4]) {
  const int n[3] = {m.ni, m.nj, m.nk};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int c[3] = {i, j, k};
    c[d] += r.off[e];
    wrap_index(c[d], n[d], m.per[d]);
    idx[e] = pidx3(m, c[0], c[1], c[2]);
  }
}

template <typename T>
__device__ __forceinline__ T dsum3(const Row<T> &r, const T *f, const size_t idx[4]) {
  T acc = T(0);
#pragma unroll
  for (int e = 0; e < 4; ++e) acc += r.w[e] * f[idx[e]];
  return r.neg ? -acc : acc;
}

// Cartesian viscous fluxes F^V_d (momentum x, y, z, energy) at one point from the primitive
// planes: gradients by D along each direction times 1/h.
template <typename T>
__device__ void visc3_at(const Dev3Mesh &m, const K3<T> &kk, const T *prim, int i, int j, int k, T Fv[3][4]) {
  const size_t p = pidx3(m, i, j, k);
  const unsigned code = m.cls[p];
  T g[4][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const Row<T> r = decode_row<T>((code >> (4 * d)) & 15u);
    size_t idx[4];
    taps3(m, i, j, k, d, r, idx);
#pragma unroll
    for (int f = 0; f < 4; ++f) g[f][d] = kk.ih[d] * dsum3(r, prim + f * m.field, idx);
  }
  const T div = g[0][0] + g[1][1] + g[2][2];
  T tau[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) tau[a][b] = kk.mu * (g[a][b] + g[b][a]) + (a == b ? kk.lam * div : T(0));
  const T vel[3] = {prim[p], prim[m.field + p], prim[2 * m.field + p]};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int c = 0; c < 3; ++c) Fv[d][c] = tau[d][c];
    Fv[d][3] = vel[0] * tau[d][0] + vel[1] * tau[d][1] + vel[2] * tau[d][2] + kk.kap * g[3][d];
  }
}

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

// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k3_prim(const Rhs3Launch a) {
  const Dev3Mesh &m = a.m;
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  if (i >= m.ni || j >= m.nj) return;
  const size_t p = pidx3(m, i, j, k);
  const T *q = static_cast<const T *>(a.q);
  T qp[5], pr[4];
#pragma unroll
  for (int v = 0; v < 5; ++v) qp[v] = q[v * m.field + p];
  prim5(qp, kc3<T>(a).gam, pr);
  T *pl = static_cast<T *>(a.prim);
#pragma unroll
  for (int f = 0; f < 4; ++f) pl[f * m.field + p] = pr[f];
}

template <typename T, bool VISC>
__global__ void __launch_bounds__(256) k3_flux(const Rhs3Launch a) {
  const Dev3Mesh &m = a.m;
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  if (i >= m.ni || j >= m.nj) return;
  const size_t p = pidx3(m, i, j, k);
  if ((m.cls[p] & 15u) == 15u) return;
  const K3<T> &kk = kc3<T>(a);
  const T *q = static_cast<const T *>(a.q);
  T qp[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qp[v] = q[v * m.field + p];
  const T ri = T(1) / qp[0];
  const T u[3] = {qp[1] * ri, qp[2] * ri, qp[3] * ri};
  const T pres = (kk.gam - T(1)) * (qp[4] - T(0.5) * (qp[1] * u[0] + qp[2] * u[1] + qp[3] * u[2]));
  T Fv[3][4];
  if (VISC) visc3_at(m, kk, static_cast<const T *>(a.prim), i, j, k, Fv);
  T *fl = static_cast<T *>(a.flux);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T F[5];
    F[0] = qp[1 + d];
#pragma unroll
    for (int c = 0; c < 3; ++c) F[1 + c] = qp[1 + c] * u[d] + (c == d ? pres : T(0));
    F[4] = (qp[4] + pres) * u[d];
    if (VISC) {
#pragma unroll
      for (int c = 0; c < 4; ++c) F[1 + c] -= Fv[d][c];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) fl[(5 * d + v) * m.field + p] = F[v];
  }
}

// One thread per SAT point, launched in 32-thread blocks so that the few hundred points of a
// background spread over the SMs.
template <typename T, bool VISC>
__global__ void __launch_bounds__(32) k3_sat(const Rhs3Launch a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.nsat) return;
  const Dev3Mesh &m = a.m;
  const K3<T> &kk = kc3<T>(a);
  const int64_t pl = a.sat_pt[s];
  const int i = (int)(pl % m.ni), j = (int)((pl / m.ni) % m.nj), k = (int)(pl / ((int64_t)m.ni * m.nj));
  const size_t p = pidx3(m, i, j, k);
  const T *q = static_cast<const T *>(a.q);
  constexpr int NRV = VISC ? kRv3 : 5;
  T rv[NRV];
#pragma unroll
  for (int c = 0; c < NRV; ++c) rv[c] = T(0);
  const int recv = a.sat_recv[s];
  if (recv >= 0) {
    const T *dv = static_cast<const T *>(a.dv);
    const T *w = static_cast<const T *>(a.dwt) + 12 * recv;
    for (int t = 0; t < 64; ++t) {  // donor point (c3 * 4 + b) * 4 + e
      const int e = t & 3, b = (t >> 2) & 3, c3 = t >> 4;
      const T wt = w[e] * w[4 + b] * w[8 + c3];
      const int d = a.didx[64 * recv + t];
#pragma unroll
      for (int c = 0; c < NRV; ++c) rv[c] += wt * dv[c * a.ndv + d];
    }
  }
  T qp[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qp[v] = q[v * m.field + p];
  T Fv[3][4] = {};
  if (VISC) visc3_at(m, kk, static_cast<const T *>(a.prim), i, j, k, Fv);
  const uint32_t code = a.sat_code[s];
  const int nt = code & 3u;
  T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
  for (int t = 0; t < nt; ++t) {
    const unsigned term = (code >> (2 + 4 * t)) & 15u;
    const int d = term & 3u, side = (term & 4u) ? -1 : 1, far = (term >> 3) & 1u;
    T kv[3] = {T(0), T(0), T(0)};
    kv[d] = kk.ih[d];
    T tgt[5], sig1 = T(0);
    const T sigI = far ? kk.sig_phys : kk.sig_int;
    if (!far) {
#pragma unroll
      for (int v = 0; v < 5; ++v) tgt[v] = rv[v];
      if (VISC) sig1 = T(0.5) * kk.mu * (kv[d] * kv[d]);
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) tgt[v] = kk.qinf[v];
    }
    T dq[5], kd[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) dq[v] = qp[v] - tgt[v];
    penalty3(qp, kk.gam, kv, side, dq, kd);
    T sat[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) sat[v] = -(sigI * kd[v] + sig1 * dq[v]) * T(1.0 / SBP_P0);
    if (VISC && !far) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const T own = kv[d] * Fv[d][c];
        const T hat = kv[d] * rv[5 + 4 * d + c];
        sat[1 + c] += T(0.5) * T(side) * (own - hat) * T(1.0 / SBP_P0);
      }
    }
    const T sc = far ? T(1) : (T)a.sat_scale[s];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += sc * sat[v];
  }
  T *satb = static_cast<T *>(a.sat);
#pragma unroll
  for (int v = 0; v < 5; ++v) satb[v * a.nsat + s] = acc[v];
}

template <typename T>
__global__ void __launch_bounds__(256) k3_update(const Rhs3Launch a) {
  const Dev3Mesh &m = a.m;
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  if (i >= m.ni || j >= m.nj) return;
  const size_t p = pidx3(m, i, j, k);
  const unsigned code = m.cls[p];
  const K3<T> &kk = kc3<T>(a);
  T rhs[5] = {T(0), T(0), T(0), T(0), T(0)};
  if ((code & 15u) != 15u) {
    const T *fl = static_cast<const T *>(a.flux);
    T dsum[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const Row<T> r = decode_row<T>((code >> (4 * d)) & 15u);
      size_t idx[4];
      taps3(m, i, j, k, d, r, idx);
#pragma unroll
      for (int v = 0; v < 5; ++v) dsum[v] += kk.ih[d] * dsum3(r, fl + (5 * d + v) * m.field, idx);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) rhs[v] = -dsum[v];
    const int row = k * m.nj + j;
    int lo = a.row_sat[row], hi = a.row_sat[row + 1];
    if (lo < hi) {
      const int64_t key = ((int64_t)k * m.nj + j) * m.ni + i;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a.sat_pt[mid] < key) lo = mid + 1;
        else hi = mid;
      }
      if (lo < a.row_sat[row + 1] && a.sat_pt[lo] == key) {
        const T *satb = static_cast<const T *>(a.sat);
#pragma unroll
        for (int v = 0; v < 5; ++v) rhs[v] += satb[v * a.nsat + lo];
      }
    }
  }
  T *out = static_cast<T *>(a.out);
  if (a.mode == 0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v * m.field + p] = rhs[v];
  } else {
    const T *q = static_cast<const T *>(a.q);
    T *qn = static_cast<T *>(a.qnext);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      out[v * m.field + p] = rhs[v];
      double acc = (double)q[v * m.field + p];
      for (int h = 0; h < a.nold; ++h) acc += a.alpha[h] * (double)static_cast<const T *>(a.hold[h])[v * m.field + p];
      acc += a.alpha[a.nold] * (double)rhs[v];
      qn[v * m.field + p] = (T)acc;
    }
  }
}

// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void set_state3(const Donor3Launch &a, int set, size_t p, T out[5]) {
  const T *q = static_cast<const T *>(a.q);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    double acc = (double)q[v * a.d.field + p];
    for (int k = 0; k < a.nb[set]; ++k) acc += a.beta[set][k] * (double)static_cast<const T *>(a.hist[k])[v * a.d.field + p];
    out[v] = (T)acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k3_donor(const Donor3Launch a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nsets * a.npts) return;
  const int set = t / a.npts, dp = t - set * a.npts;
  const Dev3Mesh &m = a.d;
  const K3<T> &kk = kd3<T>(a);
  const int64_t pl = a.pts[dp];
  const int i = (int)(pl % m.ni), j = (int)((pl / m.ni) % m.nj), k = (int)(pl / ((int64_t)m.ni * m.nj));
  const size_t p = pidx3(m, i, j, k);
  T s[5];
  set_state3(a, set, p, s);
  T *dv = static_cast<T *>(a.dv) + (size_t)set * kRv3 * a.npts;
#pragma unroll
  for (int v = 0; v < 5; ++v) dv[v * a.npts + dp] = s[v];
  if (!a.visc) return;
  // gradients of the primitives of the (extrapolated) state along each direction
  const unsigned code = m.cls[p];
  T g[4][3];
  for (int d = 0; d < 3; ++d) {
    const Row<T> r = decode_row<T>((code >> (4 * d)) & 15u);
    size_t idx[4];
    taps3(m, i, j, k, d, r, idx);
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int e = 0; e < 4; ++e) {
      T sn[5], pn[4];
      set_state3(a, set, idx[e], sn);
      prim5(sn, kk.gam, pn);
#pragma unroll
      for (int f = 0; f < 4; ++f) acc[f] += r.w[e] * pn[f];
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) g[f][d] = kk.ih[d] * (r.neg ? -acc[f] : acc[f]);
  }
  T pc[4];
  prim5(s, kk.gam, pc);
  const T div = g[0][0] + g[1][1] + g[2][2];
  T tau[3][3];
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3; ++y) tau[x][y] = kk.mu * (g[x][y] + g[y][x]) + (x == y ? kk.lam * div : T(0));
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int c = 0; c < 3; ++c) dv[(5 + 4 * d + c) * a.npts + dp] = tau[d][c];
    dv[(5 + 4 * d + 3) * a.npts + dp] = pc[0] * tau[d][0] + pc[1] * tau[d][1] + pc[2] * tau[d][2] + kk.kap * g[3][d];
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k3_gather(const Gather3Launch a) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.nrecv) return;
  const T *dv = static_cast<const T *>(a.dv);
  const T *w = static_cast<const T *>(a.dwt) + 12 * r;
  T acc[kRv3];
  for (int c = 0; c < a.nval; ++c) acc[c] = T(0);
  for (int c3 = 0; c3 < 4; ++c3)
    for (int b = 0; b < 4; ++b)
      for (int e = 0; e < 4; ++e) {
        const T wt = w[e] * w[4 + b] * w[8 + c3];
        const int d = a.didx[64 * r + (c3 * 4 + b) * 4 + e];
        for (int c = 0; c < a.nval; ++c) acc[c] += wt * dv[c * a.ndv + d];
      }
  T *qh = static_cast<T *>(a.qhat);
  for (int c = 0; c < 5; ++c) qh[c * a.nrecv + r] = acc[c];
  if (a.fvhat && a.nval > 5) {
    T *fh = static_cast<T *>(a.fvhat);
    for (int c = 5; c < a.nval; ++c) fh[(c - 5) * a.nrecv + r] = acc[c];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k3_dt(const Dev3Mesh m, K3<double> kk, double mu, double pr, const T *q,
                                             unsigned long long *out) {
  double best = DBL_MAX;
  const size_t n = (size_t)m.ni * m.nj * m.nk;
  const double s2 = kk.ih[0] * kk.ih[0] + kk.ih[1] * kk.ih[1] + kk.ih[2] * kk.ih[2];
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % m.ni), j = (int)((t / m.ni) % m.nj), k = (int)(t / ((size_t)m.ni * m.nj));
    const size_t p = pidx3(m, i, j, k);
    if ((m.cls[p] & 15u) == 15u) continue;
    const double rho = q[p];
    const double u[3] = {q[m.field + p] / rho, q[2 * m.field + p] / rho, q[3 * m.field + p] / rho};
    const double pres = (kk.gam - 1.0) * ((double)q[4 * m.field + p] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
    const double c = sqrt(kk.gam * pres / rho);
    const double inv = fabs(u[0]) * kk.ih[0] + fabs(u[1]) * kk.ih[1] + fabs(u[2]) * kk.ih[2] + c * sqrt(s2);
    const double nu = fmax(mu, kk.gam * mu / pr) / rho;
    best = fmin(best, 1.0 / (inv + 2.0 * nu * s2));
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

__global__ void k3_fill_u64(unsigned long long *p, unsigned long long v) { *p = v; }

// ---------------------------------------------------------------------------------------------
template <typename T>
static cudaError_t launch3_rhs_t(const Rhs3Launch &a, cudaStream_t s) {
  const Dev3Mesh &m = a.m;
  dim3 blk(32, 8), grid((m.ni + 31) / 32, (m.nj + 7) / 8, m.nk);
  if (a.visc) k3_prim<T><<<grid, blk, 0, s>>>(a);
  if (a.visc) k3_flux<T, true><<<grid, blk, 0, s>>>(a);
  else k3_flux<T, false><<<grid, blk, 0, s>>>(a);
  if (a.nsat > 0) {
    const int blocks = (a.nsat + 31) / 32;
    if (a.visc) k3_sat<T, true><<<blocks, 32, 0, s>>>(a);
    else k3_sat<T, false><<<blocks, 32, 0, s>>>(a);
  }
  k3_update<T><<<grid, blk, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch3_rhs(const Rhs3Launch &a, int dtype, cudaStream_t s) {
  return dtype == SBP_F64 ? launch3_rhs_t<double>(a, s) : launch3_rhs_t<float>(a, s);
}

cudaError_t launch3_donor(const Donor3Launch &a, int dtype, cudaStream_t s) {
  const int n = a.nsets * a.npts;
  if (n == 0) return cudaSuccess;
  if (dtype == SBP_F64) k3_donor<double><<<(n + 127) / 128, 128, 0, s>>>(a);
  else k3_donor<float><<<(n + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch3_gather(const Gather3Launch &a, int dtype, cudaStream_t s) {
  if (a.nrecv == 0) return cudaSuccess;
  if (dtype == SBP_F64) k3_gather<double><<<(a.nrecv + 127) / 128, 128, 0, s>>>(a);
  else k3_gather<float><<<(a.nrecv + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch3_dt(const Dev3Mesh &m, const K3<double> &k, double mu, double pr, const void *q, int dtype,
                       unsigned long long *out, cudaStream_t s) {
  double big = DBL_MAX;
  unsigned long long bits;
  memcpy(&bits, &big, sizeof(bits));
  k3_fill_u64<<<1, 1, 0, s>>>(out, bits);
  const size_t n = (size_t)m.ni * m.nj * m.nk;
  int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
  if (dtype == SBP_F64) k3_dt<double><<<blocks, 256, 0, s>>>(m, k, mu, pr, (const double *)q, out);
  else k3_dt<float><<<blocks, 256, 0, s>>>(m, k, mu, pr, (const float *)q, out);
  return cudaGetLastError();
}

}  // namespace sbp
