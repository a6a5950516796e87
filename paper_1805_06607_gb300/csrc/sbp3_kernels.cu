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
#include "sbp3_penalty.cuh"

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

// The point-wise arithmetic of the right-hand side below carries explicit roundings (mul_rn /
// fma_rn): the compiler cannot contract it differently in different kernels, so the per-point and
// the marching designs give the same bits.
template <typename T>
__device__ __forceinline__ T ke3(const T q[5], T u, T v, T w) {  // rho |u|^2
  return fma_rn(q[3], w, fma_rn(q[2], v, mul_rn(q[1], u)));
}

template <typename T>
__device__ __forceinline__ T pres3(const T q[5], T gam, T ke) {  // (gamma - 1)(rho E - ke / 2)
  return mul_rn(gam - T(1), fma_rn(T(-0.5), ke, q[4]));
}

// Primitives (u, v, w, T = gamma p / rho) of a state.
template <typename T>
__device__ __forceinline__ void prim5(const T q[5], T gam, T pr[4]) {
  const T ri = T(1) / q[0];
  const T u = mul_rn(q[1], ri), v = mul_rn(q[2], ri), w = mul_rn(q[3], ri);
  const T pres = pres3(q, gam, ke3(q, u, v, w));
  pr[0] = u;
  pr[1] = v;
  pr[2] = w;
  pr[3] = mul_rn(mul_rn(gam, pres), ri);
}

// sum_e w[e] x[e] in tap order.
template <typename T>
__device__ __forceinline__ T tap4(const T w[4], T x0, T x1, T x2, T x3) {
  return fma_rn(w[3], x3, fma_rn(w[2], x2, fma_rn(w[1], x1, mul_rn(w[0], x0))));
}

template <typename T>
__device__ __forceinline__ void central_w(T w[4]) {
  w[0] = CentralRow<T>::w0;
  w[1] = CentralRow<T>::w1;
  w[2] = CentralRow<T>::w2;
  w[3] = CentralRow<T>::w3;
}

// Viscous stresses (Stokes hypothesis, constant mu) from the gradients g[f][d] of (u, v, w, T).
template <typename T>
__device__ __forceinline__ void tau3(const K3<T> &kk, const T g[4][3], T tau[3][3]) {
  const T ld = mul_rn(kk.lam, g[0][0] + g[1][1] + g[2][2]);
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3; ++y) {
      const T sm = g[x][y] + g[y][x];
      tau[x][y] = x == y ? fma_rn(kk.mu, sm, ld) : mul_rn(kk.mu, sm);
    }
}

// Energy component of the viscous flux along d: u . tau_d + kappa dT/dx_d.
template <typename T>
__device__ __forceinline__ T evisc3(const K3<T> &kk, const T tau[3][3], const T g[4][3], const T vel[3], int d) {
  return fma_rn(kk.kap, g[3][d], fma_rn(vel[2], tau[d][2], fma_rn(vel[1], tau[d][1], mul_rn(vel[0], tau[d][0]))));
}

// F_d - F^V_d (5 components) of a point: inviscid flux along d from the state, velocity and
// pressure, minus the viscous flux (tau, gradients; VISC only).
template <typename T, bool VISC>
__device__ __forceinline__ void flux3_dir(const K3<T> &kk, const T qp[5], const T u[3], T pres, const T tau[3][3],
                                          const T g[4][3], const T vel[3], int d, T F[5]) {
  F[0] = qp[1 + d];
#pragma unroll
  for (int c = 0; c < 3; ++c) F[1 + c] = c == d ? fma_rn(qp[1 + c], u[d], pres) : mul_rn(qp[1 + c], u[d]);
  F[4] = mul_rn(qp[4] + pres, u[d]);
  if constexpr (VISC) {
#pragma unroll
    for (int c = 0; c < 3; ++c) F[1 + c] -= tau[d][c];
    F[4] -= evisc3(kk, tau, g, vel, d);
  }
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

// A derivative row applied to plane f (sign of a high-end closure included).
template <typename T>
__device__ __forceinline__ T dsum3(const Row<T> &r, const T *f, const size_t idx[4]) {
  const T acc = tap4(r.w, f[idx[0]], f[idx[1]], f[idx[2]], f[idx[3]]);
  return r.neg ? -acc : acc;
}

// Primitives (u, v, w, T) at index p: read from the primitive planes, or (FROMQ) computed from the
// state planes with prim5 (the arithmetic k3_prim applies when it writes the planes).
template <typename T, bool FROMQ>
__device__ __forceinline__ void prim_src(const T *src, size_t field, size_t p, T gam, T pv[4]) {
  if constexpr (FROMQ) {
    T qv[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qv[v] = src[v * field + p];
    prim5(qv, gam, pv);
  } else {
#pragma unroll
    for (int f = 0; f < 4; ++f) pv[f] = src[f * field + p];
  }
}

// Gradients g[f][d] of (u, v, w, T) at one point from the primitives (planes, or the state with
// FROMQ): D along each direction times 1/h.
template <typename T, bool FROMQ>
__device__ void grad3_at(const Dev3Mesh &m, const K3<T> &kk, const T *src, int i, int j, int k, T g[4][3]) {
  const unsigned code = m.cls[pidx3(m, i, j, k)];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const Row<T> r = decode_row<T>((code >> (4 * d)) & 15u);
    size_t idx[4];
    taps3(m, i, j, k, d, r, idx);
    T pv[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) prim_src<T, FROMQ>(src, m.field, idx[e], kk.gam, pv[e]);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const T acc = tap4(r.w, pv[0][f], pv[1][f], pv[2][f], pv[3][f]);
      g[f][d] = mul_rn(kk.ih[d], r.neg ? -acc : acc);
    }
  }
}

// Cartesian viscous fluxes F^V_d (momentum x, y, z, energy) at one point.
template <typename T, bool FROMQ>
__device__ void visc3_at(const Dev3Mesh &m, const K3<T> &kk, const T *src, int i, int j, int k, T Fv[3][4]) {
  T g[4][3], tau[3][3], pc[4];
  grad3_at<T, FROMQ>(m, kk, src, i, j, k, g);
  tau3(kk, g, tau);
  prim_src<T, FROMQ>(src, m.field, pidx3(m, i, j, k), kk.gam, pc);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int c = 0; c < 3; ++c) Fv[d][c] = tau[d][c];
    Fv[d][3] = evisc3(kk, tau, g, pc, d);
  }
}

// Element offsets of the interior row's taps (-2, -1, +1, +2) along each direction at (i, j, k),
// wrapped on periodic lines. Every point of class 0 takes them, so the warps of a mesh's interior
// (periodic seams included) follow one path.
__device__ __forceinline__ void central_offsets(const Dev3Mesh &m, int i, int j, int k, ptrdiff_t o[3][4]) {
  const int c[3] = {i, j, k}, n[3] = {m.ni, m.nj, m.nk};
  const ptrdiff_t st[3] = {1, (ptrdiff_t)m.pitch, (ptrdiff_t)m.pitch * m.nj};
  const int off[4] = {-2, -1, 1, 2};
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int cc = c[d] + off[e];
      wrap_index(cc, n[d], m.per[d]);
      o[d][e] = (ptrdiff_t)(cc - c[d]) * st[d];
    }
}

// The interior row applied to plane f at index p with the tap offsets o.
template <typename T>
__device__ __forceinline__ T csum3(const T *f, size_t p, const ptrdiff_t o[4]) {
  T w[4];
  central_w(w);
  return tap4(w, f[p + o[0]], f[p + o[1]], f[p + o[2]], f[p + o[3]]);
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
  const unsigned code = m.cls[p];
  if ((code & 15u) == 15u) return;
  const K3<T> &kk = kc3<T>(a);
  const T *q = static_cast<const T *>(a.q);
  T qp[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qp[v] = q[v * m.field + p];
  const T ri = T(1) / qp[0];
  const T u[3] = {mul_rn(qp[1], ri), mul_rn(qp[2], ri), mul_rn(qp[3], ri)};
  const T pres = pres3(qp, kk.gam, ke3(qp, u[0], u[1], u[2]));
  T g[4][3], tau[3][3], vel[3];
  if (VISC) {
    const T *prim = static_cast<const T *>(a.prim);
    if (code == 0u) {
      ptrdiff_t o[3][4];
      central_offsets(m, i, j, k, o);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int f = 0; f < 4; ++f) g[f][d] = mul_rn(kk.ih[d], csum3(prim + f * m.field, p, o[d]));
    } else {
      grad3_at<T, false>(m, kk, prim, i, j, k, g);
    }
    tau3(kk, g, tau);
#pragma unroll
    for (int c = 0; c < 3; ++c) vel[c] = prim[c * m.field + p];
  }
  T *fl = static_cast<T *>(a.flux);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T F[5];
    flux3_dir<T, VISC>(kk, qp, u, pres, tau, g, vel, d, F);
#pragma unroll
    for (int v = 0; v < 5; ++v) fl[(5 * d + v) * m.field + p] = F[v];
  }
}

// One thread per SAT point, launched in 32-thread blocks so that the few hundred points of a
// background spread over the SMs.
template <typename T, bool VISC, bool FROMQ>
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
      const int d = checked_index(a.didx[64 * recv + t], a.ndv, a.err);
#pragma unroll
      for (int c = 0; c < NRV; ++c) rv[c] += wt * dv[c * a.ndv + d];
    }
  }
  T qp[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qp[v] = q[v * m.field + p];
  T Fv[3][4] = {};
  if (VISC) visc3_at<T, FROMQ>(m, kk, FROMQ ? q : static_cast<const T *>(a.prim), i, j, k, Fv);
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

// Sponge layer (Sec. 5.1) at point (i, j, k), after the SAT terms: rhs -= sigma (q - qinf) with
// sigma = sponge_tab[d] for the index distance d < sponge_d to the nearest far-field face. The
// update kernels take it behind a template switch, so meshes without a sponge (the periodic
// boxes) run code without it.
template <typename T>
__device__ __forceinline__ void sponge3(const Rhs3Launch &a, const K3<T> &kk, int i, int j, int k, size_t p,
                                        T rhs[5]) {
  if (kk.sponge_d <= 0) return;
  const Dev3Mesh &m = a.m;
  int d = 1 << 30;
  if (kk.sponge_faces & 1) d = min(d, i);
  if (kk.sponge_faces & 2) d = min(d, m.ni - 1 - i);
  if (kk.sponge_faces & 4) d = min(d, j);
  if (kk.sponge_faces & 8) d = min(d, m.nj - 1 - j);
  if (kk.sponge_faces & 16) d = min(d, k);
  if (kk.sponge_faces & 32) d = min(d, m.nk - 1 - k);
  if (d >= kk.sponge_d) return;
  const T sg = kk.sponge_tab[d];
  if (sg == T(0)) return;
  const T *q = static_cast<const T *>(a.q);
#pragma unroll
  for (int v = 0; v < 5; ++v) rhs[v] = fma_rn(-sg, q[v * m.field + p] - kk.qinf[v], rhs[v]);
}

template <typename T, bool SPONGE>
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
    if (code == 0u) {
      ptrdiff_t o[3][4];
      central_offsets(m, i, j, k, o);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v) dsum[v] = fma_rn(kk.ih[d], csum3(fl + (5 * d + v) * m.field, p, o[d]), dsum[v]);
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const Row<T> r = decode_row<T>((code >> (4 * d)) & 15u);
        size_t idx[4];
        taps3(m, i, j, k, d, r, idx);
#pragma unroll
        for (int v = 0; v < 5; ++v) dsum[v] = fma_rn(kk.ih[d], dsum3(r, fl + (5 * d + v) * m.field, idx), dsum[v]);
      }
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
    if constexpr (SPONGE) sponge3(a, kk, i, j, k, p, rhs);
  }
  T *out = static_cast<T *>(a.out);
  if (a.mode == 0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v * m.field + p] = rhs[v];
  } else {
    const T *q = static_cast<const T *>(a.q);
    T *qn = static_cast<T *>(a.qnext);
    T q0[5], qv[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) q0[v] = q[v * m.field + p];
    ab_update<T, 5>(q0, a.hold, a.alpha, a.nold, m.field, p, rhs, qv, (code & 15u) != 15u ? a.err : nullptr);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      out[v * m.field + p] = rhs[v];
      qn[v * m.field + p] = qv[v];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Right-hand side marching along k (Navier-Stokes): a CTA owns a 32 x 8 tile of (i, j) columns,
// one column per thread, and a chunk of k planes.
//   k3_fluxm   primitives of the tile with a 3-point (i, j) halo in an 8-plane ring in shared
//              memory (plane k in slot k & 7), computed from the state three planes ahead of the
//              fluxes (the state of the next plane is loaded into registers while the current
//              plane's fluxes are computed); F - F^V, G - G^V, H - H^V of each point from ring
//              taps only. Replaces k3_prim + k3_flux: each point's primitives are computed
//              once per tile and no primitive planes cross HBM.
//   k3_updm    the 15 flux planes: the i-flux with a 3-point i halo and the j-flux with a
//              3-point j halo of plane k in double-buffered tiles, the k-flux of the tile's own
//              columns in an 8-plane ring, all copied one plane ahead with cp.async; then
//              k3_update's derivatives, SAT and epilogue.
// Both evaluate every point with k3_flux's / k3_update's operations in the same order, so the
// two right-hand-side designs give the same bits. Periodic wrap in i and j is resolved when the
// halo is loaded, in k by ring slots of the unwrapped plane index.
constexpr int kM3X = 32, kM3Y = 8, kM3Ring = 8;

template <typename T>
struct Flux3M {
  static constexpr int WX = kM3X + 6, WY = kM3Y + 6, WN = WX * WY, NIT = (WN + 255) / 256;
  static constexpr size_t bytes = (size_t)kM3Ring * 4 * WN * sizeof(T);
};

template <typename T>
__global__ void __launch_bounds__(256) k3_fluxm(const Rhs3Launch a, int chunk) {
  using F = Flux3M<T>;
  constexpr int WX = F::WX, WN = F::WN, NIT = F::NIT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *ring = reinterpret_cast<T *>(smem_raw);  // ring[(slot * 4 + f) * WN + w]
  const Dev3Mesh &m = a.m;
  const K3<T> &kk = kc3<T>(a);
  const T *q = static_cast<const T *>(a.q);
  T *fl = static_cast<T *>(a.flux);
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int i0 = blockIdx.x * kM3X, j0 = blockIdx.y * kM3Y;
  const int k0 = blockIdx.z * chunk, k1 = min(k0 + chunk, m.nk);
  const size_t plane = (size_t)m.nj * m.pitch;
  // this thread's window points: offset within a plane (-1 outside the mesh) and window index
  int wofs[NIT];
#pragma unroll
  for (int it = 0; it < NIT; ++it) {
    const int w = tid + 256 * it;
    wofs[it] = -1;
    if (w < WN) {
      int gi = i0 - 3 + w % WX, gj = j0 - 3 + w / WX;
      if (wrap_index(gi, m.ni, m.per[0]) & wrap_index(gj, m.nj, m.per[1])) wofs[it] = gj * m.pitch + gi;
    }
  }
  T qs[NIT][5];
  auto load_q = [&](int kp) {
    int kg = kp;
    const bool ok = wrap_index(kg, m.nk, m.per[2]);
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      if (!ok || wofs[it] < 0) continue;
      const size_t pp = (size_t)kg * plane + wofs[it];
#pragma unroll
      for (int v = 0; v < 5; ++v) qs[it][v] = q[v * m.field + pp];
    }
  };
  auto store_prims = [&](int kp) {
    int kg = kp;
    const bool ok = wrap_index(kg, m.nk, m.per[2]);
    T *sl = ring + (size_t)(kp & (kM3Ring - 1)) * 4 * WN;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      if (!ok || wofs[it] < 0) continue;
      T pv[4];
      prim5(qs[it], kk.gam, pv);
      const int w = tid + 256 * it;
#pragma unroll
      for (int f = 0; f < 4; ++f) sl[f * WN + w] = pv[f];
    }
  };
  // planes k0 - 3 .. k0 + 2 of the ring, and the state of plane k0 + 3 in registers
  for (int kp = k0 - 3; kp < k0 + 3; ++kp) {
    load_q(kp);
    store_prims(kp);
  }
  load_q(k0 + 3);
  const int gi = i0 + tx, gj = j0 + ty;
  const bool own = gi < m.ni && gj < m.nj;
  const int c = (ty + 3) * WX + tx + 3;
  for (int kq = k0; kq < k1; ++kq) {
    // slot of plane kq + 3 held plane kq - 5, which no thread reads any more: the previous
    // plane's fluxes read planes kq - 4 .. kq + 2
    store_prims(kq + 3);
    __syncthreads();
    if (kq + 1 < k1) load_q(kq + 4);
    if (!own) continue;
    const size_t p = (size_t)kq * plane + (size_t)gj * m.pitch + gi;
    const unsigned code = m.cls[p];
    if ((code & 15u) == 15u) continue;
    T qp[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qp[v] = q[v * m.field + p];
    const T ri = T(1) / qp[0];
    const T u[3] = {mul_rn(qp[1], ri), mul_rn(qp[2], ri), mul_rn(qp[3], ri)};
    const T pres = pres3(qp, kk.gam, ke3(qp, u[0], u[1], u[2]));
    // gradients of (u, v, w, T) from ring taps: grad3_at's sums
    const T *sk = ring + (size_t)(kq & (kM3Ring - 1)) * 4 * WN;
    T g[4][3];
    if (code == 0u) {
      T w[4];
      central_w(w);
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const T *pf = sk + f * WN + c;
        const T *rk = ring + (size_t)f * WN + c;
        g[f][0] = mul_rn(kk.ih[0], tap4(w, pf[-2], pf[-1], pf[1], pf[2]));
        g[f][1] = mul_rn(kk.ih[1], tap4(w, pf[-2 * WX], pf[-WX], pf[WX], pf[2 * WX]));
        g[f][2] = mul_rn(kk.ih[2], tap4(w, rk[(size_t)((kq - 2) & (kM3Ring - 1)) * 4 * WN],
                                         rk[(size_t)((kq - 1) & (kM3Ring - 1)) * 4 * WN],
                                         rk[(size_t)((kq + 1) & (kM3Ring - 1)) * 4 * WN],
                                         rk[(size_t)((kq + 2) & (kM3Ring - 1)) * 4 * WN]));
      }
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const Row<T> r = decode_row<T>((code >> (4 * d)) & 15u);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          T x[4];
#pragma unroll
          for (int e = 0; e < 4; ++e)
            x[e] = d == 0   ? sk[f * WN + c + r.off[e]]
                   : d == 1 ? sk[f * WN + c + r.off[e] * WX]
                            : ring[((size_t)((kq + r.off[e]) & (kM3Ring - 1)) * 4 + f) * WN + c];
          const T acc = tap4(r.w, x[0], x[1], x[2], x[3]);
          g[f][d] = mul_rn(kk.ih[d], r.neg ? -acc : acc);
        }
      }
    }
    T tau[3][3];
    tau3(kk, g, tau);
    const T vel[3] = {sk[c], sk[WN + c], sk[2 * WN + c]};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T Fd[5];
      flux3_dir<T, true>(kk, qp, u, pres, tau, g, vel, d, Fd);
#pragma unroll
      for (int v = 0; v < 5; ++v) fl[(5 * d + v) * m.field + p] = Fd[v];
    }
  }
}

template <typename T>
struct Upd3M {
  static constexpr int FX = kM3X + 6, FN = kM3Y * FX;   // i-flux tile: 8 rows x 38
  static constexpr int GN = (kM3Y + 6) * kM3X;          // j-flux tile: 14 rows x 32
  static constexpr int HN = kM3X * kM3Y;                // k-flux of the own columns
  static constexpr int BUF = 5 * (FN + GN);
  static constexpr size_t bytes = (size_t)(2 * BUF + kM3Ring * 5 * HN) * sizeof(T);
};

template <typename T, bool SPONGE>
__global__ void __launch_bounds__(256) k3_updm(const Rhs3Launch a, int chunk) {
  using U = Upd3M<T>;
  constexpr int FX = U::FX, FN = U::FN, GN = U::GN, HN = U::HN, BUF = U::BUF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *bufs = reinterpret_cast<T *>(smem_raw);  // [2][5 * FN (i-flux) + 5 * GN (j-flux)]
  T *hring = bufs + 2 * BUF;                   // [slot][5][HN]
  const Dev3Mesh &m = a.m;
  const K3<T> &kk = kc3<T>(a);
  const T *fl = static_cast<const T *>(a.flux);
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int i0 = blockIdx.x * kM3X, j0 = blockIdx.y * kM3Y;
  const int k0 = blockIdx.z * chunk, k1 = min(k0 + chunk, m.nk);
  const size_t plane = (size_t)m.nj * m.pitch;
  // plane offsets of this thread's items (-1 outside the mesh): i-flux tile (2), j-flux tile (2),
  // own column
  int fo[2], go[2];
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int w = tid + 256 * it;
    fo[it] = go[it] = -1;
    if (w < FN) {
      int gi = i0 - 3 + w % FX, gj = j0 + w / FX;
      if (wrap_index(gi, m.ni, m.per[0]) & (gj < m.nj)) fo[it] = gj * m.pitch + gi;
    }
    if (w < GN) {
      int gi = i0 + w % kM3X, gj = j0 - 3 + w / kM3X;
      if ((gi < m.ni) & wrap_index(gj, m.nj, m.per[1])) go[it] = gj * m.pitch + gi;
    }
  }
  const int gi = i0 + tx, gj = j0 + ty;
  const bool own = gi < m.ni && gj < m.nj;
  const int oo = own ? gj * m.pitch + gi : -1;
  auto fetch_ij = [&](int kp, int b) {  // i- and j-flux tiles of plane kp (inside the mesh)
    T *fb = bufs + b * BUF, *gb = fb + 5 * FN;
    const size_t base = (size_t)kp * plane;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int w = tid + 256 * it;
      if (fo[it] >= 0) {
#pragma unroll
        for (int v = 0; v < 5; ++v) cp_async_n<sizeof(T)>(fb + v * FN + w, fl + v * m.field + base + fo[it]);
      }
      if (go[it] >= 0) {
#pragma unroll
        for (int v = 0; v < 5; ++v) cp_async_n<sizeof(T)>(gb + v * GN + w, fl + (5 + v) * m.field + base + go[it]);
      }
    }
  };
  auto fetch_k = [&](int kp) {  // k-flux of the own column at (unwrapped) plane kp
    int kg = kp;
    if (oo < 0 || !wrap_index(kg, m.nk, m.per[2])) return;
    T *hb = hring + (size_t)(kp & (kM3Ring - 1)) * 5 * HN;
    const size_t pp = (size_t)kg * plane + oo;
#pragma unroll
    for (int v = 0; v < 5; ++v) cp_async_n<sizeof(T)>(hb + v * HN + tid, fl + (10 + v) * m.field + pp);
  };
  for (int kp = k0 - 3; kp <= k0 + 3; ++kp) fetch_k(kp);
  fetch_ij(k0, 0);
  cp_async_commit();
  const T *satb = static_cast<const T *>(a.sat);
  for (int kq = k0; kq < k1; ++kq) {
    cp_async_wait<0>();
    __syncthreads();
    // the next plane's tiles go to the other buffer (read last by plane kq - 1) and the ring
    // slot of plane kq + 4 (plane kq - 4, read last by plane kq - 1)
    if (kq + 1 < k1) {
      fetch_ij(kq + 1, (kq + 1 - k0) & 1);
      fetch_k(kq + 4);
    }
    cp_async_commit();
    if (!own) continue;
    const size_t p = (size_t)kq * plane + oo;
    const unsigned code = m.cls[p];
    const T *fb = bufs + ((kq - k0) & 1) * BUF, *gb = fb + 5 * FN;
    const int cf = ty * FX + tx + 3, cg = (ty + 3) * kM3X + tx;
    T rhs[5] = {T(0), T(0), T(0), T(0), T(0)};
    if ((code & 15u) != 15u) {
      T dsum[5] = {T(0), T(0), T(0), T(0), T(0)};
      if (code == 0u) {
        const int off[4] = {-2, -1, 1, 2};
        T w[4];
        central_w(w);
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            T x[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
              x[e] = d == 0   ? fb[v * FN + cf + off[e]]
                     : d == 1 ? gb[v * GN + cg + off[e] * kM3X]
                              : hring[((size_t)((kq + off[e]) & (kM3Ring - 1)) * 5 + v) * HN + tid];
            dsum[v] = fma_rn(kk.ih[d], tap4(w, x[0], x[1], x[2], x[3]), dsum[v]);
          }
      } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const Row<T> r = decode_row<T>((code >> (4 * d)) & 15u);
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            T x[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
              x[e] = d == 0   ? fb[v * FN + cf + r.off[e]]
                     : d == 1 ? gb[v * GN + cg + r.off[e] * kM3X]
                              : hring[((size_t)((kq + r.off[e]) & (kM3Ring - 1)) * 5 + v) * HN + tid];
            const T acc = tap4(r.w, x[0], x[1], x[2], x[3]);
            dsum[v] = fma_rn(kk.ih[d], r.neg ? -acc : acc, dsum[v]);
          }
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) rhs[v] = -dsum[v];
      const int row = kq * m.nj + gj;
      int lo = a.row_sat[row], hi = a.row_sat[row + 1];
      if (lo < hi) {
        const int64_t key = ((int64_t)kq * m.nj + gj) * m.ni + gi;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (a.sat_pt[mid] < key) lo = mid + 1;
          else hi = mid;
        }
        if (lo < a.row_sat[row + 1] && a.sat_pt[lo] == key) {
#pragma unroll
          for (int v = 0; v < 5; ++v) rhs[v] += satb[v * a.nsat + lo];
        }
      }
      if constexpr (SPONGE) sponge3(a, kk, gi, gj, kq, p, rhs);
    }
    T *out = static_cast<T *>(a.out);
    if (a.mode == 0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) out[v * m.field + p] = rhs[v];
    } else {
      const T *q = static_cast<const T *>(a.q);
      T *qn = static_cast<T *>(a.qnext);
      T q0[5], qv[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) q0[v] = q[v * m.field + p];
      ab_update<T, 5>(q0, a.hold, a.alpha, a.nold, m.field, p, rhs, qv, (code & 15u) != 15u ? a.err : nullptr);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        out[v * m.field + p] = rhs[v];
        qn[v * m.field + p] = qv[v];
      }
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void set_state3(const Donor3Launch &a, int set, size_t p, T out[5]) {
  const T *q = static_cast<const T *>(a.q);
  double acc[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) acc[v] = to_f64(q[v * a.d.field + p]);
  // each history slot's five values loaded together (the same sums in the same order)
#pragma unroll
  for (int k = 0; k < kMaxHist; ++k) {
    if (k < a.nb[set]) {
      const T *h = static_cast<const T *>(a.hist[k]) + p;
      T hv[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) hv[v] = h[v * a.d.field];
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] += a.beta[set][k] * to_f64(hv[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) out[v] = (T)acc[v];
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
    T pn[4][4];
    for (int e = 0; e < 4; ++e) {
      T sn[5];
      set_state3(a, set, idx[e], sn);
      prim5(sn, kk.gam, pn[e]);
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const T acc = tap4(r.w, pn[0][f], pn[1][f], pn[2][f], pn[3][f]);
      g[f][d] = mul_rn(kk.ih[d], r.neg ? -acc : acc);
    }
  }
  T pc[4], tau[3][3];
  prim5(s, kk.gam, pc);
  tau3(kk, g, tau);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int c = 0; c < 3; ++c) dv[(5 + 4 * d + c) * a.npts + dp] = tau[d][c];
    dv[(5 + 4 * d + 3) * a.npts + dp] = evisc3(kk, tau, g, pc, d);
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
        const int d = checked_index(a.didx[64 * r + (c3 * 4 + b) * 4 + e], a.ndv, a.err);
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
static cudaError_t march3_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k3_fluxm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Flux3M<T>::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k3_updm<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Upd3M<T>::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k3_updm<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Upd3M<T>::bytes);
  done = e == cudaSuccess;
  return e;
}

template <typename T>
static cudaError_t launch3_rhs_t(const Rhs3Launch &a, cudaStream_t s) {
  const Dev3Mesh &m = a.m;
  dim3 blk(32, 8), grid((m.ni + 31) / 32, (m.nj + 7) / 8, m.nk);
  const bool march = a.kchunk > 0;
  if (march) {
    cudaError_t e = march3_attrs<T>();
    if (e != cudaSuccess) return e;
  }
  dim3 mgrid((m.ni + kM3X - 1) / kM3X, (m.nj + kM3Y - 1) / kM3Y, march ? (m.nk + a.kchunk - 1) / a.kchunk : 1);
  if (a.visc && march) {
    k3_fluxm<T><<<mgrid, 256, Flux3M<T>::bytes, s>>>(a, a.kchunk);
  } else {
    if (a.visc) k3_prim<T><<<grid, blk, 0, s>>>(a);
    if (a.visc) k3_flux<T, true><<<grid, blk, 0, s>>>(a);
    else k3_flux<T, false><<<grid, blk, 0, s>>>(a);
  }
  if (a.nsat > 0) {
    const int blocks = (a.nsat + 31) / 32;
    if (a.visc && march) k3_sat<T, true, true><<<blocks, 32, 0, s>>>(a);
    else if (a.visc) k3_sat<T, true, false><<<blocks, 32, 0, s>>>(a);
    else k3_sat<T, false, false><<<blocks, 32, 0, s>>>(a);
  }
  const bool sponge = (sizeof(T) == 4 ? a.cf.sponge_d : a.cd.sponge_d) > 0;
  if (march && sponge) k3_updm<T, true><<<mgrid, 256, Upd3M<T>::bytes, s>>>(a, a.kchunk);
  else if (march) k3_updm<T, false><<<mgrid, 256, Upd3M<T>::bytes, s>>>(a, a.kchunk);
  else if (sponge) k3_update<T, true><<<grid, blk, 0, s>>>(a);
  else k3_update<T, false><<<grid, blk, 0, s>>>(a);
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
