// Discrete adjoint (FP64) of the right-hand side, of the interface interpolation and of the
// probe-pressure objective. The right-hand side is R(q) = -J (D_xi F^_xi + D_eta F^_eta) + SAT
// with pointwise fluxes F^(q, g) of the state and of the velocity / temperature gradients
// g = chain(D P(q)); its adjoint applies, in reverse order,
//   mu = -D^T (J lam)                          transposed SBP stencils (k_adj_mu)
//   lq += (dF^/dq)^T mu,  lg = (dF^/dg)^T mu   exact local Jacobians (k_adj_point)
//   SAT terms at boundary / receiver points    exact local Jacobians (k_adj_sat)
//   lP = D^T chain^T lg                         transposed SBP stencils (k_adj_dT)
//   lq += (dP/dq)^T lP                          exact local Jacobian (k_adj_prim)
// Local Jacobians come from forward-mode dual numbers evaluated on the same pointwise formulas
// as the forward kernels (one pass per input). All reductions are gathers (no atomics), so the
// results are deterministic.
#include <cuda_runtime.h>

#include <algorithm>

#include "sbp_dev.cuh"

namespace sbp {

// Forward-mode dual number: a value and one directional derivative.
struct Dd {
  double v, d;
  __host__ __device__ Dd(double x = 0.0, double y = 0.0) : v(x), d(y) {}
};
__device__ __forceinline__ Dd operator+(Dd a, Dd b) { return Dd(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dd operator-(Dd a, Dd b) { return Dd(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dd operator-(Dd a) { return Dd(-a.v, -a.d); }
__device__ __forceinline__ Dd operator*(Dd a, Dd b) { return Dd(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dd operator/(Dd a, Dd b) {
  double r = a.v / b.v;
  return Dd(r, (a.d - r * b.d) / b.v);
}
__device__ __forceinline__ Dd &operator+=(Dd &a, Dd b) { return a = a + b; }
__device__ __forceinline__ Dd &operator-=(Dd &a, Dd b) { return a = a - b; }
__device__ __forceinline__ Dd sqrt(Dd a) {
  double r = ::sqrt(a.v);
  return Dd(r, a.d / (2.0 * r));
}
// max(a, b) on the branch the values select; at a tie (the kink) the derivative is the mean of
// the two one-sided slopes, so that the characteristic splitting (positive part of a wave speed
// minus the positive part of its negative) still differentiates to the wave speed's derivative
// when the speed is exactly zero.
__device__ __forceinline__ Dd fmax(Dd a, Dd b) {
  return a.v > b.v ? a : (a.v < b.v ? b : Dd(a.v, 0.5 * (a.d + b.d)));
}

// ---------------------------------------------------------------------------------------------
// Pointwise functions of the forward kernels, on a generic scalar S (double or Dd).
template <typename S>
__device__ __forceinline__ void prims_of(const S q[4], double gam, S out[3]) {
  S ri = S(1.0) / q[0];
  S u = q[1] * ri, v = q[2] * ri;
  S pres = S(gam - 1.0) * (q[3] - S(0.5) * (q[1] * u + q[2] * v));
  out[0] = u;
  out[1] = v;
  out[2] = S(gam) * pres * ri;
}

template <typename S>
__device__ __forceinline__ void visc_of(const KConst<double> &k, S u, S v, const S g[6], S Fv[3], S Gv[3]) {
  S txx = S(k.mu43) * g[0] - S(k.mu23) * g[3];
  S tyy = S(k.mu43) * g[3] - S(k.mu23) * g[0];
  S txy = S(k.mu) * (g[1] + g[2]);
  Fv[0] = txx;
  Fv[1] = txy;
  Fv[2] = u * txx + v * txy + S(k.kap) * g[4];
  Gv[0] = txy;
  Gv[1] = tyy;
  Gv[2] = u * txy + v * tyy + S(k.kap) * g[5];
}

// Contravariant fluxes (F^_xi, F^_eta) of k_flux at one point.
template <typename S, bool VISC, bool CURV>
__device__ void flux_of(const KConst<double> &k, const double mt[5], const S q[4], const S g[6], S out[8]) {
  S F[4], G[4];
  if (VISC) {
    S pr[3];
    prims_of(q, k.gam, pr);
    S p = q[0] * pr[2] / S(k.gam);
    S Fv[3], Gv[3];
    visc_of(k, pr[0], pr[1], g, Fv, Gv);
    F[0] = q[1];
    F[1] = q[1] * pr[0] + p - Fv[0];
    F[2] = q[2] * pr[0] - Fv[1];
    F[3] = (q[3] + p) * pr[0] - Fv[2];
    G[0] = q[2];
    G[1] = q[1] * pr[1] - Gv[0];
    G[2] = q[2] * pr[1] + p - Gv[1];
    G[3] = (q[3] + p) * pr[1] - Gv[2];
  } else {
    S ri = S(1.0) / q[0];
    S u = q[1] * ri, v = q[2] * ri;
    S p = S(k.gam - 1.0) * (q[3] - S(0.5) * (q[1] * u + q[2] * v));
    F[0] = q[1];
    F[1] = q[1] * u + p;
    F[2] = q[2] * u;
    F[3] = (q[3] + p) * u;
    G[0] = q[2];
    G[1] = q[1] * v;
    G[2] = q[2] * v + p;
    G[3] = (q[3] + p) * v;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (CURV) {
      out[c] = S(mt[0]) * F[c] + S(mt[1]) * G[c];
      out[4 + c] = S(mt[2]) * F[c] + S(mt[3]) * G[c];
    } else {
      out[c] = S(mt[0]) * F[c];
      out[4 + c] = S(mt[3]) * G[c];
    }
  }
}

// SAT terms of one point (the forward's sat_terms) as a function of the state, the own
// gradients, the receiver values rv (state, then viscous fluxes) and the far-field state.
template <typename S, bool VISC>
__device__ void sat_of(const KConst<double> &k, const double mt[5], uint32_t code, double scale, const S q[4],
                       const S g[6], const S rv[10], const S qinf[4], S out[4]) {
  S Fv[3] = {S(0), S(0), S(0)}, Gv[3] = {S(0), S(0), S(0)};
  if (VISC) {
    S pr[3];
    prims_of(q, k.gam, pr);
    visc_of(k, pr[0], pr[1], g, Fv, Gv);
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) out[v] = S(0);
  int nt = code & 7u;
  for (int t = 0; t < nt; ++t) {
    unsigned term = (code >> (3 + 4 * t)) & 15u;
    int dir = term & 1u, side = (term & 2u) ? -1 : 1, kind = (int)(term >> 2);
    double kxd = mt[4] * mt[2 * dir], kyd = mt[4] * mt[2 * dir + 1];
    S kx(kxd), ky(kyd);
    S tgt[4];
    S sig1(0.0);
    S sigI(kind == kTermInterface ? k.sig_int : k.sig_phys);
    if (kind == kTermInterface) {
#pragma unroll
      for (int v = 0; v < 4; ++v) tgt[v] = rv[v];
      if (VISC) sig1 = S(0.5 * k.mu * (kxd * kxd + kyd * kyd));
    } else if (kind == kTermFarfield) {
#pragma unroll
      for (int v = 0; v < 4; ++v) tgt[v] = qinf[v];
    } else {
      tgt[0] = q[0];
      tgt[1] = S(0);
      tgt[2] = S(0);
      tgt[3] = q[0] * S(k.tw);
      if (VISC) sig1 = S(0.5 * k.mu * (kxd * kxd + kyd * kyd));
    }
    S dq[4], kd[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) dq[v] = q[v] - tgt[v];
    penalty_apply(q, S(k.gam), kx, ky, side, dq, kd);
    S sat[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) sat[v] = -(sigI * kd[v] + sig1 * dq[v]) * S(1.0 / SBP_P0);
    if (VISC && kind == kTermInterface) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        S own = kx * Fv[c] + ky * Gv[c];
        S hat = kx * rv[4 + c] + ky * rv[7 + c];
        sat[c + 1] += S(0.5) * S((double)side) * (own - hat) * S(1.0 / SBP_P0);
      }
    }
    S sc(kind == kTermInterface ? scale : 1.0);
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] += sc * sat[v];
  }
}

// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void metrics_at(const DevMesh &m, size_t p, double mt[5]) {
  if (m.cart) {
#pragma unroll
    for (int c = 0; c < 5; ++c) mt[c] = m.mc[c];
  } else {
    const double *met = static_cast<const double *>(m.met);
#pragma unroll
    for (int c = 0; c < 5; ++c) mt[c] = met[c * m.field + p];
  }
}

// Cartesian gradients g (6) at (i, j) of primitives (u, v, T) given point-wise by prim_at,
// through the point's derivative rows and metrics.
template <typename PF>
__device__ void grads_gen(const DevMesh &m, int i, int j, PF prim_at, double g[6]) {
  size_t p = (size_t)j * m.pitch + i;
  unsigned code = m.cls[p];
  double dxi[3] = {0, 0, 0}, deta[3] = {0, 0, 0};
  for (int dir = 0; dir < 2; ++dir) {
    int row, sgn;
    row_of(dir == 0 ? (code & 15u) : (code >> 4), row, sgn);
    for (int e = 0; e < 4; ++e) {
      double we = c_w64[row][e];
      if (we == 0.0) continue;
      int ii = i, jj = j;
      if (dir == 0) ii += sgn * c_off[row][e];
      else jj += sgn * c_off[row][e];
      wrap_index(ii, m.ni, m.per_i);
      wrap_index(jj, m.nj, m.per_j);
      double pr[3];
      prim_at((size_t)jj * m.pitch + ii, pr);
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        if (dir == 0) dxi[f] += sgn * we * pr[f];
        else deta[f] += sgn * we * pr[f];
      }
    }
  }
  double mt[5];
  metrics_at(m, p, mt);
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    if (m.cart) {
      g[2 * f] = mt[4] * mt[0] * dxi[f];
      g[2 * f + 1] = mt[4] * mt[3] * deta[f];
    } else {
      g[2 * f] = mt[4] * (mt[0] * dxi[f] + mt[2] * deta[f]);
      g[2 * f + 1] = mt[4] * (mt[1] * dxi[f] + mt[3] * deta[f]);
    }
  }
}

// Gradients of the primitives of the state q.
__device__ void grads_at(const DevMesh &m, const double *q, double gam, int i, int j, double g[6]) {
  grads_gen(m, i, j,
            [&](size_t pn, double pr[3]) {
              double qq[4] = {q[pn], q[m.field + pn], q[2 * m.field + pn], q[3 * m.field + pn]};
              prims_of(qq, gam, pr);
            },
            g);
}

// Gradients of primitives stored as 3 planes (u, v, T or their tangents).
__device__ void grads_planes(const DevMesh &m, const double *pl, int i, int j, double g[6]) {
  grads_gen(m, i, j,
            [&](size_t pn, double pr[3]) {
              pr[0] = pl[pn];
              pr[1] = pl[m.field + pn];
              pr[2] = pl[2 * m.field + pn];
            },
            g);
}

// Adjoint of the gradient chain: lg (6 Cartesian) -> adjoint of (D_xi P, D_eta P) (6 planes
// ordered u_xi, u_eta, v_xi, v_eta, T_xi, T_eta).
__device__ __forceinline__ void chain_adjoint(const double mt[5], bool cart, const double lg[6], double ldp[6]) {
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    if (cart) {
      ldp[2 * f] = mt[4] * mt[0] * lg[2 * f];
      ldp[2 * f + 1] = mt[4] * mt[3] * lg[2 * f + 1];
    } else {
      ldp[2 * f] = mt[4] * (mt[0] * lg[2 * f] + mt[1] * lg[2 * f + 1]);
      ldp[2 * f + 1] = mt[4] * (mt[2] * lg[2 * f] + mt[3] * lg[2 * f + 1]);
    }
  }
}

// Transposed stencil: the coefficient that the derivative row (direction dir) of the point at
// offset o from (i, j) gives to (i, j), and that point's index pj (0 when out of the mesh or when
// its row does not reach (i, j)). A non-zero tap has a unique offset, so at most one matches.
__device__ __forceinline__ double tcoef(const DevMesh &m, int i, int j, int dir, int o, size_t &pj) {
  const int n = dir == 0 ? m.ni : m.nj;
  const int per = dir == 0 ? m.per_i : m.per_j;
  int c = (dir == 0 ? i : j) + o;
  if (!wrap_index(c, n, per)) return 0.0;
  pj = dir == 0 ? (size_t)j * m.pitch + c : (size_t)c * m.pitch + i;
  unsigned code = m.cls[pj];
  code = dir == 0 ? (code & 15u) : (code >> 4);
  int row, sgn;
  row_of(code, row, sgn);
  double cf = 0.0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const double we = c_w64[row][e];
    if (we != 0.0 && sgn * c_off[row][e] == -o) cf = sgn * we;
  }
  return cf;
}

// mu = -D^T (J lam): 8 planes (xi: 4 variables, eta: 4 variables); each neighbour's row is
// decoded once for all variables.
__global__ void k_adj_mu(const AdjLaunch a) {
  const DevMesh &m = a.m;
  size_t n = (size_t)m.ni * m.nj;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % m.ni), j = (int)(t / m.ni);
    size_t p = (size_t)j * m.pitch + i;
    for (int dir = 0; dir < 2; ++dir) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int o = -3; o <= 3; ++o) {
        size_t pj = 0;
        const double cf = tcoef(m, i, j, dir, o, pj);
        if (cf == 0.0) continue;
        const double jac = m.cart ? m.mc[4] : static_cast<const double *>(m.met)[4 * m.field + pj];
        const double x = cf * jac;
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += x * a.lam[c * m.field + pj];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) a.mu[(dir * 4 + c) * m.field + p] = -acc[c];
    }
  }
}

template <bool VISC, bool CURV>
__global__ void k_adj_point(const AdjLaunch a) {
  const DevMesh &m = a.m;
  size_t n = (size_t)m.ni * m.nj;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % m.ni), j = (int)(t / m.ni);
    size_t p = (size_t)j * m.pitch + i;
    if ((m.cls[p] & 15u) == 15u) {
      for (int c = 0; c < 6; ++c) a.ld[c * m.field + p] = 0.0;
      continue;
    }
    double mt[5];
    metrics_at(m, p, mt);
    double q[4] = {a.q[p], a.q[m.field + p], a.q[2 * m.field + p], a.q[3 * m.field + p]};
    double g[6] = {0, 0, 0, 0, 0, 0};
    if (VISC) grads_at(m, a.q, a.k.gam, i, j, g);
    double mu[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) mu[c] = a.mu[c * m.field + p];
    constexpr int NIN = VISC ? 10 : 4;
    double lin[NIN];
    for (int s = 0; s < NIN; ++s) {
      Dd qd[4], gd[6], out[8];
#pragma unroll
      for (int b = 0; b < 4; ++b) qd[b] = Dd(q[b], s == b ? 1.0 : 0.0);
#pragma unroll
      for (int b = 0; b < 6; ++b) gd[b] = Dd(g[b], s == 4 + b ? 1.0 : 0.0);
      flux_of<Dd, VISC, CURV>(a.k, mt, qd, gd, out);
      double acc = 0.0;
#pragma unroll
      for (int o = 0; o < 8; ++o) acc += out[o].d * mu[o];
      lin[s] = acc;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) a.lq[c * m.field + p] += lin[c];
    if (VISC) {
      double lg[6], ldp[6];
#pragma unroll
      for (int b = 0; b < 6; ++b) lg[b] = lin[4 + b];
      chain_adjoint(mt, !CURV, lg, ldp);
#pragma unroll
      for (int b = 0; b < 6; ++b) a.ld[b * m.field + p] = ldp[b];
    }
  }
}

// SAT adjoint in two passes: one thread per (SAT point, input) evaluates the dual-number
// derivative of the point's SAT terms along that input (inputs: q 4, g 6, rv 10, qinf 4) and
// stores lam . dSAT/d(input); then one thread per SAT point applies the 24 values.
template <bool VISC, bool CURV>
__global__ void k_adj_sat(const AdjLaunch a) {
  const DevMesh &m = a.m;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 24 * a.nsat) return;
  const int s = t / 24, in = t - 24 * s;
  const int recv = a.sat_recv[s];
  if ((!VISC && in >= 4 && in < 10) || (recv < 0 && in >= 10 && in < 20)) {
    a.satlin[t] = 0.0;
    return;
  }
  uint32_t ij = a.sat_ij[s];
  int i = (int)(ij & 0xFFFFu), j = (int)(ij >> 16);
  size_t p = (size_t)j * m.pitch + i;
  double mt[5];
  metrics_at(m, p, mt);
  double q[4] = {a.q[p], a.q[m.field + p], a.q[2 * m.field + p], a.q[3 * m.field + p]};
  double g[6] = {0, 0, 0, 0, 0, 0};
  if (VISC) grads_at(m, a.q, a.k.gam, i, j, g);
  double rv[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (recv >= 0)
    for (int c = 0; c < 10; ++c) rv[c] = a.rv[(size_t)c * a.nrecv + recv];
  Dd qd[4], gd[6], rd[10], fd[4], out[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) qd[b] = Dd(q[b], in == b ? 1.0 : 0.0);
#pragma unroll
  for (int b = 0; b < 6; ++b) gd[b] = Dd(g[b], in == 4 + b ? 1.0 : 0.0);
#pragma unroll
  for (int b = 0; b < 10; ++b) rd[b] = Dd(rv[b], in == 10 + b ? 1.0 : 0.0);
#pragma unroll
  for (int b = 0; b < 4; ++b) fd[b] = Dd(a.k.qinf[b], in == 20 + b ? 1.0 : 0.0);
  sat_of<Dd, VISC>(a.k, mt, a.sat_code[s], a.sat_scale[s], qd, gd, rd, fd, out);
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) acc += out[c].d * a.lam[c * m.field + p];
  a.satlin[t] = acc;
}

template <bool CURV>
__global__ void k_adj_sat_apply(const AdjLaunch a) {
  const DevMesh &m = a.m;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.nsat) return;
  const double *lin = a.satlin + 24 * (size_t)s;
  uint32_t ij = a.sat_ij[s];
  int i = (int)(ij & 0xFFFFu), j = (int)(ij >> 16);
  size_t p = (size_t)j * m.pitch + i;
#pragma unroll
  for (int c = 0; c < 4; ++c) a.lq[c * m.field + p] += lin[c];
  if (a.viscous) {
    double mt[5], ldp[6];
    metrics_at(m, p, mt);
    chain_adjoint(mt, !CURV, lin + 4, ldp);
#pragma unroll
    for (int b = 0; b < 6; ++b) a.ld[b * m.field + p] += ldp[b];
  }
  const int recv = a.sat_recv[s];
  if (recv >= 0)
    for (int c = 0; c < 10; ++c) a.lrv[(size_t)c * a.nrecv + recv] = lin[10 + c];
#pragma unroll
  for (int c = 0; c < 4; ++c) a.lqinf[(size_t)4 * s + c] = lin[20 + c];
}

// lp (3 planes) = D_xi^T ld(xi) + D_eta^T ld(eta) for u, v, T.
__global__ void k_adj_dT(const DevMesh m, const double *ld, double *lp) {
  size_t n = (size_t)m.ni * m.nj;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % m.ni), j = (int)(t / m.ni);
    size_t p = (size_t)j * m.pitch + i;
    double acc[3][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    for (int dir = 0; dir < 2; ++dir)
      for (int o = -3; o <= 3; ++o) {
        size_t pj = 0;
        const double cf = tcoef(m, i, j, dir, o, pj);
        if (cf == 0.0) continue;
#pragma unroll
        for (int f = 0; f < 3; ++f) acc[f][dir] += cf * ld[(2 * f + dir) * m.field + pj];
      }
#pragma unroll
    for (int f = 0; f < 3; ++f) lp[f * m.field + p] = acc[f][0] + acc[f][1];
  }
}

// lq += (dP/dq)^T lp at active points, P = (u, v, T) of the state q.
__global__ void k_adj_prim(const DevMesh m, double gam, const double *q, const double *lp, double *lq) {
  size_t n = (size_t)m.ni * m.nj;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % m.ni), j = (int)(t / m.ni);
    size_t p = (size_t)j * m.pitch + i;
    if ((m.cls[p] & 15u) == 15u) continue;
    double l[3] = {lp[p], lp[m.field + p], lp[2 * m.field + p]};
    if (l[0] == 0.0 && l[1] == 0.0 && l[2] == 0.0) continue;
    double qv[4] = {q[p], q[m.field + p], q[2 * m.field + p], q[3 * m.field + p]};
    for (int s = 0; s < 4; ++s) {
      Dd qd[4], pr[3];
#pragma unroll
      for (int b = 0; b < 4; ++b) qd[b] = Dd(qv[b], s == b ? 1.0 : 0.0);
      prims_of(qd, gam, pr);
      lq[s * m.field + p] += pr[0].d * l[0] + pr[1].d * l[1] + pr[2].d * l[2];
    }
  }
}

cudaError_t launch_rhs_adjoint(const AdjLaunch &a, cudaStream_t s) {
  size_t n = (size_t)a.m.ni * a.m.nj;
  int blocks = (int)std::min<size_t>((n + 127) / 128, 152 * 16);
  k_adj_mu<<<blocks, 128, 0, s>>>(a);
  bool curv = !a.m.cart;
  if (a.viscous) {
    if (curv) k_adj_point<true, true><<<blocks, 128, 0, s>>>(a);
    else k_adj_point<true, false><<<blocks, 128, 0, s>>>(a);
  } else {
    if (curv) k_adj_point<false, true><<<blocks, 128, 0, s>>>(a);
    else k_adj_point<false, false><<<blocks, 128, 0, s>>>(a);
  }
  if (a.nsat > 0) {
    int sb = (24 * a.nsat + 63) / 64;
    if (a.viscous) {
      if (curv) k_adj_sat<true, true><<<sb, 64, 0, s>>>(a);
      else k_adj_sat<true, false><<<sb, 64, 0, s>>>(a);
    } else {
      if (curv) k_adj_sat<false, true><<<sb, 64, 0, s>>>(a);
      else k_adj_sat<false, false><<<sb, 64, 0, s>>>(a);
    }
    int ab = (a.nsat + 63) / 64;
    if (curv) k_adj_sat_apply<true><<<ab, 64, 0, s>>>(a);
    else k_adj_sat_apply<false><<<ab, 64, 0, s>>>(a);
  }
  if (a.viscous) {
    k_adj_dT<<<blocks, 128, 0, s>>>(a.m, a.ld, a.lp);
    k_adj_prim<<<blocks, 128, 0, s>>>(a.m, a.k.gam, a.q, a.lp, a.lq);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Receiver values -> donor points -> donor state.
__global__ void k_adj_gather_dv(const AdjDonorLaunch a) {
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < a.npts; d += gridDim.x * blockDim.x) {
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = a.inv_off[d]; t < a.inv_off[d + 1]; ++t) {
      int re = a.inv_re[t], r = re >> 4, sl = re & 15;
      double w = a.w[8 * r + (sl & 3)] * a.w[8 * r + 4 + (sl >> 2)];
      for (int c = 0; c < 10; ++c) acc[c] += w * a.lrv[(size_t)c * a.nrecv + r];
    }
    for (int c = 0; c < 10; ++c) a.ldv[(size_t)c * a.npts + d] = acc[c];
  }
}

template <bool CURV>
__global__ void k_adj_dvpoint(const AdjDonorLaunch a, int viscous) {
  const DevMesh &m = a.d;
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < a.npts; d += gridDim.x * blockDim.x) {
    uint32_t ij = a.pts[d];
    int i = (int)(ij & 0xFFFFu), j = (int)(ij >> 16);
    size_t p = (size_t)j * m.pitch + i;
    double lsv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) lsv[c] = a.ldv[(size_t)c * a.npts + d];
    if (viscous) {
      double mt[5];
      metrics_at(m, p, mt);
      double q[4] = {a.shat[p], a.shat[m.field + p], a.shat[2 * m.field + p], a.shat[3 * m.field + p]};
      double g[6];
      grads_at(m, a.shat, a.k.gam, i, j, g);
      double mu[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) mu[c] = a.ldv[(size_t)(4 + c) * a.npts + d];
      double lin[10];
      for (int s = 0; s < 10; ++s) {
        Dd qd[4], gd[6], pr[3], Fv[3], Gv[3];
#pragma unroll
        for (int b = 0; b < 4; ++b) qd[b] = Dd(q[b], s == b ? 1.0 : 0.0);
#pragma unroll
        for (int b = 0; b < 6; ++b) gd[b] = Dd(g[b], s == 4 + b ? 1.0 : 0.0);
        prims_of(qd, a.k.gam, pr);
        visc_of(a.k, pr[0], pr[1], gd, Fv, Gv);
        lin[s] = Fv[0].d * mu[0] + Fv[1].d * mu[1] + Fv[2].d * mu[2] + Gv[0].d * mu[3] + Gv[1].d * mu[4] +
                 Gv[2].d * mu[5];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) lsv[c] += lin[c];
      double ldp[6];
      chain_adjoint(mt, !CURV, lin + 4, ldp);
#pragma unroll
      for (int b = 0; b < 6; ++b) a.ld[b * m.field + p] = ldp[b];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) a.lshat[c * m.field + p] += lsv[c];
  }
}

cudaError_t launch_donor_adjoint(const AdjDonorLaunch &a, cudaStream_t s) {
  if (a.npts == 0) return cudaSuccess;
  int b = (a.npts + 127) / 128;
  k_adj_gather_dv<<<b, 128, 0, s>>>(a);
  cudaError_t e;
  if (a.viscous) {
    if ((e = cudaMemsetAsync(a.ld, 0, 6 * a.d.field * sizeof(double), s)) != cudaSuccess) return e;
  }
  if (a.d.cart) k_adj_dvpoint<false><<<b, 128, 0, s>>>(a, a.viscous ? 1 : 0);
  else k_adj_dvpoint<true><<<b, 128, 0, s>>>(a, a.viscous ? 1 : 0);
  if (a.viscous) {
    size_t n = (size_t)a.d.ni * a.d.nj;
    int blocks = (int)std::min<size_t>((n + 127) / 128, 152 * 16);
    k_adj_dT<<<blocks, 128, 0, s>>>(a.d, a.ld, a.lp);
    k_adj_prim<<<blocks, 128, 0, s>>>(a.d, a.k.gam, a.shat, a.lp, a.lshat);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Probe pressures and the adjoint seed of sum_p p_p^2 (one thread: the probes share points).
__global__ void k_probe(const DevMesh m, const double *q, int nprobe, const int *base, const double *w, double *pout,
                        double *lq, double scale, double gam) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int pr = 0; pr < nprobe; ++pr) {
    double pv = 0.0;
    for (int b = 0; b < 4; ++b)
      for (int a = 0; a < 4; ++a) {
        int ii = base[2 * pr] + a, jj = base[2 * pr + 1] + b;
        wrap_index(ii, m.ni, m.per_i);
        wrap_index(jj, m.nj, m.per_j);
        size_t p = (size_t)jj * m.pitch + ii;
        double r = q[p], u = q[m.field + p] / r, v = q[2 * m.field + p] / r;
        double pres = (gam - 1.0) * (q[3 * m.field + p] - 0.5 * r * (u * u + v * v));
        pv += w[8 * pr + a] * w[8 * pr + 4 + b] * pres;
      }
    if (pout) pout[pr] = pv;
    if (!lq) continue;
    for (int b = 0; b < 4; ++b)
      for (int a = 0; a < 4; ++a) {
        int ii = base[2 * pr] + a, jj = base[2 * pr + 1] + b;
        wrap_index(ii, m.ni, m.per_i);
        wrap_index(jj, m.nj, m.per_j);
        size_t p = (size_t)jj * m.pitch + ii;
        double r = q[p], u = q[m.field + p] / r, v = q[2 * m.field + p] / r;
        double c = scale * 2.0 * pv * w[8 * pr + a] * w[8 * pr + 4 + b] * (gam - 1.0);
        lq[p] += c * 0.5 * (u * u + v * v);
        lq[m.field + p] -= c * u;
        lq[2 * m.field + p] -= c * v;
        lq[3 * m.field + p] += c;
      }
  }
}

cudaError_t launch_probe(const DevMesh &m, const double *q, int nprobe, const int *base, const double *w,
                         double *pout, double *lq, double scale, double gamma, cudaStream_t s) {
  k_probe<<<1, 32, 0, s>>>(m, q, nprobe, base, w, pout, lq, scale, gamma);
  return cudaGetLastError();
}

}  // namespace sbp

namespace sbp {

// out = base + sum_k c[k] x[k] over n doubles (out may alias base).
__global__ void k_lincomb(double *out, const double *base, int nx, LinComb lc, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    double acc = base ? base[t] : 0.0;
    for (int k = 0; k < nx; ++k) acc += lc.c[k] * lc.x[k][t];
    out[t] = acc;
  }
}

cudaError_t launch_lincomb(double *out, const double *base, const LinComb &lc, int nx, size_t n, cudaStream_t s) {
  int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
  k_lincomb<<<blocks, 256, 0, s>>>(out, base, nx, lc, n);
  return cudaGetLastError();
}

// acc[c] += sum_s x[4 s + c], c < 4 (one block, fixed order: deterministic).
__global__ void k_sum4(const double *x, int n, double *acc) {
  __shared__ double part[256][4];
  double s4[4] = {0, 0, 0, 0};
  for (int s = threadIdx.x; s < n; s += blockDim.x)
    for (int c = 0; c < 4; ++c) s4[c] += x[4 * s + c];
  for (int c = 0; c < 4; ++c) part[threadIdx.x][c] = s4[c];
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += part[i][threadIdx.x];
    acc[threadIdx.x] += t;
  }
}

cudaError_t launch_sum4(const double *x, int n, double *acc, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_sum4<<<1, 256, 0, s>>>(x, n, acc);
  return cudaGetLastError();
}

}  // namespace sbp

// ---------------------------------------------------------------------------------------------
// Tangent (forward-mode) right-hand side: one dual pass per point along the given direction.
namespace sbp {

// pd (3 planes) = dP/dq qd for P = (u, v, T).
__global__ void k_tl_prim(const DevMesh m, double gam, const double *q, const double *qd, double *pd) {
  size_t n = (size_t)m.ni * m.nj;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % m.ni), j = (int)(t / m.ni);
    size_t p = (size_t)j * m.pitch + i;
    Dd qq[4], pr[3];
#pragma unroll
    for (int b = 0; b < 4; ++b) qq[b] = Dd(q[b * m.field + p], qd[b * m.field + p]);
    prims_of(qq, gam, pr);
#pragma unroll
    for (int f = 0; f < 3; ++f) pd[f * m.field + p] = pr[f].d;
  }
}

// Tangent of the receiver values: state part I qd, viscous part I (dF^V/dq qd + dF^V/dg gd).
template <bool VISC>
__global__ void k_tl_recv(const TlDonorLaunch a) {
  const DevMesh &m = a.d;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.nrecv; r += gridDim.x * blockDim.x) {
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) {
        int ii = a.base[2 * r] + c, jj = a.base[2 * r + 1] + b;
        wrap_index(ii, m.ni, m.per_i);
        wrap_index(jj, m.nj, m.per_j);
        size_t p = (size_t)jj * m.pitch + ii;
        double w = a.w[8 * r + c] * a.w[8 * r + 4 + b];
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] += w * a.qd[v * m.field + p];
        if (VISC) {
          double g[6], gd[6];
          grads_at(m, a.q, a.k.gam, ii, jj, g);
          grads_planes(m, a.pd, ii, jj, gd);
          Dd qq[4], gg[6], pr[3], Fv[3], Gv[3];
#pragma unroll
          for (int v = 0; v < 4; ++v) qq[v] = Dd(a.q[v * m.field + p], a.qd[v * m.field + p]);
#pragma unroll
          for (int v = 0; v < 6; ++v) gg[v] = Dd(g[v], gd[v]);
          prims_of(qq, a.k.gam, pr);
          visc_of(a.k, pr[0], pr[1], gg, Fv, Gv);
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            acc[4 + v] += w * Fv[v].d;
            acc[7 + v] += w * Gv[v].d;
          }
        }
      }
    for (int c = 0; c < 10; ++c) a.rvd[(size_t)c * a.nrecv + r] = acc[c];
  }
}

// fd (8 planes) = tangent of the contravariant fluxes.
template <bool VISC, bool CURV>
__global__ void k_tl_flux(const TlLaunch a) {
  const DevMesh &m = a.m;
  size_t n = (size_t)m.ni * m.nj;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % m.ni), j = (int)(t / m.ni);
    size_t p = (size_t)j * m.pitch + i;
    if ((m.cls[p] & 15u) == 15u) {
      for (int c = 0; c < 8; ++c) a.fd[c * m.field + p] = 0.0;
      continue;
    }
    double mt[5];
    metrics_at(m, p, mt);
    double g[6] = {0, 0, 0, 0, 0, 0}, gd[6] = {0, 0, 0, 0, 0, 0};
    if (VISC) {
      grads_at(m, a.q, a.k.gam, i, j, g);
      grads_planes(m, a.pd, i, j, gd);
    }
    Dd qq[4], gg[6], out[8];
#pragma unroll
    for (int b = 0; b < 4; ++b) qq[b] = Dd(a.q[b * m.field + p], a.qd[b * m.field + p]);
#pragma unroll
    for (int b = 0; b < 6; ++b) gg[b] = Dd(g[b], gd[b]);
    flux_of<Dd, VISC, CURV>(a.k, mt, qq, gg, out);
#pragma unroll
    for (int c = 0; c < 8; ++c) a.fd[c * m.field + p] = out[c].d;
  }
}

// out = -J (D_xi fd_xi + D_eta fd_eta) at active points, 0 in holes.
__global__ void k_tl_div(const TlLaunch a) {
  const DevMesh &m = a.m;
  size_t n = (size_t)m.ni * m.nj;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % m.ni), j = (int)(t / m.ni);
    size_t p = (size_t)j * m.pitch + i;
    unsigned code = m.cls[p];
    if ((code & 15u) == 15u) {
      for (int c = 0; c < 4; ++c) a.out[c * m.field + p] = 0.0;
      continue;
    }
    double jac = m.cart ? m.mc[4] : static_cast<const double *>(m.met)[4 * m.field + p];
    double acc[4] = {0, 0, 0, 0};
    for (int dir = 0; dir < 2; ++dir) {
      int row, sgn;
      row_of(dir == 0 ? (code & 15u) : (code >> 4), row, sgn);
      for (int e = 0; e < 4; ++e) {
        double we = c_w64[row][e];
        if (we == 0.0) continue;
        int ii = i, jj = j;
        if (dir == 0) ii += sgn * c_off[row][e];
        else jj += sgn * c_off[row][e];
        wrap_index(ii, m.ni, m.per_i);
        wrap_index(jj, m.nj, m.per_j);
        size_t pn = (size_t)jj * m.pitch + ii;
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += sgn * we * a.fd[(dir * 4 + c) * m.field + pn];
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) a.out[c * m.field + p] = -jac * acc[c];
  }
}

template <bool VISC, bool CURV>
__global__ void k_tl_sat(const TlLaunch a) {
  const DevMesh &m = a.m;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.nsat; s += gridDim.x * blockDim.x) {
    uint32_t ij = a.sat_ij[s];
    int i = (int)(ij & 0xFFFFu), j = (int)(ij >> 16);
    size_t p = (size_t)j * m.pitch + i;
    double mt[5];
    metrics_at(m, p, mt);
    double g[6] = {0, 0, 0, 0, 0, 0}, gd[6] = {0, 0, 0, 0, 0, 0};
    if (VISC) {
      grads_at(m, a.q, a.k.gam, i, j, g);
      grads_planes(m, a.pd, i, j, gd);
    }
    int recv = a.sat_recv[s];
    Dd qq[4], gg[6], rr[10], ff[4], out[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) qq[b] = Dd(a.q[b * m.field + p], a.qd[b * m.field + p]);
#pragma unroll
    for (int b = 0; b < 6; ++b) gg[b] = Dd(g[b], gd[b]);
#pragma unroll
    for (int b = 0; b < 10; ++b)
      rr[b] = recv >= 0 ? Dd(a.rv[(size_t)b * a.nrecv + recv], a.rvd[(size_t)b * a.nrecv + recv]) : Dd(0.0, 0.0);
#pragma unroll
    for (int b = 0; b < 4; ++b) ff[b] = Dd(a.k.qinf[b], a.qinfd[b]);
    sat_of<Dd, VISC>(a.k, mt, a.sat_code[s], a.sat_scale[s], qq, gg, rr, ff, out);
#pragma unroll
    for (int c = 0; c < 4; ++c) a.out[c * m.field + p] += out[c].d;
  }
}

cudaError_t launch_rhs_tangent(const TlLaunch &a, const TlDonorLaunch &dn, cudaStream_t s) {
  size_t n = (size_t)a.m.ni * a.m.nj;
  int blocks = (int)std::min<size_t>((n + 127) / 128, 152 * 16);
  if (dn.nrecv > 0) {
    if (a.viscous) {
      size_t nd = (size_t)dn.d.ni * dn.d.nj;
      int bd = (int)std::min<size_t>((nd + 127) / 128, 152 * 16);
      k_tl_prim<<<bd, 128, 0, s>>>(dn.d, dn.k.gam, dn.q, dn.qd, dn.pd);
      k_tl_recv<true><<<(dn.nrecv + 63) / 64, 64, 0, s>>>(dn);
    } else {
      k_tl_recv<false><<<(dn.nrecv + 63) / 64, 64, 0, s>>>(dn);
    }
  }
  bool curv = !a.m.cart;
  if (a.viscous) k_tl_prim<<<blocks, 128, 0, s>>>(a.m, a.k.gam, a.q, a.qd, a.pd);
  if (a.viscous) {
    if (curv) k_tl_flux<true, true><<<blocks, 128, 0, s>>>(a);
    else k_tl_flux<true, false><<<blocks, 128, 0, s>>>(a);
  } else {
    if (curv) k_tl_flux<false, true><<<blocks, 128, 0, s>>>(a);
    else k_tl_flux<false, false><<<blocks, 128, 0, s>>>(a);
  }
  k_tl_div<<<blocks, 128, 0, s>>>(a);
  if (a.nsat > 0) {
    int sb = (a.nsat + 63) / 64;
    if (a.viscous) {
      if (curv) k_tl_sat<true, true><<<sb, 64, 0, s>>>(a);
      else k_tl_sat<true, false><<<sb, 64, 0, s>>>(a);
    } else {
      if (curv) k_tl_sat<false, true><<<sb, 64, 0, s>>>(a);
      else k_tl_sat<false, false><<<sb, 64, 0, s>>>(a);
    }
  }
  return cudaGetLastError();
}

}  // namespace sbp
