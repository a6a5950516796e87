// CUDA kernels (sm_103a) of the SBP-SAT overset right-hand side and its multi-rate
// Adams-Bashforth update.
//
//  k_rhs     fused tile kernel: SBP 4-2 derivatives with segment closures of the metric-
//            weighted inviscid and viscous fluxes, SAT penalties, and (mode 1) the MRAB /
//            Adams-Bashforth state update as an epilogue (Sec. 2.2 eq. (int), Sec. 3.3).
//  k_interp  donor-cell Lagrange interpolation with the slow-state extrapolation of the MRAB
//            micro steps fused in, one half-warp per receiver (Sec. 2.2, Sec. 3.3 Step 2).
//  k_dt      stable step estimate, min-reduced over the mesh (Sec. 4.1).
//  k_metrics metric terms by the derivative operator (Sec. 2.1; setup only).
//  k_axpy    Runge-Kutta stage combinations of the bootstrap (Sec. 3.1).
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>
#include <cstring>

#include "sbp_device.h"

namespace sbp {

// ---------------------------------------------------------------------------------------------
// SBP 4-2 first derivative, every class written as four (offset, weight) pairs applied with a
// direction sign: rows 0..3 are the boundary closures of the diagonal-norm operator with norm
// H = diag(17/48, 59/48, 43/48, 49/48, 1, ...), row 4 the interior fourth-order central row,
// row 5 a hole (all zero). A closure counted from a segment's high end uses the same row with
// the offsets and the result negated.
__constant__ int8_t c_off[6][4] = {{0, 1, 2, 3}, {-1, 1, 0, 0}, {-2, -1, 1, 2}, {-3, -1, 1, 2}, {-2, -1, 1, 2},
                                   {0, 0, 0, 0}};
__constant__ double c_w64[6][4] = {{-24.0 / 17.0, 59.0 / 34.0, -4.0 / 17.0, -3.0 / 34.0},
                                   {-0.5, 0.5, 0.0, 0.0},
                                   {4.0 / 43.0, -59.0 / 86.0, 59.0 / 86.0, -4.0 / 43.0},
                                   {3.0 / 98.0, -59.0 / 98.0, 32.0 / 49.0, -4.0 / 49.0},
                                   {1.0 / 12.0, -2.0 / 3.0, 2.0 / 3.0, -1.0 / 12.0},
                                   {0.0, 0.0, 0.0, 0.0}};
__constant__ float c_w32[6][4] = {{-24.0f / 17.0f, 59.0f / 34.0f, -4.0f / 17.0f, -3.0f / 34.0f},
                                  {-0.5f, 0.5f, 0.0f, 0.0f},
                                  {4.0f / 43.0f, -59.0f / 86.0f, 59.0f / 86.0f, -4.0f / 43.0f},
                                  {3.0f / 98.0f, -59.0f / 98.0f, 32.0f / 49.0f, -4.0f / 49.0f},
                                  {1.0f / 12.0f, -2.0f / 3.0f, 2.0f / 3.0f, -1.0f / 12.0f},
                                  {0.0f, 0.0f, 0.0f, 0.0f}};
// p0 of eq. (int): first entry of the norm H (unit index spacing).
#define SBP_P0 (17.0 / 48.0)

template <typename T> __device__ __forceinline__ T wgt(int r, int e);
template <> __device__ __forceinline__ double wgt<double>(int r, int e) { return c_w64[r][e]; }
template <> __device__ __forceinline__ float wgt<float>(int r, int e) { return c_w32[r][e]; }

// (row, sign) of a 4-bit class code (kind << 2 | closure row).
__device__ __forceinline__ void row_of(unsigned code, int &row, int &sgn) {
  unsigned kind = code >> 2;
  row = kind == kInterior ? 4 : kind == kHole ? 5 : (int)(code & 3u);
  sgn = kind == kRight ? -1 : 1;
}

// Derivative along a direction with element stride st at position s of array f.
template <typename T>
__device__ __forceinline__ T dline(const T *f, int s, int st, unsigned code) {
  int row, sgn;
  row_of(code, row, sgn);
  T acc = T(0);
#pragma unroll
  for (int e = 0; e < 4; ++e) acc += wgt<T>(row, e) * f[s + sgn * c_off[row][e] * st];
  return sgn > 0 ? acc : -acc;
}

__device__ __forceinline__ bool wrap_index(int &g, int n, int per) {
  if (per) {
    if (g < 0) g += n;
    if (g >= n) g -= n;
    return true;
  }
  return g >= 0 && g < n;
}

// ---------------------------------------------------------------------------------------------
// Pointwise physics. q = (rho, rho u, rho v, rho E), p = (gamma-1)(rho E - rho |u|^2/2),
// T = gamma p / rho.
template <typename T>
__device__ __forceinline__ void inviscid_flux(const T q[4], T gam, T F[4], T G[4], T &u, T &v, T &p) {
  T ri = T(1) / q[0];
  u = q[1] * ri;
  v = q[2] * ri;
  p = (gam - T(1)) * (q[3] - T(0.5) * (q[1] * u + q[2] * v));
  F[0] = q[1];
  F[1] = q[1] * u + p;
  F[2] = q[2] * u;
  F[3] = (q[3] + p) * u;
  G[0] = q[2];
  G[1] = q[1] * v;
  G[2] = q[2] * v + p;
  G[3] = (q[3] + p) * v;
}

// Cartesian viscous fluxes (momentum x, momentum y, energy of F^V and of G^V) from the
// velocity and temperature gradients: Stokes hypothesis, constant mu, Fourier heat flux.
template <typename T>
__device__ __forceinline__ void viscous_flux(T u, T v, const T gr[6], T mu, T kap, T Fv[3], T Gv[3]) {
  // gr = (u_x, u_y, v_x, v_y, T_x, T_y)
  T div = gr[0] + gr[3];
  T txx = mu * (T(2) * gr[0]) - T(2.0 / 3.0) * mu * div;
  T tyy = mu * (T(2) * gr[3]) - T(2.0 / 3.0) * mu * div;
  T txy = mu * (gr[1] + gr[2]);
  Fv[0] = txx;
  Fv[1] = txy;
  Fv[2] = u * txx + v * txy + kap * gr[4];
  Gv[0] = txy;
  Gv[1] = tyy;
  Gv[2] = u * txy + v * tyy + kap * gr[5];
}

// K^{+/-}_k (q - target) of eq. (int), applied through the eigen-decomposition of the flux
// Jacobian in direction k at state q: the acoustic waves U +/- c|k| with strengths
// (dp +/- rho c dUn) / (2 c^2), and the entropy and shear waves at U. side = +1 keeps the
// positive eigenvalues ((|L| + L)/2), side = -1 the magnitude of the negative ones.
template <typename T>
__device__ __forceinline__ void penalty_apply(const T q[4], T gam, T kx, T ky, int side, const T dq[4], T out[4]) {
  T rho = q[0], ri = T(1) / rho, u = q[1] * ri, v = q[2] * ri;
  T k2 = u * u + v * v;
  T p = (gam - T(1)) * (q[3] - T(0.5) * rho * k2);
  T c2 = gam * p * ri, c = sqrt(c2);
  T H = (q[3] + p) * ri;
  T kn = sqrt(kx * kx + ky * ky), kinv = T(1) / kn;
  T nx = kx * kinv, ny = ky * kinv;
  T U = kx * u + ky * v, Un = U * kinv;
  T du = (dq[1] - u * dq[0]) * ri, dv = (dq[2] - v * dq[0]) * ri;
  T dp = (gam - T(1)) * (dq[3] - u * dq[1] - v * dq[2] + T(0.5) * k2 * dq[0]);
  T dUn = nx * du + ny * dv;
  T ap = (dp + rho * c * dUn) / (T(2) * c2), am = (dp - rho * c * dUn) / (T(2) * c2);
  T a0 = dq[0] - dp / c2;
  T dut = du - nx * dUn, dvt = dv - ny * dUn;
  T l0 = U, lp = U + c * kn, lm = U - c * kn;
  T f0 = side > 0 ? fmax(l0, T(0)) : fmax(-l0, T(0));
  T fp = side > 0 ? fmax(lp, T(0)) : fmax(-lp, T(0));
  T fm = side > 0 ? fmax(lm, T(0)) : fmax(-lm, T(0));
  out[0] = f0 * a0 + fp * ap + fm * am;
  out[1] = f0 * (a0 * u + rho * dut) + fp * ap * (u + c * nx) + fm * am * (u - c * nx);
  out[2] = f0 * (a0 * v + rho * dvt) + fp * ap * (v + c * ny) + fm * am * (v - c * ny);
  out[3] = f0 * (a0 * T(0.5) * k2 + rho * (u * dut + v * dvt)) + fp * ap * (H + c * Un) + fm * am * (H - c * Un);
}

// ---------------------------------------------------------------------------------------------
// Fused right-hand side. One CTA per kTileX x kTileY tile, one thread per owned point.
// Shared memory holds the state (and primitives) on the tile plus a halo of HQ points, and
// metrics, gradients and contravariant fluxes on the tile plus HB = 3 points (the reach of
// the closure rows). Halo HQ = 3 for Euler; 6 for Navier-Stokes, where the fluxes at the
// band points need gradients that reach 3 points further.
template <typename T, bool VISC, bool CURV>
struct RhsSmem {
  static constexpr int TX = kTileX, TY = kTileY, NT = TX * TY;
  static constexpr int HQ = VISC ? 6 : 3, HB = 3;
  static constexpr int RX = TX + 2 * HQ, RY = TY + 2 * HQ, RN = RX * RY;
  static constexpr int BX = TX + 2 * HB, BY = TY + 2 * HB, BN = BX * BY;
  static constexpr size_t n_q = 4 * RN, n_prim = VISC ? 3 * RN : 0, n_met = CURV ? 5 * BN : 0,
                          n_grad = VISC ? 6 * BN : 0, n_flx = 8 * BN, n_rhs = 4 * NT;
  static constexpr size_t bytes = (n_q + n_prim + n_met + n_grad + n_flx + n_rhs) * sizeof(T) + RN;
};

template <typename T, bool CURV>
__device__ __forceinline__ void load_metrics(const DevMesh &m, const T *smet, int bidx, int bn, T mt[5]) {
  if (CURV) {
#pragma unroll
    for (int c = 0; c < 5; ++c) mt[c] = smet[c * bn + bidx];
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) mt[c] = (T)m.mc[c];
  }
}

template <typename T, bool VISC, bool CURV>
__global__ void __launch_bounds__(kTileX *kTileY) k_rhs(const RhsLaunch a) {
  using S = RhsSmem<T, VISC, CURV>;
  constexpr int TX = S::TX, NT = S::NT, HQ = S::HQ, HB = S::HB, RX = S::RX, RN = S::RN, BX = S::BX,
                BN = S::BN;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sq = reinterpret_cast<T *>(smem_raw);
  T *sprim = sq + S::n_q;
  T *smet = sprim + S::n_prim;
  T *sgrad = smet + S::n_met;
  T *sflx = sgrad + S::n_grad;
  T *srhs = sflx + S::n_flx;
  uint8_t *scls = reinterpret_cast<uint8_t *>(srhs + S::n_rhs);

  const DevMesh &m = a.m;
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * S::TY;
  const T *q = static_cast<const T *>(a.q);
  const T gam = (T)a.g.gamma, mu = (T)a.g.mu, kap = (T)(a.g.mu / (a.g.pr * (a.g.gamma - 1.0)));

  // ---- stage 0: state and classes on the halo region; metrics on the band
  for (int idx = tid; idx < RN; idx += NT) {
    int gi = i0 - HQ + idx % RX, gj = j0 - HQ + idx / RX;
    bool in = wrap_index(gi, m.ni, m.per_i) & wrap_index(gj, m.nj, m.per_j);
    if (in) {
      size_t p = (size_t)gj * m.pitch + gi;
      scls[idx] = m.cls[p];
#pragma unroll
      for (int v = 0; v < 4; ++v) sq[v * RN + idx] = q[v * m.field + p];
    } else {
      scls[idx] = 0xFF;
      sq[idx] = T(1);
      sq[RN + idx] = T(0);
      sq[2 * RN + idx] = T(0);
      sq[3 * RN + idx] = T(2.5);
    }
  }
  if (CURV) {
    const T *met = static_cast<const T *>(m.met);
    for (int idx = tid; idx < BN; idx += NT) {
      int gi = i0 - HB + idx % BX, gj = j0 - HB + idx / BX;
      bool in = wrap_index(gi, m.ni, m.per_i) & wrap_index(gj, m.nj, m.per_j);
      if (in) {
        size_t p = (size_t)gj * m.pitch + gi;
#pragma unroll
        for (int c = 0; c < 5; ++c) smet[c * BN + idx] = met[c * m.field + p];
      } else {
        smet[idx] = T(1);
        smet[BN + idx] = T(0);
        smet[2 * BN + idx] = T(0);
        smet[3 * BN + idx] = T(1);
        smet[4 * BN + idx] = T(1);
      }
    }
  }
  __syncthreads();

  // ---- stage 1: primitives u, v, T on the halo region (viscous only)
  if (VISC) {
    for (int idx = tid; idx < RN; idx += NT) {
      T ri = T(1) / sq[idx];
      T u = sq[RN + idx] * ri, v = sq[2 * RN + idx] * ri;
      T p = (gam - T(1)) * (sq[3 * RN + idx] - T(0.5) * (sq[RN + idx] * u + sq[2 * RN + idx] * v));
      sprim[idx] = u;
      sprim[RN + idx] = v;
      sprim[2 * RN + idx] = gam * p * ri;
    }
    __syncthreads();
  }

  // ---- stage 2: gradients and contravariant fluxes on the band
  for (int idx = tid; idx < BN; idx += NT) {
    int bx = idx % BX, by = idx / BX;
    int r = (by + HQ - HB) * RX + (bx + HQ - HB);
    unsigned code = scls[r];
    T mt[5];
    load_metrics<T, CURV>(m, smet, idx, BN, mt);
    T qp[4] = {sq[r], sq[RN + r], sq[2 * RN + r], sq[3 * RN + r]};
    T F[4], G[4], u, v, p;
    inviscid_flux(qp, gam, F, G, u, v, p);
    if (VISC) {
      T gr[6];
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        T dxi = dline(sprim + f * RN, r, 1, code & 15u);
        T deta = dline(sprim + f * RN, r, RX, code >> 4);
        if (CURV) {
          gr[2 * f] = mt[4] * (mt[0] * dxi + mt[2] * deta);
          gr[2 * f + 1] = mt[4] * (mt[1] * dxi + mt[3] * deta);
        } else {
          gr[2 * f] = mt[4] * (mt[0] * dxi);
          gr[2 * f + 1] = mt[4] * (mt[3] * deta);
        }
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) sgrad[c * BN + idx] = gr[c];
      T Fv[3], Gv[3];
      viscous_flux(u, v, gr, mu, kap, Fv, Gv);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        F[c + 1] -= Fv[c];
        G[c + 1] -= Gv[c];
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (CURV) {
        sflx[c * BN + idx] = mt[0] * F[c] + mt[1] * G[c];
        sflx[(4 + c) * BN + idx] = mt[2] * F[c] + mt[3] * G[c];
      } else {
        sflx[c * BN + idx] = mt[0] * F[c];
        sflx[(4 + c) * BN + idx] = mt[3] * G[c];
      }
    }
  }
  __syncthreads();

  // ---- stage 3: dq/dt = -J (D_xi F^_xi + D_eta F^_eta) at the owned points
  const int lx = tid % TX, ly = tid / TX;
  const int gi = i0 + lx, gj = j0 + ly;
  const int bown = (ly + HB) * BX + (lx + HB);
  const int rown = (ly + HQ) * RX + (lx + HQ);
  {
    unsigned code = scls[rown];
    T mt[5];
    load_metrics<T, CURV>(m, smet, bown, BN, mt);
    bool hole = (code & 15u) == 0xFu;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      T d = dline(sflx + c * BN, bown, 1, code & 15u) + dline(sflx + (4 + c) * BN, bown, BX, code >> 4);
      srhs[c * NT + tid] = hole ? T(0) : -mt[4] * d;
    }
  }
  __syncthreads();

  // ---- stage 4: SAT penalties at this tile's boundary and receiver points
  {
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    const int s0 = a.tile_sat[tile], s1 = a.tile_sat[tile + 1];
    const T *qhat = static_cast<const T *>(a.qhat);
    const T *fvhat = static_cast<const T *>(a.fvhat);
    for (int s = s0 + tid; s < s1; s += NT) {
      uint32_t ij = a.sat_ij[s];
      int li = (int)(ij & 0xFFFFu) - i0, lj = (int)(ij >> 16) - j0;
      int r = (lj + HQ) * RX + (li + HQ);
      int b = (lj + HB) * BX + (li + HB);
      T mt[5];
      load_metrics<T, CURV>(m, smet, b, BN, mt);
      T qp[4] = {sq[r], sq[RN + r], sq[2 * RN + r], sq[3 * RN + r]};
      T Fv[3] = {0, 0, 0}, Gv[3] = {0, 0, 0};
      if (VISC) {
        T gr[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) gr[c] = sgrad[c * BN + b];
        viscous_flux(sprim[r], sprim[RN + r], gr, mu, kap, Fv, Gv);
      }
      uint32_t code = a.sat_code[s];
      int recv = a.sat_recv[s];
      T scale = (T)a.sat_scale[s];
      T acc[4] = {0, 0, 0, 0};
      int nt = code & 7u;
      for (int t = 0; t < nt; ++t) {
        unsigned term = (code >> (3 + 4 * t)) & 15u;
        int dir = term & 1u, side = (term & 2u) ? -1 : 1, kind = (int)(term >> 2);
        T kx = mt[4] * mt[2 * dir], ky = mt[4] * mt[2 * dir + 1];
        T tgt[4];
        T sig1 = T(0), sigI = kind == kTermInterface ? (T)a.g.sig_int : (T)a.g.sig_phys;
        if (kind == kTermInterface) {
#pragma unroll
          for (int v = 0; v < 4; ++v) tgt[v] = qhat[v * a.nrecv + recv];
          if (VISC) sig1 = T(0.5) * mu * (kx * kx + ky * ky);
        } else if (kind == kTermFarfield) {
#pragma unroll
          for (int v = 0; v < 4; ++v) tgt[v] = (T)a.g.qinf[v];
        } else {
          tgt[0] = qp[0];
          tgt[1] = T(0);
          tgt[2] = T(0);
          tgt[3] = qp[0] * (T)(a.g.twall / (a.g.gamma * (a.g.gamma - 1.0)));
          if (VISC) sig1 = T(0.5) * mu * (kx * kx + ky * ky);
        }
        T dq[4], kd[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) dq[v] = qp[v] - tgt[v];
        penalty_apply(qp, gam, kx, ky, side, dq, kd);
        T sat[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) sat[v] = -(sigI * kd[v] + sig1 * dq[v]) * T(1.0 / SBP_P0);
        if (VISC && kind == kTermInterface) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            T own = kx * Fv[c] + ky * Gv[c];
            T hat = kx * fvhat[c * a.nrecv + recv] + ky * fvhat[(3 + c) * a.nrecv + recv];
            sat[c + 1] += T(0.5) * T(side) * (own - hat) * T(1.0 / SBP_P0);
          }
        }
        T sc = kind == kTermInterface ? scale : T(1);
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] += sc * sat[v];
      }
      int o = lj * TX + li;
#pragma unroll
      for (int v = 0; v < 4; ++v) srhs[v * NT + o] += acc[v];
    }
  }
  __syncthreads();

  // ---- stage 5: epilogue
  if (gi < m.ni && gj < m.nj) {
    size_t p = (size_t)gj * m.pitch + gi;
    T *out = static_cast<T *>(a.out);
    if (a.mode == 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) out[c * m.field + p] = srhs[c * NT + tid];
    } else {
      T *qn = static_cast<T *>(a.qnext);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        T rc = srhs[c * NT + tid];
        out[c * m.field + p] = rc;
        double acc = (double)sq[c * RN + rown];
        for (int k = 0; k < a.nold; ++k) acc += a.alpha[k] * (double)static_cast<const T *>(a.hold[k])[c * m.field + p];
        acc += a.alpha[a.nold] * (double)rc;
        qn[c * m.field + p] = (T)acc;
      }
    }
  }
}

template <typename T, bool VISC, bool CURV>
static cudaError_t launch_rhs_t(const RhsLaunch &a, cudaStream_t s) {
  using S = RhsSmem<T, VISC, CURV>;
  auto kern = k_rhs<T, VISC, CURV>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((a.m.ni + S::TX - 1) / S::TX, (a.m.nj + S::TY - 1) / S::TY);
  kern<<<grid, S::NT, S::bytes, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rhs(const RhsLaunch &a, int dtype, bool viscous, cudaStream_t s) {
  bool curv = !a.m.cart;
  if (dtype == SBP_F64) {
    if (viscous) return curv ? launch_rhs_t<double, true, true>(a, s) : launch_rhs_t<double, true, false>(a, s);
    return curv ? launch_rhs_t<double, false, true>(a, s) : launch_rhs_t<double, false, false>(a, s);
  }
  if (viscous) return curv ? launch_rhs_t<float, true, true>(a, s) : launch_rhs_t<float, true, false>(a, s);
  return curv ? launch_rhs_t<float, false, true>(a, s) : launch_rhs_t<float, false, false>(a, s);
}

size_t rhs_smem_bytes(int dtype, bool viscous, bool curv) {
  if (dtype == SBP_F64) {
    if (viscous) return curv ? RhsSmem<double, true, true>::bytes : RhsSmem<double, true, false>::bytes;
    return curv ? RhsSmem<double, false, true>::bytes : RhsSmem<double, false, false>::bytes;
  }
  if (viscous) return curv ? RhsSmem<float, true, true>::bytes : RhsSmem<float, true, false>::bytes;
  return curv ? RhsSmem<float, false, true>::bytes : RhsSmem<float, false, false>::bytes;
}

// ---------------------------------------------------------------------------------------------
// Interpolation. A half-warp per receiver: lane l of the half holds donor (l & 3, l >> 2) of
// the 4x4 stencil; the weighted values are summed with shuffles.
template <typename T>
__device__ __forceinline__ void donor_state(const InterpLaunch &a, size_t p, T out[4]) {
  const T *q = static_cast<const T *>(a.q);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double acc = (double)q[v * a.d.field + p];
    for (int k = 0; k < a.nbeta; ++k) acc += a.beta[k] * (double)static_cast<const T *>(a.hist[k])[v * a.d.field + p];
    out[v] = (T)acc;
  }
}

template <typename T>
__device__ __forceinline__ void donor_prim(const InterpLaunch &a, int i, int j, T gam, T pr[3]) {
  T s[4];
  donor_state(a, (size_t)j * a.d.pitch + i, s);
  T ri = T(1) / s[0];
  T u = s[1] * ri, v = s[2] * ri;
  T p = (gam - T(1)) * (s[3] - T(0.5) * (s[1] * u + s[2] * v));
  pr[0] = u;
  pr[1] = v;
  pr[2] = gam * p * ri;
}

template <typename T, bool VISC, bool CURV>
__global__ void __launch_bounds__(256) k_interp(const InterpLaunch a) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int r = warp * 2 + (lane >> 4);
  const int l = lane & 15, da = l & 3, db = l >> 2;
  const bool valid = r < a.nrecv;
  const T gam = (T)a.g.gamma, mu = (T)a.g.mu, kap = (T)(a.g.mu / (a.g.pr * (a.g.gamma - 1.0)));
  T val[4] = {0, 0, 0, 0};
  T fv[6] = {0, 0, 0, 0, 0, 0};
  if (valid) {
    int ii = a.base[2 * r] + da, jj = a.base[2 * r + 1] + db;
    wrap_index(ii, a.d.ni, a.d.per_i);
    wrap_index(jj, a.d.nj, a.d.per_j);
    T w = (T)(a.w[8 * r + da] * a.w[8 * r + 4 + db]);
    size_t p = (size_t)jj * a.d.pitch + ii;
    T s[4];
    donor_state(a, p, s);
#pragma unroll
    for (int v = 0; v < 4; ++v) val[v] = w * s[v];
    if (VISC && a.fvhat) {
      unsigned code = a.d.cls[p];
      T dxi[3] = {0, 0, 0}, deta[3] = {0, 0, 0};
      for (int dir = 0; dir < 2; ++dir) {
        int row, sgn;
        row_of(dir == 0 ? (code & 15u) : (code >> 4), row, sgn);
        for (int e = 0; e < 4; ++e) {
          T we = wgt<T>(row, e);
          if (we == T(0)) continue;
          int ni_ = ii, nj_ = jj;
          if (dir == 0) ni_ += sgn * c_off[row][e];
          else nj_ += sgn * c_off[row][e];
          wrap_index(ni_, a.d.ni, a.d.per_i);
          wrap_index(nj_, a.d.nj, a.d.per_j);
          T pr[3];
          donor_prim(a, ni_, nj_, gam, pr);
          for (int f = 0; f < 3; ++f) {
            if (dir == 0) dxi[f] += T(sgn) * we * pr[f];
            else deta[f] += T(sgn) * we * pr[f];
          }
        }
      }
      T mt[5];
      if (CURV) {
        const T *met = static_cast<const T *>(a.d.met);
#pragma unroll
        for (int c = 0; c < 5; ++c) mt[c] = met[c * a.d.field + p];
      } else {
#pragma unroll
        for (int c = 0; c < 5; ++c) mt[c] = (T)a.d.mc[c];
      }
      T gr[6];
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        gr[2 * f] = mt[4] * (mt[0] * dxi[f] + mt[2] * deta[f]);
        gr[2 * f + 1] = mt[4] * (mt[1] * dxi[f] + mt[3] * deta[f]);
      }
      T pc[3];
      donor_prim(a, ii, jj, gam, pc);
      T Fv[3], Gv[3];
      viscous_flux(pc[0], pc[1], gr, mu, kap, Fv, Gv);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        fv[c] = w * Fv[c];
        fv[3 + c] = w * Gv[c];
      }
    }
  }
#pragma unroll
  for (int off = 8; off > 0; off >>= 1) {
#pragma unroll
    for (int v = 0; v < 4; ++v) val[v] += __shfl_xor_sync(0xffffffffu, val[v], off);
    if (VISC) {
#pragma unroll
      for (int c = 0; c < 6; ++c) fv[c] += __shfl_xor_sync(0xffffffffu, fv[c], off);
    }
  }
  if (valid && l == 0) {
    T *qh = static_cast<T *>(a.qhat);
#pragma unroll
    for (int v = 0; v < 4; ++v) qh[v * a.nrecv + r] = val[v];
    if (VISC && a.fvhat) {
      T *fh = static_cast<T *>(a.fvhat);
#pragma unroll
      for (int c = 0; c < 6; ++c) fh[c * a.nrecv + r] = fv[c];
    }
  }
}

template <typename T, bool VISC, bool CURV>
static cudaError_t launch_interp_t(const InterpLaunch &a, cudaStream_t s) {
  if (a.nrecv == 0) return cudaSuccess;
  int warps = (a.nrecv + 1) / 2;
  int blocks = (warps * 32 + 255) / 256;
  k_interp<T, VISC, CURV><<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_interp(const InterpLaunch &a, int dtype, bool viscous, cudaStream_t s) {
  bool curv = !a.d.cart;
  if (dtype == SBP_F64) {
    if (viscous) return curv ? launch_interp_t<double, true, true>(a, s) : launch_interp_t<double, true, false>(a, s);
    return curv ? launch_interp_t<double, false, true>(a, s) : launch_interp_t<double, false, false>(a, s);
  }
  if (viscous) return curv ? launch_interp_t<float, true, true>(a, s) : launch_interp_t<float, true, false>(a, s);
  return curv ? launch_interp_t<float, false, true>(a, s) : launch_interp_t<float, false, false>(a, s);
}

// ---------------------------------------------------------------------------------------------
// Time step (Sec. 4.1): dt_inv = 1/(sum_m |u . grad xi_m| + c sqrt(sum_m |grad xi_m|^2)),
// dt_visc = 1/(1/dt_inv + 2 nu* sum_m |grad xi_m|^2), nu* = max(mu, gamma mu/Pr)/rho; the
// minimum over active points is combined with atomicMin on the bit pattern (positive doubles
// order like unsigned integers).
template <typename T, bool CURV>
__global__ void __launch_bounds__(256) k_dt(const DevMesh m, Gas g, const T *q, unsigned long long *out) {
  double best = DBL_MAX;
  size_t n = (size_t)m.ni * m.nj;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % m.ni), j = (int)(t / m.ni);
    size_t p = (size_t)j * m.pitch + i;
    if ((m.cls[p] & 15u) == 15u) continue;
    double rho = q[p], u = q[m.field + p] / rho, v = q[2 * m.field + p] / rho;
    double pres = (g.gamma - 1.0) * ((double)q[3 * m.field + p] - 0.5 * rho * (u * u + v * v));
    double c = sqrt(g.gamma * pres / rho);
    double mt[5];
    if (CURV) {
      const T *met = static_cast<const T *>(m.met);
      for (int k = 0; k < 5; ++k) mt[k] = met[k * m.field + p];
    } else {
      for (int k = 0; k < 5; ++k) mt[k] = m.mc[k];
    }
    double conv = 0.0, g2 = 0.0;
    for (int d = 0; d < 2; ++d) {
      double kx = mt[4] * mt[2 * d], ky = mt[4] * mt[2 * d + 1];
      conv += fabs(u * kx + v * ky);
      g2 += kx * kx + ky * ky;
    }
    double inv = conv + c * sqrt(g2);
    double dt = 1.0 / inv;
    if (g.mu > 0.0) {
      double nu = fmax(g.mu, g.gamma * g.mu / g.pr) / rho;
      dt = fmin(dt, 1.0 / (inv + 2.0 * nu * g2));
    }
    best = fmin(best, dt);
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

__global__ void k_fill_u64(unsigned long long *p, unsigned long long v) { *p = v; }

cudaError_t launch_dt(const DevMesh &m, const Gas &g, const void *q, int dtype, unsigned long long *out,
                      cudaStream_t s) {
  double big = DBL_MAX;
  unsigned long long bits;
  memcpy(&bits, &big, sizeof(bits));
  k_fill_u64<<<1, 1, 0, s>>>(out, bits);
  size_t n = (size_t)m.ni * m.nj;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (dtype == SBP_F64) {
    if (m.cart) k_dt<double, false><<<blocks, 256, 0, s>>>(m, g, (const double *)q, out);
    else k_dt<double, true><<<blocks, 256, 0, s>>>(m, g, (const double *)q, out);
  } else {
    if (m.cart) k_dt<float, false><<<blocks, 256, 0, s>>>(m, g, (const float *)q, out);
    else k_dt<float, true><<<blocks, 256, 0, s>>>(m, g, (const float *)q, out);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Metrics (setup): x_xi, y_xi, x_eta, y_eta by the full 6-entry SBP rows (interior row over
// offsets -2..2) summed left to right with separately rounded products and sums, then
// xi_x/J = y_eta, xi_y/J = -x_eta, eta_x/J = -y_xi, eta_y/J = x_xi, J = 1 / (x_xi y_eta -
// x_eta y_xi). Coordinates across a periodic wrap are shifted by the period vector.
__constant__ double c_row6[4][6] = {{-24.0 / 17.0, 59.0 / 34.0, -4.0 / 17.0, -3.0 / 34.0, 0.0, 0.0},
                                    {-1.0 / 2.0, 0.0, 1.0 / 2.0, 0.0, 0.0, 0.0},
                                    {4.0 / 43.0, -59.0 / 86.0, 0.0, 59.0 / 86.0, -4.0 / 43.0, 0.0},
                                    {3.0 / 98.0, 0.0, -59.0 / 98.0, 0.0, 32.0 / 49.0, -4.0 / 49.0}};
__constant__ double c_int5[5] = {1.0 / 12.0, -2.0 / 3.0, 0.0, 2.0 / 3.0, -1.0 / 12.0};

__device__ double coord_at(const double *f, int ni, int i, int j, int di, int dj, int n, int dir, double sh) {
  int k = (dir == 0 ? i : j) + (dir == 0 ? di : dj);
  int w = 0;
  while (k < 0) { k += n; --w; }
  while (k >= n) { k -= n; ++w; }
  double val = dir == 0 ? f[(size_t)j * ni + k] : f[(size_t)k * ni + i];
  return __dadd_rn(val, __dmul_rn((double)w, sh));
}

__device__ double dcoord(const double *f, int ni, int nj, int i, int j, int dir, unsigned code, double sh) {
  int n = dir == 0 ? ni : nj;
  unsigned kind = code >> 2, r = code & 3u;
  double s = 0.0;
  if (kind == kInterior) {
    for (int o = -2; o <= 2; ++o) {
      if (c_int5[o + 2] == 0.0) continue;
      double v = coord_at(f, ni, i, j, dir == 0 ? o : 0, dir == 1 ? o : 0, n, dir, sh);
      s = __dadd_rn(s, __dmul_rn(c_int5[o + 2], v));
    }
  } else if (kind == kLeft) {
    for (int c = 0; c < 6; ++c) {
      if (c_row6[r][c] == 0.0) continue;
      int o = c - (int)r;
      double v = coord_at(f, ni, i, j, dir == 0 ? o : 0, dir == 1 ? o : 0, n, dir, sh);
      s = __dadd_rn(s, __dmul_rn(c_row6[r][c], v));
    }
  } else if (kind == kRight) {
    for (int c = 0; c < 6; ++c) {
      if (c_row6[r][c] == 0.0) continue;
      int o = (int)r - c;
      double v = coord_at(f, ni, i, j, dir == 0 ? o : 0, dir == 1 ? o : 0, n, dir, sh);
      s = __dsub_rn(s, __dmul_rn(c_row6[r][c], v));
    }
  }
  return s;
}

template <typename T>
__global__ void k_metrics(const DevMesh m, const double *x, const double *y, double s0, double s1, double s2,
                          double s3, T *met) {
  size_t n = (size_t)m.ni * m.nj;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % m.ni), j = (int)(t / m.ni);
    size_t p = (size_t)j * m.pitch + i;
    unsigned code = m.cls[p];
    double o[5];
    if ((code & 15u) == 15u) {
      o[0] = 1.0; o[1] = 0.0; o[2] = 0.0; o[3] = 1.0; o[4] = 1.0;
    } else {
      double x_xi = dcoord(x, m.ni, m.nj, i, j, 0, code & 15u, s0);
      double y_xi = dcoord(y, m.ni, m.nj, i, j, 0, code & 15u, s1);
      double x_eta = dcoord(x, m.ni, m.nj, i, j, 1, code >> 4, s2);
      double y_eta = dcoord(y, m.ni, m.nj, i, j, 1, code >> 4, s3);
      double jinv = __dsub_rn(__dmul_rn(x_xi, y_eta), __dmul_rn(x_eta, y_xi));
      o[0] = y_eta;
      o[1] = -x_eta;
      o[2] = -y_xi;
      o[3] = x_xi;
      o[4] = __ddiv_rn(1.0, jinv);
    }
    for (int c = 0; c < 5; ++c) met[c * m.field + p] = (T)o[c];
  }
}

cudaError_t launch_metrics(const DevMesh &m, const double *x, const double *y, const double sh[4], void *met,
                           int dtype, cudaStream_t s) {
  size_t n = (size_t)m.ni * m.nj;
  int blocks = (int)((n + 255) / 256);
  if (dtype == SBP_F64) k_metrics<double><<<blocks, 256, 0, s>>>(m, x, y, sh[0], sh[1], sh[2], sh[3], (double *)met);
  else k_metrics<float><<<blocks, 256, 0, s>>>(m, x, y, sh[0], sh[1], sh[2], sh[3], (float *)met);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_axpy(const T *y, const T *k1, double c1, const T *k2, double c2, T *yo, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    double acc = (double)y[t] + c1 * (double)k1[t];
    if (k2) acc += c2 * (double)k2[t];
    yo[t] = (T)acc;
  }
}

cudaError_t launch_axpy(const void *y, const void *k1, double c1, const void *k2, double c2, void *yo, size_t n,
                        int dtype, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (dtype == SBP_F64)
    k_axpy<double><<<blocks, 256, 0, s>>>((const double *)y, (const double *)k1, c1, (const double *)k2, c2,
                                          (double *)yo, n);
  else
    k_axpy<float><<<blocks, 256, 0, s>>>((const float *)y, (const float *)k1, c1, (const float *)k2, c2,
                                         (float *)yo, n);
  return cudaGetLastError();
}

}  // namespace sbp
