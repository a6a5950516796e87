// Device code shared by the library's CUDA translation units (sm_103a): SBP 4-2 derivative
// rows, pointwise physics, the SAT penalty, and the tile bodies of the right-hand side
// (flux_tile, update_tile) and of the donor values (donor_group), which the single-system
// kernels and the batched persistent kernel both call.
#pragma once
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
static __constant__ int8_t c_off[6][4] = SBP_ROW_OFFSETS;
static __constant__ double c_w64[6][4] = {{-24.0 / 17.0, 59.0 / 34.0, -4.0 / 17.0, -3.0 / 34.0},
                                   {-0.5, 0.5, 0.0, 0.0},
                                   {4.0 / 43.0, -59.0 / 86.0, 59.0 / 86.0, -4.0 / 43.0},
                                   {3.0 / 98.0, -59.0 / 98.0, 32.0 / 49.0, -4.0 / 49.0},
                                   {1.0 / 12.0, -2.0 / 3.0, 2.0 / 3.0, -1.0 / 12.0},
                                   {0.0, 0.0, 0.0, 0.0}};
static __constant__ float c_w32[6][4] = {{-24.0f / 17.0f, 59.0f / 34.0f, -4.0f / 17.0f, -3.0f / 34.0f},
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

// A derivative row decoded once per point and direction: tap offsets (times the direction
// sign), weights, and whether the sum is negated (a closure counted from the segment's high
// end). row_sum applies it to one plane with dline's operation order, through per-tap pointers
// shared by all planes (plane c at offset c * plane stride).
template <typename T>
struct Row {
  int off[4];
  T w[4];
  bool neg;
};

template <typename T>
__device__ __forceinline__ Row<T> decode_row(unsigned code) {
  Row<T> r;
  int row, sgn;
  row_of(code, row, sgn);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    r.off[e] = sgn * c_off[row][e];
    r.w[e] = wgt<T>(row, e);
  }
  r.neg = sgn < 0;
  return r;
}

// The same with the weights taken from a per-mesh table of scaled rows (tab[row][tap]).
template <typename T>
__device__ __forceinline__ Row<T> decode_row_w(unsigned code, const T (*tab)[4]) {
  Row<T> r;
  int row, sgn;
  row_of(code, row, sgn);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    r.off[e] = sgn * c_off[row][e];
    r.w[e] = tab[row][e];
  }
  r.neg = sgn < 0;
  return r;
}

template <typename T>
__device__ __forceinline__ T row_sum(const Row<T> &r, const T *const p[4], int plane) {
  T acc = T(0);
#pragma unroll
  for (int e = 0; e < 4; ++e) acc += r.w[e] * p[e][plane];
  return r.neg ? -acc : acc;
}

// The interior row (row 4) with its weights as compile-time constants: the same values and
// operation order as row_sum on a decoded interior row, with the taps at fixed offsets.
template <typename T>
struct CentralRow;
template <>
struct CentralRow<float> {
  static constexpr float w0 = 1.0f / 12.0f, w1 = -2.0f / 3.0f, w2 = 2.0f / 3.0f, w3 = -1.0f / 12.0f;
};
template <>
struct CentralRow<double> {
  static constexpr double w0 = 1.0 / 12.0, w1 = -2.0 / 3.0, w2 = 2.0 / 3.0, w3 = -1.0 / 12.0;
};

template <typename T>
__device__ __forceinline__ T central_sum(const T *const p[4], int plane) {
  T acc = T(0);
  acc += CentralRow<T>::w0 * p[0][plane];
  acc += CentralRow<T>::w1 * p[1][plane];
  acc += CentralRow<T>::w2 * p[2][plane];
  acc += CentralRow<T>::w3 * p[3][plane];
  return acc;
}

// The interior row with the weights w (a scaled table's row 4), taps at fixed offsets: row_sum's
// operation order.
template <typename T>
__device__ __forceinline__ T central_sum_w(const T *const p[4], int plane, const T w[4]) {
  T acc = T(0);
#pragma unroll
  for (int e = 0; e < 4; ++e) acc += w[e] * p[e][plane];
  return acc;
}

// Index g on a line of n points: wrapped once on a periodic line; false when outside the line
// (non-periodic) or more than one period away (strips wider than a small periodic mesh).
__device__ __forceinline__ bool wrap_index(int &g, int n, int per) {
  if (per) {
    if (g < 0) g += n;
    else if (g >= n) g -= n;
  }
  return (unsigned)g < (unsigned)n;
}

// Asynchronous global -> shared copies of N bytes (cp.async), their commit and wait.
template <int N>
__device__ __forceinline__ void cp_async_n(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(N));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Exact FP32 -> FP64 widening written from the IEEE 754 binary32 / binary64 layouts: the sign
// kept, the exponent re-biased by 1023 - 127 = 896, the 23 fraction bits moved to the top of the
// 52-bit fraction; zeros keep only their sign. Integer operations only, because GB300 issues the
// hardware conversion to the FP64 pipe, which the FP64 accumulations of the FP32 forms (MRAB
// update, slow-state extrapolation) already keep busy. Subnormal, infinite and NaN inputs take
// the hardware conversion. Bit-identical to (double)x for every input.
__device__ __forceinline__ double widen(float x) {
  const unsigned b = __float_as_uint(x), e = (b >> 23) & 0xFFu;
  if (e - 1u < 254u)
    return __hiloint2double((int)((b & 0x80000000u) | ((e + 896u) << 20) | ((b >> 3) & 0xFFFFFu)), (int)(b << 29));
  if ((b & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  return (double)x;
}
__device__ __forceinline__ double to_f64(float x) { return widen(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }

// Failure detection: true when a value is infinite or NaN (exponent field all ones), tested on
// the bits (integer operations, nothing issued to the FP64 pipe).
__device__ __forceinline__ bool not_finite(float x) { return (__float_as_uint(x) & 0x7F800000u) == 0x7F800000u; }
__device__ __forceinline__ bool not_finite(double x) {
  return (__double_as_longlong(x) & 0x7FF0000000000000ll) == 0x7FF0000000000000ll;
}

// Records SBP_ERR_NONFINITE in the device error word (first error wins) when a new state has a
// non-finite value or a density that is not positive: the state cannot be stepped further.
template <typename T, int NV>
__device__ __forceinline__ void flag_bad_state(const T qn[NV], int *err) {
  bool bad = !(qn[0] > T(0));
#pragma unroll
  for (int c = 1; c < NV; ++c) bad |= not_finite(qn[c]);
  if (bad && err) atomicCAS(err, 0, (int)SBP_ERR_NONFINITE);
}

// Adams-Bashforth / MRAB update of one point's NV variables (Sec. 3.1 eq. (ab_general)):
// qn = q + sum_h alpha[h] hold[h] + alpha[nold] rhs, accumulated in FP64 in that order. The
// loads of one history slot's NV values are issued together, ahead of their products. A new
// state that is not finite or has a non-positive density is flagged in *err (callers pass err
// for active points only: hole points carry no state).
template <typename T, int NV>
__device__ __forceinline__ void ab_update(const T qv[NV], const void *const *hold, const double *alpha, int nold,
                                          size_t field, size_t p, const T rhs[NV], T qn[NV], int *err) {
  double acc[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) acc[c] = to_f64(qv[c]);
#pragma unroll
  for (int h = 0; h < kMaxHist - 1; ++h) {
    if (h < nold) {
      const T *hp = static_cast<const T *>(hold[h]) + p;
      T hv[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) hv[c] = hp[c * field];
#pragma unroll
      for (int c = 0; c < NV; ++c) acc[c] += alpha[h] * to_f64(hv[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    acc[c] += alpha[nold] * to_f64(rhs[c]);
    qn[c] = (T)acc[c];
  }
  flag_bad_state<T, NV>(qn, err);
}

// Products and fused multiply-adds with a fixed rounding (never re-associated or contracted
// differently by the compiler), for expressions that several kernels must evaluate to the
// same bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Index checks of the tables the gathers follow, in builds with SBP_BOUNDS_CHECK defined: an
// index outside [0, n) records SBP_ERR_BOUNDS in *err (when given) and is replaced by 0, a valid
// entry, so that the kernel neither reads out of range nor stops. Without the flag, the indices
// are used as they are (the setup builds them in range, and the tests check the tables).
#ifdef SBP_BOUNDS_CHECK
__device__ __forceinline__ int checked_index(int d, int n, int *err) {
  if ((unsigned)d >= (unsigned)n) {
    if (err) atomicCAS(err, 0, (int)SBP_ERR_BOUNDS);
    return 0;
  }
  return d;
}
#else
__device__ __forceinline__ int checked_index(int d, int, int *) { return d; }
#endif

// a b + c d and a b + c d + e f with one fixed rounding order (fma(a, b, c d), fma(a, b,
// fma(c, d, e f))): the viscous and contravariant fluxes and the metric chain rule that every
// right-hand-side design evaluates, so that they give the same bits whatever the compiler does.
template <typename T>
__device__ __forceinline__ T dot2_rn(T a, T b, T c, T d) {
  return fma_rn(a, b, mul_rn(c, d));
}
template <typename T>
__device__ __forceinline__ T dot3_rn(T a, T b, T c, T d, T e, T f) {
  return fma_rn(a, b, fma_rn(c, d, mul_rn(e, f)));
}

// d/dx and d/dy of a field from its index-direction derivatives (chain rule with the metrics on
// curvilinear meshes; Cartesian meshes take rows already scaled by 1/h).
template <typename T, bool CURV>
__device__ __forceinline__ T grad_x(const T mt[5], T dxi, T deta) {
  return CURV ? mul_rn(mt[4], dot2_rn(mt[0], dxi, mt[2], deta)) : dxi;
}
template <typename T, bool CURV>
__device__ __forceinline__ T grad_y(const T mt[5], T dxi, T deta) {
  return CURV ? mul_rn(mt[4], dot2_rn(mt[1], dxi, mt[3], deta)) : deta;
}

// F - F^V and G - G^V of the Navier-Stokes equations at a point: state qp, velocity (u, v),
// pressure pr, Cartesian viscous fluxes Fv, Gv (momentum x, momentum y, energy).
template <typename T>
__device__ __forceinline__ void ns_flux_x(const T qp[4], T u, T pr, const T Fv[3], T Fx[4]) {
  Fx[0] = qp[1];
  Fx[1] = fma_rn(qp[1], u, pr) - Fv[0];
  Fx[2] = fma_rn(qp[2], u, -Fv[1]);
  Fx[3] = fma_rn(qp[3] + pr, u, -Fv[2]);
}
template <typename T>
__device__ __forceinline__ void ns_flux_y(const T qp[4], T v, T pr, const T Gv[3], T Gx[4]) {
  Gx[0] = qp[2];
  Gx[1] = fma_rn(qp[1], v, -Gv[0]);
  Gx[2] = fma_rn(qp[2], v, pr) - Gv[1];
  Gx[3] = fma_rn(qp[3] + pr, v, -Gv[2]);
}

// p = (gamma - 1)(rho E - (rho u u + rho v v) / 2).
template <typename T>
__device__ __forceinline__ T pressure_of(T gam, T rE, T ru, T rv, T u, T v) {
  const T ke = fma_rn(ru, u, mul_rn(rv, v));
  return mul_rn(gam - T(1), fma_rn(T(-0.5), ke, rE));
}

// ---------------------------------------------------------------------------------------------
// Pointwise physics. q = (rho, rho u, rho v, rho E), p = (gamma-1)(rho E - rho |u|^2/2),
// T = gamma p / rho.
template <typename T>
__device__ __forceinline__ void inviscid_flux(const T q[4], T gam, T F[4], T G[4], T &u, T &v, T &p) {
  T ri = T(1) / q[0];
  u = q[1] * ri;
  v = q[2] * ri;
  p = pressure_of(gam, q[3], q[1], q[2], u, v);
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
  T m23 = T(2.0 / 3.0) * mu;
  T txx = dot2_rn(mu, T(2) * gr[0], -m23, div);
  T tyy = dot2_rn(mu, T(2) * gr[3], -m23, div);
  T txy = mu * (gr[1] + gr[2]);
  Fv[0] = txx;
  Fv[1] = txy;
  Fv[2] = dot3_rn(u, txx, v, txy, kap, gr[4]);
  Gv[0] = txy;
  Gv[1] = tyy;
  Gv[2] = dot3_rn(u, txy, v, tyy, kap, gr[5]);
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
// Right-hand side in two kernels per mesh:
//  k_flux    contravariant fluxes F^_xi, F^_eta (inviscid minus viscous) at every point, written
//            to a flux buffer (8 planes) that stays in L2 for the next kernel. Navier-Stokes
//            tiles stage the primitives with a 3-point halo in shared memory for the velocity
//            and temperature gradients; each flux is computed once.
//  k_update  SBP derivatives of the fluxes (3-point halo of flux planes in shared memory),
//            -J times their sum, SAT penalties at the tile's boundary and receiver points, and
//            the epilogue (mode 0: dq/dt; mode 1: also the Adams-Bashforth / MRAB update).
template <typename T, bool CURV>
__device__ __forceinline__ void point_metrics(const DevMesh &m, int gi, int gj, T mt[5]) {
  if (CURV) {
    const T *met = static_cast<const T *>(m.met);
    size_t p = (size_t)gj * m.pitch + gi;
#pragma unroll
    for (int c = 0; c < 5; ++c) mt[c] = met[c * m.field + p];
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) mt[c] = (T)m.mc[c];
  }
}

// Primitives (u, v, T) of the conserved state (q0, q1, q2, q3).
template <typename T>
__device__ __forceinline__ void prim4(T q0, T q1, T q2, T q3, T gam, T pr[3]) {
  T ri = T(1) / q0;
  T u = q1 * ri, v = q2 * ri;
  T pres = pressure_of(gam, q3, q1, q2, u, v);
  pr[0] = u;
  pr[1] = v;
  pr[2] = gam * pres * ri;
}

template <typename T>
__device__ __forceinline__ void prim_at(const T *q, size_t field, size_t p, T gam, T pr[3]) {
  prim4(q[p], q[field + p], q[2 * field + p], q[3 * field + p], gam, pr);
}

// Kernel constants in the compute type.
template <typename T>
__device__ __forceinline__ const KConst<T> &kc(const RhsLaunch &a);
template <>
__device__ __forceinline__ const KConst<float> &kc<float>(const RhsLaunch &a) {
  return a.cf;
}
template <>
__device__ __forceinline__ const KConst<double> &kc<double>(const RhsLaunch &a) {
  return a.cd;
}

template <typename T, bool CURV>
__device__ __forceinline__ void load_met(const RhsLaunch &a, int gi, int gj, T mt[5]) {
  if (CURV) {
    const T *met = static_cast<const T *>(a.m.met);
    size_t p = (size_t)gj * a.m.pitch + gi;
#pragma unroll
    for (int c = 0; c < 5; ++c) mt[c] = met[c * a.m.field + p];
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) mt[c] = kc<T>(a).mc[c];
  }
}

// Cartesian viscous fluxes from gradients (u_x, u_y, v_x, v_y, T_x, T_y), Stokes hypothesis.
template <typename T>
__device__ __forceinline__ void visc_flux_kx(const KConst<T> &k, T u, T v, const T gr[6], T Fv[3]) {
  T txx = dot2_rn(k.mu43, gr[0], -k.mu23, gr[3]);
  T txy = k.mu * (gr[1] + gr[2]);
  Fv[0] = txx;
  Fv[1] = txy;
  Fv[2] = dot3_rn(u, txx, v, txy, k.kap, gr[4]);
}
template <typename T>
__device__ __forceinline__ void visc_flux_ky(const KConst<T> &k, T u, T v, const T gr[6], T Gv[3]) {
  T tyy = dot2_rn(k.mu43, gr[3], -k.mu23, gr[0]);
  T txy = k.mu * (gr[1] + gr[2]);
  Gv[0] = txy;
  Gv[1] = tyy;
  Gv[2] = dot3_rn(u, txy, v, tyy, k.kap, gr[5]);
}
template <typename T>
__device__ __forceinline__ void visc_flux_k(const KConst<T> &k, T u, T v, const T gr[6], T Fv[3], T Gv[3]) {
  visc_flux_kx(k, u, v, gr, Fv);
  visc_flux_ky(k, u, v, gr, Gv);
}

// Gradients of (u, v, T) at smem index r of the primitive planes (row stride rx), chain rule
// with the metrics; Cartesian meshes take the rows scaled by 1/hx, 1/hy (d/dx, d/dy directly).
template <typename T, bool CURV>
__device__ __forceinline__ void smem_grads(const RhsLaunch &a, const T *prim, int rn, int r, int rx, unsigned code,
                                           const T mt[5], T gr[6]) {
  const Row<T> ri = CURV ? decode_row<T>(code & 15u) : decode_row_w<T>(code & 15u, kc<T>(a).wx);
  const Row<T> rj = CURV ? decode_row<T>(code >> 4) : decode_row_w<T>(code >> 4, kc<T>(a).wy);
  const T *pi[4], *pj[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    pi[e] = prim + r + ri.off[e];
    pj[e] = prim + r + rj.off[e] * rx;
  }
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    T dxi = row_sum(ri, pi, f * rn);
    T deta = row_sum(rj, pj, f * rn);
    gr[2 * f] = grad_x<T, CURV>(mt, dxi, deta);
    gr[2 * f + 1] = grad_y<T, CURV>(mt, dxi, deta);
  }
}

// SAT terms of one boundary / receiver point (Sec. 2.2 eq. (int); physical forms of Sec. 5.1):
// q_p the point's state, (Fv, Gv) its Cartesian viscous fluxes; returns the sum in acc.
template <typename T, bool VISC>
__device__ void sat_terms(const RhsLaunch &a, int s, const T qp[4], const T mt[5], const T Fv[3], const T Gv[3],
                          T acc[4]) {
  const KConst<T> &k = kc<T>(a);
  const T *qhat = static_cast<const T *>(a.qhat);
  const T *fvhat = static_cast<const T *>(a.fvhat);
  const T *dw = static_cast<const T *>(a.dwt);
  uint32_t code = a.sat_code[s];
  int recv = a.sat_recv[s];
  T scale = (T)a.sat_scale[s];
  constexpr int NRV = VISC ? 10 : 4;
  T rv[NRV];
#pragma unroll
  for (int c = 0; c < NRV; ++c) rv[c] = T(0);
  if (recv >= 0) {
    if (a.dv) {
      const T *dv = static_cast<const T *>(a.dv);
      for (int e = 0; e < 16; ++e) {
        T w = dw[8 * recv + (e & 3)] * dw[8 * recv + 4 + (e >> 2)];
        int d = checked_index(a.didx[16 * recv + e], a.ndv, a.err);
#pragma unroll
        for (int c = 0; c < NRV; ++c) rv[c] += w * dv[c * a.ndv + d];
      }
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) rv[c] = qhat[c * a.nrecv + recv];
      if constexpr (VISC) {
#pragma unroll
        for (int c = 0; c < 6; ++c) rv[4 + c] = fvhat[c * a.nrecv + recv];
      }
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) acc[v] = T(0);
  int nt = code & 7u;
  for (int t = 0; t < nt; ++t) {
    unsigned term = (code >> (3 + 4 * t)) & 15u;
    int dir = term & 1u, side = (term & 2u) ? -1 : 1, kind = (int)(term >> 2);
    T kx = mt[4] * mt[2 * dir], ky = mt[4] * mt[2 * dir + 1];
    T tgt[4];
    T sig1 = T(0), sigI = kind == kTermInterface ? k.sig_int : k.sig_phys;
    if (kind == kTermInterface) {
#pragma unroll
      for (int v = 0; v < 4; ++v) tgt[v] = rv[v];
      if (VISC) sig1 = T(0.5) * k.mu * (kx * kx + ky * ky);
    } else if (kind == kTermFarfield) {
#pragma unroll
      for (int v = 0; v < 4; ++v) tgt[v] = k.qinf[v];
    } else {
      tgt[0] = qp[0];
      tgt[1] = T(0);
      tgt[2] = T(0);
      tgt[3] = qp[0] * k.tw;
      if (VISC) sig1 = T(0.5) * k.mu * (kx * kx + ky * ky);
    }
    T dq[4], kd[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) dq[v] = qp[v] - tgt[v];
    penalty_apply(qp, k.gam, kx, ky, side, dq, kd);
    T sat[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) sat[v] = -(sigI * kd[v] + sig1 * dq[v]) * T(1.0 / SBP_P0);
    if constexpr (VISC) {
      if (kind == kTermInterface) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T own = kx * Fv[c] + ky * Gv[c];
          T hat = kx * rv[4 + c] + ky * rv[7 + c];
          sat[c + 1] += T(0.5) * T(side) * (own - hat) * T(1.0 / SBP_P0);
        }
      }
    }
    T sc = kind == kTermInterface ? scale : T(1);
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[v] += sc * sat[v];
  }
}

// Sponge strength at (gi, gj): by the index distance to the nearest far-field face (0 outside
// the layer). The layer's term -sigma (q - qinf) is added after the SAT terms.
template <typename T>
__device__ __forceinline__ T sponge_sigma(const KConst<T> &k, const DevMesh &m, int gi, int gj) {
  int d = 1 << 30;
  if (k.sponge_faces & 1) d = min(d, gi);
  if (k.sponge_faces & 2) d = min(d, m.ni - 1 - gi);
  if (k.sponge_faces & 4) d = min(d, gj);
  if (k.sponge_faces & 8) d = min(d, m.nj - 1 - gj);
  return d < k.sponge_d ? k.sponge_tab[d] : T(0);
}

// SAT entries of the CTA's rows: the tile lists are grouped by 32 x 8 tiles in column-major
// tile order, so a 32 x TY block owns a contiguous range.
// A block of fewer than 8 rows gets its 8-row group's range (a superset, searched by key).
template <int TY>
__device__ __forceinline__ void tile_sat_range(const RhsLaunch &a, int bx, int by, int &s0, int &s1) {
  const int nty8 = (a.m.nj + 7) / 8;
  const int ty8 = (by * TY) / 8, ty8e = min(((by + 1) * TY + 7) / 8, nty8);
  const int id0 = bx * nty8 + ty8, id1 = bx * nty8 + ty8e;
  s0 = a.tile_sat[id0];
  s1 = a.tile_sat[id1];
}

template <typename T, bool VISC, int TY>
struct FluxTile {
  // one point per thread up to 8 rows (128 threads for 4-row tiles), kNT threads beyond
  static constexpr int TX = kTileX, NT = TX * TY < kNT ? TX * TY : kNT, PPT = TX * TY / NT;
  static constexpr int H = VISC ? 3 : 0, RX = TX + 2 * H, RY = TY + 2 * H, RN = RX * RY;
};

// Contravariant fluxes at every point of a 32 x TY tile, then the SAT terms of the tile's
// boundary and receiver points (their state, primitives and gradients are at hand here).
template <typename T, bool VISC, bool CURV, int TY>
__device__ __forceinline__ void flux_tile(const RhsLaunch &a, int bx, int by, T *prim, uint8_t *scls) {
  using F = FluxTile<T, VISC, TY>;
  constexpr int TX = F::TX, NT = F::NT, H = F::H, RX = F::RX, RN = F::RN;
  const DevMesh &m = a.m;
  const KConst<T> &k = kc<T>(a);
  const int tid = threadIdx.x;
  const int i0 = bx * TX, j0 = by * TY;
  const T *q = static_cast<const T *>(a.q);
  T *fl = static_cast<T *>(a.flux);
  if constexpr (VISC) {
    const T *pin = static_cast<const T *>(a.prim_in);
    for (int idx = tid; idx < RN; idx += NT) {
      int gi = i0 - H + idx % RX, gj = j0 - H + idx / RX;
      bool in = wrap_index(gi, m.ni, m.per_i) & wrap_index(gj, m.nj, m.per_j);
      T pr[3] = {T(0), T(0), T(1)};
      uint8_t c = 0xFF;
      if (in) {
        size_t p = (size_t)gj * m.pitch + gi;
        if (pin) {
          pr[0] = pin[p];
          pr[1] = pin[m.field + p];
          pr[2] = pin[2 * m.field + p];
        } else {
          prim_at(q, m.field, p, k.gam, pr);
        }
        c = m.cls[p];
      }
      prim[idx] = pr[0];
      prim[RN + idx] = pr[1];
      prim[2 * RN + idx] = pr[2];
      scls[idx] = c;
    }
    __syncthreads();
  }
#pragma unroll
  for (int kk = 0; kk < F::PPT; ++kk) {
    const int li = tid % TX, lj = tid / TX + kk * (NT / TX);
    const int gi = i0 + li, gj = j0 + lj;
    if (gi >= m.ni || gj >= m.nj) continue;
    const size_t p = (size_t)gj * m.pitch + gi;
    T qp[4] = {q[p], q[m.field + p], q[2 * m.field + p], q[3 * m.field + p]};
    T mt[5];
    load_met<T, CURV>(a, gi, gj, mt);
    T u, v, pr;
    T Fx[4], Gx[4];
    if constexpr (VISC) {
      const int r = (lj + H) * RX + (li + H);
      u = prim[r];
      v = prim[RN + r];
      pr = pressure_of(k.gam, qp[3], qp[1], qp[2], u, v);  // prim_at's pressure
      T gr[6];
      smem_grads<T, CURV>(a, prim, RN, r, RX, scls[r], mt, gr);
      T Fv[3], Gv[3];
      visc_flux_k(k, u, v, gr, Fv, Gv);
      ns_flux_x(qp, u, pr, Fv, Fx);
      ns_flux_y(qp, v, pr, Gv, Gx);
    } else {
      inviscid_flux(qp, k.gam, Fx, Gx, u, v, pr);
    }
    // contravariant fluxes on curvilinear meshes; Cartesian meshes keep F and G (the update's
    // scaled rows give d/dx, d/dy)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      fl[c * m.field + p] = CURV ? dot2_rn(mt[0], Fx[c], mt[1], Gx[c]) : Fx[c];
      fl[(4 + c) * m.field + p] = CURV ? dot2_rn(mt[2], Fx[c], mt[3], Gx[c]) : Gx[c];
    }
  }
  // SAT terms of this tile's boundary / receiver points (one thread per point)
  int s0, s1;
  tile_sat_range<TY>(a, bx, by, s0, s1);
  T *satb = static_cast<T *>(a.sat);
  for (int s = s0 + tid; s < s1; s += NT) {
    uint32_t ij = a.sat_ij[s];
    int gi = (int)(ij & 0xFFFFu), gj = (int)(ij >> 16);
    // tiles of fewer than 8 rows share their 8-row group's SAT range: each takes its own rows
    if (TY < 8 && (gj < j0 || gj >= j0 + TY)) continue;
    size_t p = (size_t)gj * m.pitch + gi;
    T qp[4] = {q[p], q[m.field + p], q[2 * m.field + p], q[3 * m.field + p]};
    T mt[5];
    load_met<T, CURV>(a, gi, gj, mt);
    T Fv[3] = {0, 0, 0}, Gv[3] = {0, 0, 0};
    if constexpr (VISC) {
      const int r = (gj - j0 + H) * RX + (gi - i0 + H);
      T gr[6];
      smem_grads<T, CURV>(a, prim, RN, r, RX, scls[r], mt, gr);
      visc_flux_k(k, prim[r], prim[RN + r], gr, Fv, Gv);
    }
    T acc[4];
    sat_terms<T, VISC>(a, s, qp, mt, Fv, Gv, acc);
#pragma unroll
    for (int c = 0; c < 4; ++c) satb[c * a.nsat + s] = acc[c];
  }
}

template <typename T, int TY>
struct UpdTile {
  static constexpr int TX = kTileX, NT = TX * TY < kNT ? TX * TY : kNT, PPT = TX * TY / NT;
  static constexpr int RX = TX + 6, RY = TY + 6, RN = RX * RY;
  static constexpr size_t bytes = (size_t)(8 * RN) * sizeof(T);
};

// SBP derivatives of the fluxes, the tile's SAT terms, and the epilogue.
template <typename T, bool VISC, bool CURV, int TY>
__device__ __forceinline__ void update_tile(const RhsLaunch &a, int bx, int by, T *sf) {
  using U = UpdTile<T, TY>;
  constexpr int TX = U::TX, NT = U::NT, RX = U::RX, RN = U::RN;
  const DevMesh &m = a.m;
  const int tid = threadIdx.x;
  const int i0 = bx * TX, j0 = by * TY;
  const T *q = static_cast<const T *>(a.q);
  const T *fl = static_cast<const T *>(a.flux);
  const T *satb = static_cast<const T *>(a.sat);

  for (int idx = tid; idx < RN; idx += NT) {
    int gi = i0 - 3 + idx % RX, gj = j0 - 3 + idx / RX;
    bool in = wrap_index(gi, m.ni, m.per_i) & wrap_index(gj, m.nj, m.per_j);
    size_t p = in ? (size_t)gj * m.pitch + gi : 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) sf[c * RN + idx] = in ? fl[c * m.field + p] : T(0);
  }
  __syncthreads();
  int s0, s1;
  tile_sat_range<TY>(a, bx, by, s0, s1);
#pragma unroll
  for (int kk = 0; kk < U::PPT; ++kk) {
    const int li = tid % TX, lj = tid / TX + kk * (NT / TX);
    const int gi = i0 + li, gj = j0 + lj;
    if (gi >= m.ni || gj >= m.nj) continue;
    const size_t p = (size_t)gj * m.pitch + gi;
    unsigned code = m.cls[p];
    const int r = (lj + 3) * RX + (li + 3);
    T rhs[4] = {T(0), T(0), T(0), T(0)};
    if ((code & 15u) != 15u) {
      const Row<T> ri = CURV ? decode_row<T>(code & 15u) : decode_row_w<T>(code & 15u, kc<T>(a).wx);
      const Row<T> rj = CURV ? decode_row<T>(code >> 4) : decode_row_w<T>(code >> 4, kc<T>(a).wy);
      const T *pi[4], *pj[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        pi[e] = sf + r + ri.off[e];
        pj[e] = sf + r + rj.off[e] * RX;
      }
      if (CURV) {
        const T jac = static_cast<const T *>(m.met)[4 * m.field + p];
#pragma unroll
        for (int c = 0; c < 4; ++c) rhs[c] = -jac * (row_sum(ri, pi, c * RN) + row_sum(rj, pj, (4 + c) * RN));
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) rhs[c] = -(row_sum(ri, pi, c * RN) + row_sum(rj, pj, (4 + c) * RN));
      }
      if (s0 < s1) {
        // the tile's SAT entries are sorted by (j, i): binary search for this point
        uint32_t key = (uint32_t)gi | ((uint32_t)gj << 16);
        int lo = s0, hi = s1;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          uint32_t km = a.sat_ij[mid];
          if ((km >> 16) < (key >> 16) || ((km >> 16) == (key >> 16) && (km & 0xFFFFu) < (key & 0xFFFFu))) lo = mid + 1;
          else hi = mid;
        }
        if (lo < s1 && a.sat_ij[lo] == key) {
#pragma unroll
          for (int c = 0; c < 4; ++c) rhs[c] += satb[c * a.nsat + lo];
        }
      }
      if (kc<T>(a).sponge_d > 0) {
        const T sg = sponge_sigma(kc<T>(a), m, gi, gj);
        if (sg != T(0)) {
#pragma unroll
          for (int c = 0; c < 4; ++c) rhs[c] = fma_rn(-sg, q[c * m.field + p] - kc<T>(a).qinf[c], rhs[c]);
        }
      }
    }
    T *out = static_cast<T *>(a.out);
    if (a.mode == 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) out[c * m.field + p] = rhs[c];
    } else {
      T *qn = static_cast<T *>(a.qnext);
      T q0[4], qv[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) q0[c] = q[c * m.field + p];
      ab_update<T, 4>(q0, a.hold, a.alpha, a.nold, m.field, p, rhs, qv, (code & 15u) != 15u ? a.err : nullptr);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        out[c * m.field + p] = rhs[c];
        qn[c * m.field + p] = qv[c];
      }
      if (VISC && a.prim_out) {
        // the next right-hand side's primitives of this point (prim_at's arithmetic)
        T pr[3];
        prim4(qv[0], qv[1], qv[2], qv[3], kc<T>(a).gam, pr);
        T *po = static_cast<T *>(a.prim_out);
#pragma unroll
        for (int f = 0; f < 3; ++f) po[f * m.field + p] = pr[f];
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Donor-point values for the fused gather of k_rhs. One thread per (extrapolation set, distinct
// donor point): the state q + sum_k beta_k hist_k (FP64 accumulation; Sec. 3.3 Step 2 for the
// slow extrapolant at a micro time) and, for Navier-Stokes, the Cartesian viscous fluxes of that
// state by the donor mesh's own SBP derivatives.
template <typename T>
__device__ __forceinline__ void set_state(const DonorLaunch &a, int set, size_t p, T out[4]) {
  const T *q = static_cast<const T *>(a.q);
  double acc[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) acc[v] = to_f64(q[v * a.d.field + p]);
  // each history slot's four values loaded together (the same sums in the same order)
#pragma unroll
  for (int k = 0; k < kMaxHist; ++k) {
    if (k < a.nb[set]) {
      const T *h = static_cast<const T *>(a.hist[k]) + p;
      T hv[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) hv[v] = h[v * a.d.field];
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[v] += a.beta[set][k] * to_f64(hv[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) out[v] = (T)acc[v];
}

// Primitives (u, v, T) of an extrapolated donor state with one fixed rounding order, so that
// the single-system kernel and the batched persistent kernel give the same bits whatever the
// compiler contracts.
template <typename T>
__device__ __forceinline__ void donor_prims(const T s[4], T gam, T pr[3]) {
  const T ri = T(1) / s[0];
  pr[0] = mul_rn(s[1], ri);
  pr[1] = mul_rn(s[2], ri);
  const T ke = fma_rn(s[1], s[1], mul_rn(s[2], s[2]));
  pr[2] = mul_rn(mul_rn(mul_rn(gam, gam - T(1)), fma_rn(mul_rn(T(-0.5), ke), ri, s[3])), ri);
}

// Navier-Stokes donor values of one (set, donor point) pair by a 16-lane group; every lane of
// the warp must call this (shuffles), with valid = false for lanes past the end. The weighted
// taps are rounded products, so the butterfly's sums take no contraction either.
template <typename T, bool CURV>
__device__ __forceinline__ void donor_group(const DonorLaunch &a, int pair, bool valid);

template <typename T, bool CURV>
__device__ __forceinline__ void donor_group(const DonorLaunch &a, int pair, bool valid) {
  {
    const int l = threadIdx.x & 15;
    const int set = valid ? pair / a.npts : 0, d = valid ? pair - set * a.npts : 0;
    const uint32_t ij = valid ? a.pts[d] : 0u;
    const int ii = (int)(ij & 0xFFFFu), jj = (int)(ij >> 16);
    const size_t p = (size_t)jj * a.d.pitch + ii;
    const unsigned code = valid ? a.d.cls[p] : 0xFFu;
    const T gam = (T)a.g.gamma;
    int pi = ii, pj = jj, dir = 2;
    T w = T(0);
    if (l >= 1 && l <= 8) {
      dir = l <= 4 ? 0 : 1;
      int row, sgn;
      row_of(dir == 0 ? (code & 15u) : (code >> 4), row, sgn);
      const int e = (l - 1) & 3;
      w = T(sgn) * wgt<T>(row, e);
      const int off = sgn * c_off[row][e];
      if (dir == 0) pi += off;
      else pj += off;
      wrap_index(pi, a.d.ni, a.d.per_i);
      wrap_index(pj, a.d.nj, a.d.per_j);
    }
    const bool act = valid && (l == 0 || w != T(0));
    T s[4] = {T(1), T(0), T(0), T(2.5)};
    if (act) set_state(a, set, (size_t)pj * a.d.pitch + pi, s);
    T pr[3];
    donor_prims(s, gam, pr);
    T cx[3], cy[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      cx[f] = (act && dir == 0) ? mul_rn(w, pr[f]) : T(0);
      cy[f] = (act && dir == 1) ? mul_rn(w, pr[f]) : T(0);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        cx[f] += __shfl_xor_sync(0xffffffffu, cx[f], o);
        cy[f] += __shfl_xor_sync(0xffffffffu, cy[f], o);
      }
    }
    if (valid && l == 0) {
      const int st = a.stride ? a.stride : a.npts;
      T *dv = static_cast<T *>(a.dv) + (size_t)set * 10 * st;
#pragma unroll
      for (int v = 0; v < 4; ++v) dv[v * st + d] = s[v];
      const T mu = (T)a.g.mu, kap = (T)(a.g.mu / (a.g.pr * (a.g.gamma - 1.0)));
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
        gr[2 * f] = grad_x<T, true>(mt, cx[f], cy[f]);
        gr[2 * f + 1] = grad_y<T, true>(mt, cx[f], cy[f]);
      }
      T Fv[3], Gv[3];
      viscous_flux(pr[0], pr[1], gr, mu, kap, Fv, Gv);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dv[(4 + c) * st + d] = Fv[c];
        dv[(7 + c) * st + d] = Gv[c];
      }
    }
  }
}

}  // namespace sbp
