// CUDA kernels (sm_103a) besides the right-hand side: interpolation to receivers, donor values
// of the MRAB micro steps, the time-step reduction, metrics and Runge-Kutta stage combinations.
//
//  k_interp      donor-cell Lagrange interpolation with the slow-state extrapolation, one
//                half-warp per receiver (Sec. 2.2, Sec. 3.3 Step 2).
//  k_donor_vals  per distinct donor point: extrapolated state and viscous fluxes (Sec. 3.3).
//  k_dt          stable step estimate, min-reduced over the mesh (Sec. 4.1).
//  k_metrics     metric terms by the derivative operator (Sec. 2.1; setup only).
//  k_axpy        Runge-Kutta stage combinations of the bootstrap (Sec. 3.1).
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>
#include <cstring>

#include "sbp_dev.cuh"

namespace sbp {

// ---------------------------------------------------------------------------------------------
// Interpolation. A half-warp per receiver: lane l of the half holds donor (l & 3, l >> 2) of
// the 4x4 stencil; the weighted values are summed with shuffles.
template <typename T>
__device__ __forceinline__ void donor_state(const InterpLaunch &a, size_t p, T out[4]) {
  const T *q = static_cast<const T *>(a.q);
  double acc[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) acc[v] = to_f64(q[v * a.d.field + p]);
  // each history slot's four values loaded together (the same sums in the same order)
#pragma unroll
  for (int k = 0; k < kMaxHist; ++k) {
    if (k < a.nbeta) {
      const T *h = static_cast<const T *>(a.hist[k]) + p;
      T hv[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) hv[v] = h[v * a.d.field];
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[v] += a.beta[k] * to_f64(hv[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) out[v] = (T)acc[v];
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
        gr[2 * f] = grad_x<T, true>(mt, dxi[f], deta[f]);
        gr[2 * f + 1] = grad_y<T, true>(mt, dxi[f], deta[f]);
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

template <typename T, bool VISC, bool CURV>
__global__ void __launch_bounds__(128) k_donor_vals(const DonorLaunch a) {
  const int n = a.nsets * a.npts;
  if constexpr (VISC) {
    const int pair = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
    donor_group<T, CURV>(a, pair, pair < n);
    return;
  } else {
    // Euler: one thread per (set, donor point)
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int set = t / a.npts, d = t - set * a.npts;
    const uint32_t ij = a.pts[d];
    const size_t p = (size_t)(ij >> 16) * a.d.pitch + (ij & 0xFFFFu);
    const int st = a.stride ? a.stride : a.npts;
    T *dv = static_cast<T *>(a.dv) + (size_t)set * 10 * st;
    T s[4];
    set_state(a, set, p, s);
#pragma unroll
    for (int v = 0; v < 4; ++v) dv[v * st + d] = s[v];
  }
}

// Navier-Stokes: a 16-lane group per (set, donor point). Lane 0 holds the point itself, lanes
// 1-4 the xi-stencil and lanes 5-8 the eta-stencil points of its derivative classes; every lane
// evaluates the extrapolated state and primitives of its point, and the stencil-weighted
// primitives are summed over the group with shuffles.
template <typename T, bool VISC, bool CURV>
static cudaError_t launch_donor_vals_t(const DonorLaunch &a, cudaStream_t s) {
  long n = (long)a.nsets * a.npts;
  if (n == 0) return cudaSuccess;
  long threads = VISC ? 16 * n : n;
  k_donor_vals<T, VISC, CURV><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_donor_vals(const DonorLaunch &a, int dtype, bool viscous, cudaStream_t s) {
  bool curv = !a.d.cart;
  if (dtype == SBP_F64) {
    if (viscous)
      return curv ? launch_donor_vals_t<double, true, true>(a, s) : launch_donor_vals_t<double, true, false>(a, s);
    return curv ? launch_donor_vals_t<double, false, true>(a, s) : launch_donor_vals_t<double, false, false>(a, s);
  }
  if (viscous)
    return curv ? launch_donor_vals_t<float, true, true>(a, s) : launch_donor_vals_t<float, true, false>(a, s);
  return curv ? launch_donor_vals_t<float, false, true>(a, s) : launch_donor_vals_t<float, false, false>(a, s);
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
    double acc = to_f64(y[t]) + c1 * to_f64(k1[t]);
    if (k2) acc += c2 * to_f64(k2[t]);
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


// y = (double)x through widen() (the conversion of the FP32 forms' FP64 accumulations).
__global__ void k_widen(const float *x, double *y, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = widen(x[t]);
}

cudaError_t launch_widen(const float *x, double *y, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_widen<<<blocks, 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

// Adams-Bashforth state update without a new right-hand side (the slow step of the
// slowest-first MRAB variants, whose newest history value already exists):
// out = q + sum_k alpha_k hist_k in history order, FP64 accumulation.
template <typename T>
__global__ void k_ab_combine(const T *q, const ABCombine c, T *out, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    double acc = to_f64(q[t]);
    for (int k = 0; k < c.nh; ++k) acc += c.alpha[k] * to_f64(static_cast<const T *>(c.hist[k])[t]);
    out[t] = (T)acc;
  }
}

cudaError_t launch_ab_combine(const void *q, const ABCombine &c, void *out, size_t n, int dtype, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (dtype == SBP_F64) k_ab_combine<double><<<blocks, 256, 0, s>>>((const double *)q, c, (double *)out, n);
  else k_ab_combine<float><<<blocks, 256, 0, s>>>((const float *)q, c, (float *)out, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Element-type dispatch of the right-hand-side and batch launchers (instantiated per type in
// their own translation units so that they compile in parallel).
cudaError_t launch_rhs_f32(const RhsLaunch &a, bool viscous, cudaStream_t s);
cudaError_t launch_rhs_f64(const RhsLaunch &a, bool viscous, cudaStream_t s);
cudaError_t launch_batch_f32(const BatchSubstep &b, int grid, bool viscous, bool curv_fine, int ty, cudaStream_t s);
cudaError_t launch_batch_f64(const BatchSubstep &b, int grid, bool viscous, bool curv_fine, int ty, cudaStream_t s);
cudaError_t batch_grid_f32(bool viscous, bool curv_fine, int ty, int *grid);
cudaError_t batch_grid_f64(bool viscous, bool curv_fine, int ty, int *grid);

cudaError_t launch_rhs(const RhsLaunch &a, int dtype, bool viscous, cudaStream_t s) {
  return dtype == SBP_F64 ? launch_rhs_f64(a, viscous, s) : launch_rhs_f32(a, viscous, s);
}

cudaError_t launch_batch_substep(const BatchSubstep &b, int grid, int dtype, bool viscous, bool curv_fine, int ty,
                                 cudaStream_t s) {
  return dtype == SBP_F64 ? launch_batch_f64(b, grid, viscous, curv_fine, ty, s)
                          : launch_batch_f32(b, grid, viscous, curv_fine, ty, s);
}

cudaError_t batch_grid_size(int dtype, bool viscous, bool curv_fine, int ty, int *grid) {
  return dtype == SBP_F64 ? batch_grid_f64(viscous, curv_fine, ty, grid) : batch_grid_f32(viscous, curv_fine, ty, grid);
}

}  // namespace sbp
