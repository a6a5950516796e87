// Single-pass right-hand side by column marching (k_col): each thread owns one mesh column and a
// CTA of NT threads a strip of NT - 12 output columns (plus 6 halo columns per side); the CTA
// marches up a chunk of rows one row per tick. The j-direction stencils read their taps from
// per-thread register windows of the last rows (primitives, contravariant fluxes F^_eta, class
// bytes), the i-direction stencils from one shared-memory row per stage, so a point costs few
// shared-memory operations and no ring-index arithmetic. Per tick, with L the row loaded:
//   P  primitives (u, v, T) of row L: registers (window of 8 rows) and a shared row
//   G  i-gradients of the primitives at row L (window of 4 rows)
//   F  contravariant fluxes of row F = L - 3 (j-gradients from the primitive window): F^_xi to a
//      shared row, F^_eta to a window of 8 rows; the i-divergence of F^_xi at row F (window of 4)
//   O  row O = L - 6: -J (D_xi F^_xi + D_eta F^_eta) with the j-divergence from the F^_eta
//      window, SAT terms (from k_sat), sponge, epilogue (dq/dt, or the MRAB update)
// Every point takes the same floating-point operations in the same order as the kernel pair
// and the marching kernel (flux_tile / update_tile / march_*_point), so all designs give the
// same bits. The windows are indexed by compile-time slots: the tick loop is unrolled by 8.
#pragma once
#include "sbp_dev.cuh"
#include "sbp_march_impl.cuh"  // k_sat, kNoCls

namespace sbp {

template <typename T, bool VISC, bool CURV, int NT_>
struct Col {
  static constexpr int NT = NT_, W = NT - 12;  // threads, output columns per strip
};

// Register windows of one thread. Slot s of an 8-row window holds row r with (r & 7) == s; of a
// 4-row window, (r & 3) == s.
template <typename T>
struct ColWin {
  T p[3][8];      // primitives u, v, T
  T q[4][4];      // conserved state: q[slot][variable]
  unsigned c[8];  // class byte (kNoCls: no point)
  T gi[4][3];     // i-gradients (d/dxi, Cartesian d/dx) of u, v, T: gi[slot][field]
  T fe[4][8];     // F^_eta (Cartesian: G): fe[variable][slot]
  T di[4][4];     // i-divergence of F^_xi: di[slot][variable]
  T qn[4];        // the next row's state, loaded one tick ahead
  unsigned cn;
};

// Tap of an 8-row window at row base + off (off in -3..3), slot of base known at compile time.
template <int B, typename V>
__device__ __forceinline__ V win_tap(const V (&w)[8], int off) {
  switch (off) {
    case -3: return w[(B + 5) & 7];
    case -2: return w[(B + 6) & 7];
    case -1: return w[(B + 7) & 7];
    case 1: return w[(B + 1) & 7];
    case 2: return w[(B + 2) & 7];
    case 3: return w[(B + 3) & 7];
    default: return w[B & 7];
  }
}

// row_sum / central_sum over window taps (the same operation order: acc = 0, then the four taps
// in order, negated for a closure counted from the segment's high end).
template <typename T>
__device__ __forceinline__ T taps_sum(const Row<T> &r, const T t[4]) {
  T acc = T(0);
#pragma unroll
  for (int e = 0; e < 4; ++e) acc += r.w[e] * t[e];
  return r.neg ? -acc : acc;
}
template <typename T>
__device__ __forceinline__ T central_taps(const T t[4]) {
  T acc = T(0);
  acc += CentralRow<T>::w0 * t[0];
  acc += CentralRow<T>::w1 * t[1];
  acc += CentralRow<T>::w2 * t[2];
  acc += CentralRow<T>::w3 * t[3];
  return acc;
}
template <typename T>
__device__ __forceinline__ T central_taps_w(const T t[4], const T w[4]) {
  T acc = T(0);
#pragma unroll
  for (int e = 0; e < 4; ++e) acc += w[e] * t[e];
  return acc;
}

// O: the output of row O (slots O8, O4 of its class byte / i-divergence; the F^_eta taps at
// O - 3 .. O + 3 are the window rows): -J (D_xi F^_xi + D_eta F^_eta) (Cartesian: -(d/dx F +
// d/dy G)), the SAT terms, the sponge term, then dq/dt or the MRAB update (march_tile's epilogue).
template <typename T, bool VISC, bool CURV, int NT, int O8, int O4>
__device__ __forceinline__ void col_output(const RhsLaunch &a, const ColWin<T> &w, int O, int j0, int j1, int t,
                                           int gu, int gi) {
  const DevMesh &m = a.m;
  const KConst<T> &k = kc<T>(a);
  if (t < 6 || t >= NT - 6 || O < j0 || O >= j1 || gu >= m.ni || gi < 0) return;
  const int gj = O;
  const size_t p = (size_t)gj * m.pitch + gi;
  const unsigned code = w.c[O8];
  const T *q = static_cast<const T *>(a.q);
  T rhs[4] = {T(0), T(0), T(0), T(0)};
  if ((code & 15u) != 15u) {
    const unsigned cj = code >> 4;
    T dj[4];
    if (cj == 0u) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const T tp[4] = {w.fe[c][(O8 + 6) & 7], w.fe[c][(O8 + 7) & 7], w.fe[c][(O8 + 1) & 7], w.fe[c][(O8 + 2) & 7]};
        dj[c] = CURV ? central_taps(tp) : central_taps_w(tp, k.wy[4]);
      }
    } else {
      const Row<T> rj = CURV ? decode_row<T>(cj) : decode_row_w<T>(cj, k.wy);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        T tp[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) tp[e] = win_tap<O8>(w.fe[c], rj.off[e]);
        dj[c] = taps_sum(rj, tp);
      }
    }
    if (CURV) {
      const T jac = static_cast<const T *>(m.met)[4 * m.field + p];
#pragma unroll
      for (int c = 0; c < 4; ++c) rhs[c] = -jac * (w.di[O4][c] + dj[c]);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) rhs[c] = -(w.di[O4][c] + dj[c]);
    }
    // SAT points are boundary or receiver points: a closure row in some direction
    if (code != 0u) {
      const int nty8 = (m.nj + 7) / 8;
      const int tile = (gi / kTileX) * nty8 + gj / 8;
      const int s0 = a.tile_sat[tile], s1 = a.tile_sat[tile + 1];
      if (s0 < s1) {
        const uint32_t key = (uint32_t)gi | ((uint32_t)gj << 16);
        int lo = s0, hi = s1;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          const uint32_t km = a.sat_ij[mid];
          if ((km >> 16) < (key >> 16) || ((km >> 16) == (key >> 16) && (km & 0xFFFFu) < (key & 0xFFFFu)))
            lo = mid + 1;
          else
            hi = mid;
        }
        if (lo < s1 && a.sat_ij[lo] == key) {
          const T *satb = static_cast<const T *>(a.sat);
#pragma unroll
          for (int c = 0; c < 4; ++c) rhs[c] += satb[c * a.nsat + lo];
        }
      }
    }
    if (k.sponge_d > 0) {
      const T sg = sponge_sigma(k, m, gi, gj);
      if (sg != T(0)) {
#pragma unroll
        for (int c = 0; c < 4; ++c) rhs[c] = fma_rn(-sg, q[c * m.field + p] - k.qinf[c], rhs[c]);
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
  }
}

// The tick of load row L (L & 7 == PH). t: the thread's window column, gu its unwrapped mesh
// column, gi the wrapped one (-1 outside the mesh); rows [j0, j1) are this CTA's output rows.
template <typename T, bool VISC, bool CURV, int NT, int PH>
__device__ __forceinline__ void col_tick(const RhsLaunch &a, ColWin<T> &w, int L, int j0, int j1, int t, int gu,
                                         int gi, T *sp, T *sf) {
  const DevMesh &m = a.m;
  const KConst<T> &k = kc<T>(a);
  const T *q = static_cast<const T *>(a.q);
  constexpr int S8 = PH & 7, S4 = PH & 3;          // slots of row L
  constexpr int F8 = (PH + 5) & 7, F4 = (PH + 1) & 3;  // row F = L - 3
  constexpr int O8 = (PH + 2) & 7, O4 = (PH + 2) & 3;  // row O = L - 6
  // P: row L from the prefetched registers; the prefetch of row L + 1
#pragma unroll
  for (int v = 0; v < 4; ++v) w.q[S4][v] = w.qn[v];
  w.c[S8] = w.cn;
  {
    int gj = L + 1;
    w.cn = kNoCls;
    if (gi >= 0 && L + 1 < j1 + 6 && wrap_index(gj, m.nj, m.per_j)) {
      const size_t p = (size_t)gj * m.pitch + gi;
#pragma unroll
      for (int v = 0; v < 4; ++v) w.qn[v] = q[v * m.field + p];
      w.cn = m.cls[p];
    }
  }
  if constexpr (VISC) {
    T pr[3] = {T(0), T(0), T(1)};
    if (w.c[S8] != kNoCls) prim4(w.q[S4][0], w.q[S4][1], w.q[S4][2], w.q[S4][3], k.gam, pr);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      w.p[f][S8] = pr[f];
      sp[f * NT + t] = pr[f];
    }
  }
  __syncthreads();
  // G: i-gradients of the primitives at row L (flux columns)
  if constexpr (VISC) {
    if (t >= 3 && t < NT - 3) {
      const unsigned ci = w.c[S8] & 15u;
      if (ci == 0u) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          const T tp[4] = {sp[f * NT + t - 2], sp[f * NT + t - 1], sp[f * NT + t + 1], sp[f * NT + t + 2]};
          w.gi[S4][f] = CURV ? central_taps(tp) : central_taps_w(tp, k.wx[4]);
        }
      } else {
        const Row<T> ri = CURV ? decode_row<T>(ci) : decode_row_w<T>(ci, k.wx);
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          T tp[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) tp[e] = sp[f * NT + t + ri.off[e]];
          w.gi[S4][f] = taps_sum(ri, tp);
        }
      }
    }
  }
  // F: contravariant fluxes of row F = L - 3
  {
    const int F = L - 3;
    int gj = F;
    const bool act = t >= 3 && t < NT - 3 && w.c[F8] != kNoCls && F >= j0 - 3 && F < j1 + 3 &&
                     wrap_index(gj, m.nj, m.per_j);
    T fx[4] = {T(0), T(0), T(0), T(0)}, fy[4] = {T(0), T(0), T(0), T(0)};
    if (act) {
      const unsigned code = w.c[F8];
      T qp[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) qp[v] = w.q[F4][v];
      T mt[5];
      load_met<T, CURV>(a, gi, gj, mt);
      T u, v, pr, Fx[4], Gx[4];
      if constexpr (VISC) {
        u = w.p[0][F8];
        v = w.p[1][F8];
        pr = pressure_of(k.gam, qp[3], qp[1], qp[2], u, v);  // prim_at's pressure
        const unsigned cj = code >> 4;
        T gr[6];
        if (cj == 0u) {
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            const T tp[4] = {w.p[f][(F8 + 6) & 7], w.p[f][(F8 + 7) & 7], w.p[f][(F8 + 1) & 7], w.p[f][(F8 + 2) & 7]};
            const T deta = CURV ? central_taps(tp) : central_taps_w(tp, k.wy[4]);
            const T dxi = w.gi[F4][f];
            if (CURV) {
              gr[2 * f] = grad_x<T, true>(mt, dxi, deta);
              gr[2 * f + 1] = grad_y<T, true>(mt, dxi, deta);
            } else {
              gr[2 * f] = dxi;
              gr[2 * f + 1] = deta;
            }
          }
        } else {
          const Row<T> rj = CURV ? decode_row<T>(cj) : decode_row_w<T>(cj, k.wy);
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            T tp[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) tp[e] = win_tap<F8>(w.p[f], rj.off[e]);
            const T deta = taps_sum(rj, tp);
            const T dxi = w.gi[F4][f];
            if (CURV) {
              gr[2 * f] = grad_x<T, true>(mt, dxi, deta);
              gr[2 * f + 1] = grad_y<T, true>(mt, dxi, deta);
            } else {
              gr[2 * f] = dxi;
              gr[2 * f + 1] = deta;
            }
          }
        }
        T Fv[3], Gv[3];
        visc_flux_k(k, u, v, gr, Fv, Gv);
        ns_flux_x(qp, u, pr, Fv, Fx);
        ns_flux_y(qp, v, pr, Gv, Gx);
      } else {
        inviscid_flux(qp, k.gam, Fx, Gx, u, v, pr);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        fx[c] = CURV ? dot2_rn(mt[0], Fx[c], mt[1], Gx[c]) : Fx[c];
        fy[c] = CURV ? dot2_rn(mt[2], Fx[c], mt[3], Gx[c]) : Gx[c];
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      sf[c * NT + t] = fx[c];
      w.fe[c][F8] = fy[c];
    }
  }
  __syncthreads();
  // i-divergence of F^_xi at row F (output columns)
  if (t >= 6 && t < NT - 6) {
    const unsigned ci = w.c[F8] & 15u;
    if (ci == 0u) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const T tp[4] = {sf[c * NT + t - 2], sf[c * NT + t - 1], sf[c * NT + t + 1], sf[c * NT + t + 2]};
        w.di[F4][c] = CURV ? central_taps(tp) : central_taps_w(tp, k.wx[4]);
      }
    } else {
      const Row<T> ri = CURV ? decode_row<T>(ci) : decode_row_w<T>(ci, k.wx);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        T tp[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) tp[e] = sf[c * NT + t + ri.off[e]];
        w.di[F4][c] = taps_sum(ri, tp);
      }
    }
  }
  col_output<T, VISC, CURV, NT, O8, O4>(a, w, L - 6, j0, j1, t, gu, gi);
}

// One strip (blockIdx.x) x chunk (blockIdx.y) per CTA of NT threads; rows are loaded from
// j0 - 6 to j1 + 5, in groups of 8 ticks whose register-window slots are compile-time.
template <typename T, bool VISC, bool CURV, int NT>
__global__ void __launch_bounds__(NT) k_col(const RhsLaunch a, int chunk) {
  __shared__ T sp[VISC ? 3 * NT : 1];
  __shared__ T sf[4 * NT];
  const DevMesh &m = a.m;
  const int t = threadIdx.x;
  const int i0 = blockIdx.x * Col<T, VISC, CURV, NT>::W;
  const int j0 = blockIdx.y * chunk, j1 = min(j0 + chunk, m.nj);
  const int gu = i0 - 6 + t;
  int gi = gu;
  if (!wrap_index(gi, m.ni, m.per_i)) gi = -1;
  ColWin<T> w;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    w.c[s] = kNoCls;
#pragma unroll
    for (int f = 0; f < 3; ++f) w.p[f][s] = T(0);
#pragma unroll
    for (int c = 0; c < 4; ++c) w.fe[c][s] = T(0);
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
#pragma unroll
    for (int c = 0; c < 4; ++c) w.q[s][c] = w.di[s][c] = T(0);
#pragma unroll
    for (int f = 0; f < 3; ++f) w.gi[s][f] = T(0);
  }
  const int Ls = j0 - 6, Le = j1 + 6;  // load rows
  {
    const T *q = static_cast<const T *>(a.q);
    int gj = Ls;
    w.cn = kNoCls;
#pragma unroll
    for (int v = 0; v < 4; ++v) w.qn[v] = T(0);
    if (gi >= 0 && wrap_index(gj, m.nj, m.per_j)) {
      const size_t p = (size_t)gj * m.pitch + gi;
#pragma unroll
      for (int v = 0; v < 4; ++v) w.qn[v] = q[v * m.field + p];
      w.cn = m.cls[p];
    }
  }
  T *spp = sp, *sfp = sf;
  for (int Lg = (Ls >> 3) << 3; Lg < Le; Lg += 8) {
#define SBP_COL_TICK(PH)                                                                         \
    if (Lg + PH >= Ls && Lg + PH < Le) col_tick<T, VISC, CURV, NT, PH>(a, w, Lg + PH, j0, j1, t, gu, gi, spp, sfp);
    SBP_COL_TICK(0)
    SBP_COL_TICK(1)
    SBP_COL_TICK(2)
    SBP_COL_TICK(3)
    SBP_COL_TICK(4)
    SBP_COL_TICK(5)
    SBP_COL_TICK(6)
    SBP_COL_TICK(7)
#undef SBP_COL_TICK
  }
}

template <typename T, bool VISC, bool CURV, int NT>
static cudaError_t launch_col_nt(const RhsLaunch &a, cudaStream_t s) {
  if (a.m.ni < NT || a.chunk < 1) return cudaErrorInvalidValue;
  if (a.nsat > 0) {
    k_sat<T, VISC, CURV><<<(a.nsat + 127) / 128, 128, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  constexpr int W = Col<T, VISC, CURV, NT>::W;
  dim3 grid((a.m.ni + W - 1) / W, (a.m.nj + a.chunk - 1) / a.chunk);
  k_col<T, VISC, CURV, NT><<<grid, NT, 0, s>>>(a, a.chunk);
  return cudaGetLastError();
}

template <typename T, bool VISC, bool CURV>
static cudaError_t launch_col_w(const RhsLaunch &a, cudaStream_t s) {
  if (a.strip == kColW128) return launch_col_nt<T, VISC, CURV, 128>(a, s);
  if (a.strip == kColW256) return launch_col_nt<T, VISC, CURV, 256>(a, s);
  return cudaErrorInvalidValue;
}

}  // namespace sbp
