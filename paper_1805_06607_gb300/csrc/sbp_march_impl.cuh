// Single-pass right-hand side of one mesh: a CTA owns a strip of W = kMarchW columns and a chunk of
// rows and marches up the chunk R = 4 rows at a time, keeping the rows its stencils still need
// in 16-row ring buffers in shared memory: the state, the metrics and the class bytes of the
// window columns [i0 - 6, i0 + W + 6) (copied one tick ahead with cp.async, so the copies of the
// next rows overlap this tick's arithmetic), the primitives and the contravariant fluxes.
// Per tick (rows counted from the tick's base row b):
//   P  primitives (u, v, T) of rows [b, b + R)                  (Navier-Stokes only)
//   F  contravariant fluxes of rows [b - 3, b + R - 3)           (gradients from P's ring)
//   O  SBP derivatives + SAT + epilogue of rows [b - 6, b + R - 6) (derivatives from F's ring)
// so every point's flux is computed once per strip (plus 3 halo columns per side) and the
// state, metrics and right-hand side cross HBM once. The per-point arithmetic is the split
// kernels' (flux_tile, update_tile) operation for operation, so both paths give the same bits;
// points whose rows are interior in both directions take the central stencil with its weights
// and offsets as constants. The SAT terms come from k_sat (one thread per boundary / receiver
// point) launched first.
#pragma once
#include "sbp_dev.cuh"

namespace sbp {

constexpr int kRing = 16;  // rows per ring buffer (a power of two: slot = row & 15)
constexpr unsigned kNoCls = 0x100u;  // "no class byte fetched" (outside the mesh)

template <typename T, bool VISC, bool CURV>
struct March {
  static constexpr int W = kMarchW, NT = 256, R = NT / W;
  static constexpr int PW = W + 12, FW = W + 6;
  static constexpr int QR = 4 * kRing * PW;                // state ring
  static constexpr int MR = CURV ? 5 * kRing * PW : 0;     // metric ring
  static constexpr int PR = VISC ? 3 * kRing * PW : 0;     // primitive ring
  static constexpr int FR = 8 * kRing * FW;                // flux ring
  static constexpr size_t bytes = (size_t)(QR + MR + PR + FR) * sizeof(T) + (size_t)kRing * PW;
  // ring rows live at once: q and metrics from the rows O reads (b - 6) to the prefetched
  // rows (b + 2R); primitives and fluxes R + 6
  static_assert(2 * R + 6 <= kRing && R + 6 <= kRing, "ring too short");
};

// SAT terms of every boundary / receiver point into a.sat, with the point's gradients from a
// local copy of the primitives on its stencil cross (the arithmetic of flux_tile's SAT tail).
template <typename T, bool VISC, bool CURV>
__device__ __forceinline__ void sat_point(const RhsLaunch &a, int s) {
  const DevMesh &m = a.m;
  const KConst<T> &k = kc<T>(a);
  const T *q = static_cast<const T *>(a.q);
  T *satb = static_cast<T *>(a.sat);
  uint32_t ij = a.sat_ij[s];
  int gi = (int)(ij & 0xFFFFu), gj = (int)(ij >> 16);
  size_t p = (size_t)gj * m.pitch + gi;
  T qp[4] = {q[p], q[m.field + p], q[2 * m.field + p], q[3 * m.field + p]};
  T mt[5];
  load_met<T, CURV>(a, gi, gj, mt);
  T Fv[3] = {0, 0, 0}, Gv[3] = {0, 0, 0};
  if constexpr (VISC) {
    constexpr int RX = 7, RN = 49, RC = 3 * RX + 3;
    T loc[3 * RN];
    for (int d = -3; d <= 3; ++d)
      for (int dir = 0; dir < 2; ++dir) {
        if (dir == 1 && d == 0) continue;
        int ii = gi + (dir == 0 ? d : 0), jj = gj + (dir == 1 ? d : 0);
        bool in = wrap_index(ii, m.ni, m.per_i) & wrap_index(jj, m.nj, m.per_j);
        T pr[3] = {T(0), T(0), T(1)};
        if (in) prim_at(q, m.field, (size_t)jj * m.pitch + ii, k.gam, pr);
        int r = RC + (dir == 0 ? d : d * RX);
        loc[r] = pr[0];
        loc[RN + r] = pr[1];
        loc[2 * RN + r] = pr[2];
      }
    T gr[6];
    smem_grads<T, CURV>(a, loc, RN, RC, RX, m.cls[p], mt, gr);
    visc_flux_k(k, loc[RC], loc[RN + RC], gr, Fv, Gv);
  }
  T acc[4];
  sat_terms<T, VISC>(a, s, qp, mt, Fv, Gv, acc);
#pragma unroll
  for (int c = 0; c < 4; ++c) satb[c * a.nsat + s] = acc[c];
}

template <typename T, bool VISC, bool CURV>
__global__ void __launch_bounds__(128) k_sat(const RhsLaunch a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < a.nsat) sat_point<T, VISC, CURV>(a, s);
}

// A thread's items of a window stage with `width` columns per row (R rows): row in the tick,
// ring column, and the wrapped mesh column (-1 outside the mesh or past the items). The same
// every tick, so they are worked out once per CTA.
struct WinItem {
  int rr, cc, gi;
};

template <int R, int NT>
__device__ __forceinline__ void win_items(const DevMesh &m, int width, int col0, WinItem it[2]) {
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int idx = threadIdx.x + k * NT;
    it[k].rr = idx / width;
    it[k].cc = idx - it[k].rr * width;
    int gi = col0 + it[k].cc;
    it[k].gi = (idx < R * width && wrap_index(gi, m.ni, m.per_i)) ? gi : -1;
  }
}

// Copies of rows [r0, r0 + R) of the window into the state / metric rings (cp.async) and
// class bytes into registers (cls[] per item; kNoCls where the point is outside the mesh).
template <typename T, bool VISC, bool CURV>
__device__ __forceinline__ void march_fetch(const RhsLaunch &a, const WinItem wi[2], int r0, int rmax, T *qr,
                                            T *mr, unsigned cls[2]) {
  using M = March<T, VISC, CURV>;
  constexpr int R = M::R, PW = M::PW, NT = M::NT;
  const DevMesh &m = a.m;
  const T *q = static_cast<const T *>(a.q);
  const T *met = static_cast<const T *>(m.met);
  static_assert(R * PW <= 2 * NT, "two items per thread");
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    cls[it] = kNoCls;
    const int gi = wi[it].gi, cc = wi[it].cc;
    const int row = r0 + wi[it].rr;
    int gj = row;
    if (gi < 0 || row >= rmax || !wrap_index(gj, m.nj, m.per_j)) continue;
    const size_t p = (size_t)gj * m.pitch + gi;
    const int o = (row & (kRing - 1)) * PW + cc;
#pragma unroll
    for (int v = 0; v < 4; ++v) cp_async_n<sizeof(T)>(qr + v * kRing * PW + o, q + v * m.field + p);
    if (CURV) {
#pragma unroll
      for (int c = 0; c < 5; ++c) cp_async_n<sizeof(T)>(mr + c * kRing * PW + o, met + c * m.field + p);
    }
    cls[it] = m.cls[p];
  }
}

template <typename T, bool VISC, bool CURV>
__device__ __forceinline__ void march_store_cls(const WinItem wi[2], int r0, uint8_t *cr, const unsigned cls[2]) {
  using M = March<T, VISC, CURV>;
  constexpr int PW = M::PW;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    if (cls[it] == kNoCls) continue;
    cr[((r0 + wi[it].rr) & (kRing - 1)) * PW + wi[it].cc] = (uint8_t)cls[it];
  }
}

// Contravariant fluxes of one point (ring row `row`, window column pc) into the flux ring;
// INT: the point is interior in both directions (central stencil as constants). The state and
// metric rings have QW columns per row with the window's column 0 at ring column qsh (QW = PW,
// qsh = 0 for the cp.async-staged kernel); the primitive ring has PW.
template <typename T, bool VISC, bool CURV, bool INT, int QW = March<T, VISC, CURV>::PW>
__device__ __forceinline__ void march_flux_point(const RhsLaunch &a, const T *qr, const T *mr, const T *prim, T *fr,
                                                 int row, int pc, unsigned code, int qsh = 0) {
  using M = March<T, VISC, CURV>;
  constexpr int PW = M::PW, FW = M::FW;
  const KConst<T> &k = kc<T>(a);
  const int sl = row & (kRing - 1), o = sl * PW + pc, qo = sl * QW + pc + qsh;
  T qp[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) qp[v] = qr[v * kRing * QW + qo];
  T mt[5];
  if (CURV) {
#pragma unroll
    for (int c = 0; c < 5; ++c) mt[c] = mr[c * kRing * QW + qo];
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) mt[c] = k.mc[c];
  }
  T u, v, pr;
  T Fx[4], Gx[4];
  if constexpr (VISC) {
    u = prim[o];
    v = prim[kRing * PW + o];
    pr = pressure_of(k.gam, qp[3], qp[1], qp[2], u, v);  // prim_at's pressure
    const T *pi[4], *pj[4];
    Row<T> ri, rj;
    if (INT) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int off = e < 2 ? e - 2 : e - 1;
        pi[e] = prim + o + off;
        pj[e] = prim + ((row + off) & (kRing - 1)) * PW + pc;
      }
    } else {
      ri = CURV ? decode_row<T>(code & 15u) : decode_row_w<T>(code & 15u, k.wx);
      rj = CURV ? decode_row<T>(code >> 4) : decode_row_w<T>(code >> 4, k.wy);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        pi[e] = prim + o + ri.off[e];
        pj[e] = prim + ((row + rj.off[e]) & (kRing - 1)) * PW + pc;
      }
    }
    T gr[6];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      if (CURV) {
        T dxi = INT ? central_sum(pi, f * kRing * PW) : row_sum(ri, pi, f * kRing * PW);
        T deta = INT ? central_sum(pj, f * kRing * PW) : row_sum(rj, pj, f * kRing * PW);
        gr[2 * f] = grad_x<T, true>(mt, dxi, deta);
        gr[2 * f + 1] = grad_y<T, true>(mt, dxi, deta);
      } else {
        gr[2 * f] = INT ? central_sum_w(pi, f * kRing * PW, k.wx[4]) : row_sum(ri, pi, f * kRing * PW);
        gr[2 * f + 1] = INT ? central_sum_w(pj, f * kRing * PW, k.wy[4]) : row_sum(rj, pj, f * kRing * PW);
      }
    }
    T Fv[3], Gv[3];
    visc_flux_k(k, u, v, gr, Fv, Gv);
    ns_flux_x(qp, u, pr, Fv, Fx);
    ns_flux_y(qp, v, pr, Gv, Gx);
  } else {
    inviscid_flux(qp, k.gam, Fx, Gx, u, v, pr);
  }
  const int fo = sl * FW + pc - 3;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    fr[c * kRing * FW + fo] = CURV ? dot2_rn(mt[0], Fx[c], mt[1], Gx[c]) : Fx[c];
    fr[(4 + c) * kRing * FW + fo] = CURV ? dot2_rn(mt[2], Fx[c], mt[3], Gx[c]) : Gx[c];
  }
}

// -J (D_xi F^_xi + D_eta F^_eta) of one point from the flux ring (flux column fc); on Cartesian
// meshes -(d/dx F + d/dy G) with the scaled rows of k.
template <typename T, bool CURV, bool INT>
__device__ __forceinline__ void march_div_point(const KConst<T> &k, const T *fr, int FW, int row, int fc,
                                                unsigned code, T jac, T rhs[4]) {
  const int sl = row & (kRing - 1), o = sl * FW + fc;
  const T *pi[4], *pj[4];
  Row<T> ri, rj;
  if (INT) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int off = e < 2 ? e - 2 : e - 1;
      pi[e] = fr + o + off;
      pj[e] = fr + ((row + off) & (kRing - 1)) * FW + fc;
    }
  } else {
    ri = CURV ? decode_row<T>(code & 15u) : decode_row_w<T>(code & 15u, k.wx);
    rj = CURV ? decode_row<T>(code >> 4) : decode_row_w<T>(code >> 4, k.wy);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      pi[e] = fr + o + ri.off[e];
      pj[e] = fr + ((row + rj.off[e]) & (kRing - 1)) * FW + fc;
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (CURV) {
      const T di = INT ? central_sum(pi, c * kRing * FW) : row_sum(ri, pi, c * kRing * FW);
      const T dj = INT ? central_sum(pj, (4 + c) * kRing * FW) : row_sum(rj, pj, (4 + c) * kRing * FW);
      rhs[c] = -jac * (di + dj);
    } else {
      const T di = INT ? central_sum_w(pi, c * kRing * FW, k.wx[4]) : row_sum(ri, pi, c * kRing * FW);
      const T dj = INT ? central_sum_w(pj, (4 + c) * kRing * FW, k.wy[4]) : row_sum(rj, pj, (4 + c) * kRing * FW);
      rhs[c] = -(di + dj);
    }
  }
}

// One strip (bx) x chunk (by) of the mesh, by one CTA of 256 threads with M::bytes of shared
// memory at smem_raw (the body of k_march, also run by the batched persistent kernel).
template <typename T, bool VISC, bool CURV>
__device__ __forceinline__ void march_tile(const RhsLaunch &a, int bx, int by, int chunk, unsigned char *smem_raw) {
  using M = March<T, VISC, CURV>;
  constexpr int W = M::W, R = M::R, PW = M::PW, FW = M::FW, NT = M::NT;
  T *qr = reinterpret_cast<T *>(smem_raw);
  T *mr = qr + M::QR;
  T *prim = mr + M::MR;
  T *fr = prim + M::PR;
  uint8_t *cr = reinterpret_cast<uint8_t *>(fr + M::FR);
  const DevMesh &m = a.m;
  const KConst<T> &k = kc<T>(a);
  const int tid = threadIdx.x;
  const int i0 = bx * W;
  const int j0 = by * chunk, j1 = min(j0 + chunk, m.nj);
  const T *q = static_cast<const T *>(a.q);
  const T *satb = static_cast<const T *>(a.sat);
  const int nty8 = (m.nj + 7) / 8;
  const int rmax = j1 + 6;  // rows of the window: [j0 - 6, j1 + 6)

  WinItem pw[2], fw[2];  // items of the P-wide (fetch, primitives) and F-wide (fluxes) stages
  win_items<R, NT>(m, PW, i0 - 6, pw);
  win_items<R, NT>(m, FW, i0 - 3, fw);
  unsigned cls[2];
  march_fetch<T, VISC, CURV>(a, pw, j0 - 6, rmax, qr, mr, cls);
  cp_async_commit();
  march_store_cls<T, VISC, CURV>(pw, j0 - 6, cr, cls);

  for (int b = j0 - 6; b - 6 < j1; b += R) {
    // this tick's rows have landed (issued one tick ago) and every thread is done with the
    // previous tick; then the next tick's rows go in flight during this tick's arithmetic
    // (their ring slots belong to rows no stage of this tick reads)
    cp_async_wait<0>();
    __syncthreads();
    march_fetch<T, VISC, CURV>(a, pw, b + R, rmax, qr, mr, cls);
    cp_async_commit();
    if constexpr (VISC) {
      // P: primitives of rows [b, b + R)
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int row = b + pw[it].rr;
        const int o = (row & (kRing - 1)) * PW + pw[it].cc;
        int gj = row;
        if (pw[it].gi < 0 || row >= rmax || !wrap_index(gj, m.nj, m.per_j)) continue;
        T pr[3];
        prim4(qr[o], qr[kRing * PW + o], qr[2 * kRing * PW + o], qr[3 * kRing * PW + o], k.gam, pr);
#pragma unroll
        for (int f = 0; f < 3; ++f) prim[f * kRing * PW + o] = pr[f];
      }
      __syncthreads();
    }
    // F: contravariant fluxes of rows [b - 3, b + R - 3), window columns [3, W + 9)
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int row = b - 3 + fw[it].rr;
      int gj = row;
      if (fw[it].gi < 0 || row < j0 - 3 || row >= j1 + 3 || !wrap_index(gj, m.nj, m.per_j)) continue;
      const int pc = fw[it].cc + 3;
      const unsigned code = cr[(row & (kRing - 1)) * PW + pc];
      if (code == 0u) march_flux_point<T, VISC, CURV, true>(a, qr, mr, prim, fr, row, pc, code);
      else march_flux_point<T, VISC, CURV, false>(a, qr, mr, prim, fr, row, pc, code);
    }
    __syncthreads();
    // O: rows [b - 6, b + R - 6), one point per thread
    {
      const int rr = tid / W, cc = tid - rr * W;
      const int gj = b - 6 + rr, gi = i0 + cc;
      if (rr < R && gj >= j0 && gj < j1 && gi < m.ni) {
        const size_t p = (size_t)gj * m.pitch + gi;
        const int o = (gj & (kRing - 1)) * PW + cc + 6;
        const unsigned code = cr[o];
        T rhs[4] = {T(0), T(0), T(0), T(0)};
        if ((code & 15u) != 15u) {
          const T jac = CURV ? mr[4 * kRing * PW + o] : k.mc[4];
          if (code == 0u) march_div_point<T, CURV, true>(k, fr, FW, gj, cc + 3, code, jac, rhs);
          else march_div_point<T, CURV, false>(k, fr, FW, gj, cc + 3, code, jac, rhs);
          // SAT points are boundary or receiver points: a closure row in some direction
          const int tile = (gi / kTileX) * nty8 + gj / 8;
          const int s0 = code != 0u ? a.tile_sat[tile] : 0, s1 = code != 0u ? a.tile_sat[tile + 1] : 0;
          if (s0 < s1) {
            const uint32_t key = (uint32_t)gi | ((uint32_t)gj << 16);
            int lo = s0, hi = s1;
            while (lo < hi) {
              int mid = (lo + hi) >> 1;
              uint32_t km = a.sat_ij[mid];
              if ((km >> 16) < (key >> 16) || ((km >> 16) == (key >> 16) && (km & 0xFFFFu) < (key & 0xFFFFu)))
                lo = mid + 1;
              else
                hi = mid;
            }
            if (lo < s1 && a.sat_ij[lo] == key) {
#pragma unroll
              for (int c = 0; c < 4; ++c) rhs[c] += satb[c * a.nsat + lo];
            }
          }
          if (k.sponge_d > 0) {
            const T sg = sponge_sigma(k, m, gi, gj);
            if (sg != T(0)) {
#pragma unroll
              for (int c = 0; c < 4; ++c) rhs[c] = fma_rn(-sg, qr[c * kRing * PW + o] - k.qinf[c], rhs[c]);
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
          for (int c = 0; c < 4; ++c) q0[c] = qr[c * kRing * PW + o];
          ab_update<T, 4>(q0, a.hold, a.alpha, a.nold, m.field, p, rhs, qv, (code & 15u) != 15u ? a.err : nullptr);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            out[c * m.field + p] = rhs[c];
            qn[c * m.field + p] = qv[c];
          }
        }
      }
    }
    // class bytes of the prefetched rows; their slots are not read by this tick's stages
    march_store_cls<T, VISC, CURV>(pw, b + R, cr, cls);
  }
  cp_async_wait<0>();
}

template <typename T, bool VISC, bool CURV>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (CURV ? 2 : 3) : 1) k_march(const RhsLaunch a, int chunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  march_tile<T, VISC, CURV>(a, blockIdx.x, blockIdx.y, chunk, smem_raw);
}

template <typename T, bool VISC, bool CURV>
static cudaError_t launch_march_vc(const RhsLaunch &a, cudaStream_t s) {
  using M = March<T, VISC, CURV>;
  auto km = k_march<T, VISC, CURV>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(km, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)M::bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (a.nsat > 0) {
    k_sat<T, VISC, CURV><<<(a.nsat + 127) / 128, 128, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int chunk = a.chunk;
  dim3 grid((a.m.ni + M::W - 1) / M::W, (a.m.nj + chunk - 1) / chunk);
  km<<<grid, M::NT, M::bytes, s>>>(a, chunk);
  return cudaGetLastError();
}

template <typename T, bool VISC, bool CURV>
static cudaError_t launch_march_w(const RhsLaunch &a, cudaStream_t s) {
  if (a.strip != kMarchW) return cudaErrorInvalidValue;
  return launch_march_vc<T, VISC, CURV>(a, s);
}

}  // namespace sbp
