// The marching right-hand-side kernel (sbp_march_impl.cuh) with its state and metric rows staged
// by TMA tensor copies: per tick one thread issues, for each of the 4 state planes (and the 5
// metric planes of a curvilinear mesh), one cp.async.bulk.tensor copy of a box of 72 columns x
// 4 rows (the window's 70 columns rounded out to 16-byte boundaries) into the ring, completing
// on an mbarrier that every thread waits on one tick later. This replaces the per-thread
// cp.async addressing of the window (two items per thread, nine planes each) by nine copies per
// CTA and tick. The ring rows of the state and metrics are kTmaW = 72 columns wide (a 4-row box
// lands as 4 consecutive rows), the window's column 0 at ring column sh = (i0 - 6) mod 4 (FP32;
// 0 in FP64); ring slots count rows from the chunk's first window row so that every 4-row box
// lands in one slot group. Boxes read zeros outside the mesh; where a periodic direction wraps
// (the first and last strip of a periodic i direction, the rows past a periodic j seam) the
// threads overwrite those entries from the wrapped rows and columns after the copy has landed.
// The primitives, fluxes, class bytes, SAT values and the per-point arithmetic are the
// cp.async kernel's, so both kernels give the same bits.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include "sbp_march_impl.cuh"

namespace sbp {

constexpr int kTmaW = 72;              // ring columns of the staged planes (box width)
constexpr long kTmaSpins = 1L << 20;   // polls of the copy's mbarrier before giving up
constexpr unsigned kTmaPollNs = 1000;  // suspend-time hint of one poll

template <typename T, bool VISC, bool CURV>
struct MarchTma {
  using B = March<T, VISC, CURV>;
  static constexpr int W = B::W, NT = B::NT, R = B::R, PW = B::PW, FW = B::FW, QW = kTmaW;
  static constexpr int NQ = 4 + (CURV ? 5 : 0);     // planes staged per row group
  static constexpr int QR = 4 * kRing * QW;          // state ring
  static constexpr int MR = CURV ? 5 * kRing * QW : 0;
  static constexpr int PR = B::PR, FR = B::FR;
  static constexpr size_t cls_off = (size_t)(QR + MR + PR + FR) * sizeof(T);
  static constexpr size_t bar_off = (cls_off + (size_t)kRing * PW + 15) / 16 * 16;
  static constexpr size_t bytes = bar_off + 16;
  static constexpr unsigned tx = (unsigned)(NQ * R * QW * sizeof(T));  // bytes per row group
  static_assert(R == 4 && kRing % R == 0, "row groups of 4 ring slots");
  static_assert((R * QW * sizeof(T)) % 128 == 0 && (kRing * QW * sizeof(T)) % 128 == 0,
                "every box lands on a 128-byte boundary");
  // kMarchW is even, so the window start i0 - 6 is even: sh <= 2 in FP32, 0 in FP64
  static_assert(kMarchW % 2 == 0 && PW + (sizeof(T) == 4 ? 2 : 0) <= QW, "box covers the window");
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kTmaPollNs)
      : "memory");
  return done != 0;
}

// Polls the mbarrier's phase `parity` at most kTmaSpins times (each poll suspends the thread for
// at most about kTmaPollNs), about a second in all; false when it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
  for (long it = 0; it < kTmaSpins; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Orders this thread's earlier generic-proxy accesses of shared memory before later async-proxy
// (TMA) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Class bytes of rows [r0, r0 + R) of the window into registers (march_fetch's class part).
template <typename T, bool VISC, bool CURV>
__device__ __forceinline__ void march_fetch_cls(const RhsLaunch &a, const WinItem wi[2], int r0, int rmax,
                                                unsigned cls[2]) {
  const DevMesh &m = a.m;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    cls[it] = kNoCls;
    const int gi = wi[it].gi;
    const int row = r0 + wi[it].rr;
    int gj = row;
    if (gi < 0 || row >= rmax || !wrap_index(gj, m.nj, m.per_j)) continue;
    cls[it] = m.cls[(size_t)gj * m.pitch + gi];
  }
}

// One strip (blockIdx.x) x chunk (blockIdx.y) of the mesh by one CTA of 256 threads.
template <typename T, bool VISC, bool CURV>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (CURV ? 2 : 3) : 1)
    k_march_tma(const RhsLaunch a, int chunk, const __grid_constant__ CUtensorMap tq,
                const __grid_constant__ CUtensorMap tm) {
  using M = MarchTma<T, VISC, CURV>;
  constexpr int W = M::W, R = M::R, PW = M::PW, FW = M::FW, NT = M::NT, QW = M::QW;
  extern __shared__ __align__(128) unsigned char smem_tma[];  // its own name: 128-byte alignment
  unsigned char *smem_raw = smem_tma;
  T *qr = reinterpret_cast<T *>(smem_raw);
  T *mr = qr + M::QR;
  T *prim = mr + M::MR;
  T *fr = prim + M::PR;
  uint8_t *cr = smem_raw + M::cls_off;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + M::bar_off);
  const DevMesh &m = a.m;
  const KConst<T> &k = kc<T>(a);
  const T *q = static_cast<const T *>(a.q);
  const T *met = static_cast<const T *>(m.met);
  const T *satb = static_cast<const T *>(a.sat);
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * W;
  const int j0 = blockIdx.y * chunk, j1 = min(j0 + chunk, m.nj);
  const int rb = j0 - 6, rmax = j1 + 6;  // window rows [j0 - 6, j1 + 6); ring slot = (row - rb) & 15
  constexpr int AL = 16 / (int)sizeof(T);
  const int x0 = (i0 - 6) & ~(AL - 1), sh = (i0 - 6) - x0;
  const bool seam_i = m.per_i && (i0 - 6 < 0 || i0 - 6 + PW > m.ni);
  const int nty8 = (m.nj + 7) / 8;
  if (smem_u32(smem_raw) & 127u) {  // the boxes need 128-byte aligned destinations
    if (tid == 0 && a.err) atomicCAS(a.err, 0, (int)SBP_ERR_BOUNDS);
    return;
  }

  WinItem pw[2], fw[2];
  win_items<R, NT>(m, PW, i0 - 6, pw);
  win_items<R, NT>(m, FW, i0 - 3, fw);
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  // rows [r0, r0 + R) of the state (and metric) planes into their ring slot group
  auto issue = [&](int r0) {
    if (tid == 0) {
      fence_proxy_async_smem();
      mbar_expect_tx(bar, M::tx);
      const int g = ((r0 - rb) & (kRing - 1)) * QW;
#pragma unroll
      for (int v = 0; v < 4; ++v) tma_load_3d(qr + v * kRing * QW + g, &tq, x0, r0, v, bar);
      if (CURV) {
#pragma unroll
        for (int c = 0; c < 5; ++c) tma_load_3d(mr + c * kRing * QW + g, &tm, x0, r0, c, bar);
      }
    }
  };
  auto store_cls = [&](int r0, const unsigned c[2]) {
#pragma unroll
    for (int it = 0; it < 2; ++it)
      if (c[it] != kNoCls) cr[((r0 + pw[it].rr - rb) & (kRing - 1)) * PW + pw[it].cc] = (uint8_t)c[it];
  };
  unsigned cls[2];
  march_fetch_cls<T, VISC, CURV>(a, pw, j0 - 6, rmax, cls);
  issue(j0 - 6);
  store_cls(j0 - 6, cls);

  unsigned phase = 0;
  for (int b = j0 - 6; b - 6 < j1; b += R) {
    // this tick's rows have landed (issued one tick ago) and every thread is done with the
    // previous tick
    const bool ok = mbar_wait_bounded(bar, phase);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        if (a.err) atomicCAS(a.err, 0, (int)SBP_ERR_TIMEOUT);
        mbar_wait_bounded(bar, phase ^ 1u);  // one more bounded wait for the copy in flight
      }
      return;
    }
    // entries a box read as zeros where a periodic direction wraps
    if (seam_i || (m.per_j && (b < 0 || b + R > m.nj))) {
      for (int idx = tid; idx < R * PW; idx += NT) {
        const int rr = idx / PW, cc = idx - rr * PW;
        int gi = i0 - 6 + cc, gj = b + rr;
        const bool wrapped = (m.per_i && (gi < 0 || gi >= m.ni)) || (m.per_j && (gj < 0 || gj >= m.nj));
        if (!wrapped || !wrap_index(gi, m.ni, m.per_i) || !wrap_index(gj, m.nj, m.per_j)) continue;
        const size_t p = (size_t)gj * m.pitch + gi;
        const int o = ((b + rr - rb) & (kRing - 1)) * QW + cc + sh;
#pragma unroll
        for (int v = 0; v < 4; ++v) qr[v * kRing * QW + o] = q[v * m.field + p];
        if (CURV) {
#pragma unroll
          for (int c = 0; c < 5; ++c) mr[c * kRing * QW + o] = met[c * m.field + p];
        }
      }
      fence_proxy_async_smem();  // before a later copy into these slots
      __syncthreads();
    }
    // the next tick's rows go in flight during this tick's arithmetic (their ring slots belong to
    // rows no stage of this tick reads)
    if (b + R < rmax) issue(b + R);
    march_fetch_cls<T, VISC, CURV>(a, pw, b + R, rmax, cls);
    if constexpr (VISC) {
      // P: primitives of rows [b, b + R)
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int row = b + pw[it].rr;
        int gj = row;
        if (pw[it].gi < 0 || row >= rmax || !wrap_index(gj, m.nj, m.per_j)) continue;
        const int sl = (row - rb) & (kRing - 1);
        const int po = sl * PW + pw[it].cc, qo = sl * QW + pw[it].cc + sh;
        T pr[3];
        prim4(qr[qo], qr[kRing * QW + qo], qr[2 * kRing * QW + qo], qr[3 * kRing * QW + qo], k.gam, pr);
#pragma unroll
        for (int f = 0; f < 3; ++f) prim[f * kRing * PW + po] = pr[f];
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
      const unsigned code = cr[((row - rb) & (kRing - 1)) * PW + pc];
      if (code == 0u) march_flux_point<T, VISC, CURV, true, QW>(a, qr, mr, prim, fr, row - rb, pc, code, sh);
      else march_flux_point<T, VISC, CURV, false, QW>(a, qr, mr, prim, fr, row - rb, pc, code, sh);
    }
    __syncthreads();
    // O: rows [b - 6, b + R - 6), one point per thread
    {
      const int rr = tid / W, cc = tid - rr * W;
      const int gj = b - 6 + rr, gi = i0 + cc;
      if (rr < R && gj >= j0 && gj < j1 && gi < m.ni) {
        const size_t p = (size_t)gj * m.pitch + gi;
        const int sl = (gj - rb) & (kRing - 1);
        const int o = sl * PW + cc + 6, qo = sl * QW + cc + 6 + sh;
        const unsigned code = cr[o];
        T rhs[4] = {T(0), T(0), T(0), T(0)};
        if ((code & 15u) != 15u) {
          const T jac = CURV ? mr[4 * kRing * QW + qo] : k.mc[4];
          if (code == 0u) march_div_point<T, CURV, true>(k, fr, FW, gj - rb, cc + 3, code, jac, rhs);
          else march_div_point<T, CURV, false>(k, fr, FW, gj - rb, cc + 3, code, jac, rhs);
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
              for (int c = 0; c < 4; ++c) rhs[c] = fma_rn(-sg, qr[c * kRing * QW + qo] - k.qinf[c], rhs[c]);
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
          for (int c = 0; c < 4; ++c) q0[c] = qr[c * kRing * QW + qo];
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
    store_cls(b + R, cls);
  }
}

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point query: no link to
// the driver library); null when the driver does not provide it.
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult res;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &res) ==
            cudaSuccess &&
        res == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// A tensor map over `planes` planes of the mesh's layout at base: dimensions (ni, nj, planes),
// strides (pitch, field) elements, boxes of kTmaW x 4 x 1, zeros outside.
template <typename T>
inline bool plane_tensor_map(CUtensorMap *map, const void *base, const DevMesh &m, int planes) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15u)) return false;
  const cuuint64_t dim[3] = {(cuuint64_t)m.ni, (cuuint64_t)m.nj, (cuuint64_t)planes};
  const cuuint64_t stride[2] = {(cuuint64_t)m.pitch * sizeof(T), (cuuint64_t)m.field * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)kTmaW, 4u, 1u};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  return enc(map, sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
             const_cast<void *>(base), dim, stride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The marching kernel with TMA staging (chunk = a.chunk without kStageTma); falls back to the
// cp.async-staged kernel (the same bits) when a tensor map cannot be made (no encoder in the
// driver, a state not 16-byte aligned).
template <typename T, bool VISC, bool CURV>
static cudaError_t launch_march_tma(const RhsLaunch &a, cudaStream_t s) {
  using M = MarchTma<T, VISC, CURV>;
  alignas(64) CUtensorMap tq, tm;
  const bool maps = plane_tensor_map<T>(&tq, a.q, a.m, 4) && (!CURV || plane_tensor_map<T>(&tm, a.m.met, a.m, 5));
  if (!maps) {
    RhsLaunch b = a;
    b.chunk = a.chunk & (kStageTma - 1);
    return launch_march_vc<T, VISC, CURV>(b, s);
  }
  if (!CURV) tm = tq;
  auto km = k_march_tma<T, VISC, CURV>;
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
  const int chunk = a.chunk & (kStageTma - 1);
  dim3 grid((a.m.ni + M::W - 1) / M::W, (a.m.nj + chunk - 1) / chunk);
  km<<<grid, M::NT, M::bytes, s>>>(a, chunk, tq, tm);
  return cudaGetLastError();
}

}  // namespace sbp
