// Batched persistent micro step over many overset systems (one cooperative launch); included once
// per element type by sbp_batch_f32.cu and sbp_batch_f64.cu.
#pragma once
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>
#include <cstring>

#include "sbp_dev.cuh"
#include "sbp_march_impl.cuh"

namespace sbp {

// ---------------------------------------------------------------------------------------------
// Batched persistent substep: one cooperative launch advances every member system of a batch
// through one micro step (Sec. 3.3) in three phases separated by grid barriers: donor values of
// all receiving meshes, contravariant fluxes of all tiles, then SBP derivatives + SAT +
// Adams-Bashforth update of all tiles. Work items index per-mesh descriptors in device memory.

// Grid barrier for a cooperative launch (all CTAs resident). The spin is bounded: after
// kBarrierSpins polls the CTA records SBP_ERR_TIMEOUT in *err and the barrier returns false,
// so a broken launch ends instead of hanging the device.
constexpr unsigned kBarrierSpins = 4u << 20;  // with 256 ns sleeps: about one second

static __device__ bool grid_barrier(unsigned *count, volatile unsigned *gen, unsigned nblocks, int *err,
                                    unsigned max_spins = kBarrierSpins) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned g = *gen;
    __threadfence();
    if (atomicAdd(count, 1u) == nblocks - 1) {
      *count = 0;
      __threadfence();
      atomicAdd((unsigned *)gen, 1u);
    } else {
      unsigned spins = 0;
      while (*gen == g) {
        if (++spins > max_spins || *(volatile int *)err) {
          atomicCAS(err, 0, (int)SBP_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename T, bool VISC, bool CURVF, int TY>
struct BatchSmem {
  static constexpr size_t flux = VISC ? 3 * FluxTile<T, VISC, TY>::RN * sizeof(T) + FluxTile<T, VISC, TY>::RN : 16;
  static constexpr size_t upd = UpdTile<T, TY>::bytes;
  static constexpr size_t bytes = flux > upd ? flux : upd;
};

// Phase 1 of a batched micro step: donor values of all receiving meshes (VISC: 16-lane groups,
// two per warp; Euler: one thread per (set, donor point) pair).
template <typename T, bool VISC>
__device__ __forceinline__ void batch_donor_phase(const BatchSubstep &b) {
  const DonorLaunch *dl = static_cast<const DonorLaunch *>(b.dl);
  const int total = b.dl_off[b.n_dl];
  if (total > 0) {
    const int lanes = VISC ? 16 : 1;
    const int per_warp = 32 / lanes;
    const int nwarps = gridDim.x * (kNT / 32);
    const int warp = blockIdx.x * (kNT / 32) + (threadIdx.x >> 5);
    const int sub = (threadIdx.x & 31) / lanes;
    for (int w0 = warp * per_warp; w0 < total; w0 += nwarps * per_warp) {
      const int g = w0 + sub;
      const bool valid = g < total;
      int lo = 0, hi = b.n_dl;  // descriptor: last offset <= g
      while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (b.dl_off[mid] <= g) lo = mid;
        else hi = mid;
      }
      const DonorLaunch &a = dl[lo];
      const int pair = g - b.dl_off[lo];
      if constexpr (VISC) {
        if (a.d.cart) donor_group<T, false>(a, pair, valid);
        else donor_group<T, true>(a, pair, valid);
      } else if (valid) {
        const int set = pair / a.npts, d = pair - set * a.npts;
        const uint32_t ij = a.pts[d];
        const size_t p = (size_t)(ij >> 16) * a.d.pitch + (ij & 0xFFFFu);
        const int sd = a.stride ? a.stride : a.npts;
        T *dv = static_cast<T *>(a.dv) + (size_t)set * 10 * sd;
        T st[4];
        set_state(a, set, p, st);
#pragma unroll
        for (int v = 0; v < 4; ++v) dv[v * sd + d] = st[v];
      }
    }
  }
}

template <typename T, bool VISC, bool CURVF, int TY>
__global__ void __launch_bounds__(kNT, sizeof(T) == 4 ? (VISC ? 3 : 4) : (VISC ? 1 : 2)) k_batch_substep(const BatchSubstep b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using F = FluxTile<T, VISC, TY>;
  T *prim = reinterpret_cast<T *>(smem_raw);
  uint8_t *scls = reinterpret_cast<uint8_t *>(prim + (VISC ? 3 * F::RN : 0));
  T *sf = reinterpret_cast<T *>(smem_raw);
  const RhsLaunch *rl = static_cast<const RhsLaunch *>(b.rl);

  batch_donor_phase<T, VISC>(b);
  if (!grid_barrier(b.bar_count, b.bar_gen, gridDim.x, b.err)) return;
  // phase 2: fluxes (and SAT terms) of every tile
  for (int it = blockIdx.x; it < b.n_items; it += gridDim.x) {
    const int4 w = b.items[it];
    __syncthreads();
    if (w.w) flux_tile<T, VISC, CURVF, TY>(rl[w.x], w.y, w.z, prim, scls);
    else flux_tile<T, VISC, false, TY>(rl[w.x], w.y, w.z, prim, scls);
  }
  if (!grid_barrier(b.bar_count, b.bar_gen, gridDim.x, b.err)) return;
  // phase 3: derivatives, SAT, update
  for (int it = blockIdx.x; it < b.n_items; it += gridDim.x) {
    const int4 w = b.items[it];
    __syncthreads();
    if (w.w) update_tile<T, VISC, CURVF, TY>(rl[w.x], w.y, w.z, sf);
    else update_tile<T, VISC, false, TY>(rl[w.x], w.y, w.z, sf);
  }
}

// The same micro step with the single-pass right-hand side (march_tile, kMarchW-column strips of
// b.chunk rows): donor values; SAT values of every boundary / receiver point of all meshes;
// then the strips. The SAT phase replaces k_sat, the strips k_march.
template <typename T, bool VISC, bool CURVF>
struct BatchMarchSmem {
  static constexpr size_t a = March<T, VISC, false>::bytes, c = March<T, VISC, CURVF>::bytes;
  static constexpr size_t bytes = a > c ? a : c;
};

template <typename T, bool VISC, bool CURVF>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (CURVF ? 2 : 3) : 1) k_batch_march(const BatchSubstep b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const RhsLaunch *rl = static_cast<const RhsLaunch *>(b.rl);
  batch_donor_phase<T, VISC>(b);
  if (!grid_barrier(b.bar_count, b.bar_gen, gridDim.x, b.err)) return;
  const int nsat = b.sat_off[b.n_rl];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nsat; g += gridDim.x * blockDim.x) {
    int lo = 0, hi = b.n_rl;  // descriptor: last offset <= g
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (b.sat_off[mid] <= g) lo = mid;
      else hi = mid;
    }
    if (b.rl_curv[lo]) sat_point<T, VISC, CURVF>(rl[lo], g - b.sat_off[lo]);
    else sat_point<T, VISC, false>(rl[lo], g - b.sat_off[lo]);
  }
  if (!grid_barrier(b.bar_count, b.bar_gen, gridDim.x, b.err)) return;
  for (int it = blockIdx.x; it < b.n_items; it += gridDim.x) {
    const int4 w = b.items[it];
    __syncthreads();
    if (w.w) march_tile<T, VISC, CURVF>(rl[w.x], w.y, w.z, b.chunk, smem_raw);
    else march_tile<T, VISC, false>(rl[w.x], w.y, w.z, b.chunk, smem_raw);
  }
}

template <typename T, bool VISC, bool CURVF>
static cudaError_t launch_batch_m(const BatchSubstep &b, int grid, cudaStream_t s) {
  auto kern = k_batch_march<T, VISC, CURVF>;
  using S = BatchMarchSmem<T, VISC, CURVF>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (grid <= 0) return cudaErrorInvalidValue;
  BatchSubstep bb = b;
  void *args[] = {&bb};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(256), args, S::bytes, s);
}

template <typename T, bool VISC, bool CURVF>
static cudaError_t batch_grid_m(int *grid) {
  auto kern = k_batch_march<T, VISC, CURVF>;
  using S = BatchMarchSmem<T, VISC, CURVF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, S::bytes)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  *grid = per_sm * sms;
  return cudaSuccess;
}

template <typename T, bool VISC, bool CURVF, int TY>
static cudaError_t launch_batch_t(const BatchSubstep &b, int grid, cudaStream_t s) {
  auto kern = k_batch_substep<T, VISC, CURVF, TY>;
  using S = BatchSmem<T, VISC, CURVF, TY>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (grid <= 0) return cudaErrorInvalidValue;
  BatchSubstep bb = b;
  void *args[] = {&bb};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(kNT), args, S::bytes, s);
}

template <typename T, bool VISC, bool CURVF, int TY>
static cudaError_t batch_grid_t(int *grid) {
  auto kern = k_batch_substep<T, VISC, CURVF, TY>;
  using S = BatchSmem<T, VISC, CURVF, TY>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNT, S::bytes)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  *grid = per_sm * sms;
  return cudaSuccess;
}

// ty = rows per work item: 8 or 16 for the flux / derivative tile pair; 32 or more for the
// single-pass strips (Euler).
template <typename T>
cudaError_t launch_batch_typed(const BatchSubstep &b, int grid, bool viscous, bool curv_fine, int ty, cudaStream_t s) {
  if (ty >= 32) {
    if (viscous) return cudaErrorInvalidValue;
    return curv_fine ? launch_batch_m<T, false, true>(b, grid, s) : launch_batch_m<T, false, false>(b, grid, s);
  }
  if (ty != 8 && ty != 16) return cudaErrorInvalidValue;
#define SBP_B(V, C) (ty == 8 ? launch_batch_t<T, V, C, 8>(b, grid, s) : launch_batch_t<T, V, C, 16>(b, grid, s))
  if (viscous) return curv_fine ? SBP_B(true, true) : SBP_B(true, false);
  return curv_fine ? SBP_B(false, true) : SBP_B(false, false);
#undef SBP_B
}

template <typename T>
cudaError_t batch_grid_typed(bool viscous, bool curv_fine, int ty, int *grid) {
  if (ty >= 32) {
    if (viscous) return cudaErrorInvalidValue;
    return curv_fine ? batch_grid_m<T, false, true>(grid) : batch_grid_m<T, false, false>(grid);
  }
  if (ty != 8 && ty != 16) return cudaErrorInvalidValue;
#define SBP_G(V, C) (ty == 8 ? batch_grid_t<T, V, C, 8>(grid) : batch_grid_t<T, V, C, 16>(grid))
  if (viscous) return curv_fine ? SBP_G(true, true) : SBP_G(true, false);
  return curv_fine ? SBP_G(false, true) : SBP_G(false, false);
#undef SBP_G
}

}  // namespace sbp
