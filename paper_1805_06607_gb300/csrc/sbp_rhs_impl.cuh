// Right-hand-side kernels of one mesh, k_flux then k_update (tile bodies in sbp_dev.cuh); included
// once per element type by sbp_rhs_f32.cu and sbp_rhs_f64.cu.
#pragma once
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>
#include <cstring>

#include "sbp_dev.cuh"
#include "sbp_march_impl.cuh"
#include "sbp_march_tma.cuh"
#include "sbp_col_impl.cuh"

namespace sbp {

// At least 4 (FP32) / 3 (FP64) resident CTAs per SM: caps the registers that the SAT tail
// (taken by boundary tiles only) would otherwise claim for the whole kernel.
// The tile of this CTA under the launch's tile box; false: the CTA has no tile (mode 2, inside).
__device__ __forceinline__ bool box_tile(const TileBox &b, int &bx, int &by) {
  bx = blockIdx.x;
  by = blockIdx.y;
  if (b.mode == 1) {
    bx += b.x0;
    by += b.y0;
  } else if (b.mode == 2) {
    return !(bx >= b.x0 && bx < b.x1 && by >= b.y0 && by < b.y1);
  }
  return true;
}

// The grid of a launch over a tile box of a full grid nx x ny.
static inline dim3 box_grid(const TileBox &b, int nx, int ny) {
  return b.mode == 1 ? dim3((unsigned)(b.x1 - b.x0), (unsigned)(b.y1 - b.y0)) : dim3((unsigned)nx, (unsigned)ny);
}

template <typename T, bool VISC, bool CURV, int TY>
__global__ void __launch_bounds__(FluxTile<T, VISC, TY>::NT, (sizeof(T) == 4 ? 4 : 3) * kNT / FluxTile<T, VISC, TY>::NT)
    k_flux(const RhsLaunch a) {
  using F = FluxTile<T, VISC, TY>;
  __shared__ T prim[VISC ? 3 * F::RN : 1];
  __shared__ uint8_t scls[VISC ? F::RN : 1];
  int bx, by;
  if (!box_tile(a.fbox, bx, by)) return;
  flux_tile<T, VISC, CURV, TY>(a, bx, by, prim, scls);
}

template <typename T, bool VISC, bool CURV, int TY>
__global__ void __launch_bounds__(UpdTile<T, TY>::NT) k_update(const RhsLaunch a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int bx, by;
  if (!box_tile(a.ubox, bx, by)) return;
  update_tile<T, VISC, CURV, TY>(a, bx, by, reinterpret_cast<T *>(smem_raw));
}

template <typename T, bool VISC, bool CURV, int TY>
static cudaError_t launch_flux_t(const RhsLaunch &a, cudaStream_t s) {
  dim3 grid = box_grid(a.fbox, (a.m.ni + kTileX - 1) / kTileX, (a.m.nj + TY - 1) / TY);
  k_flux<T, VISC, CURV, TY><<<grid, FluxTile<T, VISC, TY>::NT, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T, bool VISC, bool CURV, int TY>
static cudaError_t launch_update_t(const RhsLaunch &a, cudaStream_t s) {
  using U = UpdTile<T, TY>;
  auto ku = k_update<T, VISC, CURV, TY>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(ku, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)U::bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid = box_grid(a.ubox, (a.m.ni + kTileX - 1) / kTileX, (a.m.nj + TY - 1) / TY);
  ku<<<grid, U::NT, U::bytes, s>>>(a);
  return cudaGetLastError();
}

// The flux kernel with rows_per_cta (4, 8, 16, 32) rows per CTA, then the update kernel with
// rows_upd (4, 8, 16, 32; 0: the same).
template <typename T, bool VISC, bool CURV>
static cudaError_t launch_rhs_ty(const RhsLaunch &a, cudaStream_t s) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (a.rows_per_cta) {
    case 4: e = launch_flux_t<T, VISC, CURV, 4>(a, s); break;
    case 8: e = launch_flux_t<T, VISC, CURV, 8>(a, s); break;
    case 16: e = launch_flux_t<T, VISC, CURV, 16>(a, s); break;
    case 32: e = launch_flux_t<T, VISC, CURV, 32>(a, s); break;
  }
  if (e != cudaSuccess) return e;
  switch (a.rows_upd ? a.rows_upd : a.rows_per_cta) {
    case 4: return launch_update_t<T, VISC, CURV, 4>(a, s);
    case 8: return launch_update_t<T, VISC, CURV, 8>(a, s);
    case 16: return launch_update_t<T, VISC, CURV, 16>(a, s);
    case 32: return launch_update_t<T, VISC, CURV, 32>(a, s);
  }
  return cudaErrorInvalidValue;
}

// Launch for one element type T, dispatched on physics and metric kind.
template <typename T>
cudaError_t launch_rhs_typed(const RhsLaunch &a, bool viscous, cudaStream_t s) {
  bool curv = !a.m.cart;
  if (a.strip == kColW128 || a.strip == kColW256) {
    if (viscous) return curv ? launch_col_w<T, true, true>(a, s) : launch_col_w<T, true, false>(a, s);
    return curv ? launch_col_w<T, false, true>(a, s) : launch_col_w<T, false, false>(a, s);
  }
  if (a.strip && (a.chunk & kStageTma)) {
    if (a.strip != kMarchW) return cudaErrorInvalidValue;
    if (viscous) return curv ? launch_march_tma<T, true, true>(a, s) : launch_march_tma<T, true, false>(a, s);
    return curv ? launch_march_tma<T, false, true>(a, s) : launch_march_tma<T, false, false>(a, s);
  }
  if (a.strip) {
    if (viscous) return curv ? launch_march_w<T, true, true>(a, s) : launch_march_w<T, true, false>(a, s);
    return curv ? launch_march_w<T, false, true>(a, s) : launch_march_w<T, false, false>(a, s);
  }
  if (viscous) return curv ? launch_rhs_ty<T, true, true>(a, s) : launch_rhs_ty<T, true, false>(a, s);
  return curv ? launch_rhs_ty<T, false, true>(a, s) : launch_rhs_ty<T, false, false>(a, s);
}

}  // namespace sbp
