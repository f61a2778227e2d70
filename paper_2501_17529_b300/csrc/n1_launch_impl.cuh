// Launchers of the FP32 fused N-1 kernel k_n1_reg, templated on the Phi_f build
// (TC = false: FFMA2 on the CUDA cores; TC = true: split-BF16x3 on the tensor
// cores).  Included by n1_launch.cu and n1_launch_tc.cu, which instantiate one
// build each (the kernels have many template instances).
#pragma once

#include "n1_launch.cuh"
#include "n1_reg.cuh"

namespace dcf {

template <bool TC, int TT, int RMAX, bool OVL = true>
int launch_tma_t(const N1Maps& maps, const Args& a, dim3 grid, cudaStream_t st, int t0) {
  static uint64_t attr = 0;
  if constexpr (TT >= 4) {  // register-tiled kernel
    using L = RegLayout<TT, RMAX, false, TC>;
    if constexpr (OVL && !TC) {  // the tracking variant: each maximum's tile for the top-k cases
      if (a.tile) {
        static uint64_t attr_t = 0;
        if (smem_attr_once(k_n1_reg<TT, RMAX, true, false, false, true>, L::kBytes, attr_t) != cudaSuccess)
          return DCFLOW_ERR_CUDA;
        k_n1_reg<TT, RMAX, true, false, false, true><<<grid, RegTile<TT>::NT, L::kBytes, st>>>(maps, a, t0, SelArgs{});
        return 0;
      }
    }
    if (smem_attr_once(k_n1_reg<TT, RMAX, OVL, false, TC>, L::kBytes, attr) != cudaSuccess) return DCFLOW_ERR_CUDA;
    k_n1_reg<TT, RMAX, OVL, false, TC><<<grid, RegTile<TT>::NT, L::kBytes, st>>>(maps, a, t0, SelArgs{});
  } else {  // one timestep: one thread per contingency
    using L = TmaLayout<TT, RMAX>;
    if (smem_attr_once(k_n1_tma<TT, RMAX, 1, OVL>, L::kBytes, attr) != cudaSuccess) return DCFLOW_ERR_CUDA;
    k_n1_tma<TT, RMAX, 1, OVL><<<grid, kCB, L::kBytes, st>>>(maps, a, t0);
  }
  return 0;
}

template <bool TC>
int launch_tma_screen_k(const N1Maps& maps, const Args& a, int RMAX, dim3 grid, cudaStream_t st, int t0) {
  if (RMAX == 4) return launch_tma_t<TC, 32, 4, false>(maps, a, grid, st, t0);
  if (RMAX == 8) return launch_tma_t<TC, 32, 8, false>(maps, a, grid, st, t0);
  return launch_tma_t<TC, 32, 16, false>(maps, a, grid, st, t0);
}

template <bool TC, int RMAX>
int launch_tma_r(const N1Maps& maps, const Args& a, int TT, dim3 grid, cudaStream_t st, int t0) {
  switch (TT) {
    case 1:
      if constexpr (!TC) return launch_tma_t<TC, 1, RMAX>(maps, a, grid, st, t0);
      return DCFLOW_ERR_INVALID_ARG;  // one-timestep passes keep the FFMA build (dispatched before)
    case 4: return launch_tma_t<TC, 4, RMAX>(maps, a, grid, st, t0);
    case 8: return launch_tma_t<TC, 8, RMAX>(maps, a, grid, st, t0);
    case 16: return launch_tma_t<TC, 16, RMAX>(maps, a, grid, st, t0);
    case 24: return launch_tma_t<TC, 24, RMAX>(maps, a, grid, st, t0);
    default: return launch_tma_t<TC, 32, RMAX>(maps, a, grid, st, t0);
  }
}

template <bool TC>
int launch_tma_k(const N1Maps& maps, const Args& a, int RMAX, int TT, dim3 grid, cudaStream_t st, int t0) {
  if (RMAX == 4) return launch_tma_r<TC, 4>(maps, a, TT, grid, st, t0);
  if (RMAX == 8) return launch_tma_r<TC, 8>(maps, a, TT, grid, st, t0);
  return launch_tma_r<TC, 16>(maps, a, TT, grid, st, t0);
}

// selected-contingency mode (screened N-1), TT >= 4
template <bool TC, int TT, int RMAX>
int launch_reg_sel_t(const N1Maps& maps, const Args& a, const SelArgs& sel, int items, cudaStream_t st, int t0) {
  using L = RegLayout<TT, RMAX, true, TC>;
  static uint64_t attr = 0;
  if (smem_attr_once(k_n1_reg<TT, RMAX, true, true, TC>, L::kBytes, attr) != cudaSuccess) return DCFLOW_ERR_CUDA;
  k_n1_reg<TT, RMAX, true, true, TC><<<items, RegTile<TT>::NT, L::kBytes, st>>>(maps, a, t0, sel);
  return 0;
}
template <bool TC, int RMAX>
int launch_reg_sel_r(const N1Maps& maps, const Args& a, const SelArgs& sel, int TT, int items, cudaStream_t st,
                     int t0) {
  switch (TT) {
    case 4: return launch_reg_sel_t<TC, 4, RMAX>(maps, a, sel, items, st, t0);
    case 8: return launch_reg_sel_t<TC, 8, RMAX>(maps, a, sel, items, st, t0);
    case 16: return launch_reg_sel_t<TC, 16, RMAX>(maps, a, sel, items, st, t0);
    case 24: return launch_reg_sel_t<TC, 24, RMAX>(maps, a, sel, items, st, t0);
    default: return launch_reg_sel_t<TC, 32, RMAX>(maps, a, sel, items, st, t0);
  }
}
template <bool TC>
int launch_reg_sel_k(const N1Maps& maps, const Args& a, const SelArgs& sel, int RMAX, int TT, int items,
                     cudaStream_t st, int t0) {
  if (RMAX == 4) return launch_reg_sel_r<TC, 4>(maps, a, sel, TT, items, st, t0);
  if (RMAX == 8) return launch_reg_sel_r<TC, 8>(maps, a, sel, TT, items, st, t0);
  return launch_reg_sel_r<TC, 16>(maps, a, sel, TT, items, st, t0);
}

// every topology's valid contingencies, compacted: grid (blocks per topology, slots)
template <bool TC, int TT, int RMAX, bool OVL>
int launch_reg_cmp_t(const N1Maps& maps, const Args& a, const SelArgs& sel, dim3 grid, cudaStream_t st, int t0) {
  using L = RegLayout<TT, RMAX, true, TC>;
  static uint64_t attr = 0;
  if (smem_attr_once(k_n1_reg<TT, RMAX, OVL, true, TC>, L::kBytes, attr) != cudaSuccess) return DCFLOW_ERR_CUDA;
  k_n1_reg<TT, RMAX, OVL, true, TC><<<grid, RegTile<TT>::NT, L::kBytes, st>>>(maps, a, t0, sel);
  return 0;
}
template <bool TC, int RMAX>
int launch_reg_cmp_r(const N1Maps& maps, const Args& a, const SelArgs& sel, int TT, bool ovl, dim3 grid,
                     cudaStream_t st, int t0) {
  if (!ovl) return launch_reg_cmp_t<TC, 32, RMAX, false>(maps, a, sel, grid, st, t0);
  switch (TT) {
    case 4: return launch_reg_cmp_t<TC, 4, RMAX, true>(maps, a, sel, grid, st, t0);
    case 8: return launch_reg_cmp_t<TC, 8, RMAX, true>(maps, a, sel, grid, st, t0);
    case 16: return launch_reg_cmp_t<TC, 16, RMAX, true>(maps, a, sel, grid, st, t0);
    case 24: return launch_reg_cmp_t<TC, 24, RMAX, true>(maps, a, sel, grid, st, t0);
    default: return launch_reg_cmp_t<TC, 32, RMAX, true>(maps, a, sel, grid, st, t0);
  }
}
template <bool TC>
int launch_reg_cmp_k(const N1Maps& maps, const Args& a, const SelArgs& sel, int RMAX, int TT, bool ovl, dim3 grid,
                     cudaStream_t st, int t0) {
  if (RMAX == 4) return launch_reg_cmp_r<TC, 4>(maps, a, sel, TT, ovl, grid, st, t0);
  if (RMAX == 8) return launch_reg_cmp_r<TC, 8>(maps, a, sel, TT, ovl, grid, st, t0);
  return launch_reg_cmp_r<TC, 16>(maps, a, sel, TT, ovl, grid, st, t0);
}

}  // namespace dcf
