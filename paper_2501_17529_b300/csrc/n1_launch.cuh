// Launchers of the FP32 fused N-1 kernels (k_n1_reg, k_n1_tma) and the
// tensor maps they read.  Kept in their own translation unit: the kernels have
// many template instances (timesteps per pass x rank class x variant).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "args.cuh"
#include "n1_types.cuh"

namespace dcf {

// Row-major FP32 tensor of `rank` dims (innermost first); strides in bytes for dims 1..rank-1.
// swizzle128: the box lands with 128-byte swizzling (its inner extent is then
// 128 bytes and the destination 1024-byte aligned): 16-byte chunk c of box
// row y sits at chunk c ^ (y % 8).
int encode_map(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
               const uint32_t* box, bool swizzle128 = false);
// tc: the Phi_f tile on the tensor cores (split BF16x3; the maps then carry
// the BF16 Z rows and a Phi tile 68 columns wide) instead of FFMA2.
// every contingency column, TT timesteps per pass (TT = 1: one thread per
// contingency, always the FFMA build)
int launch_tma(const N1Maps& maps, const Args& a, int RMAX, int TT, dim3 grid, cudaStream_t st, int t0, bool tc);
// metric-first screening of candidates: maximum only, 32 timesteps per pass
int launch_tma_screen(const N1Maps& maps, const Args& a, int RMAX, dim3 grid, cudaStream_t st, int t0, bool tc);
// selected contingencies (screened N-1): one block per work item
int launch_reg_sel(const N1Maps& maps, const Args& a, const SelArgs& sel, int RMAX, int TT, int items,
                   cudaStream_t st, int t0, bool tc);
// every topology's compacted valid contingencies
int launch_reg_cmp(const N1Maps& maps, const Args& a, const SelArgs& sel, int RMAX, int TT, bool ovl, dim3 grid,
                   cudaStream_t st, int t0, bool tc);

// templated bodies (n1_launch_impl.cuh), one instance set per build
template <bool TC>
int launch_tma_k(const N1Maps& maps, const Args& a, int RMAX, int TT, dim3 grid, cudaStream_t st, int t0);
template <bool TC>
int launch_tma_screen_k(const N1Maps& maps, const Args& a, int RMAX, dim3 grid, cudaStream_t st, int t0);
template <bool TC>
int launch_reg_sel_k(const N1Maps& maps, const Args& a, const SelArgs& sel, int RMAX, int TT, int items,
                     cudaStream_t st, int t0);
template <bool TC>
int launch_reg_cmp_k(const N1Maps& maps, const Args& a, const SelArgs& sel, int RMAX, int TT, bool ovl, dim3 grid,
                     cudaStream_t st, int t0);

}  // namespace dcf
