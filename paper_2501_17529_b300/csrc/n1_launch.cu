// Launchers of the FP32 fused N-1 kernels (declarations in n1_launch.cuh).
#include <string>

#include <cudaTypedefs.h>

#include "n1_launch.cuh"
#include "n1_reg.cuh"

namespace dcf {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

int encode_map(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
               const uint32_t* box) {
  auto fn = tensor_map_encoder();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return DCFLOW_ERR_CUDA;
  }
  cuuint64_t d[5], s[4];
  cuuint32_t b[5], e[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    e[i] = 1;
    if (i + 1 < rank) s[i] = strides[i];
  }
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<void*>(base), d, s, b, e,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return DCFLOW_ERR_CUDA;
  }
  return 0;
}

template <int TT, int RMAX, bool OVL = true>
int launch_tma_t(const N1Maps& maps, const Args& a, dim3 grid, cudaStream_t st, int t0) {
  static uint64_t attr = 0;
  if constexpr (TT >= 4) {  // register-tiled kernel
    using L = RegLayout<TT, RMAX>;
    if (smem_attr_once(k_n1_reg<TT, RMAX, OVL>, L::kBytes, attr) != cudaSuccess) return DCFLOW_ERR_CUDA;
    k_n1_reg<TT, RMAX, OVL><<<grid, RegTile<TT>::NT, L::kBytes, st>>>(maps, a, t0, SelArgs{});
  } else {  // one timestep: one thread per contingency
    using L = TmaLayout<TT, RMAX>;
    if (smem_attr_once(k_n1_tma<TT, RMAX, 1, OVL>, L::kBytes, attr) != cudaSuccess) return DCFLOW_ERR_CUDA;
    k_n1_tma<TT, RMAX, 1, OVL><<<grid, kCB, L::kBytes, st>>>(maps, a, t0);
  }
  return 0;
}

int launch_tma_screen(const N1Maps& maps, const Args& a, int RMAX, dim3 grid, cudaStream_t st, int t0) {
  if (RMAX == 4) return launch_tma_t<32, 4, false>(maps, a, grid, st, t0);
  if (RMAX == 8) return launch_tma_t<32, 8, false>(maps, a, grid, st, t0);
  return launch_tma_t<32, 16, false>(maps, a, grid, st, t0);
}

template <int RMAX>
int launch_tma_r(const N1Maps& maps, const Args& a, int TT, dim3 grid, cudaStream_t st, int t0) {
  switch (TT) {
    case 1: return launch_tma_t<1, RMAX>(maps, a, grid, st, t0);
    case 4: return launch_tma_t<4, RMAX>(maps, a, grid, st, t0);
    case 8: return launch_tma_t<8, RMAX>(maps, a, grid, st, t0);
    case 16: return launch_tma_t<16, RMAX>(maps, a, grid, st, t0);
    case 24: return launch_tma_t<24, RMAX>(maps, a, grid, st, t0);
    default: return launch_tma_t<32, RMAX>(maps, a, grid, st, t0);
  }
}

// selected-contingency mode (screened N-1), FP32, TT >= 4
template <int TT, int RMAX>
int launch_reg_sel_t(const N1Maps& maps, const Args& a, const SelArgs& sel, int items, cudaStream_t st, int t0) {
  using L = RegLayout<TT, RMAX, true>;
  static uint64_t attr = 0;
  if (smem_attr_once(k_n1_reg<TT, RMAX, true, true>, L::kBytes, attr) != cudaSuccess) return DCFLOW_ERR_CUDA;
  k_n1_reg<TT, RMAX, true, true><<<items, RegTile<TT>::NT, L::kBytes, st>>>(maps, a, t0, sel);
  return 0;
}
template <int RMAX>
int launch_reg_sel_r(const N1Maps& maps, const Args& a, const SelArgs& sel, int TT, int items, cudaStream_t st,
                     int t0) {
  switch (TT) {
    case 4: return launch_reg_sel_t<4, RMAX>(maps, a, sel, items, st, t0);
    case 8: return launch_reg_sel_t<8, RMAX>(maps, a, sel, items, st, t0);
    case 16: return launch_reg_sel_t<16, RMAX>(maps, a, sel, items, st, t0);
    case 24: return launch_reg_sel_t<24, RMAX>(maps, a, sel, items, st, t0);
    default: return launch_reg_sel_t<32, RMAX>(maps, a, sel, items, st, t0);
  }
}
int launch_reg_sel(const N1Maps& maps, const Args& a, const SelArgs& sel, int RMAX, int TT, int items,
                   cudaStream_t st, int t0) {
  if (RMAX == 4) return launch_reg_sel_r<4>(maps, a, sel, TT, items, st, t0);
  if (RMAX == 8) return launch_reg_sel_r<8>(maps, a, sel, TT, items, st, t0);
  return launch_reg_sel_r<16>(maps, a, sel, TT, items, st, t0);
}

// every topology's valid contingencies, compacted: grid (blocks per topology, slots)
template <int TT, int RMAX, bool OVL>
int launch_reg_cmp_t(const N1Maps& maps, const Args& a, const SelArgs& sel, dim3 grid, cudaStream_t st, int t0) {
  using L = RegLayout<TT, RMAX, true>;
  static uint64_t attr = 0;
  if (smem_attr_once(k_n1_reg<TT, RMAX, OVL, true>, L::kBytes, attr) != cudaSuccess) return DCFLOW_ERR_CUDA;
  k_n1_reg<TT, RMAX, OVL, true><<<grid, RegTile<TT>::NT, L::kBytes, st>>>(maps, a, t0, sel);
  return 0;
}
template <int RMAX>
int launch_reg_cmp_r(const N1Maps& maps, const Args& a, const SelArgs& sel, int TT, bool ovl, dim3 grid,
                     cudaStream_t st, int t0) {
  if (!ovl) return launch_reg_cmp_t<32, RMAX, false>(maps, a, sel, grid, st, t0);
  switch (TT) {
    case 4: return launch_reg_cmp_t<4, RMAX, true>(maps, a, sel, grid, st, t0);
    case 8: return launch_reg_cmp_t<8, RMAX, true>(maps, a, sel, grid, st, t0);
    case 16: return launch_reg_cmp_t<16, RMAX, true>(maps, a, sel, grid, st, t0);
    case 24: return launch_reg_cmp_t<24, RMAX, true>(maps, a, sel, grid, st, t0);
    default: return launch_reg_cmp_t<32, RMAX, true>(maps, a, sel, grid, st, t0);
  }
}
int launch_reg_cmp(const N1Maps& maps, const Args& a, const SelArgs& sel, int RMAX, int TT, bool ovl, dim3 grid,
                   cudaStream_t st, int t0) {
  if (RMAX == 4) return launch_reg_cmp_r<4>(maps, a, sel, TT, ovl, grid, st, t0);
  if (RMAX == 8) return launch_reg_cmp_r<8>(maps, a, sel, TT, ovl, grid, st, t0);
  return launch_reg_cmp_r<16>(maps, a, sel, TT, ovl, grid, st, t0);
}

int launch_tma(const N1Maps& maps, const Args& a, int RMAX, int TT, dim3 grid, cudaStream_t st, int t0) {
  if (RMAX == 4) return launch_tma_r<4>(maps, a, TT, grid, st, t0);
  if (RMAX == 8) return launch_tma_r<8>(maps, a, TT, grid, st, t0);
  return launch_tma_r<16>(maps, a, TT, grid, st, t0);
}

}  // namespace dcf
