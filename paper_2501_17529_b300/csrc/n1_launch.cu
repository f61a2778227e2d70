// Launchers of the FP32 fused N-1 kernels (declarations in n1_launch.cuh):
// the tensor maps, the dispatch between the two Phi_f builds, and the
// instances of the FFMA2 build (the tensor-core build: n1_launch_tc.cu).
#include <string>

#include <cudaTypedefs.h>

#include "n1_launch_impl.cuh"

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
               const uint32_t* box, bool swizzle128) {
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
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return DCFLOW_ERR_CUDA;
  }
  return 0;
}

// the tensor-core build is instantiated in n1_launch_tc.cu only
extern template int launch_tma_screen_k<true>(const N1Maps&, const Args&, int, dim3, cudaStream_t, int);
extern template int launch_tma_k<true>(const N1Maps&, const Args&, int, int, dim3, cudaStream_t, int);
extern template int launch_reg_sel_k<true>(const N1Maps&, const Args&, const SelArgs&, int, int, int, cudaStream_t,
                                           int);
extern template int launch_reg_cmp_k<true>(const N1Maps&, const Args&, const SelArgs&, int, int, bool, dim3,
                                           cudaStream_t, int);

template int launch_tma_screen_k<false>(const N1Maps&, const Args&, int, dim3, cudaStream_t, int);
template int launch_tma_k<false>(const N1Maps&, const Args&, int, int, dim3, cudaStream_t, int);
template int launch_reg_sel_k<false>(const N1Maps&, const Args&, const SelArgs&, int, int, int, cudaStream_t, int);
template int launch_reg_cmp_k<false>(const N1Maps&, const Args&, const SelArgs&, int, int, bool, dim3, cudaStream_t,
                                     int);

int launch_tma(const N1Maps& maps, const Args& a, int RMAX, int TT, dim3 grid, cudaStream_t st, int t0, bool tc) {
  if (tc && TT >= 4) return launch_tma_k<true>(maps, a, RMAX, TT, grid, st, t0);
  return launch_tma_k<false>(maps, a, RMAX, TT, grid, st, t0);
}

int launch_tma_screen(const N1Maps& maps, const Args& a, int RMAX, dim3 grid, cudaStream_t st, int t0, bool tc) {
  return tc ? launch_tma_screen_k<true>(maps, a, RMAX, grid, st, t0)
            : launch_tma_screen_k<false>(maps, a, RMAX, grid, st, t0);
}

int launch_reg_sel(const N1Maps& maps, const Args& a, const SelArgs& sel, int RMAX, int TT, int items,
                   cudaStream_t st, int t0, bool tc) {
  return tc ? launch_reg_sel_k<true>(maps, a, sel, RMAX, TT, items, st, t0)
            : launch_reg_sel_k<false>(maps, a, sel, RMAX, TT, items, st, t0);
}

int launch_reg_cmp(const N1Maps& maps, const Args& a, const SelArgs& sel, int RMAX, int TT, bool ovl, dim3 grid,
                   cudaStream_t st, int t0, bool tc) {
  return tc ? launch_reg_cmp_k<true>(maps, a, sel, RMAX, TT, ovl, grid, st, t0)
            : launch_reg_cmp_k<false>(maps, a, sel, RMAX, TT, ovl, grid, st, t0);
}

}  // namespace dcf
