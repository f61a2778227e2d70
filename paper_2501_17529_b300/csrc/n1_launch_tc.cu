// Instances of the FP32 fused N-1 kernel with the split-BF16x3 tensor-core
// Phi_f build (the dispatch lives in n1_launch.cu).
#include "n1_launch_impl.cuh"

namespace dcf {

template int launch_tma_screen_k<true>(const N1Maps&, const Args&, int, dim3, cudaStream_t, int);
template int launch_tma_k<true>(const N1Maps&, const Args&, int, int, dim3, cudaStream_t, int);
template int launch_reg_sel_k<true>(const N1Maps&, const Args&, const SelArgs&, int, int, int, cudaStream_t, int);
template int launch_reg_cmp_k<true>(const N1Maps&, const Args&, const SelArgs&, int, int, bool, dim3, cudaStream_t,
                                    int);

}  // namespace dcf
