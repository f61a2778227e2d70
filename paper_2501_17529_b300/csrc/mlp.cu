// Tensor-core building blocks of the learned contingency screener.
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "internal.cuh"
#include "tc_gemm.cuh"

namespace dcf {

static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
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

// 2-D bf16 K-major operand [rows x K] (row pitch ld elements) as 64 x 128 boxes with 128-byte swizzle.
static int bf16_operand_map(CUtensorMap* m, const void* base, int rows, int K, int ld) {
  auto fn = encoder();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return DCFLOW_ERR_CUDA;
  }
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * 2) % 16) {
    set_error("tensor-core GEMM operand must be 16-byte aligned with a 16-byte row pitch");
    return DCFLOW_ERR_INVALID_ARG;
  }
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {tc::BK, tc::BM};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (bf16) failed: " + std::to_string((int)r));
    return DCFLOW_ERR_CUDA;
  }
  return 0;
}

// D[M x N] = A[M x K] B[N x K]^T (+ bias) (ReLU) on the tensor cores.
int gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K, const float* bias, bool relu,
              void* D, int ldd, bool out_bf16, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0 || M % tc::BM || N % tc::BN || K % tc::BK) {
    set_error("tensor-core GEMM needs M, N multiples of 128 and K a multiple of 64");
    return DCFLOW_ERR_INVALID_ARG;
  }
  CUtensorMap ma, mb;
  int rc = bf16_operand_map(&ma, A, M, K, lda);
  if (!rc) rc = bf16_operand_map(&mb, B, N, K, ldb);
  if (rc) return rc;
  static bool attr = false;
  if (!attr) {
    DCF_CUDA(cudaFuncSetAttribute(tc::k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes));
    attr = true;
  }
  tc::GemmArgs g{M, N, K, bias, relu ? 1 : 0, D, ldd, out_bf16 ? 1 : 0, err};
  tc::k_gemm_bf16<<<dim3(N / tc::BN, M / tc::BM), 128, tc::kSmemBytes, st>>>(ma, mb, g);
  DCF_CHECK_LAUNCH();
  return 0;
}

}  // namespace dcf

using namespace dcf;

extern "C" int dcflow_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B,
                                int32_t ldb, const float* bias, int32_t relu, void* D, int32_t ldd, int32_t out_bf16,
                                void* stream) {
  static std::mutex mu;
  static int* d_err = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!d_err) {
      if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) {
        set_error("dcflow_gemm_bf16: allocation of the error word failed");
        return DCFLOW_ERR_OOM;
      }
      cudaMemset(d_err, 0, sizeof(int));
    }
  }
  if (!A || !B || !D) {
    set_error("dcflow_gemm_bf16: null operand");
    return DCFLOW_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = gemm_bf16(A, lda, B, ldb, M, N, K, bias, relu != 0, D, ldd, out_bf16 != 0, d_err, st);
  if (rc) return rc;
  int h = 0;
  DCF_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DCF_CUDA(cudaStreamSynchronize(st));
  if (h) {
    cudaMemsetAsync(d_err, 0, sizeof(int), st);
    set_error("dcflow_gemm_bf16: a bounded device wait expired");
    return DCFLOW_ERR_TIMEOUT;
  }
  return DCFLOW_OK;
}
