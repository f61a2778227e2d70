// Host entry points of the FP64 dense kernels (blocked Cholesky and solves).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dcf {
// C -= op(A) op(B) for row-major padded matrices (M, N multiples of 64, K of 16).
int dgemm_sub(bool ta, bool tb, bool lower, int M, int N, int K, const double* A, int lda,
              const double* B, int ldb, double* C, int ldc, cudaStream_t st, int64_t* launches);
// In-place lower Cholesky of the padded SPD matrix A (npad x npad); d_info != 0 on failure.
int cholesky(double* A, int npad, int* d_info, cudaStream_t st, int64_t* launches);
// R (npad x ncol, leading dimension ldr) <- (L L^T)^{-1} R; ncol a multiple of 64.
int chol_solve(const double* L, int npad, double* R, int ldr, int ncol, cudaStream_t st, int64_t* launches);
}  // namespace dcf
