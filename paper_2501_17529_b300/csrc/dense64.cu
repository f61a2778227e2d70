// FP64 dense kernels for the one-time base factorisation (Sec. II, Def. 2 /
// Eq. (1)): the reduced nodal susceptance matrix B' is factored as L L^T by a
// blocked right-looking Cholesky, and many right-hand sides are solved with
// blocked forward / backward substitution.  All matrices are row-major and
// padded to multiples of kNB = 64 (padding carries an identity block), so no
// tile is ragged.  B300 has a weak FP64 pipe; these kernels run once per
// grid / study and are not on the per-batch path.
#include "internal.cuh"
#include "dense64.cuh"

namespace dcf {

// C[M x N] -= op(A)[M x K] * op(B)[K x N]; M, N multiples of 64, K of 16.
// A(m,k) = TA ? A[k*lda + m] : A[m*lda + k];  B(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n].
// LOWER: skip output tiles strictly above the block diagonal (square C).
template <bool TA, bool TB, bool LOWER>
__global__ __launch_bounds__(256) void k_dgemm_sub(int M, int N, int K, const double* __restrict__ A,
                                                  int lda, const double* __restrict__ B, int ldb,
                                                  double* __restrict__ C, int ldc) {
  if (LOWER && blockIdx.x > blockIdx.y) return;
  __shared__ double As[16][64];
  __shared__ double Bs[16][64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = tid + q * 256;  // 0..1023
      if (!TA) {
        int m = idx >> 4, k = idx & 15;
        As[k][m] = A[(size_t)(m0 + m) * lda + k0 + k];
      } else {
        int k = idx >> 6, m = idx & 63;
        As[k][m] = A[(size_t)(k0 + k) * lda + m0 + m];
      }
      if (!TB) {
        int k = idx >> 6, n = idx & 63;
        Bs[k][n] = B[(size_t)(k0 + k) * ldb + n0 + n];
      } else {
        int n = idx >> 4, k = idx & 15;
        Bs[k][n] = B[(size_t)(n0 + n) * ldb + k0 + k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double* c = C + (size_t)(m0 + ty + 16 * i) * ldc + n0 + tx + 16 * j;
      *c -= acc[i][j];
    }
}

// Cholesky of the 64x64 diagonal block kb (lower); info <- 1 + row of a
// non-positive pivot (the matrix is not positive definite).
__global__ __launch_bounds__(256) void k_potrf_diag(double* A, int lda, int kb, int* info) {
  __shared__ double a[64][65];
  double* blk = A + (size_t)kb * 64 * lda + kb * 64;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < 4096; idx += 256) a[idx >> 6][idx & 63] = blk[(size_t)(idx >> 6) * lda + (idx & 63)];
  __syncthreads();
  for (int k = 0; k < 64; ++k) {
    if (tid == 0) {
      double d = a[k][k];
      if (!(d > 0.0)) {
        atomicCAS(info, 0, 1 + kb * 64 + k);
        d = 1.0;
      }
      a[k][k] = sqrt(d);
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < 64; i += 256) a[i][k] /= a[k][k];
    __syncthreads();
    const int m = 63 - k;
    for (int idx = tid; idx < m * m; idx += 256) {
      int i = k + 1 + idx / m, j = k + 1 + idx % m;
      if (j <= i) a[i][j] = fma(-a[i][k], a[j][k], a[i][j]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < 4096; idx += 256) {
    int i = idx >> 6, j = idx & 63;
    blk[(size_t)i * lda + j] = (j <= i) ? a[i][j] : 0.0;
  }
}

// Panel: A[ib][kb] <- A[ib][kb] * L_kk^{-T} for ib = kb+1+blockIdx.x (one thread per row).
__global__ __launch_bounds__(64) void k_trsm_panel(double* A, int lda, int kb) {
  __shared__ double Lk[64][65];
  __shared__ double X[64][65];
  const int ib = kb + 1 + blockIdx.x, r = threadIdx.x;
  const double* lk = A + (size_t)kb * 64 * lda + kb * 64;
  double* xb = A + (size_t)ib * 64 * lda + kb * 64;
  for (int idx = r; idx < 4096; idx += 64) {
    Lk[idx >> 6][idx & 63] = lk[(size_t)(idx >> 6) * lda + (idx & 63)];
    X[idx >> 6][idx & 63] = xb[(size_t)(idx >> 6) * lda + (idx & 63)];
  }
  __syncthreads();
  for (int j = 0; j < 64; ++j) {
    double s = X[r][j];
    for (int p = 0; p < j; ++p) s = fma(-X[r][p], Lk[j][p], s);
    X[r][j] = s / Lk[j][j];
  }
  __syncthreads();
  for (int idx = r; idx < 4096; idx += 64) xb[(size_t)(idx >> 6) * lda + (idx & 63)] = X[idx >> 6][idx & 63];
}

// Forward substitution on block row kb of the right-hand sides: R_kb <- L_kk^{-1} R_kb.
__global__ __launch_bounds__(64) void k_trsm_fwd(const double* L, int ldl, int kb, double* R, int ldr) {
  __shared__ double Lk[64][64];
  const double* lk = L + (size_t)kb * 64 * ldl + kb * 64;
  for (int idx = threadIdx.x; idx < 4096; idx += 64) Lk[idx >> 6][idx & 63] = lk[(size_t)(idx >> 6) * ldl + (idx & 63)];
  __syncthreads();
  double* rc = R + (size_t)kb * 64 * ldr + blockIdx.x * 64 + threadIdx.x;
  double z[64];
#pragma unroll
  for (int i = 0; i < 64; ++i) z[i] = rc[(size_t)i * ldr];
#pragma unroll
  for (int i = 0; i < 64; ++i) {
    double s = z[i];
#pragma unroll
    for (int p = 0; p < i; ++p) s = fma(-Lk[i][p], z[p], s);
    z[i] = s / Lk[i][i];
  }
#pragma unroll
  for (int i = 0; i < 64; ++i) rc[(size_t)i * ldr] = z[i];
}

// Backward substitution on block row kb: R_kb <- L_kk^{-T} R_kb.
__global__ __launch_bounds__(64) void k_trsm_bwd(const double* L, int ldl, int kb, double* R, int ldr) {
  __shared__ double Lk[64][64];
  const double* lk = L + (size_t)kb * 64 * ldl + kb * 64;
  for (int idx = threadIdx.x; idx < 4096; idx += 64) Lk[idx >> 6][idx & 63] = lk[(size_t)(idx >> 6) * ldl + (idx & 63)];
  __syncthreads();
  double* rc = R + (size_t)kb * 64 * ldr + blockIdx.x * 64 + threadIdx.x;
  double z[64];
#pragma unroll
  for (int i = 0; i < 64; ++i) z[i] = rc[(size_t)i * ldr];
#pragma unroll
  for (int i = 63; i >= 0; --i) {
    double s = z[i];
#pragma unroll
    for (int p = i + 1; p < 64; ++p) s = fma(-Lk[p][i], z[p], s);
    z[i] = s / Lk[i][i];
  }
#pragma unroll
  for (int i = 0; i < 64; ++i) rc[(size_t)i * ldr] = z[i];
}

int dgemm_sub(bool ta, bool tb, bool lower, int M, int N, int K, const double* A, int lda,
              const double* B, int ldb, double* C, int ldc, cudaStream_t st, int64_t* launches) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  dim3 grid(N / 64, M / 64);
  if (!ta && tb && lower) k_dgemm_sub<false, true, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc);
  else if (!ta && !tb) k_dgemm_sub<false, false, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc);
  else if (ta && !tb) k_dgemm_sub<true, false, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc);
  else if (!ta && tb) k_dgemm_sub<false, true, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc);
  else return DCFLOW_ERR_INVALID_ARG;
  ++*launches;
  DCF_CHECK_LAUNCH();
  return 0;
}

int cholesky(double* A, int npad, int* d_info, cudaStream_t st, int64_t* launches) {
  const int nb = npad / 64;
  for (int kb = 0; kb < nb; ++kb) {
    k_potrf_diag<<<1, 256, 0, st>>>(A, npad, kb, d_info);
    ++*launches;
    DCF_CHECK_LAUNCH();
    if (kb + 1 < nb) {
      k_trsm_panel<<<nb - kb - 1, 64, 0, st>>>(A, npad, kb);
      ++*launches;
      DCF_CHECK_LAUNCH();
      const int m = (nb - kb - 1) * 64;
      double* a21 = A + (size_t)(kb + 1) * 64 * npad + kb * 64;
      double* a22 = A + (size_t)(kb + 1) * 64 * npad + (kb + 1) * 64;
      int rc = dgemm_sub(false, true, true, m, m, 64, a21, npad, a21, npad, a22, npad, st, launches);
      if (rc) return rc;
    }
  }
  return 0;
}

int chol_solve(const double* L, int npad, double* R, int ldr, int ncol, cudaStream_t st, int64_t* launches) {
  const int nb = npad / 64;
  if (ncol <= 0) return 0;
  for (int kb = 0; kb < nb; ++kb) {
    k_trsm_fwd<<<ncol / 64, 64, 0, st>>>(L, npad, kb, R, ldr);
    ++*launches;
    DCF_CHECK_LAUNCH();
    if (kb + 1 < nb) {
      int rc = dgemm_sub(false, false, false, (nb - kb - 1) * 64, ncol, 64,
                         L + (size_t)(kb + 1) * 64 * npad + kb * 64, npad,
                         R + (size_t)kb * 64 * ldr, ldr, R + (size_t)(kb + 1) * 64 * ldr, ldr, st, launches);
      if (rc) return rc;
    }
  }
  for (int kb = nb - 1; kb >= 0; --kb) {
    k_trsm_bwd<<<ncol / 64, 64, 0, st>>>(L, npad, kb, R, ldr);
    ++*launches;
    DCF_CHECK_LAUNCH();
    if (kb > 0) {
      // R[0:kb] -= (L[kb, 0:kb])^T * R_kb
      int rc = dgemm_sub(true, false, false, kb * 64, ncol, 64, L + (size_t)kb * 64 * npad, npad,
                         R + (size_t)kb * 64 * ldr, ldr, R, ldr, st, launches);
      if (rc) return rc;
    }
  }
  return 0;
}

}  // namespace dcf
