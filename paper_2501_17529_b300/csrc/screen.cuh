// Learned contingency screener: model state and the pieces shared between the
// training entry points (mlp.cu) and the screened solve (solve.cu).
//
// Network (F inputs, H = 256 hidden, C outputs, BF16 operands on the tensor
// cores, FP32 accumulation and FP32 master weights with Adam moments):
//   h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2), z = h2 W3^T + b3.
// Features of one (topology, timestep): the M signed N-0 loadings
// p_f[l] / limit_l (Eq. (2) on the modified topology), then one bit per
// incident branch of every split-capable substation (ascending bus id, then
// ascending branch id: the order of the busbar masks of Sec. III-A), 1 if the
// branch sits on busbar B; zero padding up to Fp = round_up(F, 128).
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace dcf {

constexpr int kScreenHidden = 256;
enum : int { kW1 = 0, kB1, kW2, kB2, kW3, kB3, kNumScreenTensors };

// One tensor-core GEMM D = A B^T with the epilogue options of k_gemm_bf16.
struct GemmSpec {
  const void* A = nullptr;
  int lda = 0;
  const void* B = nullptr;
  int ldb = 0;
  int M = 0, N = 0, K = 0;
  const float* bias = nullptr;
  bool relu = false;
  const __nv_bfloat16* mask = nullptr;
  int ldm = 0;
  void* D = nullptr;
  int ldd = 0;
  bool out_bf16 = false;
  __nv_bfloat16* Dt = nullptr;
  int lddt = 0;
  int splits = 1;          // split-K factor (FP32 output without epilogue options only)
  float* part = nullptr;   // splits * M * ldd floats of scratch when splits > 1
};
int gemm_run(const GemmSpec& s, int* err, cudaStream_t st);

// Order-preserving key of a float: larger value <=> larger unsigned key.
__device__ __forceinline__ uint32_t float_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// k-th largest of the warp's 32 * NPL keys (lane owns elements lane + 32 i);
// warp-uniform result built bit by bit from the top: the largest x with
// #{key >= x} >= k.  Also returns #{key > x}.
template <int NPL>
__device__ __forceinline__ void warp_kth_key(const uint32_t (&key)[NPL], int k, uint32_t& thr, int& n_above) {
  uint32_t prefix = 0;
#pragma unroll 1
  for (int bit = 31; bit >= 0; --bit) {
    const uint32_t cand = prefix | (1u << bit);
    int cnt = 0;
#pragma unroll
    for (int i = 0; i < NPL; ++i) cnt += key[i] >= cand;
#pragma unroll
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (cnt >= k) prefix = cand;
  }
  thr = prefix;
  int cnt = 0;
#pragma unroll
  for (int i = 0; i < NPL; ++i) cnt += key[i] > prefix;
#pragma unroll
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  n_above = cnt;
}

// Membership of the top k (ties at the threshold to the lower element index).
template <int NPL>
__device__ __forceinline__ void warp_top_k(const uint32_t (&key)[NPL], int k, bool (&sel)[NPL], uint32_t& thr) {
  int above;
  warp_kth_key<NPL>(key, k, thr, above);
  const int lane = threadIdx.x & 31;
  int need = k - above;  // elements equal to the threshold still to take, lowest index first
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const bool eq = key[i] == thr;
    const uint32_t b = __ballot_sync(0xffffffffu, eq);
    const int rank = __popc(b & ((1u << lane) - 1u));
    sel[i] = key[i] > thr || (eq && rank < need);
    need -= __popc(b);
    if (need < 0) need = 0;
  }
}

}  // namespace dcf

struct dcflow_screen {
  dcflow_ctx* ctx = nullptr;
  int dev = 0;
  int M = 0, C = 0, F = 0, Fp = 0, H = dcf::kScreenHidden, Cp = 0, V = 0, max_rows = 0;
  int64_t t = 0;  // Adam steps taken
  float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  dcf::DevBuf foff;  // int[V]: offset of bus v's split bits among the features (-1: not split-capable)
  dcf::DevBuf prm[dcf::kNumScreenTensors], grd[dcf::kNumScreenTensors];
  dcf::DevBuf mom[dcf::kNumScreenTensors], vel[dcf::kNumScreenTensors];
  dcf::DevBuf wb[3], wt[3];  // BF16 W_i [out x in] and W_i^T [in x out]
  // training activations, max_rows rows
  dcf::DevBuf Xb, Xt, Yb, H1, H1t, H2, H2t, Z, dZ, dZt, dH2, dH2t, dH1t, part, err;
  // inference activations of the screened solve (grown on demand)
  dcf::DevBuf iX, iH1, iH2, iZ;
  int rows(int k) const { return (k == dcf::kW1 || k == dcf::kB1 || k == dcf::kW2 || k == dcf::kB2) ? H : Cp; }
  int cols(int k) const { return k == dcf::kW1 ? Fp : ((k == dcf::kW2 || k == dcf::kW3) ? H : 1); }
  int logical_rows(int k) const { return (k == dcf::kW3 || k == dcf::kB3) ? C : H; }
  int logical_cols(int k) const { return k == dcf::kW1 ? F : ((k == dcf::kW2 || k == dcf::kW3) ? H : 1); }
};
