// Tensor-core GEMM host side and the learned contingency screener: model
// state, training (forward, binary cross-entropy, backward, Adam) and
// inference entry points of the C ABI.
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "screen.cuh"
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

// 2-D bf16 K-major operand [rows x K] (row pitch ld elements) as 64 x box_rows boxes with 128-byte swizzle.
static int bf16_operand_map(CUtensorMap* m, const void* base, int rows, int K, int ld, int box_rows) {
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
  cuuint32_t box[2] = {tc::BK, (cuuint32_t)box_rows};
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

__global__ void k_splitk_reduce(const float* __restrict__ part, int S, int M, int N, int ld, float* __restrict__ D) {
  const size_t n = (size_t)M * ld;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if ((int)(i % ld) >= N) continue;
    float s = 0.f;
    for (int z = 0; z < S; ++z) s += part[z * n + i];
    D[i] = s;
  }
}

int gemm_run(const GemmSpec& s, int* err, cudaStream_t st) {
  if (s.M <= 0 || s.N <= 0 || s.K <= 0 || s.M % tc::BM || s.N % 128 || s.splits < 1 ||
      s.K % (tc::BK * s.splits)) {
    set_error("tensor-core GEMM needs M, N multiples of 128 and K a multiple of 64 x splits");
    return DCFLOW_ERR_INVALID_ARG;
  }
  if (s.splits > 1 && (s.out_bf16 || s.bias || s.relu || s.mask || s.Dt || !s.part || !s.D)) {
    set_error("split-K GEMM: FP32 output without epilogue options, with scratch");
    return DCFLOW_ERR_INVALID_ARG;
  }
  if ((s.mask && (s.ldm % 8 || (reinterpret_cast<uintptr_t>(s.mask) & 15))) ||
      (s.D && (s.ldd % 4 || (reinterpret_cast<uintptr_t>(s.D) & 15)))) {
    set_error("tensor-core GEMM: D and mask need 16-byte aligned rows");
    return DCFLOW_ERR_INVALID_ARG;
  }
  // the wide tile where it still gives at least 120 CTAs
  const bool wide = s.N % 256 == 0 && (int64_t)(s.M / 128) * (s.N / 256) * s.splits >= 120;
  const int BN = wide ? 256 : 128;
  CUtensorMap ma, mb;
  int rc = bf16_operand_map(&ma, s.A, s.M, s.K, s.lda, tc::BM);
  if (!rc) rc = bf16_operand_map(&mb, s.B, s.N, s.K, s.ldb, BN);
  if (rc) return rc;
  static uint64_t attr128 = 0, attr256 = 0;
  DCF_CUDA(smem_attr_once(tc::k_gemm_bf16<128>, tc::Cfg<128>::kSmemBytes, attr128));
  DCF_CUDA(smem_attr_once(tc::k_gemm_bf16<256>, tc::Cfg<256>::kSmemBytes, attr256));
  tc::GemmArgs g{};
  g.M = s.M;
  g.N = s.N;
  g.K = s.K;
  g.bias = s.bias;
  g.relu = s.relu ? 1 : 0;
  g.mask = s.mask;
  g.ldm = s.ldm;
  g.D = s.splits > 1 ? static_cast<void*>(s.part) : s.D;
  g.ldd = s.ldd;
  g.out_bf16 = s.out_bf16 ? 1 : 0;
  g.Dt = s.Dt;
  g.lddt = s.lddt;
  g.split_stride = (long long)s.M * s.ldd;
  g.err = err;
  if (wide)
    tc::k_gemm_bf16<256><<<dim3(s.N / 256, s.M / tc::BM, s.splits), 128, tc::Cfg<256>::kSmemBytes, st>>>(ma, mb, g);
  else
    tc::k_gemm_bf16<128><<<dim3(s.N / 128, s.M / tc::BM, s.splits), 128, tc::Cfg<128>::kSmemBytes, st>>>(ma, mb, g);
  DCF_CHECK_LAUNCH();
  if (s.splits > 1) {
    k_splitk_reduce<<<592, 256, 0, st>>>(s.part, s.splits, s.M, s.N, s.ldd, static_cast<float*>(s.D));
    DCF_CHECK_LAUNCH();
  }
  return 0;
}

// ---------------------------------------------------------------------------
// screener kernels
// ---------------------------------------------------------------------------
// Row gather with an optional transposed copy: dst[r, :] = src[idx[r], :]
// (idx null: row r itself) for r < n, zero rows for n <= r < rows; dstT[c, r]
// mirrors dst.  32 x 32 tiles through shared memory keep both stores coalesced.
template <class E>
__global__ void k_gather_rows(const E* __restrict__ src, int64_t lds, const int* __restrict__ idx, int n, int rows,
                              int cols, E* __restrict__ dst, int ldd, E* __restrict__ dstT, int lddt) {
  __shared__ E tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    E v{};
    if (r < n && c < cols) v = src[(size_t)(idx ? idx[r] : r) * lds + c];
    if (r < rows && c < cols) dst[(size_t)r * ldd + c] = v;
    tile[i][threadIdx.x] = v;
  }
  if (!dstT) return;
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dstT[(size_t)c * lddt + r] = tile[threadIdx.x][i];
  }
}

// Binary cross-entropy with logits, mean over n rows x C outputs:
// dz = (sigmoid(z) - y) / (n C) (zero on padding), stored in BF16 row-major and
// transposed; the loss sum goes to *loss.
__global__ void k_bce(const float* __restrict__ Z, int ldz, const uint8_t* __restrict__ Y, int ldy, int n, int rows,
                      int C, int Cp, float scale, __nv_bfloat16* __restrict__ dZ, __nv_bfloat16* __restrict__ dZt,
                      float* __restrict__ loss) {
  __shared__ float tile[32][33];
  __shared__ float red[8];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  float acc = 0.f;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    float d = 0.f;
    if (r < n && c < C) {
      const float z = Z[(size_t)r * ldz + c];
      const float y = (float)Y[(size_t)r * ldy + c];
      const float sp = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
      acc += sp - y * z;
      d = (1.f / (1.f + expf(-z)) - y) * scale;
    }
    if (r < rows && c < Cp) dZ[(size_t)r * Cp + c] = __float2bfloat16_rn(d);
    tile[i][threadIdx.x] = d;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < Cp && r < rows) dZt[(size_t)c * rows + r] = __float2bfloat16_rn(tile[threadIdx.x][i]);
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) red[threadIdx.y] = acc;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)blockDim.y; ++w) s += red[w];
    atomicAdd(loss, s * scale);
  }
}

// out[r] = sum_k A[r, k] (BF16 rows, FP32 sum): the bias gradients from the
// transposed output gradients.  One warp per row.
__global__ void k_rowsum(const __nv_bfloat16* __restrict__ A, int R, int K, int lda, float* __restrict__ out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= R) return;
  float s = 0.f;
  for (int k = lane; k < K; k += 32) s += __bfloat162float(A[(size_t)w * lda + k]);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[w] = s;
}

// Adam (bias-corrected) on the logical part of a [rows x cols] tensor with row
// pitch ld; refreshes the BF16 copy (and its transpose) of a weight matrix.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int lrows, int lcols, int ld, int rows, float lr, float b1, float b2,
                       float eps, float bc1, float bc2, __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wt) {
  const size_t n = (size_t)lrows * lcols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / lcols), c = (int)(e % lcols);
    const size_t i = (size_t)r * ld + c;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
    if (wb) wb[i] = __float2bfloat16_rn(pi);
    if (wt) wt[(size_t)c * rows + r] = __float2bfloat16_rn(pi);
  }
}

__global__ void k_to_bf16(const float* __restrict__ p, int rows, int cols, __nv_bfloat16* __restrict__ wb,
                          __nv_bfloat16* __restrict__ wt) {
  const size_t n = (size_t)rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e % cols);
    const __nv_bfloat16 h = __float2bfloat16_rn(p[e]);
    if (wb) wb[e] = h;
    if (wt) wt[(size_t)c * rows + r] = h;
  }
}

// Labels: y[r, c] = 1 iff c is among the k largest cmax[r, :] (ties to the
// lower c) and cmax[r, c] > 1.  One warp per row; padding columns are zero.
template <int NPL>
__global__ void k_labels(const float* __restrict__ cmax, int64_t rows, int C, int k, uint8_t* __restrict__ Y,
                         int64_t ldy) {
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  uint32_t key[NPL];
  float val[NPL];
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const int c = lane + 32 * i;
    val[i] = c < C ? cmax[r * C + c] : -1.f;
    key[i] = c < C ? float_key(val[i]) : 0u;
  }
  bool sel[NPL];
  uint32_t thr;
  warp_top_k<NPL>(key, k < C ? k : C, sel, thr);
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const int c = lane + 32 * i;
    if (c < ldy) Y[r * ldy + c] = (c < C && sel[i] && val[i] > 1.f) ? 1 : 0;
  }
}

// Counter-based normal numbers for the initial weights: SplitMix64 of
// (seed, tensor, index), two uniforms, Box-Muller.
static uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
static double normal_at(uint64_t seed, int tensor, uint64_t i) {
  const uint64_t a = splitmix64(seed ^ ((uint64_t)tensor << 56) ^ (2 * i));
  const uint64_t b = splitmix64(seed ^ ((uint64_t)tensor << 56) ^ (2 * i + 1));
  const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0);  // (0, 1]
  const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

static int refresh_bf16(dcflow_screen* s, int k, cudaStream_t st) {
  const int w = k / 2;
  if (k % 2) return 0;
  k_to_bf16<<<296, 256, 0, st>>>(s->prm[k].as<float>(), s->rows(k), s->cols(k), s->wb[w].as<__nv_bfloat16>(),
                                 w ? s->wt[w].as<__nv_bfloat16>() : nullptr);
  DCF_CHECK_LAUNCH();
  return 0;
}

static int check_err(dcflow_screen* s, cudaStream_t st) {
  int h = 0;
  DCF_CUDA(cudaMemcpyAsync(&h, s->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  DCF_CUDA(cudaStreamSynchronize(st));
  if (h) {
    DCF_CUDA(cudaMemsetAsync(s->err.p, 0, sizeof(int), st));
    set_error("screener: a bounded device wait of a tensor-core GEMM expired");
    return DCFLOW_ERR_TIMEOUT;
  }
  return 0;
}

// Forward (and optionally backward) of n rows gathered from X (and Y).
static int screen_pass(dcflow_screen* s, const void* X, int64_t ldx, const uint8_t* Y, int64_t ldy, const int* rows,
                       int n, bool backward, float* loss, cudaStream_t st) {
  using bf = __nv_bfloat16;
  const int B = (int)round_up(n, 128), Fp = s->Fp, H = s->H, Cp = s->Cp;
  int* err = s->err.as<int>();
  {
    dim3 blk(32, 8), grd((Fp + 31) / 32, B / 32);
    k_gather_rows<bf><<<grd, blk, 0, st>>>(static_cast<const bf*>(X), ldx, rows, n, B, Fp, s->Xb.as<bf>(), Fp,
                                           backward ? s->Xt.as<bf>() : nullptr, B);
    DCF_CHECK_LAUNCH();
    if (backward) {
      dim3 gy((Cp + 31) / 32, B / 32);
      k_gather_rows<uint8_t><<<gy, blk, 0, st>>>(Y, ldy, rows, n, B, Cp, s->Yb.as<uint8_t>(), Cp, nullptr, 0);
      DCF_CHECK_LAUNCH();
    }
  }
  GemmSpec g1;
  g1.A = s->Xb.p; g1.lda = Fp; g1.B = s->wb[0].p; g1.ldb = Fp; g1.M = B; g1.N = H; g1.K = Fp;
  g1.bias = s->prm[kB1].as<float>(); g1.relu = true; g1.D = s->H1.p; g1.ldd = H; g1.out_bf16 = true;
  if (backward) { g1.Dt = s->H1t.as<bf>(); g1.lddt = B; }
  int rc = gemm_run(g1, err, st);
  if (rc) return rc;
  GemmSpec g2;
  g2.A = s->H1.p; g2.lda = H; g2.B = s->wb[1].p; g2.ldb = H; g2.M = B; g2.N = H; g2.K = H;
  g2.bias = s->prm[kB2].as<float>(); g2.relu = true; g2.D = s->H2.p; g2.ldd = H; g2.out_bf16 = true;
  if (backward) { g2.Dt = s->H2t.as<bf>(); g2.lddt = B; }
  if ((rc = gemm_run(g2, err, st))) return rc;
  GemmSpec g3;
  g3.A = s->H2.p; g3.lda = H; g3.B = s->wb[2].p; g3.ldb = H; g3.M = B; g3.N = Cp; g3.K = H;
  g3.bias = s->prm[kB3].as<float>(); g3.D = s->Z.p; g3.ldd = Cp;
  if ((rc = gemm_run(g3, err, st))) return rc;
  if (!backward) return 0;
  {
    dim3 blk(32, 8), grd(Cp / 32, B / 32);
    k_bce<<<grd, blk, 0, st>>>(s->Z.as<float>(), Cp, s->Yb.as<uint8_t>(), Cp, n, B, s->C, Cp,
                               1.f / ((float)n * (float)s->C), s->dZ.as<bf>(), s->dZt.as<bf>(), loss);
    DCF_CHECK_LAUNCH();
  }
  // split-K for the weight gradients (K = batch rows): enough CTAs for the SMs
  auto splits_for = [&](int M, int N) {
    int sp = 1;
    const int tiles = (M / 128) * (N / 128);
    while (tiles * sp * 2 <= 148 && (B / 64) % (sp * 2) == 0 && sp < 16) sp *= 2;
    return sp;
  };
  GemmSpec g4;  // dW3 = dZ^T H2
  g4.A = s->dZt.p; g4.lda = B; g4.B = s->H2t.p; g4.ldb = B; g4.M = Cp; g4.N = H; g4.K = B;
  g4.D = s->grd[kW3].p; g4.ldd = H; g4.splits = splits_for(Cp, H); g4.part = s->part.as<float>();
  if ((rc = gemm_run(g4, err, st))) return rc;
  GemmSpec g5;  // dH2 = (dZ W3) * relu'(a2)
  g5.A = s->dZ.p; g5.lda = Cp; g5.B = s->wt[2].p; g5.ldb = Cp; g5.M = B; g5.N = H; g5.K = Cp;
  g5.mask = s->H2.as<bf>(); g5.ldm = H; g5.D = s->dH2.p; g5.ldd = H; g5.out_bf16 = true;
  g5.Dt = s->dH2t.as<bf>(); g5.lddt = B;
  if ((rc = gemm_run(g5, err, st))) return rc;
  GemmSpec g6;  // dW2 = dH2^T H1
  g6.A = s->dH2t.p; g6.lda = B; g6.B = s->H1t.p; g6.ldb = B; g6.M = H; g6.N = H; g6.K = B;
  g6.D = s->grd[kW2].p; g6.ldd = H; g6.splits = splits_for(H, H); g6.part = s->part.as<float>();
  if ((rc = gemm_run(g6, err, st))) return rc;
  GemmSpec g7;  // dH1 = (dH2 W2) * relu'(a1), kept transposed only
  g7.A = s->dH2.p; g7.lda = H; g7.B = s->wt[1].p; g7.ldb = H; g7.M = B; g7.N = H; g7.K = H;
  g7.mask = s->H1.as<bf>(); g7.ldm = H; g7.Dt = s->dH1t.as<bf>(); g7.lddt = B;
  if ((rc = gemm_run(g7, err, st))) return rc;
  GemmSpec g8;  // dW1 = dH1^T X
  g8.A = s->dH1t.p; g8.lda = B; g8.B = s->Xt.p; g8.ldb = B; g8.M = H; g8.N = Fp; g8.K = B;
  g8.D = s->grd[kW1].p; g8.ldd = Fp; g8.splits = splits_for(H, Fp); g8.part = s->part.as<float>();
  if ((rc = gemm_run(g8, err, st))) return rc;
  const int wpb = 8;
  k_rowsum<<<(Cp + wpb - 1) / wpb, 32 * wpb, 0, st>>>(s->dZt.as<bf>(), Cp, B, B, s->grd[kB3].as<float>());
  k_rowsum<<<(H + wpb - 1) / wpb, 32 * wpb, 0, st>>>(s->dH2t.as<bf>(), H, B, B, s->grd[kB2].as<float>());
  k_rowsum<<<(H + wpb - 1) / wpb, 32 * wpb, 0, st>>>(s->dH1t.as<bf>(), H, B, B, s->grd[kB1].as<float>());
  DCF_CHECK_LAUNCH();
  return 0;
}

static int screen_adam(dcflow_screen* s, float lr, cudaStream_t st) {
  s->t += 1;
  const float bc1 = 1.f - (float)std::pow((double)s->beta1, (double)s->t);
  const float bc2 = 1.f - (float)std::pow((double)s->beta2, (double)s->t);
  for (int k = 0; k < kNumScreenTensors; ++k) {
    const int w = k / 2;
    const bool mat = k % 2 == 0;
    k_adam<<<592, 256, 0, st>>>(s->prm[k].as<float>(), s->grd[k].as<float>(), s->mom[k].as<float>(),
                                s->vel[k].as<float>(), s->logical_rows(k), s->logical_cols(k), s->cols(k), s->rows(k),
                                lr, s->beta1, s->beta2, s->eps, bc1, bc2,
                                mat ? s->wb[w].as<__nv_bfloat16>() : nullptr,
                                (mat && w) ? s->wt[w].as<__nv_bfloat16>() : nullptr);
    DCF_CHECK_LAUNCH();
  }
  return 0;
}

}  // namespace dcf

using namespace dcf;

extern "C" int dcflow_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B,
                                int32_t ldb, const float* bias, int32_t relu, void* D, int32_t ldd, int32_t out_bf16,
                                void* stream) {
  static std::mutex mu;
  static int* d_errs[64] = {};  // one error word per device
  int dev = 0;
  DCF_CUDA(cudaGetDevice(&dev));
  if (dev >= 64) {
    set_error("dcflow_gemm_bf16: device index above 63");
    return DCFLOW_ERR_INVALID_ARG;
  }
  int* d_err = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!d_errs[dev]) {
      if (cudaMalloc(&d_errs[dev], sizeof(int)) != cudaSuccess) {
        d_errs[dev] = nullptr;
        set_error("dcflow_gemm_bf16: allocation of the error word failed");
        return DCFLOW_ERR_OOM;
      }
      cudaMemset(d_errs[dev], 0, sizeof(int));
    }
    d_err = d_errs[dev];
  }
  if (!A || !B || !D) {
    set_error("dcflow_gemm_bf16: null operand");
    return DCFLOW_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  GemmSpec s;
  s.A = A; s.lda = lda; s.B = B; s.ldb = ldb; s.M = M; s.N = N; s.K = K;
  s.bias = bias; s.relu = relu != 0; s.D = D; s.ldd = ldd; s.out_bf16 = out_bf16 != 0;
  int rc = gemm_run(s, d_err, st);
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

extern "C" int dcflow_screen_create(dcflow_ctx* ctx, int32_t max_rows, uint64_t seed, dcflow_screen** out) {
  if (!ctx || !out) {
    set_error("dcflow_screen_create: null argument");
    return DCFLOW_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (!ctx->has_study) {
    set_error("dcflow_screen_create: no study bound (dcflow_set_study)");
    return DCFLOW_ERR_NO_STUDY;
  }
  if (max_rows < 128 || max_rows % 128 || max_rows > (1 << 20)) {
    set_error("dcflow_screen_create: max_rows must be a multiple of 128 in [128, 2^20]");
    return DCFLOW_ERR_INVALID_ARG;
  }
  if (ctx->C < 1 || ctx->C > 2048) {
    set_error("dcflow_screen_create: the study needs 1 to 2048 contingencies");
    return DCFLOW_ERR_INVALID_ARG;
  }
  DCF_CUDA(cudaSetDevice(ctx->dev));
  auto* s = new dcflow_screen();
  s->ctx = ctx;
  s->dev = ctx->dev;
  s->V = ctx->V;
  s->M = ctx->M;
  s->C = ctx->C;
  s->Cp = (int)round_up(ctx->C, 128);
  s->max_rows = max_rows;
  std::vector<int> foff(ctx->V, -1);
  int nbits = 0;
  for (int v = 0; v < ctx->V; ++v)
    if (ctx->h_split_ok[v]) {
      foff[v] = ctx->M + nbits;
      nbits += ctx->h_inc_ptr[v + 1] - ctx->h_inc_ptr[v];
    }
  s->F = ctx->M + nbits;
  s->Fp = (int)round_up(s->F, 128);
  auto fail = [&](int rc) {
    dcflow_screen_destroy(s);
    return rc;
  };
  const int H = s->H, Fp = s->Fp, Cp = s->Cp, B = max_rows;
  const size_t bf = 2;
  if (s->foff.ensure(sizeof(int) * ctx->V) || s->err.ensure(sizeof(int))) return fail(DCFLOW_ERR_OOM);
  for (int k = 0; k < kNumScreenTensors; ++k) {
    const size_t n = (size_t)s->rows(k) * s->cols(k) * sizeof(float);
    if (s->prm[k].ensure(n) || s->grd[k].ensure(n) || s->mom[k].ensure(n) || s->vel[k].ensure(n))
      return fail(DCFLOW_ERR_OOM);
  }
  for (int w = 0; w < 3; ++w) {
    const size_t n = (size_t)s->rows(2 * w) * s->cols(2 * w) * bf;
    if (s->wb[w].ensure(n) || (w && s->wt[w].ensure(n))) return fail(DCFLOW_ERR_OOM);
  }
  size_t part = std::max<size_t>((size_t)16 * Cp * H, (size_t)16 * H * Fp) * sizeof(float);
  if (s->Xb.ensure((size_t)B * Fp * bf) || s->Xt.ensure((size_t)B * Fp * bf) || s->Yb.ensure((size_t)B * Cp) ||
      s->H1.ensure((size_t)B * H * bf) || s->H1t.ensure((size_t)B * H * bf) || s->H2.ensure((size_t)B * H * bf) ||
      s->H2t.ensure((size_t)B * H * bf) || s->Z.ensure((size_t)B * Cp * 4) || s->dZ.ensure((size_t)B * Cp * bf) ||
      s->dZt.ensure((size_t)B * Cp * bf) || s->dH2.ensure((size_t)B * H * bf) || s->dH2t.ensure((size_t)B * H * bf) ||
      s->dH1t.ensure((size_t)B * H * bf) || s->part.ensure(part))
    return fail(DCFLOW_ERR_OOM);
  // He-normal weights (std sqrt(2 / fan_in)) on the logical part, zero padding;
  // b3 starts at the log-odds of 64 positives in C
  std::vector<float> h;
  for (int k = 0; k < kNumScreenTensors; ++k) {
    const int R = s->rows(k), Cc = s->cols(k), lr = s->logical_rows(k), lc = s->logical_cols(k);
    h.assign((size_t)R * Cc, 0.f);
    if (k % 2 == 0) {
      const double sd = std::sqrt(2.0 / lc);
      for (int r = 0; r < lr; ++r)
        for (int c = 0; c < lc; ++c) h[(size_t)r * Cc + c] = (float)(sd * normal_at(seed, k, (uint64_t)r * lc + c));
    } else if (k == kB3) {
      const double prior = std::min(0.5, 64.0 / s->C);
      for (int r = 0; r < lr; ++r) h[r] = (float)std::log(prior / (1.0 - prior));
    }
    if (cudaMemcpy(s->prm[k].p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(s->grd[k].p, 0, h.size() * sizeof(float)) != cudaSuccess ||
        cudaMemset(s->mom[k].p, 0, h.size() * sizeof(float)) != cudaSuccess ||
        cudaMemset(s->vel[k].p, 0, h.size() * sizeof(float)) != cudaSuccess) {
      set_error("dcflow_screen_create: parameter upload failed");
      return fail(DCFLOW_ERR_CUDA);
    }
  }
  if (cudaMemcpy(s->foff.p, foff.data(), sizeof(int) * ctx->V, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->err.p, 0, sizeof(int)) != cudaSuccess) {
    set_error("dcflow_screen_create: upload failed");
    return fail(DCFLOW_ERR_CUDA);
  }
  for (int k = 0; k < kNumScreenTensors; k += 2) {
    int rc = refresh_bf16(s, k, 0);
    if (rc) return fail(rc);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error("dcflow_screen_create: initialisation failed");
    return fail(DCFLOW_ERR_CUDA);
  }
  *out = s;
  return DCFLOW_OK;
}

extern "C" void dcflow_screen_destroy(dcflow_screen* s) {
  if (!s) return;
  DevBuf* b[] = {&s->foff, &s->Xb, &s->Xt, &s->Yb, &s->H1, &s->H1t, &s->H2, &s->H2t, &s->Z, &s->dZ, &s->dZt,
                 &s->dH2, &s->dH2t, &s->dH1t, &s->part, &s->err, &s->iX, &s->iH1, &s->iH2, &s->iZ};
  for (auto* x : b) x->release();
  for (int k = 0; k < kNumScreenTensors; ++k) {
    s->prm[k].release();
    s->grd[k].release();
    s->mom[k].release();
    s->vel[k].release();
  }
  for (int w = 0; w < 3; ++w) {
    s->wb[w].release();
    s->wt[w].release();
  }
  delete s;
}

extern "C" int dcflow_screen_dims(const dcflow_screen* s, int32_t* F, int32_t* F_pad, int32_t* H, int32_t* C,
                                  int32_t* C_pad) {
  if (!s) return DCFLOW_ERR_INVALID_ARG;
  if (F) *F = s->F;
  if (F_pad) *F_pad = s->Fp;
  if (H) *H = s->H;
  if (C) *C = s->C;
  if (C_pad) *C_pad = s->Cp;
  return DCFLOW_OK;
}

static int check_rows(const dcflow_screen* s, const void* X, int64_t ldx, const int32_t* rows, int32_t n,
                      const char* who) {
  if (!X || n < 1 || n > s->max_rows || ldx < s->Fp || ldx % 8) {
    set_error(std::string(who) + ": need X, 1 <= n <= max_rows and ldx >= F_pad, ldx % 8 == 0");
    return DCFLOW_ERR_INVALID_ARG;
  }
  (void)rows;
  return 0;
}

extern "C" int dcflow_screen_backward(dcflow_screen* s, const void* X, int64_t ldx, const uint8_t* Y, int64_t ldy,
                                      const int32_t* rows, int32_t n, float* loss, void* stream) {
  if (!s) return DCFLOW_ERR_INVALID_ARG;
  int rc = check_rows(s, X, ldx, rows, n, "dcflow_screen_backward");
  if (rc) return rc;
  if (!Y || ldy < s->Cp || !loss) {
    set_error("dcflow_screen_backward: need Y with ldy >= C_pad and a loss word");
    return DCFLOW_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = screen_pass(s, X, ldx, Y, ldy, rows, n, true, loss, st))) return rc;
  return check_err(s, st);
}

extern "C" int dcflow_screen_adam(dcflow_screen* s, float lr, void* stream) {
  if (!s || !(lr >= 0.f)) return DCFLOW_ERR_INVALID_ARG;
  return screen_adam(s, lr, (cudaStream_t)stream);
}

extern "C" int dcflow_screen_train_step(dcflow_screen* s, const void* X, int64_t ldx, const uint8_t* Y, int64_t ldy,
                                        const int32_t* rows, int32_t n, float lr, float* loss, void* stream) {
  if (!s) return DCFLOW_ERR_INVALID_ARG;
  int rc = check_rows(s, X, ldx, rows, n, "dcflow_screen_train_step");
  if (rc) return rc;
  if (!Y || ldy < s->Cp || !loss || !(lr >= 0.f)) {
    set_error("dcflow_screen_train_step: need Y with ldy >= C_pad, a loss word and lr >= 0");
    return DCFLOW_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = screen_pass(s, X, ldx, Y, ldy, rows, n, true, loss, st))) return rc;
  return screen_adam(s, lr, st);
}

extern "C" int dcflow_screen_check(dcflow_screen* s, void* stream) {
  if (!s) return DCFLOW_ERR_INVALID_ARG;
  return check_err(s, (cudaStream_t)stream);
}

__global__ void k_copy_logits(const float* __restrict__ Z, int ldz, int n, int C, float* __restrict__ out,
                              int64_t ldo) {
  const int r = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x)
    if (r < n) out[r * ldo + c] = Z[(size_t)r * ldz + c];
}

extern "C" int dcflow_screen_logits(dcflow_screen* s, const void* X, int64_t ldx, int64_t n_rows, float* Z,
                                    int64_t ldz, void* stream) {
  if (!s) return DCFLOW_ERR_INVALID_ARG;
  if (!X || !Z || n_rows < 0 || ldx < s->Fp || ldx % 8 || ldz < s->C) {
    set_error("dcflow_screen_logits: need X (ldx >= F_pad, ldx % 8 == 0) and Z (ldz >= C)");
    return DCFLOW_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const auto* Xb = static_cast<const __nv_bfloat16*>(X);
  for (int64_t r0 = 0; r0 < n_rows; r0 += s->max_rows) {
    const int n = (int)std::min<int64_t>(s->max_rows, n_rows - r0);
    int rc = screen_pass(s, Xb + r0 * ldx, ldx, nullptr, 0, nullptr, n, false, nullptr, st);
    if (rc) return rc;
    k_copy_logits<<<dim3((s->C + 255) / 256, n), 256, 0, st>>>(s->Z.as<float>(), s->Cp, n, s->C, Z + r0 * ldz, ldz);
    DCF_CHECK_LAUNCH();
  }
  return check_err(s, st);
}

extern "C" int dcflow_screen_labels(dcflow_screen* s, const float* cont_max, int64_t n_rows, int32_t k, uint8_t* Y,
                                    int64_t ldy, void* stream) {
  if (!s || !cont_max || !Y || n_rows < 0 || k < 1 || ldy < s->C) {
    set_error("dcflow_screen_labels: need cont_max, Y (ldy >= C), k >= 1");
    return DCFLOW_ERR_INVALID_ARG;
  }
  if (n_rows == 0) return DCFLOW_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int C = s->C;
  const unsigned grid = (unsigned)((n_rows * 32 + 255) / 256);
  if (C <= 256) k_labels<8><<<grid, 256, 0, st>>>(cont_max, n_rows, C, k, Y, ldy);
  else if (C <= 512) k_labels<16><<<grid, 256, 0, st>>>(cont_max, n_rows, C, k, Y, ldy);
  else if (C <= 1024) k_labels<32><<<grid, 256, 0, st>>>(cont_max, n_rows, C, k, Y, ldy);
  else k_labels<64><<<grid, 256, 0, st>>>(cont_max, n_rows, C, k, Y, ldy);
  DCF_CHECK_LAUNCH();
  return DCFLOW_OK;
}

extern "C" int dcflow_screen_get(const dcflow_screen* s, int32_t tensor, int32_t kind, float* host) {
  if (!s || tensor < 0 || tensor >= kNumScreenTensors || kind < 0 || kind > 3 || !host) {
    set_error("dcflow_screen_get: tensor in [0, 6), kind in [0, 4), host buffer");
    return DCFLOW_ERR_INVALID_ARG;
  }
  const DevBuf* src[] = {&s->prm[tensor], &s->grd[tensor], &s->mom[tensor], &s->vel[tensor]};
  const int R = s->logical_rows(tensor), Cl = s->logical_cols(tensor), ld = s->cols(tensor);
  DCF_CUDA(cudaSetDevice(s->dev));
  DCF_CUDA(cudaDeviceSynchronize());
  DCF_CUDA(cudaMemcpy2D(host, sizeof(float) * Cl, src[kind]->p, sizeof(float) * ld, sizeof(float) * Cl, R,
                        cudaMemcpyDeviceToHost));
  return DCFLOW_OK;
}

extern "C" int dcflow_screen_set(dcflow_screen* s, int32_t tensor, int32_t kind, const float* host) {
  if (!s || tensor < 0 || tensor >= kNumScreenTensors || kind < 0 || kind > 3 || !host) {
    set_error("dcflow_screen_set: tensor in [0, 6), kind in [0, 4), host buffer");
    return DCFLOW_ERR_INVALID_ARG;
  }
  DevBuf* dst[] = {&s->prm[tensor], &s->grd[tensor], &s->mom[tensor], &s->vel[tensor]};
  const int R = s->logical_rows(tensor), Cl = s->logical_cols(tensor), ld = s->cols(tensor);
  DCF_CUDA(cudaSetDevice(s->dev));
  DCF_CUDA(cudaDeviceSynchronize());
  DCF_CUDA(cudaMemcpy2D(dst[kind]->p, sizeof(float) * ld, host, sizeof(float) * Cl, sizeof(float) * Cl, R,
                        cudaMemcpyHostToDevice));
  if (kind == 0) {
    int rc = refresh_bf16(s, tensor, 0);
    if (rc) return rc;
    DCF_CUDA(cudaDeviceSynchronize());
  }
  return DCFLOW_OK;
}

extern "C" int dcflow_screen_adam_step(dcflow_screen* s, int64_t* t, int32_t set) {
  if (!s || !t) return DCFLOW_ERR_INVALID_ARG;
  if (set) {
    if (*t < 0) return DCFLOW_ERR_INVALID_ARG;
    s->t = *t;
  } else {
    *t = s->t;
  }
  return DCFLOW_OK;
}
