// dcflow_base_ptdf_noalloc: base PTDF rows without any device allocation.
//
// Some callers cannot allocate device memory: code that runs inside a
// memory-pool or arena it does not own, tight real-time loops that must not
// hit the driver allocator, or hosts whose allocator is owned by another
// framework.  This entry point serves them: it computes the same rows as
// dcflow_base_ptdf, but its solve workspace and its copy of the row list live
// in one file-scope device array of fixed size (kScratchBytes), so the call
// never allocates.  The caller passes the row list (host) and the output
// (device) exactly as for dcflow_base_ptdf.
//
// The array is part of the loaded library: every GPU that loads it holds the
// array until the process exits.  All calls share it and it keeps the last
// call's contents, so the parts that must start at zero are cleared on every
// call, and two calls that overlap on the GPU (different streams, or another
// host thread) race on it: serialise them.
#include <mutex>

#include "dense64.cuh"
#include "internal.cuh"

namespace dcf {

constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB: rows list + npad x round_up(rows, 64) doubles

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// RHS column i = C'[branch_i, :]^T (+1 at the from bus, -1 at the to bus, slack dropped).
__global__ void k_noalloc_rhs(int nr, const int* rows, const int* f, const int* t, const int* rid, double* R,
                              int ldr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  int l = rows[i];
  int a = rid[f[l]], c = rid[t[l]];
  if (a >= 0) R[(size_t)a * ldr + i] += 1.0;
  if (c >= 0) R[(size_t)c * ldr + i] -= 1.0;
}

// out[i][n] = b_{rows_i} Y[rid(n)][i] (0 at the slack).
__global__ void k_noalloc_rows(int nr, int V, const int* rows, const double* b, const int* rid, const double* Y,
                               int ldy, double* out) {
  __shared__ double tile[32][33];
  const int n0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int n = n0 + k, i = i0 + threadIdx.x;
    double v = 0.0;
    if (n < V && i < nr) {
      int rr = rid[n];
      v = rr >= 0 ? Y[(size_t)rr * ldy + i] : 0.0;
    }
    tile[k][threadIdx.x] = v;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int i = i0 + k, n = n0 + threadIdx.x;
    if (i < nr && n < V) out[(size_t)i * V + n] = b[rows[i]] * tile[threadIdx.x][k];
  }
}

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (the entry point switches to its context's device
// before asking).
static std::mutex g_mu;
static void* g_addr[128];
static bool g_have[128];

static int scratch_address(void** out) {
  int dev = 0;
  DCF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) {
    set_error("dcflow_base_ptdf_noalloc: device ordinal out of range");
    return DCFLOW_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_have[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error(std::string("dcflow_base_ptdf_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return DCFLOW_ERR_CUDA;
    }
    g_addr[dev] = p;
    g_have[dev] = true;
  }
  *out = g_addr[dev];
  return 0;
}

}  // namespace dcf

using namespace dcf;

// Bytes of the fixed array one call needs: the row list (rounded to 256 B) and
// the (n_bus - 1, padded to 64) x (n_rows, padded to 64) FP64 solve workspace.
static size_t noalloc_bytes(const dcflow_ctx* ctx, int32_t n_rows) {
  const size_t rows_bytes = round_up((int64_t)n_rows * (int64_t)sizeof(int), 256);
  const size_t y_bytes = (size_t)ctx->npad * (size_t)round_up(n_rows, 64) * sizeof(double);
  return rows_bytes + y_bytes;
}

extern "C" int dcflow_base_ptdf_noalloc(dcflow_ctx* ctx, const int32_t* rows, int32_t n_rows, double* out,
                                        void* stream) {
  if (!ctx || n_rows < 0 || (n_rows > 0 && (!rows || !out))) {
    set_error("dcflow_base_ptdf_noalloc: invalid arguments");
    return DCFLOW_ERR_INVALID_ARG;
  }
  if (n_rows == 0) return DCFLOW_OK;
  for (int i = 0; i < n_rows; ++i)
    if (rows[i] < 0 || rows[i] >= ctx->E) {
      set_error("dcflow_base_ptdf_noalloc: row out of range");
      return DCFLOW_ERR_INVALID_ARG;
    }
  const size_t need = noalloc_bytes(ctx, n_rows);
  if (need > kScratchBytes) {
    set_error("dcflow_base_ptdf_noalloc: needs " + std::to_string(need) + " bytes of scratch, the fixed array holds " +
              std::to_string(kScratchBytes) + " (fewer rows per call, or dcflow_base_ptdf)");
    return DCFLOW_ERR_INVALID_ARG;
  }
  // the context's device, whichever device the caller has current (restored on return)
  DeviceGuard dg(ctx->dev);
  if (dg.err != cudaSuccess) {
    set_error(std::string("dcflow_base_ptdf_noalloc: cudaSetDevice: ") + cudaGetErrorString(dg.err));
    return DCFLOW_ERR_CUDA;
  }
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* p = static_cast<unsigned char*>(base);
  int* d_rows = reinterpret_cast<int*>(p);
  double* Y = reinterpret_cast<double*>(p + round_up((int64_t)n_rows * (int64_t)sizeof(int), 256));
  const int ldy = (int)round_up(n_rows, 64);
  DCF_CUDA(cudaMemcpyAsync(d_rows, rows, sizeof(int) * (size_t)n_rows, cudaMemcpyHostToDevice, st));
  // the right-hand sides are accumulated into the workspace: clear it every call
  DCF_CUDA(cudaMemsetAsync(Y, 0, (size_t)ctx->npad * ldy * sizeof(double), st));
  k_noalloc_rhs<<<(n_rows + 127) / 128, 128, 0, st>>>(n_rows, d_rows, ctx->f.as<int>(), ctx->t.as<int>(),
                                                        ctx->rid.as<int>(), Y, ldy);
  DCF_CHECK_LAUNCH();
  int64_t launches = 1;
  rc = chol_solve(ctx->L.as<double>(), ctx->npad, Y, ldy, ldy, st, &launches);
  if (rc) return rc;
  dim3 grid((ctx->V + 31) / 32, (n_rows + 31) / 32);
  k_noalloc_rows<<<grid, dim3(32, 8), 0, st>>>(n_rows, ctx->V, d_rows, ctx->b.as<double>(), ctx->rid.as<int>(), Y,
                                              ldy, out);
  DCF_CHECK_LAUNCH();
  return DCFLOW_OK;
}
