// Context lifetime, error strings and device-buffer helpers of the C ABI.
#include <string>

#include "internal.cuh"

namespace dcf {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int DevBuf::ensure(size_t need) {
  if (need <= bytes && p) return 0;
  release();
  if (need == 0) need = 1;
  if (cudaMalloc(&p, need) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    bytes = 0;
    set_error("device allocation of " + std::to_string(need) + " bytes failed");
    return DCFLOW_ERR_OOM;
  }
  bytes = need;
  return 0;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

}  // namespace dcf

extern "C" void dcflow_destroy(dcflow_ctx* ctx) {
  if (!ctx) return;
  dcf::DevBuf* bufs[] = {&ctx->f, &ctx->t, &ctx->b, &ctx->inc_ptr, &ctx->inc_list, &ctx->rid, &ctx->L, &ctx->info,
                         &ctx->nidx, &ctx->split_ok, &ctx->out_ok, &ctx->monN, &ctx->contN, &ctx->cpos_of_mon, &ctx->mpos_of_cont,
                         &ctx->inv_lim, &ctx->bN, &ctx->PhiN, &ctx->PhiNf, &ctx->bNf, &ctx->p0f, &ctx->PtdfN, &ctx->PhiMC, &ctx->Y, &ctx->p0, &ctx->dp,
                         &ctx->rank, &ctx->status, &ctx->perm, &ctx->hist, &ctx->hist_host, &ctx->err, &ctx->pool, &ctx->var_k, &ctx->PhiCM, &ctx->cont_pos, &ctx->cont_inv,
                         &ctx->cm_scratch, &ctx->of_cmax, &ctx->of_top, &ctx->gen_cols,
                         &ctx->multi_ptr, &ctx->multiN, &ctx->multi_mpos, &ctx->PhiMO};
  for (auto* b : bufs) b->release();
  ctx->bufs[0].release_all();
  ctx->bufs[1].release_all();
  cudaEvent_t evs[] = {ctx->ev_ready, ctx->ev_prep[0], ctx->ev_prep[1], ctx->ev_free[0], ctx->ev_free[1]};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  delete ctx;
}

extern "C" int64_t dcflow_last_launch_count(const dcflow_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" const char* dcflow_strerror(int code) {
  switch (code) {
    case DCFLOW_OK: return "ok";
    case DCFLOW_ERR_INVALID_ARG: return "invalid argument";
    case DCFLOW_ERR_GRID_DISCONNECTED: return "base grid is not connected";
    case DCFLOW_ERR_OOM: return "device memory exhausted";
    case DCFLOW_ERR_CUDA: return "CUDA error";
    case DCFLOW_ERR_TIMEOUT: return "bounded device wait expired";
    case DCFLOW_ERR_NO_STUDY: return "no study bound to the context";
    case DCFLOW_ERR_SINGULAR: return "base susceptance matrix is not positive definite";
    default: return "unknown error";
  }
}

extern "C" const char* dcflow_last_error(void) { return dcf::g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// failure-path self-test: one block waits on an mbarrier that nothing ever
// completes, with the bounded wait of the N-1 kernels; when the budget runs
// out it records the expiry in an error word and returns.  The host reads the
// word: DCFLOW_ERR_TIMEOUT, and the context stays usable.
// ---------------------------------------------------------------------------
#include "args.cuh"
#include "n1_tma.cuh"

namespace dcf {
__global__ void k_wait_selftest(int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);  // one arrival expected; none ever comes
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool got = mbar_wait(smem_u32(&bar), 0);
  if (__syncthreads_or(!got) && threadIdx.x == 0) atomicExch(err, 1);
}
}  // namespace dcf

extern "C" int dcflow_selftest_bounded_wait(dcflow_ctx* ctx, void* stream) {
  if (!ctx) return DCFLOW_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  dcf::DevBuf e;
  if (e.ensure(sizeof(int))) return DCFLOW_ERR_OOM;
  int h = 0;
  cudaError_t rc = cudaMemsetAsync(e.p, 0, sizeof(int), st);
  if (rc == cudaSuccess) {
    dcf::k_wait_selftest<<<1, 32, 0, st>>>(e.as<int>());
    rc = cudaGetLastError();
  }
  if (rc == cudaSuccess) rc = cudaMemcpyAsync(&h, e.p, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (rc == cudaSuccess) rc = cudaStreamSynchronize(st);
  e.release();
  if (rc != cudaSuccess) {
    dcf::set_error(std::string("dcflow_selftest_bounded_wait: ") + cudaGetErrorString(rc));
    return DCFLOW_ERR_CUDA;
  }
  if (h) {
    dcf::set_error("dcflow_selftest_bounded_wait: the bounded wait expired as designed");
    return DCFLOW_ERR_TIMEOUT;
  }
  return DCFLOW_OK;
}
