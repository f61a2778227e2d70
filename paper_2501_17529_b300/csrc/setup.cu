// Grid setup and study tables.
//
// dcflow_setup   : validate the grid, build B' (Sec. II, Def. 1, slack row and
//                  column removed) and factor it once in FP64.
// dcflow_set_study: restrict the PTDF to the needed branches N (monitored,
//                  contingency, switchable and outage-candidate branches; the
//                  row restriction of Sec. II) with one multi-RHS solve
//                  Y = B'^{-1} C_N'^T, then
//                    Phi[l, c]  = b_l (Y[f_l, c] - Y[t_l, c])   (l, c in N)
//                    PTDF[l, n] = b_l Y[n, l]                   (l in N)
//                  Phi[l, c] = PTDF[l, f_c] - PTDF[l, t_c] is the numerator of
//                  the LODF (Def. 3) and the operand of every topology update.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "dense64.cuh"
#include "internal.cuh"

namespace dcf {

// Row i of B' (one thread per non-slack bus): diagonal sum of incident b,
// off-diagonal -b per branch (parallel branches add up), in incident order.
__global__ void k_build_lap(int V, const int* inc_ptr, const int* inc_list, const int* f, const int* t,
                            const double* b, const int* rid, int npad, double* A) {
  int bus = blockIdx.x * blockDim.x + threadIdx.x;
  if (bus >= V) return;
  int i = rid[bus];
  if (i < 0) return;
  double* row = A + (size_t)i * npad;
  for (int k = inc_ptr[bus]; k < inc_ptr[bus + 1]; ++k) {
    int l = inc_list[k];
    int other = (f[l] == bus) ? t[l] : f[l];
    row[i] += b[l];
    int j = rid[other];
    if (j >= 0) row[j] -= b[l];
  }
}

__global__ void k_pad_identity(int n, int npad, double* A) {
  int i = n + blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npad) A[(size_t)i * npad + i] = 1.0;
}

// RHS column i = C'[branch_i, :]^T: +1 at the from bus, -1 at the to bus (slack dropped).
__global__ void k_branch_rhs(int nb, const int* branches, const int* f, const int* t, const int* rid,
                             double* R, int ldr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int l = branches[i];
  int a = rid[f[l]], c = rid[t[l]];
  if (a >= 0) R[(size_t)a * ldr + i] += 1.0;
  if (c >= 0) R[(size_t)c * ldr + i] -= 1.0;
}

// Phi[i][j] = b_{N_i} (Y[f_{N_i}][j] - Y[t_{N_i}][j]) for i, j < nn.
__global__ void k_phi_rows(int nn, const int* N, const int* f, const int* t, const double* b, const int* rid,
                           const double* Y, int ldy, double* Phi) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (j >= nn) return;
  int l = N[i];
  int a = rid[f[l]], c = rid[t[l]];
  double ya = a >= 0 ? Y[(size_t)a * ldy + j] : 0.0;
  double yc = c >= 0 ? Y[(size_t)c * ldy + j] : 0.0;
  Phi[(size_t)i * nn + j] = b[l] * (ya - yc);
}

// out[i][n] = b_{rows_i} Y[rid(n)][i] (0 at the slack): tiled transpose with scaling.
__global__ void k_ptdf_rows(int nr, int V, const int* rows, const double* b, const int* rid, const double* Y,
                            int ldy, double* out) {
  __shared__ double tile[32][33];
  const int n0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  // load: threads walk i (contiguous in Y) for a fixed bus n
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

// PhiMC[l][c] = Phi[monN_l][contN_c] / limit_l in the working precision (row stride ldc >= C).
template <class Real>
__global__ void k_phi_mc(int M, int C, int ldc, int nn, const int* monN, const int* contN, const double* inv_lim,
                         const double* Phi, Real* out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int l = blockIdx.y;
  if (c >= ldc) return;
  out[(size_t)l * ldc + c] = (c < C) ? (Real)(Phi[(size_t)monN[l] * nn + contN[c]] * inv_lim[l]) : (Real)0;
}

}  // namespace dcf

using namespace dcf;

static int upload(DevBuf& d, const void* h, size_t bytes) {
  if (d.ensure(bytes ? bytes : 1)) return DCFLOW_ERR_OOM;
  if (bytes) DCF_CUDA(cudaMemcpy(d.p, h, bytes, cudaMemcpyHostToDevice));
  return 0;
}

// Solve Y = B'^{-1} C'_{rows}^T for the given branches into ctx->Y (npad x round_up(nr, 64)).
static int solve_branch_columns(dcflow_ctx* ctx, const int* d_rows, int nr, int* ldy_out, cudaStream_t st) {
  const int ldy = (int)round_up(std::max(nr, 1), 64);
  if (ctx->Y.ensure((size_t)ctx->npad * ldy * sizeof(double))) return DCFLOW_ERR_OOM;
  DCF_CUDA(cudaMemsetAsync(ctx->Y.p, 0, (size_t)ctx->npad * ldy * sizeof(double), st));
  k_branch_rhs<<<(nr + 127) / 128, 128, 0, st>>>(nr, d_rows, ctx->f.as<int>(), ctx->t.as<int>(),
                                                   ctx->rid.as<int>(), ctx->Y.as<double>(), ldy);
  ++ctx->launches;
  DCF_CHECK_LAUNCH();
  int rc = chol_solve(ctx->L.as<double>(), ctx->npad, ctx->Y.as<double>(), ldy, ldy, st, &ctx->launches);
  if (rc) return rc;
  *ldy_out = ldy;
  return 0;
}

extern "C" void dcflow_default_options(dcflow_options* opt) {
  if (!opt) return;
  opt->precision = DCFLOW_FP32;
  opt->device = -1;
  opt->chunk_topo = 0;
  opt->island_tol = 1e-9;
  opt->compact_n1 = 0;
  opt->autotune = 0;
  opt->autotune_sample = 0;
  opt->tie_band = 0.0;
  opt->output_first = 0;
}

extern "C" int dcflow_setup(dcflow_ctx** out, int32_t n_bus, int32_t n_branch, const int32_t* from,
                            const int32_t* to, const double* b, int32_t slack, const dcflow_options* opt) {
  if (!out || !from || !to || !b || n_bus < 2 || n_branch < 1 || slack < 0 || slack >= n_bus) {
    set_error("dcflow_setup: invalid sizes, pointers or slack");
    return DCFLOW_ERR_INVALID_ARG;
  }
  *out = nullptr;
  dcflow_options o;
  dcflow_default_options(&o);
  if (opt) o = *opt;
  if (o.island_tol <= 0) o.island_tol = 1e-9;
  if (o.autotune_sample <= 0) o.autotune_sample = 2048;
  if (o.precision != DCFLOW_FP64 && o.precision != DCFLOW_FP32 && o.precision != DCFLOW_BF16X3) {
    set_error("dcflow_setup: unknown precision");
    return DCFLOW_ERR_INVALID_ARG;
  }
  for (int l = 0; l < n_branch; ++l) {
    if (from[l] < 0 || from[l] >= n_bus || to[l] < 0 || to[l] >= n_bus || from[l] == to[l] ||
        !(b[l] > 0.0) || !std::isfinite(b[l])) {
      set_error("dcflow_setup: branch " + std::to_string(l) + " has a bad endpoint or susceptance");
      return DCFLOW_ERR_INVALID_ARG;
    }
  }
  // connectivity (union-find on the host)
  {
    std::vector<int> par(n_bus);
    std::iota(par.begin(), par.end(), 0);
    auto find = [&](int x) {
      while (par[x] != x) x = par[x] = par[par[x]];
      return x;
    };
    int comps = n_bus;
    for (int l = 0; l < n_branch; ++l) {
      int a = find(from[l]), c = find(to[l]);
      if (a != c) {
        par[a] = c;
        --comps;
      }
    }
    if (comps != 1) {
      set_error("dcflow_setup: the base grid is not connected");
      return DCFLOW_ERR_GRID_DISCONNECTED;
    }
  }
  dcflow_ctx* ctx = new dcflow_ctx();
  ctx->opt = o;
  auto fail = [&](int rc) {
    dcflow_destroy(ctx);
    return rc;
  };
  if (o.device >= 0) {
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) {
      set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
      return fail(DCFLOW_ERR_CUDA);
    }
  }
  cudaGetDevice(&ctx->dev);
  ctx->V = n_bus;
  ctx->E = n_branch;
  ctx->slack = slack;
  ctx->n = n_bus - 1;
  ctx->npad = (int)round_up(ctx->n, kNB);
  ctx->hf.assign(from, from + n_branch);
  ctx->ht.assign(to, to + n_branch);
  ctx->hb.assign(b, b + n_branch);
  // incident lists, ascending branch id (the split-mask bit order)
  std::vector<std::vector<int>> inc(n_bus);
  for (int l = 0; l < n_branch; ++l) {
    inc[from[l]].push_back(l);
    inc[to[l]].push_back(l);
  }
  ctx->h_inc_ptr.assign(n_bus + 1, 0);
  for (int v = 0; v < n_bus; ++v) ctx->h_inc_ptr[v + 1] = ctx->h_inc_ptr[v] + (int)inc[v].size();
  ctx->h_inc_list.reserve(2 * n_branch);
  for (int v = 0; v < n_bus; ++v) ctx->h_inc_list.insert(ctx->h_inc_list.end(), inc[v].begin(), inc[v].end());
  std::vector<int> rid(n_bus);
  for (int v = 0, k = 0; v < n_bus; ++v) rid[v] = (v == slack) ? -1 : k++;

  int rc;
  if ((rc = upload(ctx->f, from, sizeof(int) * n_branch))) return fail(rc);
  if ((rc = upload(ctx->t, to, sizeof(int) * n_branch))) return fail(rc);
  if ((rc = upload(ctx->b, b, sizeof(double) * n_branch))) return fail(rc);
  if ((rc = upload(ctx->inc_ptr, ctx->h_inc_ptr.data(), sizeof(int) * (n_bus + 1)))) return fail(rc);
  if ((rc = upload(ctx->inc_list, ctx->h_inc_list.data(), sizeof(int) * ctx->h_inc_list.size()))) return fail(rc);
  if ((rc = upload(ctx->rid, rid.data(), sizeof(int) * n_bus))) return fail(rc);
  const size_t abytes = (size_t)ctx->npad * ctx->npad * sizeof(double);
  if (ctx->L.ensure(abytes) || ctx->info.ensure(sizeof(int)) || ctx->err.ensure(sizeof(int))) return fail(DCFLOW_ERR_OOM);
  if (cudaMemset(ctx->err.p, 0, sizeof(int)) != cudaSuccess) {
    set_error("dcflow_setup: memset failed");
    return fail(DCFLOW_ERR_CUDA);
  }
  cudaStream_t st = 0;
  if (cudaMemsetAsync(ctx->L.p, 0, abytes, st) != cudaSuccess || cudaMemsetAsync(ctx->info.p, 0, sizeof(int), st) != cudaSuccess) {
    set_error("dcflow_setup: memset failed");
    return fail(DCFLOW_ERR_CUDA);
  }
  k_build_lap<<<(n_bus + 127) / 128, 128, 0, st>>>(n_bus, ctx->inc_ptr.as<int>(), ctx->inc_list.as<int>(),
                                                    ctx->f.as<int>(), ctx->t.as<int>(), ctx->b.as<double>(),
                                                    ctx->rid.as<int>(), ctx->npad, ctx->L.as<double>());
  if (ctx->npad > ctx->n) k_pad_identity<<<1, 64, 0, st>>>(ctx->n, ctx->npad, ctx->L.as<double>());
  if (cudaGetLastError() != cudaSuccess) {
    set_error("dcflow_setup: launch failed");
    return fail(DCFLOW_ERR_CUDA);
  }
  if ((rc = cholesky(ctx->L.as<double>(), ctx->npad, ctx->info.as<int>(), st, &ctx->launches))) return fail(rc);
  int info = 0;
  if (cudaMemcpy(&info, ctx->info.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    set_error("dcflow_setup: factorisation failed");
    return fail(DCFLOW_ERR_CUDA);
  }
  if (info != 0) {
    set_error("dcflow_setup: B' is not positive definite at row " + std::to_string(info - 1));
    return fail(DCFLOW_ERR_SINGULAR);
  }
  *out = ctx;
  return DCFLOW_OK;
}

extern "C" int dcflow_base_ptdf(dcflow_ctx* ctx, const int32_t* rows, int32_t n_rows, double* out, void* stream) {
  if (!ctx || (n_rows > 0 && (!rows || !out)) || n_rows < 0) {
    set_error("dcflow_base_ptdf: invalid arguments");
    return DCFLOW_ERR_INVALID_ARG;
  }
  if (n_rows == 0) return DCFLOW_OK;
  for (int i = 0; i < n_rows; ++i)
    if (rows[i] < 0 || rows[i] >= ctx->E) {
      set_error("dcflow_base_ptdf: row out of range");
      return DCFLOW_ERR_INVALID_ARG;
    }
  DeviceGuard dg(ctx->dev);  // the context's device for this call
  if (dg.err != cudaSuccess) {
    set_error(std::string("dcflow_base_ptdf: cudaSetDevice: ") + cudaGetErrorString(dg.err));
    return DCFLOW_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf d_rows;
  int rc = 0;
  if (d_rows.ensure(sizeof(int) * n_rows)) return DCFLOW_ERR_OOM;
  if (cudaMemcpyAsync(d_rows.p, rows, sizeof(int) * n_rows, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    d_rows.release();
    set_error("dcflow_base_ptdf: copy failed");
    return DCFLOW_ERR_CUDA;
  }
  int ldy = 0;
  rc = solve_branch_columns(ctx, d_rows.as<int>(), n_rows, &ldy, st);
  if (!rc) {
    dim3 grid((ctx->V + 31) / 32, (n_rows + 31) / 32);
    k_ptdf_rows<<<grid, dim3(32, 8), 0, st>>>(n_rows, ctx->V, d_rows.as<int>(), ctx->b.as<double>(),
                                             ctx->rid.as<int>(), ctx->Y.as<double>(), ldy, out);
    ++ctx->launches;
    if (cudaGetLastError() != cudaSuccess) rc = DCFLOW_ERR_CUDA;
  }
  cudaStreamSynchronize(st);  // d_rows is freed below
  d_rows.release();
  return rc;
}

// Phi[mon, o] / limit for every multi-outage entry o, transposed [entries][Mpad]
// (zero padding rows): a set's columns are contiguous over the monitored rows.
template <class Real>
__global__ void k_phi_multi(int M, int Mp, int NN, const int* __restrict__ monN, const int* __restrict__ multiN,
                            const double* __restrict__ inv_lim, const double* __restrict__ PhiN,
                            Real* __restrict__ PhiMO) {
  const int e = blockIdx.y, l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= Mp) return;
  PhiMO[(size_t)e * Mp + l] = l < M ? (Real)(PhiN[(size_t)monN[l] * NN + multiN[e]] * inv_lim[l]) : (Real)0;
}

// Bridges of the base multigraph (iterative Tarjan low-link over edge ids, so
// that a parallel branch is never a bridge).
static std::vector<char> base_bridges(int V, int E, const std::vector<int>& f, const std::vector<int>& t) {
  std::vector<std::vector<std::pair<int, int>>> adj(V);
  for (int l = 0; l < E; ++l) {
    adj[f[l]].push_back({t[l], l});
    adj[t[l]].push_back({f[l], l});
  }
  std::vector<int> disc(V, -1), low(V, 0), pedge(V, -1), it(V, 0);
  std::vector<char> br(E, 0);
  int timer = 0;
  for (int r = 0; r < V; ++r) {
    if (disc[r] >= 0) continue;
    std::vector<int> stack{r};
    disc[r] = low[r] = timer++;
    while (!stack.empty()) {
      const int u = stack.back();
      if (it[u] < (int)adj[u].size()) {
        const auto [w, l] = adj[u][it[u]++];
        if (l == pedge[u]) continue;
        if (disc[w] < 0) {
          pedge[w] = l;
          disc[w] = low[w] = timer++;
          stack.push_back(w);
        } else {
          low[u] = std::min(low[u], disc[w]);
        }
      } else {
        stack.pop_back();
        if (pedge[u] >= 0) {
          const int p = f[pedge[u]] == u ? t[pedge[u]] : f[pedge[u]];
          low[p] = std::min(low[p], low[u]);
          if (low[u] > disc[p]) br[pedge[u]] = 1;
        }
      }
    }
  }
  return br;
}

extern "C" int dcflow_set_study(dcflow_ctx* ctx, const dcflow_study* s) {
  if (!ctx || !s || s->n_mon < 1 || s->n_cont < 0 || !s->mon || (s->n_cont > 0 && !s->cont) || !s->limit) {
    set_error("dcflow_set_study: invalid arguments");
    return DCFLOW_ERR_INVALID_ARG;
  }
  DeviceGuard dg(ctx->dev);  // the context's device for this call
  if (dg.err != cudaSuccess) {
    set_error(std::string("dcflow_set_study: cudaSetDevice: ") + cudaGetErrorString(dg.err));
    return DCFLOW_ERR_CUDA;
  }
  const int E = ctx->E, V = ctx->V;
  std::vector<char> is_mon(E, 0), is_cont(E, 0), need(E, 0);
  for (int i = 0; i < s->n_mon; ++i) {
    int l = s->mon[i];
    if (l < 0 || l >= E || is_mon[l] || !(s->limit[l] > 0.0) || !std::isfinite(s->limit[l])) {
      set_error("dcflow_set_study: bad or duplicate monitored branch / limit");
      return DCFLOW_ERR_INVALID_ARG;
    }
    is_mon[l] = 1;
    need[l] = 1;
  }
  for (int i = 0; i < s->n_cont; ++i) {
    int l = s->cont[i];
    if (l < 0 || l >= E || is_cont[l]) {
      set_error("dcflow_set_study: bad or duplicate contingency branch");
      return DCFLOW_ERR_INVALID_ARG;
    }
    is_cont[l] = 1;
    need[l] = 1;
  }
  std::vector<uint8_t> split_ok(V, 0);
  if (s->split_bus) {
    for (int i = 0; i < s->n_split_bus; ++i) {
      int v = s->split_bus[i];
      if (v < 0 || v >= V) {
        set_error("dcflow_set_study: split bus out of range");
        return DCFLOW_ERR_INVALID_ARG;
      }
      split_ok[v] = 1;
    }
  } else {
    std::fill(split_ok.begin(), split_ok.end(), 1);
  }
  for (int v = 0; v < V; ++v)
    if (split_ok[v])
      for (int k = ctx->h_inc_ptr[v]; k < ctx->h_inc_ptr[v + 1]; ++k) need[ctx->h_inc_list[k]] = 1;
  std::vector<uint8_t> out_ok(E, 0);  // branches a batch may take out
  if (s->outage_cand) {
    for (int i = 0; i < s->n_outage_cand; ++i) {
      int l = s->outage_cand[i];
      if (l < 0 || l >= E) {
        set_error("dcflow_set_study: outage candidate out of range");
        return DCFLOW_ERR_INVALID_ARG;
      }
      need[l] = 1;
      out_ok[l] = 1;
    }
  } else {
    std::fill(need.begin(), need.end(), 1);
    std::fill(out_ok.begin(), out_ok.end(), 1);
  }
  const int n_multi = s->n_multi > 0 ? s->n_multi : 0;
  std::vector<int> mptr(1, 0), mbr;
  if (n_multi > 0) {  // multi-outage sets: 1 to 4 distinct branches each
    if (!s->multi_ptr || !s->multi_branch || s->multi_ptr[0] != 0 || n_multi > kMaxMultiSets) {
      set_error("dcflow_set_study: multi-outage sets need multi_ptr (from 0) and multi_branch, at most 262,140 sets");
      return DCFLOW_ERR_INVALID_ARG;
    }
    for (int m = 0; m < n_multi; ++m) {
      const int a0 = s->multi_ptr[m], a1 = s->multi_ptr[m + 1];
      if (a1 - a0 < 1 || a1 - a0 > 4) {
        set_error("dcflow_set_study: a multi-outage set has 1 to 4 branches");
        return DCFLOW_ERR_INVALID_ARG;
      }
      for (int k = a0; k < a1; ++k) {
        const int l = s->multi_branch[k];
        if (l < 0 || l >= E) {
          set_error("dcflow_set_study: multi-outage branch out of range");
          return DCFLOW_ERR_INVALID_ARG;
        }
        for (int k2 = a0; k2 < k; ++k2)
          if (s->multi_branch[k2] == l) {
            set_error("dcflow_set_study: a multi-outage set repeats a branch");
            return DCFLOW_ERR_INVALID_ARG;
          }
        need[l] = 1;
        mbr.push_back(l);
      }
      mptr.push_back((int)mbr.size());
    }
  }
  ctx->has_study = false;
  ctx->M = s->n_mon;
  ctx->C = s->n_cont;
  ctx->h_mon.assign(s->mon, s->mon + s->n_mon);
  {  // internal order: base-grid bridges last (they island every topology)
    const std::vector<char> br = base_bridges(V, E, ctx->hf, ctx->ht);
    ctx->h_cont.clear();
    ctx->h_cont_pos.clear();
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i < s->n_cont; ++i)
        if ((br[s->cont[i]] != 0) == (pass == 1)) {
          ctx->h_cont.push_back(s->cont[i]);
          ctx->h_cont_pos.push_back(i);
        }
    ctx->C_eff = 0;
    for (int i = 0; i < s->n_cont; ++i) ctx->C_eff += br[s->cont[i]] == 0;
  }
  ctx->h_N.clear();
  ctx->h_nidx.assign(E, -1);
  for (int l = 0; l < E; ++l)
    if (need[l]) {
      ctx->h_nidx[l] = (int)ctx->h_N.size();
      ctx->h_N.push_back(l);
    }
  const int NN = (int)ctx->h_N.size();
  ctx->NN = NN;
  const int M = ctx->M, C = ctx->C;
  std::vector<int> monN(M), contN(std::max(C, 1)), cpos(M, -1), mpos(std::max(C, 1), -1);
  std::vector<int> pos_in_cont(E, -1), pos_in_mon(E, -1);
  for (int i = 0; i < C; ++i) pos_in_cont[ctx->h_cont[i]] = i;
  for (int i = 0; i < M; ++i) pos_in_mon[ctx->h_mon[i]] = i;
  std::vector<double> inv_lim(M);
  for (int i = 0; i < M; ++i) {
    monN[i] = ctx->h_nidx[ctx->h_mon[i]];
    cpos[i] = pos_in_cont[ctx->h_mon[i]];
    inv_lim[i] = 1.0 / s->limit[ctx->h_mon[i]];
  }
  for (int i = 0; i < C; ++i) {
    contN[i] = ctx->h_nidx[ctx->h_cont[i]];
    mpos[i] = pos_in_mon[ctx->h_cont[i]];
  }
  int rc;
  if ((rc = upload(ctx->nidx, ctx->h_nidx.data(), sizeof(int) * E))) return rc;
  if ((rc = upload(ctx->split_ok, split_ok.data(), V))) return rc;
  if ((rc = upload(ctx->out_ok, out_ok.data(), E))) return rc;
  if ((rc = upload(ctx->monN, monN.data(), sizeof(int) * M))) return rc;
  if ((rc = upload(ctx->contN, contN.data(), sizeof(int) * contN.size()))) return rc;
  if ((rc = upload(ctx->cpos_of_mon, cpos.data(), sizeof(int) * M))) return rc;
  if ((rc = upload(ctx->mpos_of_cont, mpos.data(), sizeof(int) * mpos.size()))) return rc;
  if ((rc = upload(ctx->inv_lim, inv_lim.data(), sizeof(double) * M))) return rc;
  {
    std::vector<int> pos(std::max(C, 1), 0), inv(std::max(C, 1), 0);
    for (int i = 0; i < C; ++i) {
      pos[i] = ctx->h_cont_pos[i];
      inv[ctx->h_cont_pos[i]] = i;
    }
    if ((rc = upload(ctx->cont_pos, pos.data(), sizeof(int) * pos.size()))) return rc;
    if ((rc = upload(ctx->cont_inv, inv.data(), sizeof(int) * inv.size()))) return rc;
  }
  {
    std::vector<double> bN(NN);
    for (int i = 0; i < NN; ++i) bN[i] = ctx->hb[ctx->h_N[i]];
    if ((rc = upload(ctx->bN, bN.data(), sizeof(double) * NN))) return rc;
  }
  DevBuf d_N;
  if ((rc = upload(d_N, ctx->h_N.data(), sizeof(int) * NN))) return rc;
  cudaStream_t st = 0;
  int ldy = 0;
  rc = solve_branch_columns(ctx, d_N.as<int>(), NN, &ldy, st);
  if (rc) {
    d_N.release();
    return rc;
  }
  if (ctx->PhiN.ensure((size_t)NN * NN * sizeof(double)) || ctx->PtdfN.ensure((size_t)NN * V * sizeof(double))) {
    d_N.release();
    return DCFLOW_ERR_OOM;
  }
  k_phi_rows<<<dim3((NN + 127) / 128, NN), 128, 0, st>>>(NN, d_N.as<int>(), ctx->f.as<int>(), ctx->t.as<int>(),
                                                         ctx->b.as<double>(), ctx->rid.as<int>(), ctx->Y.as<double>(),
                                                         ldy, ctx->PhiN.as<double>());
  k_ptdf_rows<<<dim3((V + 31) / 32, (NN + 31) / 32), dim3(32, 8), 0, st>>>(
      NN, V, d_N.as<int>(), ctx->b.as<double>(), ctx->rid.as<int>(), ctx->Y.as<double>(), ldy, ctx->PtdfN.as<double>());
  ctx->launches += 2;
  const size_t rs = ctx->opt.precision == DCFLOW_FP64 ? sizeof(double) : sizeof(float);
  if (ctx->opt.precision != DCFLOW_FP64) {  // float copies for the FP32 form's row operands
    if (ctx->PhiNf.ensure((size_t)NN * NN * sizeof(float)) || ctx->bNf.ensure((size_t)NN * sizeof(float))) {
      d_N.release();
      return DCFLOW_ERR_OOM;
    }
    k_to_float<<<(unsigned)std::min<size_t>(((size_t)NN * NN + 255) / 256, 148 * 64), 256, 0, st>>>(
        ctx->PhiN.as<double>(), ctx->PhiNf.as<float>(), (size_t)NN * NN);
    k_to_float<<<(NN + 255) / 256, 256, 0, st>>>(ctx->bN.as<double>(), ctx->bNf.as<float>(), (size_t)NN);
    ctx->launches += 2;
  }
  ctx->ldc = (int)round_up(std::max(C, 1), 4);
  if (ctx->PhiMC.ensure((size_t)M * ctx->ldc * rs)) {
    d_N.release();
    return DCFLOW_ERR_OOM;
  }
  if (C > 0) {
    dim3 g((ctx->ldc + 127) / 128, M);
    if (ctx->opt.precision == DCFLOW_FP64)
      k_phi_mc<double><<<g, 128, 0, st>>>(M, C, ctx->ldc, NN, ctx->monN.as<int>(), ctx->contN.as<int>(),
                                         ctx->inv_lim.as<double>(), ctx->PhiN.as<double>(), ctx->PhiMC.as<double>());
    else
      k_phi_mc<float><<<g, 128, 0, st>>>(M, C, ctx->ldc, NN, ctx->monN.as<int>(), ctx->contN.as<int>(),
                                        ctx->inv_lim.as<double>(), ctx->PhiN.as<double>(), ctx->PhiMC.as<float>());
    ++ctx->launches;
  }
  ctx->n_multi = n_multi;
  ctx->n_multi_ent = (int)mbr.size();
  if (n_multi > 0) {  // per entry: needed-row index, monitored position, Phi[mon, entry] / limit
    const int nE = (int)mbr.size(), Mp = (int)round_up(M, 16);
    std::vector<int> mN(nE), mmp(nE);
    for (int e = 0; e < nE; ++e) {
      mN[e] = ctx->h_nidx[mbr[e]];
      mmp[e] = pos_in_mon[mbr[e]];
    }
    if ((rc = upload(ctx->multi_ptr, mptr.data(), sizeof(int) * mptr.size())) ||
        (rc = upload(ctx->multiN, mN.data(), sizeof(int) * nE)) ||
        (rc = upload(ctx->multi_mpos, mmp.data(), sizeof(int) * nE))) {
      d_N.release();
      return rc;
    }
    if (ctx->PhiMO.ensure((size_t)nE * Mp * rs)) {
      d_N.release();
      return DCFLOW_ERR_OOM;
    }
    const dim3 g((Mp + 127) / 128, nE);
    if (ctx->opt.precision == DCFLOW_FP64)
      k_phi_multi<double><<<g, 128, 0, st>>>(M, Mp, NN, ctx->monN.as<int>(), ctx->multiN.as<int>(),
                                             ctx->inv_lim.as<double>(), ctx->PhiN.as<double>(),
                                             ctx->PhiMO.as<double>());
    else
      k_phi_multi<float><<<g, 128, 0, st>>>(M, Mp, NN, ctx->monN.as<int>(), ctx->multiN.as<int>(),
                                            ctx->inv_lim.as<double>(), ctx->PhiN.as<double>(),
                                            ctx->PhiMO.as<float>());
    ++ctx->launches;
  }
  cudaError_t e = cudaStreamSynchronize(st);
  d_N.release();
  ctx->Y.release();
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    set_error(std::string("dcflow_set_study: ") + cudaGetErrorString(e));
    return DCFLOW_ERR_CUDA;
  }
  ctx->h_split_ok = split_ok;
  ctx->phicm_ready = false;
  ctx->has_study = true;
  return DCFLOW_OK;
}
