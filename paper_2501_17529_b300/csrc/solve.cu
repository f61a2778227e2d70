// Per-batch path of dcflow_solve_batch.
//
// Every topology tau (splits t_b and outages t_d, Sec. III-A) is expressed as
// r = k_s + k_o modifications of the base grid.  Modification j injects a
// fictitious transfer into the base network:
//   split j  (substation A, moved set M_j, beta_j = sum_{M_j} b):
//            W[:, j] = sigma_m b_m / beta_j on the moved branches m, Sigma[:, j] = sigma_m
//            (sigma_m = +1 if the from end of m moves to the new busbar, else -1);
//   outage c: W[:, j] = Sigma[:, j] = e_c.
// With the base branch-to-branch factors Phi[l, c] = PTDF[l, f_c] - PTDF[l, t_c]
// (the LODF numerator of Def. 3):
//   Z = (I - Phi) W,  K = Sigma^T Z   (r x r, FP64),
//   p_f = p0 - Z K^{-1} Sigma^T p0                      (N-0 flows, Eq. (2)),
//   Phi_f[:, c] = Phi[:, c] - Z K^{-1} (Sigma^T Phi[:, c] - s_c)
// where s_c[j] = sigma of c in split j (0 for outage rows).  This is the
// simultaneous form of the BSDF update (Def. 5-6, Eq. (7)) and of the MODF
// (Def. 4): K = Sigma^T (I - Phi) W generalises both denominators, its
// natural-order LU pivots are the sequential BSDF / LODF denominators
// (in [0, 1], zero exactly when the topology islands), and the outaged rows
// of p_f vanish (the MODF rows O := -I).  The N-1 of the updated topology then
// follows Def. 3 / Eq. (5):
//   p_n1[c][l] = p_f[l] + Phi_f[l, c] p_f[c] / (1 - Phi_f[c, c]),  LODF[c, c] = -1,
// reduced on the fly to max |p_n1| / limit (agg_m), its arg-max and the
// overload sum.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cudaTypedefs.h>

#include "args.cuh"
#include "bf16x3.cuh"
#include "internal.cuh"
#include "screen.cuh"

namespace dcf {

// ---------------------------------------------------------------------------
// decode: topology vectors -> modification list
// ---------------------------------------------------------------------------
template <bool WRITE>
__device__ int decode_topology(const GridDev& g, const BatchDev& in, int tau, int* r_out, int* ks_out, int* en,
                               int8_t* es, double* ew, int16_t* mp) {
  const int s0 = in.split_ptr[tau], s1 = in.split_ptr[tau + 1];
  const int o0 = in.out_ptr[tau], o1 = in.out_ptr[tau + 1];
  *r_out = 0;
  *ks_out = 0;
  if (s1 < s0 || o1 < o0) return ST_INVALID;
  int r = 0, ne = 0;
  for (int k = s0; k < s1; ++k) {
    const int A = in.split_sub[k];
    if (A < 0 || A >= g.V || !g.split_ok[A]) return ST_INVALID;
    for (int k2 = s0; k2 < k; ++k2)
      if (in.split_sub[k2] == A) return ST_INVALID;
    const uint64_t m = in.split_mask[k];
    const int p0 = g.inc_ptr[A], deg = g.inc_ptr[A + 1] - p0;
    if (deg > 64 || (deg < 64 && (m >> deg) != 0)) return ST_INVALID;
    const int nb = __popcll(m);
    if (nb == 0 || nb == deg) continue;  // one busbar empty: no split
    if (r >= kRMax || ne + nb > kEntMax) return ST_INVALID;
    double beta = 0.0;
    for (int j = 0; j < deg; ++j)
      if ((m >> j) & 1ull) {
        const int l = g.inc_list[p0 + j];
        if (g.nidx[l] < 0) return ST_INVALID;
        beta += g.b[l];
      }
    if (WRITE) mp[r] = (int16_t)ne;
    for (int j = 0; j < deg; ++j)
      if ((m >> j) & 1ull) {
        const int l = g.inc_list[p0 + j];
        const int sg = (g.f[l] == A) ? 1 : -1;
        if (WRITE) {
          en[ne] = g.nidx[l];
          es[ne] = (int8_t)sg;
          ew[ne] = sg * g.b[l] / beta;
        }
        ++ne;
      }
    ++r;
  }
  const int ks = r;
  for (int k = o0; k < o1; ++k) {
    const int c = in.out_branch[k];
    if (c < 0 || c >= g.E || !g.out_ok[c] || g.nidx[c] < 0) return ST_INVALID;
    for (int k2 = o0; k2 < k; ++k2)
      if (in.out_branch[k2] == c) return ST_INVALID;
    if (r >= kRMax || ne >= kEntMax) return ST_INVALID;
    if (WRITE) {
      mp[r] = (int16_t)ne;
      en[ne] = g.nidx[c];
      es[ne] = 1;
      ew[ne] = 1.0;
    }
    ++ne;
    ++r;
  }
  if (WRITE) mp[r] = (int16_t)ne;
  *r_out = r;
  *ks_out = ks;
  return ST_OK;
}

__global__ void k_rank(GridDev g, BatchDev in, int n_topo, int8_t* rank) {
  const int tau = blockIdx.x * blockDim.x + threadIdx.x;
  if (tau >= n_topo) return;
  int r, ks;
  int st = decode_topology<false>(g, in, tau, &r, &ks, nullptr, nullptr, nullptr, nullptr);
  rank[tau] = (int8_t)(st == ST_OK ? r : -1);
}

__global__ void k_decode(GridDev g, BatchDev in, const int* perm, Args a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.nq) return;
  const int tau = perm[q];
  int r, ks;
  int st = decode_topology<true>(g, in, tau, &r, &ks, a.ent_n + (size_t)q * kEntMax, a.ent_s + (size_t)q * kEntMax,
                                 a.ent_w + (size_t)q * kEntMax, a.mod_ptr + (size_t)q * (kRMax + 1));
  QInfo qi;
  qi.tau = tau;
  qi.r = r;
  qi.ks = ks;
  qi.status = st;
  a.qi[q] = qi;
}

// ---------------------------------------------------------------------------
// base flows p0 = PTDF[N, :] P_t (Eq. (2)), one warp per needed branch
// ---------------------------------------------------------------------------
__global__ void k_p0(int NN, int V, int T, int ldp, const double* __restrict__ ptdf, const double* __restrict__ inj,
                     double* __restrict__ p0) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= NN) return;
  const double* row = ptdf + (size_t)warp * V;
  for (int t0 = 0; t0 < T; t0 += 8) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int n = lane; n < V; n += 32) {
      const double pv = row[n];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (t0 + k < T) acc[k] = fma(pv, inj[(size_t)(t0 + k) * V + n], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      double v = acc[k];
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && t0 + k < T) p0[(size_t)warp * ldp + t0 + k] = v;
    }
  }
}

// Columns T.. of p0 for the injection-candidate pool: the base flow change of
// one unit injected at each pool bus (a PTDF column, Eq. (3)); the rank-r
// update then turns them into the topology's own PTDF columns.
__global__ void k_p0_pool(int NN, int V, int T, int R, int ldp, const int* __restrict__ pool,
                          const double* __restrict__ ptdf, double* __restrict__ p0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NN) return;
  for (int k = 0; k < R; ++k) p0[(size_t)i * ldp + T + k] = ptdf[(size_t)i * V + pool[k]];
}

// ---------------------------------------------------------------------------
// r x r system per topology: K, natural-order LU (pivot test), K^{-1},
// alpha = K^{-1} Sigma^T p0, Vt = K^{-1} (Sigma^T Phi[:, cont] - s)
// ---------------------------------------------------------------------------
struct EntSmem {
  int en[kEntMax];
  double ew[kEntMax];
  double ewb[kEntMax];  // ew / b of the entry's branch
  float ewf[kEntMax], ewbf[kEntMax];  // the same in FP32 (no per-use conversion on the FP64 pipe)
  int8_t es[kEntMax];
  double esd[kEntMax];  // es as double (int-to-double conversions run on the FP64 pipe: once per entry)
  int mp[kRMax + 1];
};

__device__ void load_entries(EntSmem& S, const Args& a, int q, int r) {
  for (int i = threadIdx.x; i <= r; i += blockDim.x) S.mp[i] = a.mod_ptr[(size_t)q * (kRMax + 1) + i];
  __syncthreads();
  const int ne = S.mp[r];
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    S.en[e] = a.ent_n[(size_t)q * kEntMax + e];
    S.ew[e] = a.ent_w[(size_t)q * kEntMax + e];
    S.ewb[e] = S.ew[e] / a.bN[S.en[e]];
    S.ewf[e] = (float)S.ew[e];
    S.ewbf[e] = (float)S.ewb[e];
    S.es[e] = a.ent_s[(size_t)q * kEntMax + e];
    S.esd[e] = (double)S.es[e];
  }
  __syncthreads();
}

// Z[row, j] = W[row, j] - sum_{q in mod j} w_q Phi[row, m_q], reading row m_q
// of Phi instead of column m_q: by reciprocity Phi[l, m] b_m = Phi[m, l] b_l,
// so threads with consecutive rows read consecutive addresses (FP64)
__device__ __forceinline__ double z_entry_col(const EntSmem& S, const double* PhiN, int NN, const double* bN,
                                              int row, int j) {
  double z = 0.0, wdiag = 0.0;
  for (int e = S.mp[j]; e < S.mp[j + 1]; ++e) {
    const int m = S.en[e];
    const double w = S.ew[e];
    z = fma(S.ewb[e], PhiN[(size_t)m * NN + row], z);
    if (m == row) wdiag += w;
  }
  return fma(-bN[row], z, wdiag);
}

// The same in the working precision (monitored rows of the FP32 form; the
// denominators keep the FP64 version)
template <class Real>
__device__ __forceinline__ Real z_entry_col_r(const EntSmem& S, const double* PhiN, int NN, const double* bN,
                                              int row, int j) {
  Real z = 0, wdiag = 0;
  for (int e = S.mp[j]; e < S.mp[j + 1]; ++e) {
    const int m = S.en[e];
    z = fma((Real)S.ewb[e], (Real)PhiN[(size_t)m * NN + row], z);
    if (m == row) wdiag += (Real)S.ew[e];
  }
  return fma(-(Real)bN[row], z, wdiag);
}

// The same from float copies of Phi and b (FP32 form, monitored rows)
__device__ __forceinline__ float z_entry_col_f(const EntSmem& S, const float* PhiNf, int NN, const float* bNf, int row,
                                               int j) {
  float z = 0.f, wdiag = 0.f;
  for (int e = S.mp[j]; e < S.mp[j + 1]; ++e) {
    const int m = S.en[e];
    z = fmaf(S.ewbf[e], PhiNf[(size_t)m * NN + row], z);
    if (m == row) wdiag += S.ewf[e];
  }
  return fmaf(-bNf[row], z, wdiag);
}

// Z[row, j] = W[row, j] - sum_{q in mod j} w_q Phi[row, m_q]  (FP64)
__device__ __forceinline__ double z_entry(const EntSmem& S, const double* PhiRow, int row, int j) {
  double z = 0.0;
  for (int e = S.mp[j]; e < S.mp[j + 1]; ++e) {
    const int m = S.en[e];
    const double w = S.ew[e];
    z = fma(-w, PhiRow[m], z);
    if (m == row) z += w;
  }
  return z;
}

// Vt[j][c] = K^{-1} (Sigma^T Phi[:, c] - s_c) for the topology's R modifications (FP64), and
// its working-precision copy; rows R .. RMAX - 1 are written as zeros
template <class Real, int R, int RMAX>
__device__ __forceinline__ void vt_cols(const EntSmem& S, const Args& a, int q, int ks,
                                        const double (*Ki)[kRMax + 1]) {
  const int C = a.C;
  Real* VtR = static_cast<Real*>(a.VtR);
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const int nc = a.contN[c];
    double v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      double acc = 0.0;
      for (int e = S.mp[i]; e < S.mp[i + 1]; ++e) {
        const int m = S.en[e];
        acc = fma(S.esd[e], a.PhiN[(size_t)m * a.NN + nc], acc);
        if (i < ks && m == nc) acc -= S.esd[e];
      }
      v[i] = acc;
    }
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
      double x = 0.0;
      if (j < R) {
#pragma unroll
        for (int i = 0; i < R; ++i) x = fma(Ki[j][i], v[i], x);
      }
      const size_t o = ((size_t)q * kRMax + j) * C + c;
      a.Vt64[o] = x;
      VtR[o] = (j < R) ? (Real)x : (Real)0;  // no conversion for the zero rows
    }
  }
}

template <class Real, int R, int RMAX>
__device__ __forceinline__ void vt_rank(int r, const EntSmem& S, const Args& a, int q, int ks,
                                        const double (*Ki)[kRMax + 1]) {
  if constexpr (R <= RMAX) {
    if (r == R) vt_cols<Real, R, RMAX>(S, a, q, ks, Ki);
    else vt_rank<Real, R + 1, RMAX>(r, S, a, q, ks, Ki);
  }
}

template <class Real, int RMAX>
__global__ __launch_bounds__(128) void k_small(Args a) {
  const int q = blockIdx.x;
  __shared__ EntSmem S;
  __shared__ double K[kRMax][kRMax + 1];
  __shared__ double Ki[kRMax][kRMax + 1];
  __shared__ int bad;
  const QInfo qi = a.qi[q];
  if (qi.status != ST_OK) return;
  const int r = qi.r, ks = qi.ks, tid = threadIdx.x;
  load_entries(S, a, q, r);
  for (int p = tid; p < r * r; p += blockDim.x) {
    const int i = p / r, j = p % r;
    double acc = 0.0;
    for (int e = S.mp[i]; e < S.mp[i + 1]; ++e) {
      const int m = S.en[e];
      acc = fma(S.esd[e], z_entry(S, a.PhiN + (size_t)m * a.NN, m, j), acc);
    }
    K[i][j] = acc;
  }
  if (tid == 0) bad = 0;
  for (int p = tid; p < kRMax * (kRMax + 1); p += blockDim.x) (&Ki[0][0])[p] = 0.0;
  __syncthreads();
  if (tid < 32) {
    int isl = 0;
    for (int k = 0; k < r; ++k) {
      const double piv = K[k][k];
      if (!(fabs(piv) > a.tol)) {
        isl = 1;
        break;
      }
      __syncwarp();
      const int i = tid;
      if (i > k && i < r) {
        const double fct = K[i][k] / piv;
        K[i][k] = fct;
        for (int j = k + 1; j < r; ++j) K[i][j] = fma(-fct, K[k][j], K[i][j]);
      }
      __syncwarp();
    }
    if (!isl && tid < r) {
      const int j = tid;
      double y[RMAX];
#pragma unroll
      for (int i = 0; i < RMAX; ++i) {
        if (i < r) {
          double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
          for (int p = 0; p < i; ++p) s = fma(-K[i][p], y[p], s);
          y[i] = s;
        }
      }
#pragma unroll
      for (int i = RMAX - 1; i >= 0; --i) {
        if (i < r) {
          double s = y[i];
#pragma unroll
          for (int p = i + 1; p < RMAX; ++p)
            if (p < r) s = fma(-K[i][p], y[p], s);
          y[i] = s / K[i][i];
        }
      }
#pragma unroll
      for (int i = 0; i < RMAX; ++i)
        if (i < r) Ki[i][j] = y[i];
    }
    if (tid == 0) bad = isl;
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) a.qi[q].status = ST_ISLAND;
    return;
  }
  double* Kinv = a.Kinv + (size_t)q * kRMax * kRMax;
  for (int p = tid; p < kRMax * kRMax; p += blockDim.x) {
    const int i = p / kRMax, j = p % kRMax;
    Kinv[p] = (i < r && j < r) ? Ki[i][j] : 0.0;
  }
  // alpha[j][t]
  const int T = a.T;
  for (int t = tid; t < T; t += blockDim.x) {
    double bv[RMAX];
#pragma unroll
    for (int i = 0; i < RMAX; ++i) {
      double acc = 0.0;
      if (i < r)
        for (int e = S.mp[i]; e < S.mp[i + 1]; ++e) acc = fma(S.esd[e], a.p0[(size_t)S.en[e] * T + t], acc);
      bv[i] = acc;
    }
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
      double x = 0.0;
#pragma unroll
      for (int i = 0; i < RMAX; ++i) x = fma(Ki[j][i], bv[i], x);  // Ki is zero outside r x r
      a.alpha[((size_t)q * kRMax + j) * T + t] = x;
    }
  }
  // Vt[j][c] at the topology's exact rank (uniform over the block; the rank classes pad r
  // up to RMAX, and the padded multiply-adds would be FP64 work), zero rows r .. RMAX - 1
  vt_rank<Real, 1, RMAX>(r, S, a, q, ks, Ki);
}

// ---------------------------------------------------------------------------
// rows: Z, N-0 flows, scaled operands of the N-1 kernel, FP64 denominators
// ---------------------------------------------------------------------------
// Per-topology operands of the N-1 kernels, all row-strided by Mpad:
//   Zs   [kRMax][Mpad]  Z[l, j] / limit_l          (zero rows for outaged l)
//   ptil [T][Mpad]      p_f[l, t] / limit_l        (zero for outaged l)
//   meta [4][Mpad]      row 0: -den_c / limit_l on the row of contingency c,
//                       row 1: 1 (0 for an outaged l), row 2: position of l in
//                       the contingency list as int bits (-1 if none), row 3: 0
template <class Real, int RMAX>
__global__ __launch_bounds__(128) void k_rows(Args a, Real* __restrict__ zcd, const float* __restrict__ p0f,
                                              const float* __restrict__ PhiNf, const float* __restrict__ bNf) {
  const int q = blockIdx.x;
  __shared__ EntSmem S;
  __shared__ int outN[kRMax];
  __shared__ int nout;
  __shared__ int nisl;
  extern __shared__ unsigned char dyn[];
  Real* alph = reinterpret_cast<Real*>(dyn);  // [kRMax][T]
  const QInfo qi = a.qi[q];
  if (qi.status != ST_OK) return;
  const int r = qi.r, ks = qi.ks, tid = threadIdx.x, T = a.T, M = a.M, C = a.C, NN = a.NN, Mp = a.Mpad;
  load_entries(S, a, q, r);
  if (tid == 0) {
    nout = r - ks;
    nisl = 0;
  }
  for (int i = tid; i < r - ks; i += blockDim.x) outN[i] = S.en[S.mp[ks + i]];
  for (int p = tid; p < RMAX * T; p += blockDim.x) alph[p] = (Real)a.alpha[(size_t)q * kRMax * T + p];
  __syncthreads();
  Real* Zs = static_cast<Real*>(a.Zs) + (size_t)q * kRMax * Mp;
  Real* ptil = static_cast<Real*>(a.ptil) + (size_t)q * T * Mp;
  Real* meta = static_cast<Real*>(a.diagv) + (size_t)q * 4 * Mp;
  Real* sv = static_cast<Real*>(a.s) + (size_t)q * T * C;
  const int tau = qi.tau;
  for (int l = tid; l < M; l += blockDim.x) {
    const int nl = a.monN[l];
    bool outd = false;
    for (int k = 0; k < nout; ++k) outd |= (outN[k] == nl);
    Real z[RMAX];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
      if constexpr (sizeof(Real) == 4) z[j] = (j < r) ? z_entry_col_f(S, PhiNf, NN, bNf, nl, j) : 0.f;
      else z[j] = (j < r) ? z_entry_col_r<Real>(S, a.PhiN, NN, a.bN, nl, j) : (Real)0;
    }
    const Real il = (Real)a.inv_lim[l];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) Zs[(size_t)j * Mp + l] = outd ? (Real)0 : z[j] * il;
    if constexpr (sizeof(Real) == 4) {
      if (a.Zbf) {  // BF16x3 form: the same row split into BF16 hi / lo pairs for the tensor-core build
        constexpr int KB = TcK<RMAX>::KB;
        uint32_t* zr = a.Zbf + ((size_t)q * Mp + l) * KB;
#pragma unroll
        for (int j2 = 0; j2 < KB / 2; ++j2) {
          const float x0 = (2 * j2 < RMAX && !outd) ? (float)(z[min(2 * j2, RMAX - 1)] * il) : 0.f;
          const float x1 = (2 * j2 + 1 < RMAX && !outd) ? (float)(z[min(2 * j2 + 1, RMAX - 1)] * il) : 0.f;
          uint32_t hi, lo;
          bf16_split2(x0, x1, hi, lo);
          zr[j2] = hi;
          zr[KB / 2 + j2] = lo;
        }
      }
    }
    meta[l] = (Real)0;
    meta[Mp + l] = outd ? (Real)0 : (Real)1;
    if (sizeof(Real) == 4) {
      reinterpret_cast<int*>(meta)[2 * Mp + l] = a.cpos[l];
    } else {
      meta[2 * Mp + l] = (Real)a.cpos[l];
    }
    meta[3 * Mp + l] = (Real)0;
    for (int t = 0; t < T; ++t) {
      Real pf;
      if constexpr (sizeof(Real) == 4) pf = p0f[(size_t)nl * T + t];
      else pf = a.p0[(size_t)nl * T + t];
#pragma unroll
      for (int j = 0; j < RMAX; ++j) pf = fma(-z[j], alph[j * T + t], pf);
      ptil[(size_t)t * Mp + l] = outd ? (Real)0 : pf * il;
      if (a.out.n0_flow) a.out.n0_flow[((size_t)tau * T + t) * M + l] = outd ? 0.0 : (double)pf;
    }
  }
  __syncthreads();
  const double* Vt64 = a.Vt64 + (size_t)q * kRMax * C;
  int my_isl = 0;
  for (int c = tid; c < C; c += blockDim.x) {
    const int nc = a.contN[c];
    bool outd = false;
    for (int k = 0; k < nout; ++k) outd |= (outN[k] == nc);
    const double* prow = a.PhiN + (size_t)nc * NN;
    double z[RMAX];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) z[j] = (j < r) ? z_entry_col(S, a.PhiN, NN, a.bN, nc, j) : 0.0;
    double phicc = prow[nc];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) phicc = fma(-z[j], Vt64[(size_t)j * C + c], phicc);
    const double den = 1.0 - phicc;
    const bool ok = !outd && den > a.tol;
    my_isl += (!outd && !ok);
    a.valid[(size_t)q * C + c] = ok;
    const int mp = a.mpos[c];
    if (mp >= 0) meta[mp] = (Real)(-den * a.inv_lim[mp]);
    // the denominator is FP64; its reciprocal only needs the working precision
    const Real invd = ok ? (Real)1 / (Real)den : (Real)0;
    if (zcd)  // Z[c, :] / den_c for the injection-topology candidates
#pragma unroll
      for (int j = 0; j < RMAX; ++j) zcd[((size_t)q * kRMax + j) * C + c] = (Real)z[j] * invd;
    Real zr[RMAX];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) zr[j] = (Real)z[j];
    for (int t = 0; t < T; ++t) {
      Real pf;
      if constexpr (sizeof(Real) == 4) pf = p0f[(size_t)nc * T + t];
      else pf = a.p0[(size_t)nc * T + t];
#pragma unroll
      for (int j = 0; j < RMAX; ++j) pf = fma(-zr[j], alph[j * T + t], pf);
      sv[(size_t)t * C + c] = pf * invd;
    }
  }
  if (my_isl) atomicAdd(&nisl, my_isl);
  __syncthreads();
  if (tid == 0) a.nisl[q] = nisl;
  // N-0 maximum loading per timestep (one warp per timestep)
  if (a.out.n0_max_loading) {
    const int lane = tid & 31, nw = blockDim.x >> 5;
    for (int t = tid >> 5; t < T; t += nw) {
      Real m = 0;  // the working precision per row (B300's FP64 rate is far below FP32)
      for (int l = lane; l < M; l += 32) m = fmax(m, fabs(ptil[(size_t)t * Mp + l]));
      for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) a.out.n0_max_loading[(size_t)tau * T + t] = (double)m;
    }
  }
}

// ---------------------------------------------------------------------------
// fused N-1 (Def. 3, Eq. (5)) with in-register max / overload reduction
// ---------------------------------------------------------------------------
template <class Real>
struct Acc;

template <>
struct Acc<float> {
  // overload term via a saturating FMA: sat((|v| - 1) 2^-20) = max(0, |v| - 1) 2^-20 for |v| < 2^20 + 1
  static __device__ __forceinline__ void add(float& mx, float& ov, float v) {
    const float av = fabsf(v);
    mx = fmaxf(mx, av);
    ov += __saturatef(fmaf(av, 0x1p-20f, -0x1p-20f));
  }
  static __device__ __forceinline__ double ovl_scale() { return 1048576.0; }
};

template <>
struct Acc<double> {
  // the running maximum through the bit patterns shifted past the sign on the
  // integer pipe (magnitudes order like these unsigned integers; a masked sign
  // bit would become a double fabs), max(|v| - 1, 0) by its sign bit: of the
  // FP64 pipe only the two additions remain (B300's FP64 rate is low)
  static __device__ __forceinline__ void add(double& mx, double& ov, double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) << 1;
    if (b > ((unsigned long long)__double_as_longlong(mx) << 1)) mx = __longlong_as_double((long long)(b >> 1));
    const double d = fabs(v) - 1.0;
    ov += __double_as_longlong(d) < 0 ? 0.0 : d;
  }
  static __device__ __forceinline__ double ovl_scale() { return 1.0; }
};

// Phi_f[l, c] / limit_l for one (l, c): shared by the N-1 kernel and the
// final arg-max pass so both see bit-identical values.
template <class Real, int RMAX>
__device__ __forceinline__ Real phi_entry(Real base, const Real* zrow, const Real* vt, Real rm, int cp, int c, Real dg) {
  Real p = base;
#pragma unroll
  for (int j = 0; j < RMAX; ++j) p = fma(-zrow[j], vt[j], p);
  p = p * rm;
  return (cp == c) ? dg : p;
}

// The same at the topology's exact rank r <= RMAX: the rank class pads Z and Vt
// with zero rows, whose terms are exact zeros (at most the sign of a zero Phi_f
// entry differs, which no |v| sees)
template <class Real, int RMAX>
__device__ __forceinline__ Real phi_entry_r(Real base, const Real* zrow, const Real* vt, Real rm, int cp, int c, Real dg,
                                            int r) {
  Real p = base;
#pragma unroll
  for (int j = 0; j < RMAX; ++j) {
    if (j >= r) break;
    p = fma(-zrow[j], vt[j], p);
  }
  p = p * rm;
  return (cp == c) ? dg : p;
}

// Fused N-1 (Def. 3, Eq. (5)) of one topology x 64 contingencies (one per
// thread) x TT timesteps, LT monitored rows at a time staged in shared memory:
// the FP64 form, and the FP32 form where the register-tiled kernel does not
// apply.  Per (contingency, timestep) the maximum loading and the overload sum;
// in FP64 the overload terms are computed only for the tiles whose maximum
// exceeds 1 (queued per warp), in the same order as a per-entry sum, and Phi_f
// is built at the exact rank.
template <class Real, int TT, int RMAX, int LT>
__global__ __launch_bounds__(64) void k_n1(Args a, int t0_base) {
  const int t0 = t0_base + (int)blockIdx.z * TT;  // grid z: the passes over TT timesteps each
  const int q = blockIdx.y;
  const QInfo qi = a.qi[q];
  if (qi.status != ST_OK) return;
  const int tid = threadIdx.x, M = a.M, C = a.C, T = a.T;
  const int c = blockIdx.x * 64 + tid;
  const bool cin = c < C;
  const int cc = cin ? c : C - 1;
  __shared__ Real zs[LT][RMAX];
  __shared__ Real pt[LT][TT];
  __shared__ Real dg[LT], rm[LT];
  __shared__ int cp[LT];
  // FP64 form: the overload term only for the (contingency, timestep) items whose tile maximum
  // exceeds 1, queued per warp and served by all its lanes (B300's FP64 pipe is the scarce unit)
  constexpr bool kQ = sizeof(Real) == 8;
  __shared__ Real ph_s[kQ ? LT : 1][64];
  __shared__ Real ov_s[kQ ? TT : 1][64];
  __shared__ uint16_t qu_s[kQ ? 2 : 1][kQ ? 32 * TT : 1];
  const int Mp = a.Mpad;
  const Real* PhiMC = static_cast<const Real*>(a.PhiMC);
  const Real* Zs = static_cast<const Real*>(a.Zs) + (size_t)q * kRMax * Mp;
  const Real* ptil = static_cast<const Real*>(a.ptil) + (size_t)q * T * Mp;
  const Real* meta = static_cast<const Real*>(a.diagv) + (size_t)q * 4 * Mp;
  const Real* VtR = static_cast<const Real*>(a.VtR) + (size_t)q * kRMax * C;
  const Real* sv = static_cast<const Real*>(a.s) + (size_t)q * T * C;
  Real vt[RMAX];
#pragma unroll
  for (int j = 0; j < RMAX; ++j) vt[j] = VtR[(size_t)j * C + cc];
  Real s[TT], mx[TT], ov[TT];
#pragma unroll
  for (int t = 0; t < TT; ++t) {
    s[t] = (cin && t0 + t < T) ? sv[(size_t)(t0 + t) * C + cc] : (Real)0;
    mx[t] = 0;
    ov[t] = 0;
    if constexpr (kQ) ov_s[t][tid] = (Real)0;
  }
  for (int l0 = 0; l0 < M; l0 += LT) {
    __syncthreads();
    for (int idx = tid; idx < LT * RMAX; idx += 64) {
      const int i = idx % LT, j = idx / LT, l = l0 + i;
      zs[i][j] = (l < M) ? Zs[(size_t)j * Mp + l] : (Real)0;
    }
    for (int idx = tid; idx < LT * TT; idx += 64) {
      const int i = idx % LT, t = idx / LT, l = l0 + i;
      pt[i][t] = (l < M && t0 + t < T) ? ptil[(size_t)(t0 + t) * Mp + l] : (Real)0;
    }
    for (int i = tid; i < LT; i += 64) {
      const int l = l0 + i;
      dg[i] = (l < M) ? meta[l] : (Real)0;
      rm[i] = (l < M) ? meta[Mp + l] : (Real)0;
      cp[i] = (l < M) ? a.cpos[l] : -1;
    }
    __syncthreads();
    Real phi[LT];
#pragma unroll
    for (int i = 0; i < LT; ++i) {
      const int l = l0 + i;
      const Real base = (l < M) ? PhiMC[(size_t)l * a.ldc + cc] : (Real)0;
      if constexpr (kQ) phi[i] = phi_entry_r<Real, RMAX>(base, zs[i], vt, rm[i], cp[i], c, dg[i], qi.r);
      else phi[i] = phi_entry<Real, RMAX>(base, zs[i], vt, rm[i], cp[i], c, dg[i]);
    }
    if constexpr (kQ) {
#pragma unroll
      for (int i = 0; i < LT; ++i) ph_s[i][tid] = phi[i];
      const int lane = tid & 31, wq = tid >> 5;
      const uint32_t lt = (1u << lane) - 1u;
      int n = 0;
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        const Real st = s[t];
        // the tile's maximum |v| as bits shifted past the sign (magnitudes order like these
        // unsigned integers); a masked sign bit would become a double fabs on the FP64 pipe
        unsigned long long tb = 0;
#pragma unroll
        for (int i = 0; i < LT; ++i) {
          const unsigned long long b = (unsigned long long)__double_as_longlong(fma(phi[i], st, pt[i][t])) << 1;
          tb = b > tb ? b : tb;
        }
        if (tb > ((unsigned long long)__double_as_longlong(mx[t]) << 1)) mx[t] = __longlong_as_double((long long)(tb >> 1));
        const bool hit = tb > (0x3ff0000000000000ull << 1);  // some |v| > 1 in the tile
        const uint32_t m = __ballot_sync(0xffffffffu, hit);
        if (hit) qu_s[wq][n + __popc(m & lt)] = (uint16_t)((lane << 8) | t);
        n += __popc(m);
      }
      if (n) {
        __syncwarp();
        for (int jq = lane; jq < n; jq += 32) {  // the 8 rows of one queued item, in row order
          const int item = qu_s[wq][jq], src = (wq << 5) | (item >> 8), t = item & 255;
          const int cs = blockIdx.x * 64 + src;
          const Real st = (cs < C && t0 + t < T) ? sv[(size_t)(t0 + t) * C + cs] : (Real)0;
          Real o = ov_s[t][src];
#pragma unroll
          for (int i = 0; i < LT; ++i) {
            const double d = fabs(fma(ph_s[i][src], st, pt[i][t])) - 1.0;
            o += __double_as_longlong(d) < 0 ? 0.0 : d;
          }
          ov_s[t][src] = o;
        }
        __syncwarp();
      }
    } else {
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        const Real st = s[t];
#pragma unroll
        for (int i = 0; i < LT; ++i) Acc<Real>::add(mx[t], ov[t], fma(phi[i], st, pt[i][t]));
      }
    }
  }
  if constexpr (kQ) {
    __syncthreads();
#pragma unroll
    for (int t = 0; t < TT; ++t) ov[t] = ov_s[t][tid];
  }
  // reduce the 64 contingencies of this block: max (ties: lowest c) and overload sum
  const bool ok = cin && a.valid[(size_t)q * C + c];
  if (a.out.n1_cont_max && cin) {
#pragma unroll
    for (int t = 0; t < TT; ++t)
      if (t0 + t < T) a.out.n1_cont_max[((size_t)qi.tau * T + t0 + t) * C + a.cont_pos[c]] = ok ? (float)mx[t] : -1.f;
  }
  if (a.cmr && cin) {  // working-precision maxima for the final pass's tie band
#pragma unroll
    for (int t = 0; t < TT; ++t)
      if (t0 + t < T) static_cast<Real*>(a.cmr)[((size_t)q * T + t0 + t) * C + c] = ok ? mx[t] : (Real)-1;
  }
  __shared__ Real rv[2];  // maxima compared in the working precision (no FP64-pipe work in the FP32 form)
  __shared__ double ro[2];
  __shared__ int ra[2];
  __shared__ Real r2[2];
  const int lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int t = 0; t < TT; ++t) {
    if (t0 + t < T) {  // uniform over the block
      Real v = ok ? mx[t] : (Real)-1;
      Real w2 = (Real)-1;  // the second largest of the lanes merged so far
      int arg = ok ? c : 0x7fffffff;
      double o = ok ? (double)ov[t] * Acc<Real>::ovl_scale() : 0.0;
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        const Real v2 = __shfl_xor_sync(0xffffffffu, v, off);
        const Real s2 = __shfl_xor_sync(0xffffffffu, w2, off);
        const int a2 = __shfl_xor_sync(0xffffffffu, arg, off);
        o += __shfl_xor_sync(0xffffffffu, o, off);
        w2 = fmax(fmax(w2, s2), fmin(v, v2));
        if (v2 > v || (v2 == v && a2 < arg)) {
          v = v2;
          arg = a2;
        }
      }
      if (lane == 0) {
        rv[w] = v;
        ra[w] = arg;
        ro[w] = o;
        r2[w] = w2;
      }
      __syncthreads();
      if (tid == 0) {
        Real bv = rv[0];
        int ba = ra[0];
        const Real b2 = fmax(fmax(r2[0], r2[1]), fmin(rv[0], rv[1]));
        if (rv[1] > bv || (rv[1] == bv && ra[1] < ba)) {
          bv = rv[1];
          ba = ra[1];
        }
        const size_t o2 = ((size_t)q * T + t0 + t) * a.ncb + blockIdx.x;
        static_cast<Real*>(a.pmax)[o2] = bv;
        a.parg[o2] = (bv < (Real)0) ? -1 : ba;
        a.povl[o2] = ro[0] + ro[1];
        if (a.p2max) static_cast<Real*>(a.p2max)[o2] = b2;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// final: combine the contingency blocks (one warp per timestep), locate the
// worst monitored branch by recomputing the winning contingency's column with
// the same arithmetic as the N-1 kernel, write every output of the topology
// ---------------------------------------------------------------------------
template <class Real, int RMAX>
__global__ __launch_bounds__(128) void k_final(Args a, const int* __restrict__ nsel, const Real* __restrict__ PhiCM,
                                               int col_room) {
  const int q = blockIdx.x;
  const QInfo qi = a.qi[q];
  const int tau = qi.tau, T = a.T, M = a.M, C = a.C, Mp = a.Mpad, tid = threadIdx.x;
  const int lane = tid & 31, nw = blockDim.x >> 5;
  const dcflow_results& o = a.out;
  if (tid == 0) {
    o.island_flag[tau] = (uint8_t)qi.status;
    o.n_island_cont[tau] = (qi.status == ST_OK) ? a.nisl[q] : 0;
  }
  if (qi.status != ST_OK) {
    for (int t = tid; t < T; t += blockDim.x) {
      const size_t k = (size_t)tau * T + t;
      o.n1_max_loading[k] = 0.0;
      o.overload_sum[k] = 0.0;
      o.worst_cont[k] = -1;
      if (o.worst_mon) o.worst_mon[k] = -1;
      if (o.best_var) o.best_var[k] = -1;
      if (o.n0_max_loading) o.n0_max_loading[k] = 0.0;
    }
    if (o.n0_flow)
      for (size_t k = tid; k < (size_t)T * M; k += blockDim.x) o.n0_flow[(size_t)tau * T * M + k] = 0.0;
    if (o.n1_cont_max)
      for (size_t k = tid; k < (size_t)T * C; k += blockDim.x) o.n1_cont_max[(size_t)tau * T * C + k] = -1.f;
    return;
  }
  if (o.n1_cont_max && !nsel)  // contingencies beyond the N-1 range: base-grid bridges, never valid
    for (int k = tid; k < (C - a.C_eff) * T; k += blockDim.x) {
      const int t = k / (C - a.C_eff), c = a.C_eff + k % (C - a.C_eff);
      o.n1_cont_max[((size_t)tau * T + t) * C + a.cont_pos[c]] = -1.f;
    }
  const Real* Zs = static_cast<const Real*>(a.Zs) + (size_t)q * kRMax * Mp;
  const Real* ptil = static_cast<const Real*>(a.ptil) + (size_t)q * T * Mp;
  const Real* meta = static_cast<const Real*>(a.diagv) + (size_t)q * 4 * Mp;
  const Real* VtR = static_cast<const Real*>(a.VtR) + (size_t)q * kRMax * C;
  const Real* sv = static_cast<const Real*>(a.s) + (size_t)q * T * C;
  const Real eps = (Real)a.tie_eps;  // the tie band, eps * max(best, 1), in the working precision
  // the short remainder of the contingency range (no N-1 block of its own): its
  // Phi_f columns, built once with the N-1 kernels' arithmetic into shared memory
  // ([column][monitored row]), then applied to every timestep below
  extern __shared__ __align__(16) unsigned char fin_dyn[];
  Real* s_rem = reinterpret_cast<Real*>(fin_dyn);
  const int c_rem = nsel ? a.C_eff : a.c_rem, n_rem = a.C_eff - c_rem;
  // the worst contingency of every timestep, and one Phi_f column (after the
  // remainder columns) when the launch gave it room: the worst monitored branch
  // of all timesteps that share a worst contingency comes from one column build
  __shared__ int s_wc[256];
  Real* s_col = col_room ? s_rem + (size_t)n_rem * M : nullptr;
  if (n_rem > 0) {
    for (int i = tid; i < n_rem * M; i += blockDim.x) {
      const int c = c_rem + i / M, l = i % M;
      Real vt[RMAX], zr[RMAX];
#pragma unroll
      for (int j = 0; j < RMAX; ++j) {
        vt[j] = VtR[(size_t)j * C + c];
        zr[j] = Zs[(size_t)j * Mp + l];
      }
      s_rem[i] = phi_entry<Real, RMAX>(PhiCM[(size_t)c * Mp + l], zr, vt, meta[Mp + l], a.cpos[l], c, meta[l]);
    }
    __syncthreads();
  }
  for (int t = tid >> 5; t < T; t += nw) {
    Real bv = (Real)-1;  // maxima compared in the working precision
    double ovl = 0.0;
    int ba = 0x7fffffff;
    const int nb = nsel ? (nsel[q] + 63) / 64 : a.ncb;  // blocks of selected contingencies, or all
    for (int b = lane; b < nb; b += 32) {
      const size_t k = ((size_t)q * T + t) * a.ncb + b;
      const Real v = static_cast<const Real*>(a.pmax)[k];
      const int ar = a.parg[k];
      if (ar >= 0 && (v > bv || (v == bv && ar < ba))) {
        bv = v;
        ba = ar;
      }
      ovl += a.povl[k];
    }
    for (int off = 16; off; off >>= 1) {
      const Real v2 = __shfl_xor_sync(0xffffffffu, bv, off);
      const int a2 = __shfl_xor_sync(0xffffffffu, ba, off);
      ovl += __shfl_xor_sync(0xffffffffu, ovl, off);
      if (v2 > bv || (v2 == bv && a2 < ba)) {
        bv = v2;
        ba = a2;
      }
    }
    // the remainder columns at this timestep (their maxima kept for the tie band);
    // their overload terms summed in the working precision, one conversion per
    // column (B300 runs FP64 arithmetic and conversions at a small fraction of
    // the FP32 rate)
    Real vrem[4] = {(Real)-1, (Real)-1, (Real)-1, (Real)-1};
    for (int c = c_rem; c < a.C_eff; ++c) {
      const bool okc = a.valid[(size_t)q * C + c];
      Real vr = (Real)0;
      if (okc) {
        const Real st = sv[(size_t)t * C + c];
        const Real* ph = s_rem + (size_t)(c - c_rem) * M;
        Real ov = (Real)0;
#pragma unroll 4
        for (int l = lane; l < M; l += 32) {  // 4 rows' loads in flight per lane
          const Real x = fabs(fma(ph[l], st, ptil[(size_t)t * Mp + l]));
          vr = fmax(vr, x);
          if (x > (Real)1) ov += x - (Real)1;
        }
        for (int off = 16; off; off >>= 1) {
          vr = fmax(vr, __shfl_xor_sync(0xffffffffu, vr, off));
          ov += __shfl_xor_sync(0xffffffffu, ov, off);
        }
        if (vr > bv || (vr == bv && c < ba)) {
          bv = vr;
          ba = c;
        }
        ovl += (double)ov;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (j == c - c_rem) vrem[j] = vr;
      }
      if (lane == 0 && o.n1_cont_max)
        o.n1_cont_max[((size_t)tau * T + t) * C + a.cont_pos[c]] = okc ? (float)vr : -1.f;
      if (lane == 0 && a.cmr) static_cast<Real*>(a.cmr)[((size_t)q * T + t) * C + c] = okc ? vr : (Real)-1;
    }
    int c = (ba == 0x7fffffff) ? -1 : ba;
    if (c >= 0 && !nsel) {
      // tie band: the lowest contingency position whose maximum loading lies within
      // eps * max(best, 1) of the best (internal order is the caller's order up to
      // the base-grid bridges, which are never valid).  Each block's best within the
      // band is a candidate; only a block whose second largest maximum also lies in
      // the band needs the scan over the per-contingency maxima.
      const Real thr = bv - eps * fmax(bv, (Real)1);
      int cand = 0x7fffffff;
      bool amb = a.p2max == nullptr;
      for (int b = lane; b < nb; b += 32) {
        const size_t k = ((size_t)q * T + t) * a.ncb + b;
        const int ar = a.parg[k];
        if (ar >= 0 && static_cast<const Real*>(a.pmax)[k] >= thr) cand = min(cand, ar);
        if (a.p2max && static_cast<const Real*>(a.p2max)[k] >= thr) amb = true;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < n_rem && vrem[j] >= thr) cand = min(cand, c_rem + j);
      for (int off = 16; off; off >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, off));
      if (!__any_sync(0xffffffffu, amb)) {
        c = cand;  // the best itself lies in the band
      } else if (a.cmr) {
        __syncwarp();  // the remainder maxima written by lane 0 above
        const Real* cr = static_cast<const Real*>(a.cmr) + ((size_t)q * T + t) * C;
        int pos = -1;
        for (int p0 = 0; p0 < a.C_eff && pos < 0; p0 += 32) {
          const int p = p0 + lane;
          const unsigned m = __ballot_sync(0xffffffffu, p < a.C_eff && cr[p] >= thr);
          if (m) pos = p0 + __ffs(m) - 1;
        }
        if (pos >= 0) c = pos;
      }
    }
    if (lane == 0) {
      const size_t k = (size_t)tau * T + t;
      o.n1_max_loading[k] = c >= 0 ? (double)bv : 0.0;
      o.overload_sum[k] = ovl;
      o.worst_cont[k] = c >= 0 ? a.cont_pos[c] : -1;  // the caller's position
      if (o.best_var) o.best_var[k] = a.best_u ? a.best_u[(size_t)q * T + t] : -1;
    }
    if (lane == 0) s_wc[t] = c;
    if (o.worst_mon && !s_col) {
      // the worst contingency's column: its maximum, then the lowest monitored
      // position within the tie band of that maximum
      int arg = 0x7fffffff;
      if (c >= 0) {
        Real vt[RMAX];
#pragma unroll
        for (int j = 0; j < RMAX; ++j) vt[j] = VtR[(size_t)j * C + c];
        const Real st = sv[(size_t)t * C + c];
        auto entry = [&](int l) {
          Real zr[RMAX];
#pragma unroll
          for (int j = 0; j < RMAX; ++j) zr[j] = Zs[(size_t)j * Mp + l];
          const Real ph = phi_entry<Real, RMAX>(PhiCM[(size_t)c * Mp + l], zr, vt, meta[Mp + l], a.cpos[l], c, meta[l]);
          return fabs(fma(ph, st, ptil[(size_t)t * Mp + l]));
        };
        Real v = (Real)-1;
        for (int l = lane; l < M; l += 32) v = fmax(v, entry(l));
        for (int off = 16; off; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
        const Real thr = v - eps * fmax(v, (Real)1);
        for (int l = lane; l < M; l += 32)
          if (entry(l) >= thr) {
            arg = l;
            break;
          }
        for (int off = 16; off; off >>= 1) arg = min(arg, __shfl_xor_sync(0xffffffffu, arg, off));
      }
      if (lane == 0) o.worst_mon[(size_t)tau * T + t] = (c >= 0) ? arg : -1;
    }
  }
  if (!o.worst_mon || !s_col) return;
  __syncthreads();
  // per distinct worst contingency (block-uniform, timestep order): its Phi_f column
  // once into shared memory, then every timestep with that worst contingency: one
  // pass keeping each lane's two largest loadings decides the tie band unless some
  // lane holds two values inside it (then a second pass finds the lowest position)
  const int warp = tid >> 5;
  for (int t0 = 0; t0 < T; ++t0) {
    const int c = s_wc[t0];
    bool first = true;
    for (int t1 = 0; t1 < t0 && first; ++t1) first = s_wc[t1] != c;
    if (!first) continue;
    if (c < 0) {  // no valid contingency at these timesteps
      for (int t = t0 + tid; t < T; t += blockDim.x)
        if (s_wc[t] == c) o.worst_mon[(size_t)tau * T + t] = -1;
      continue;
    }
    {
      Real vt[RMAX];
#pragma unroll
      for (int j = 0; j < RMAX; ++j) vt[j] = VtR[(size_t)j * C + c];
      for (int l = tid; l < M; l += blockDim.x) {
        Real zr[RMAX];
#pragma unroll
        for (int j = 0; j < RMAX; ++j) zr[j] = Zs[(size_t)j * Mp + l];
        s_col[l] = phi_entry<Real, RMAX>(PhiCM[(size_t)c * Mp + l], zr, vt, meta[Mp + l], a.cpos[l], c, meta[l]);
      }
    }
    __syncthreads();
    int k = 0;  // the matching timesteps, dealt out to the warps in turn
    for (int t = t0; t < T; ++t) {
      if (s_wc[t] != c) continue;
      if ((k++ % nw) != warp) continue;
      const Real st = sv[(size_t)t * C + c];
      const Real* pt = ptil + (size_t)t * Mp;
      Real v1 = (Real)-1, v2 = (Real)-1;
      int i1 = 0x7fffffff;
#pragma unroll 4
      for (int l = lane; l < M; l += 32) {  // 4 rows' loads in flight per lane
        const Real x = fabs(fma(s_col[l], st, pt[l]));
        if (x > v1) {
          v2 = v1;
          v1 = x;
          i1 = l;
        } else if (x > v2) {
          v2 = x;
        }
      }
      Real v = v1;
      for (int off = 16; off; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
      const Real thr = v - eps * fmax(v, (Real)1);
      int arg = v1 >= thr ? i1 : 0x7fffffff;
      if (__any_sync(0xffffffffu, v2 >= thr)) {  // two candidates in one lane: its lowest in the band
        arg = 0x7fffffff;
        for (int l = lane; l < M; l += 32)
          if (fabs(fma(s_col[l], st, pt[l])) >= thr) {
            arg = l;
            break;
          }
      }
      for (int off = 16; off; off >>= 1) arg = min(arg, __shfl_xor_sync(0xffffffffu, arg, off));
      if (lane == 0) o.worst_mon[(size_t)tau * T + t] = arg;
    }
    __syncthreads();  // before the next column overwrites s_col
  }
}

// ---------------------------------------------------------------------------
// injection candidates T_i (Sec. III-A, Eq. (8)), metric-first (Sec. III-C):
// expand every (timestep, candidate) into a virtual timestep, screen them with
// the max-only N-1 kernel, keep the argmin, gather its operands
// ---------------------------------------------------------------------------
// Candidate u adds sum_k d_k e_{pool_k}; by linearity (Eq. (3)) its scaled N-0
// flows are p~[t] + sum_k d_k p~[T + k] and its N-1 weights s[t] + sum_k d_k s[T + k]
// (the pool columns went through the same rank-r update as the timesteps).
template <class Real>
__global__ void k_var_expand(Args ap, int T, int U, const int* __restrict__ var_ptr, const int* __restrict__ var_k,
                             const double* __restrict__ var_delta, Real* __restrict__ ptv, Real* __restrict__ svv) {
  const int q = blockIdx.y;
  if (ap.qi[q].status != ST_OK) return;
  const int vt = blockIdx.x, t = vt / U, u = vt % U;
  const int Text = ap.T, Mp = ap.Mpad, M = ap.M, C = ap.C, TV = T * U;
  const Real* pt = static_cast<const Real*>(ap.ptil) + (size_t)q * Text * Mp;
  const Real* sv = static_cast<const Real*>(ap.s) + (size_t)q * Text * C;
  Real* po = ptv + ((size_t)q * TV + vt) * Mp;
  Real* so = svv + ((size_t)q * TV + vt) * C;
  const int k0 = var_ptr[u], k1 = var_ptr[u + 1];
  // the candidate's entries, staged once per block in the working precision (the per-row
  // conversions would otherwise occupy the FP64 pipe)
  constexpr int kStage = 64;
  __shared__ Real d_s[kStage];
  __shared__ int k_s[kStage];
  for (int k = k0 + threadIdx.x; k < k1 && k < k0 + kStage; k += blockDim.x) {
    d_s[k - k0] = (Real)var_delta[k];
    k_s[k - k0] = var_k[k];
  }
  __syncthreads();
  const int ns = min(k1 - k0, kStage);
  for (int l = threadIdx.x; l < M; l += blockDim.x) {
    Real v = pt[(size_t)t * Mp + l];
    for (int k = 0; k < ns; ++k) v = fma(d_s[k], pt[(size_t)(T + k_s[k]) * Mp + l], v);
    for (int k = k0 + ns; k < k1; ++k) v = fma((Real)var_delta[k], pt[(size_t)(T + var_k[k]) * Mp + l], v);
    po[l] = v;
  }
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    Real v = sv[(size_t)t * C + c];
    for (int k = 0; k < ns; ++k) v = fma(d_s[k], sv[(size_t)(T + k_s[k]) * C + c], v);
    for (int k = k0 + ns; k < k1; ++k) v = fma((Real)var_delta[k], sv[(size_t)(T + var_k[k]) * C + c], v);
    so[c] = v;
  }
}

// ---------------------------------------------------------------------------
// injection topologies t_i (Sec. III-A): the busbar of every injection at a
// split substation.  Moving injections of power q_i onto busbar B of split i
// changes only the right-hand side of that split's row of the r x r system:
// Sigma^T p_f = q instead of 0, so alpha' = alpha - K^{-1} q and
//   p_f' = p_f + Z K^{-1} q,   s' = s + (Z[c, :] / den_c) K^{-1} q.
// Z, K and Phi_f stay those of the branch topology: a candidate is a rank-r
// correction of the N-0 operands, then the candidate machinery of Eq. (8)
// (screen on the maximum, argmin, full N-1 of the winner) runs unchanged.
// ---------------------------------------------------------------------------
// Per slot: the eligible injections (at an effective split's bus, ascending
// index, at most 64) and their split rows; a topology with no candidate or a
// mask bit beyond its eligible injections becomes invalid.
__global__ __launch_bounds__(128) void k_ti_decode(GridDev g, BatchDev in, Args a, int n_inj,
                                                   const int* __restrict__ inj_bus, const int* __restrict__ ti_ptr,
                                                   const uint64_t* __restrict__ ti_mask, int* __restrict__ tiel,
                                                   int* __restrict__ tirow, int* __restrict__ nel) {
  __shared__ int sbus[kRMax];
  __shared__ int nsb, cnt;
  __shared__ int wcnt[4];
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  QInfo qi = a.qi[q];
  if (qi.status != ST_OK) {
    if (tid == 0) nel[q] = 0;
    return;
  }
  const int tau = qi.tau;
  if (tid == 0) {  // effective splits in decode order (the rows i < ks)
    int k = 0;
    for (int e = in.split_ptr[tau]; e < in.split_ptr[tau + 1]; ++e) {
      const int A = in.split_sub[e];
      const int deg = g.inc_ptr[A + 1] - g.inc_ptr[A], nb = __popcll(in.split_mask[e]);
      if (nb == 0 || nb == deg) continue;
      if (k < kRMax) sbus[k] = A;
      ++k;
    }
    nsb = k < kRMax ? k : kRMax;
    cnt = 0;
  }
  __syncthreads();
  for (int e0 = 0; e0 < n_inj; e0 += blockDim.x) {  // stable compaction, ascending injection index
    if (cnt >= 64) break;  // uniform: read after a barrier
    const int e = e0 + tid;
    int row = -1;
    if (e < n_inj) {
      const int b = inj_bus[e];
      for (int i = 0; i < nsb; ++i)
        if (sbus[i] == b) row = i;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, row >= 0);
    if (lane == 0) wcnt[wp] = __popc(bal);
    __syncthreads();
    int off = cnt + __popc(bal & ((1u << lane) - 1u));
    for (int w = 0; w < wp; ++w) off += wcnt[w];
    if (row >= 0 && off < 64) {
      tiel[(size_t)q * 64 + off] = e;
      tirow[(size_t)q * 64 + off] = row;
    }
    __syncthreads();
    if (tid == 0) cnt += wcnt[0] + wcnt[1] + wcnt[2] + wcnt[3];
    __syncthreads();
  }
  const int ne = cnt < 64 ? cnt : 64;
  const int u0 = ti_ptr[tau], u1 = ti_ptr[tau + 1];
  int bad = u1 <= u0;
  for (int u = u0 + tid; u < u1; u += blockDim.x) bad |= ne < 64 && (ti_mask[u] >> ne) != 0ull;
  bad = __syncthreads_or(bad);
  if (tid == 0) {
    nel[q] = ne;
    if (bad) {
      qi.status = ST_INVALID;
      a.qi[q] = qi;
    }
  }
}

// Operands of every (timestep, candidate): the rank-r correction above.  One
// block per (topology, timestep) and its candidates in groups of 16: the
// moved powers q and K^{-1} q of a group are formed in parallel, then each
// row's operands are loaded once for the group's 16 output rows (the kernel
// is bound by writing them).  A topology with fewer candidates than U repeats
// its first one (an exact tie that the argmin resolves to the original).  Rank
// positions r <= j < RMAX carry zero weights, which leave every sum exact.
template <class Real, int RMAX>
__global__ __launch_bounds__(256) void k_ti_expand(Args ap, int T, int U, const int* __restrict__ ti_ptr,
                                                   const uint64_t* __restrict__ ti_mask,
                                                   const double* __restrict__ inj_p, int n_inj,
                                                   const int* __restrict__ tiel, const int* __restrict__ tirow,
                                                   const int* __restrict__ nel, const Real* __restrict__ zcd,
                                                   Real* __restrict__ ptv, Real* __restrict__ svv) {
  constexpr int UG = 16;
  const int q = blockIdx.y, t = blockIdx.x;
  const QInfo qi = ap.qi[q];
  if (qi.status != ST_OK) return;
  __shared__ double qv[UG][kRMax];
  __shared__ Real w_s[UG][RMAX];
  __shared__ int row_s[64];
  __shared__ double ip_s[64];  // power of the topology's j-th eligible injection at timestep t
  const int Mp = ap.Mpad, M = ap.M, C = ap.C, TV = T * U, r = qi.r, ks = qi.ks, tid = threadIdx.x;
  const int u0 = ti_ptr[qi.tau], nu = ti_ptr[qi.tau + 1] - u0;
  const int ne = nel[q];
  for (int j = tid; j < ne; j += blockDim.x) {
    row_s[j] = tirow[(size_t)q * 64 + j];
    ip_s[j] = inj_p[(size_t)t * n_inj + tiel[(size_t)q * 64 + j]];
  }
  const double* Kinv = ap.Kinv + (size_t)q * kRMax * kRMax;
  const Real* pt = static_cast<const Real*>(ap.ptil) + (size_t)q * T * Mp;
  const Real* sv = static_cast<const Real*>(ap.s) + (size_t)q * T * C;
  const Real* Zs = static_cast<const Real*>(ap.Zs) + (size_t)q * kRMax * Mp;
  const Real* zc = zcd + (size_t)q * kRMax * C;
  for (int ug = 0; ug < U; ug += UG) {
    const int un = min(UG, U - ug);
    __syncthreads();  // the injections are staged; the previous group's weights are consumed
    for (int p = tid; p < UG * kRMax; p += blockDim.x) {  // q_i: power moved onto busbar B of split i
      const int uu = p / kRMax, i = p % kRMax, u = ug + uu;
      double acc = 0.0;
      if (uu < un && i < ks) {
        const uint64_t m = ti_mask[u0 + (u < nu ? u : 0)];
        for (int j = 0; j < ne; ++j)
          if (((m >> j) & 1ull) && row_s[j] == i) acc += ip_s[j];
      }
      qv[uu][i] = acc;
    }
    __syncthreads();
    for (int p = tid; p < UG * RMAX; p += blockDim.x) {  // w = K^{-1} q (only the split rows of q are nonzero)
      const int uu = p / RMAX, jj = p % RMAX;
      double x = 0.0;
      for (int i = 0; i < ks; ++i) x = fma(Kinv[jj * kRMax + i], qv[uu][i], x);
      w_s[uu][jj] = jj < r ? (Real)x : (Real)0;
    }
    __syncthreads();
    Real* po = ptv + ((size_t)q * TV + (size_t)t * U + ug) * Mp;
    Real* so = svv + ((size_t)q * TV + (size_t)t * U + ug) * C;
    for (int l = tid; l < M; l += blockDim.x) {
      Real z[RMAX];
#pragma unroll
      for (int j = 0; j < RMAX; ++j) z[j] = Zs[(size_t)j * Mp + l];  // zero rows beyond the rank
      const Real p0 = pt[(size_t)t * Mp + l];
      for (int uu = 0; uu < un; ++uu) {
        Real v = p0;
#pragma unroll
        for (int j = 0; j < RMAX; ++j) v = fma(z[j], w_s[uu][j], v);
        po[(size_t)uu * Mp + l] = v;
      }
    }
    for (int c = tid; c < C; c += blockDim.x) {
      Real z[RMAX];
#pragma unroll
      for (int j = 0; j < RMAX; ++j) z[j] = zc[(size_t)j * C + c];
      const Real s0 = sv[(size_t)t * C + c];
      for (int uu = 0; uu < un; ++uu) {
        Real v = s0;
#pragma unroll
        for (int j = 0; j < RMAX; ++j) v = fma(z[j], w_s[uu][j], v);
        so[(size_t)uu * C + c] = v;
      }
    }
  }
}

// argmin over candidates of the screened maximum loading (ties: lowest index);
// one warp per (slot, timestep)
template <class Real>
__global__ void k_var_select(Args av, int T, int U, int* __restrict__ best_u) {
  const int q = blockIdx.x, t = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (t >= T) return;
  if (av.qi[q].status != ST_OK) {
    if (lane == 0) best_u[(size_t)q * T + t] = -1;
    return;
  }
  const int TV = T * U;
  auto cand_max = [&](int u) {  // the candidate's maximum loading over the contingency blocks
    Real v = (Real)-1;
    for (int b = 0; b < av.ncb; ++b) {
      const size_t k = ((size_t)q * TV + (size_t)t * U + u) * av.ncb + b;
      if (av.parg[k] >= 0) v = fmax(v, static_cast<const Real*>(av.pmax)[k]);
    }
    return v < (Real)0 ? (Real)0 : v;  // no valid contingency: loading 0
  };
  Real bv = (Real)1e30;  // compared in the working precision
  for (int u = lane; u < U; u += 32) bv = fmin(bv, cand_max(u));
  for (int off = 16; off; off >>= 1) bv = fmin(bv, __shfl_xor_sync(0xffffffffu, bv, off));
  // Eq. (8): the lowest candidate index within the tie band of the smallest maximum
  const Real thr = bv + (Real)(av.tie_eps * fmax((double)bv, 1.0));
  int bu = 0x7fffffff;
  for (int u = lane; u < U; u += 32)
    if (cand_max(u) <= thr) {
      bu = u;
      break;
    }
  for (int off = 16; off; off >>= 1) bu = min(bu, __shfl_xor_sync(0xffffffffu, bu, off));
  if (lane == 0) best_u[(size_t)q * T + t] = bu;
}

// operands of the chosen candidate for the full N-1 pass, and its N-0 outputs
template <class Real>
__global__ void k_var_gather(Args af, int U, const Real* __restrict__ ptv, const Real* __restrict__ svv) {
  const int q = blockIdx.y, t = blockIdx.x;
  const QInfo qi = af.qi[q];
  if (qi.status != ST_OK) return;
  const int T = af.T, Mp = af.Mpad, M = af.M, C = af.C, TV = T * U;
  const int u = af.best_u[(size_t)q * T + t];
  const Real* pi = ptv + ((size_t)q * TV + (size_t)t * U + u) * Mp;
  const Real* si = svv + ((size_t)q * TV + (size_t)t * U + u) * C;
  Real* po = static_cast<Real*>(af.ptil) + ((size_t)q * T + t) * Mp;
  Real* so = static_cast<Real*>(af.s) + ((size_t)q * T + t) * C;
  Real m = 0;
  for (int l = threadIdx.x; l < M; l += blockDim.x) {
    const Real v = pi[l];
    po[l] = v;
    m = fmax(m, fabs(v));
    if (af.out.n0_flow) af.out.n0_flow[((size_t)qi.tau * T + t) * M + l] = (double)v / af.inv_lim[l];
  }
  for (int c = threadIdx.x; c < C; c += blockDim.x) so[c] = si[c];
  if (af.out.n0_max_loading) {
    __shared__ Real red[32];
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      Real x = red[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) x = fmax(x, red[w]);
      af.out.n0_max_loading[(size_t)qi.tau * T + t] = (double)x;
    }
  }
}


// ---------------------------------------------------------------------------
// learned screener in the loop (no counterpart in the paper): features of
// every (topology, timestep), top-k of the network's scores, the union over a
// topology's timesteps, then Eq. (5) over that union only
// ---------------------------------------------------------------------------
// Feature row (layout in screen.cuh): p_f / limit of the monitored branches,
// then the busbar bits of the topology's splits; zero for a topology that
// islands or is invalid.  Rows q T + t of the chunk, or tau T + t.
template <class Real>
__global__ void k_features(Args a, GridDev g, BatchDev in, const int* __restrict__ foff, int Fp,
                           __nv_bfloat16* __restrict__ X, int64_t ldx, int by_tau, uint8_t* __restrict__ status) {
  const int q = blockIdx.x;
  const QInfo qi = a.qi[q];
  const int T = a.T, M = a.M, Mp = a.Mpad;
  const bool ok = qi.status == ST_OK;
  const Real* ptil = static_cast<const Real*>(a.ptil) + (size_t)q * T * Mp;
  if (status && threadIdx.x == 0) status[qi.tau] = (uint8_t)qi.status;
  const int64_t r0 = by_tau ? (int64_t)qi.tau * T : (int64_t)q * T;
  for (int t = 0; t < T; ++t) {
    __nv_bfloat16* x = X + (r0 + t) * ldx;
    for (int i = threadIdx.x; i < Fp; i += blockDim.x)
      x[i] = __float2bfloat16_rn((ok && i < M) ? (float)ptil[(size_t)t * Mp + i] : 0.f);
  }
  __syncthreads();
  if (!ok) return;
  for (int k = in.split_ptr[qi.tau]; k < in.split_ptr[qi.tau + 1]; ++k) {
    const int sub = in.split_sub[k];
    const uint64_t mask = in.split_mask[k];
    const int o = foff[sub];
    if (o < 0) continue;
    const int deg = g.inc_ptr[sub + 1] - g.inc_ptr[sub];
    for (int idx = threadIdx.x; idx < deg * T; idx += blockDim.x) {
      const int j = idx % deg, t = idx / deg;
      X[(r0 + t) * ldx + o + j] = __float2bfloat16_rn((float)((mask >> j) & 1ull));
    }
  }
}

// Top k of the scores of every (topology, timestep) row (one warp per row,
// ties to the lower contingency position); the union over the timesteps of a
// topology goes to a bit mask, the request for the full N-1 to fb[q] when the
// k-th score still exceeds the fallback threshold.
template <int NPL>
__global__ void k_select(const QInfo* __restrict__ qinfo, int nq, int T, int C, const float* __restrict__ Z,
                         int ldz, int k, uint32_t fb_key, uint32_t min_key, uint32_t* __restrict__ selmask, int W,
                         uint8_t* __restrict__ fb, int32_t* __restrict__ pred) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= (int64_t)nq * T) return;
  const int q = (int)(row / T), t = (int)(row % T);
  const QInfo qi = qinfo[q];
  int32_t* pr = pred ? pred + ((int64_t)qi.tau * T + t) * k : nullptr;
  if (qi.status != ST_OK) {  // nothing is evaluated: an all -1 row
    if (pr)
      for (int j = lane; j < k; j += 32) pr[j] = -1;
    return;
  }
  uint32_t key[NPL];
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const int c = lane + 32 * i;
    key[i] = c < C ? float_key(Z[row * ldz + c]) : 0u;
  }
  const int kk = k < C ? k : C;
  bool sel[NPL];
  uint32_t thr;
  warp_top_k<NPL>(key, kk, sel, thr);
  int off = 0;
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const uint32_t b = __ballot_sync(0xffffffffu, sel[i]);
    // the evaluated set: the top k, and every score above the minimum logit (not reported in pred)
    const uint32_t bx = __ballot_sync(0xffffffffu, lane + 32 * i < C && key[i] > min_key);
    if (lane == 0 && (b | bx)) atomicOr(&selmask[(size_t)q * W + i], b | bx);
    if (pr && sel[i]) pr[off + __popc(b & ((1u << lane) - 1u))] = lane + 32 * i;
    off += __popc(b);
  }
  if (pr)
    for (int j = kk + lane; j < k; j += 32) pr[j] = -1;
  if (lane == 0 && thr > fb_key) fb[q] = 1;
}

// Per topology (one warp): the selected contingencies in ascending order
// (all of them after a fallback), their count, and one work item per
// 64 of them for the N-1 kernel.
// Every valid contingency of a topology (not outaged, not islanding it; the
// base-grid bridges are already outside [0, C_eff)), compacted in internal
// order for the grid mode of the register-tiled N-1 kernel, so that the
// contingencies a topology's splits turn into bridges are never computed.
// Their per-contingency maxima (when requested) are -1 here.  One warp per slot.
__global__ void k_valid_compact(Args a, int* __restrict__ csel, int* __restrict__ nsel) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (q >= a.nq) return;
  const QInfo qi = a.qi[q];
  if (qi.status != ST_OK) {
    if (lane == 0) nsel[q] = 0;
    return;
  }
  const int C = a.C, T = a.T;
  const uint8_t* valid = a.valid + (size_t)q * C;
  float* cm = a.out.n1_cont_max;
  int base = 0;
  for (int c0 = 0; c0 < a.C_eff; c0 += 32) {
    const int c = c0 + lane;
    const bool v = c < a.C_eff && valid[c];
    const uint32_t m = __ballot_sync(0xffffffffu, v);
    if (v) csel[(size_t)q * C + base + __popc(m & ((1u << lane) - 1u))] = c;
    base += __popc(m);
    if (cm && c < a.C_eff && !v)
      for (int t = 0; t < T; ++t) cm[((size_t)qi.tau * T + t) * C + a.cont_pos[c]] = -1.f;
    if (a.cmr && c < a.C_eff && !v)  // the tie band's maxima (FP32 forms): skipped
      for (int t = 0; t < T; ++t) static_cast<float*>(a.cmr)[((size_t)q * T + t) * C + c] = -1.f;
  }
  if (lane == 0) nsel[q] = base;
}

__global__ void k_compact(const QInfo* __restrict__ qinfo, int nq, int C, int C_eff, const int* __restrict__ cont_inv,
                          int W, const uint32_t* __restrict__ selmask, const uint8_t* __restrict__ fb,
                          int* __restrict__ csel, int* __restrict__ nsel, int* __restrict__ work,
                          int* __restrict__ nwork, int32_t* __restrict__ n_eval, uint8_t* __restrict__ fb_out,
                          uint32_t* __restrict__ ev_out) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (q >= nq) return;
  const QInfo qi = qinfo[q];
  const bool ok = qi.status == ST_OK;
  const bool full = ok && fb[q];
  int base = 0;
  if (ok) {
    for (int w0 = 0; w0 < W; w0 += 32) {
      const int w = w0 + lane;
      uint32_t word = 0;
      if (w < W) {
        word = full ? 0xffffffffu : selmask[(size_t)q * W + w];
        const int rem = C - 32 * w;
        if (rem < 32) word &= (1u << rem) - 1u;
        for (uint32_t x = word; x; x &= x - 1u)  // base-grid bridges are never evaluated
          if (cont_inv[32 * w + __ffs(x) - 1] >= C_eff) word &= ~(1u << (__ffs(x) - 1));
        if (ev_out) ev_out[(size_t)qi.tau * W + w] = word;  // the evaluated set, caller's positions
      }
      const int cnt = __popc(word);
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      int pos = base + incl - cnt;
      while (word) {
        const int bit = __ffs(word) - 1;
        word &= word - 1u;
        csel[(size_t)q * C + pos++] = cont_inv[32 * w + bit];  // ascending: the order keeps the caller's
      }
      base += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  if (!ok && ev_out)  // islanded or invalid: nothing evaluated
    for (int w = lane; w < W; w += 32) ev_out[(size_t)qi.tau * W + w] = 0u;
  if (lane == 0) {
    nsel[q] = base;
    const int nb = (base + 63) / 64;
    if (nb) {
      const int w = atomicAdd(nwork, nb);
      for (int j = 0; j < nb; ++j) work[w + j] = q * 64 + j;
    }
    if (n_eval) n_eval[qi.tau] = base;
    if (fb_out) fb_out[qi.tau] = full ? 1 : 0;
  }
}

// Phi[mon, cont] / limit transposed to [cont][Mpad] (zero padding rows) for
// the selected-contingency N-1: a contingency's column becomes contiguous.
template <class Real>
__global__ void k_phi_cm(const Real* __restrict__ PhiMC, int M, int C, int ldc, int Mp, Real* __restrict__ PhiCM) {
  __shared__ Real tile[32][33];
  const int l0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int l = l0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (l < M && c < C) ? PhiMC[(size_t)l * ldc + c] : (Real)0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, l = l0 + threadIdx.x;
    if (c < C && l < Mp) PhiCM[(size_t)c * Mp + l] = tile[threadIdx.x][i];
  }
}

// Eq. (5) over the selected contingencies of each work item (topology, 64 of
// its selected contingencies), one contingency per thread; the same arithmetic
// and partial-result layout as the all-contingency kernel, with Phi read as
// contiguous rows of the transposed factors.  Blocks loop over the work list.
template <class Real, int TT, int RMAX, int LT>
__global__ __launch_bounds__(64) void k_n1_sel(Args a, const Real* __restrict__ PhiCM, const int* __restrict__ csel,
                                               const int* __restrict__ nsel, const int* __restrict__ work,
                                               const int* __restrict__ nwork, int t0) {
  const int tid = threadIdx.x, M = a.M, C = a.C, T = a.T, Mp = a.Mpad;
  __shared__ __align__(16) Real zs[LT][RMAX];
  __shared__ __align__(16) Real pt[LT][TT];
  __shared__ Real dg[LT], rm[LT];
  __shared__ int cp[LT];
  __shared__ Real rv[2];  // maxima compared in the working precision (no FP64-pipe work in the FP32 form)
  __shared__ double ro[2];
  __shared__ int ra[2];
  const int total = *nwork;
  for (int wi = blockIdx.x; wi < total; wi += gridDim.x) {
    const int item = work[wi], q = item >> 6, cb = item & 63;
    const QInfo qi = a.qi[q];
    const int jj = cb * 64 + tid;
    const bool cin = jj < nsel[q];
    const int c = csel[(size_t)q * C + (cin ? jj : 0)];
    const Real* Zs = static_cast<const Real*>(a.Zs) + (size_t)q * kRMax * Mp;
    const Real* ptil = static_cast<const Real*>(a.ptil) + (size_t)q * T * Mp;
    const Real* meta = static_cast<const Real*>(a.diagv) + (size_t)q * 4 * Mp;
    const Real* VtR = static_cast<const Real*>(a.VtR) + (size_t)q * kRMax * C;
    const Real* sv = static_cast<const Real*>(a.s) + (size_t)q * T * C;
    const Real* prow = PhiCM + (size_t)c * Mp;
    Real vt[RMAX];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) vt[j] = VtR[(size_t)j * C + c];
    Real s[TT], mx[TT], ov[TT];
#pragma unroll
    for (int t = 0; t < TT; ++t) {
      s[t] = (cin && t0 + t < T) ? sv[(size_t)(t0 + t) * C + c] : (Real)0;
      mx[t] = 0;
      ov[t] = 0;
    }
    for (int l0 = 0; l0 < M; l0 += LT) {
      __syncthreads();
      for (int idx = tid; idx < LT * RMAX; idx += 64) {
        const int i = idx % LT, j = idx / LT, l = l0 + i;
        zs[i][j] = (l < M) ? Zs[(size_t)j * Mp + l] : (Real)0;
      }
      for (int idx = tid; idx < LT * TT; idx += 64) {
        const int i = idx % LT, t = idx / LT, l = l0 + i;
        pt[i][t] = (l < M && t0 + t < T) ? ptil[(size_t)(t0 + t) * Mp + l] : (Real)0;
      }
      for (int i = tid; i < LT; i += 64) {
        const int l = l0 + i;
        dg[i] = (l < M) ? meta[l] : (Real)0;
        rm[i] = (l < M) ? meta[Mp + l] : (Real)0;
        cp[i] = (l < M) ? a.cpos[l] : -1;
      }
      __syncthreads();
      Real base[LT];  // l0 + LT <= Mp: the padded rows of PhiCM are zero
      if constexpr (sizeof(Real) == 4) {
#pragma unroll
        for (int i = 0; i < LT; i += 4) {
          const float4 v = *reinterpret_cast<const float4*>(prow + l0 + i);
          base[i] = v.x;
          base[i + 1] = v.y;
          base[i + 2] = v.z;
          base[i + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < LT; i += 2) {
          const double2 v = *reinterpret_cast<const double2*>(prow + l0 + i);
          base[i] = v.x;
          base[i + 1] = v.y;
        }
      }
      Real phi[LT];
#pragma unroll
      for (int i = 0; i < LT; ++i) phi[i] = phi_entry<Real, RMAX>(base[i], zs[i], vt, rm[i], cp[i], c, dg[i]);
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        const Real st = s[t];
#pragma unroll
        for (int i = 0; i < LT; ++i) Acc<Real>::add(mx[t], ov[t], fma(phi[i], st, pt[i][t]));
      }
    }
    const bool ok = cin && a.valid[(size_t)q * C + c];
    if (a.out.n1_cont_max && cin) {
#pragma unroll
      for (int t = 0; t < TT; ++t)
        if (t0 + t < T) a.out.n1_cont_max[((size_t)qi.tau * T + t0 + t) * C + a.cont_pos[c]] = ok ? (float)mx[t] : -1.f;
    }
    const int lane = tid & 31, w = tid >> 5;
#pragma unroll
    for (int t = 0; t < TT; ++t) {
      if (t0 + t < T) {  // uniform over the block
        Real v = ok ? mx[t] : (Real)-1;
        int arg = ok ? c : 0x7fffffff;
        double o = ok ? (double)ov[t] * Acc<Real>::ovl_scale() : 0.0;
#pragma unroll
        for (int off = 16; off; off >>= 1) {
          const Real v2 = __shfl_xor_sync(0xffffffffu, v, off);
          const int a2 = __shfl_xor_sync(0xffffffffu, arg, off);
          o += __shfl_xor_sync(0xffffffffu, o, off);
          if (v2 > v || (v2 == v && a2 < arg)) {
            v = v2;
            arg = a2;
          }
        }
        if (lane == 0) {
          rv[w] = v;
          ra[w] = arg;
          ro[w] = o;
        }
        __syncthreads();
        if (tid == 0) {
          Real bv = rv[0];
          int ba = ra[0];
          if (rv[1] > bv || (rv[1] == bv && ra[1] < ba)) {
            bv = rv[1];
            ba = ra[1];
          }
          const size_t o2 = ((size_t)q * T + t0 + t) * a.ncb + cb;
          static_cast<Real*>(a.pmax)[o2] = bv;
          a.parg[o2] = (bv < (Real)0) ? -1 : ba;
          a.povl[o2] = ro[0] + ro[1];
        }
        __syncthreads();
      }
    }
  }
}


// ---------------------------------------------------------------------------
// sparse worst results (agg_i, Sec. III-A): per (topology, timestep) the top k
// N-1 cases by maximum loading, each with its most loaded monitored branch,
// from the per-contingency maxima of the N-1 kernel (one warp per timestep)
// ---------------------------------------------------------------------------
// The top kk <= 32 of a warp's keys by (key descending, position ascending), as
// warp_top_k selects them, when few keys reach the kk-th largest lane maximum:
// the kk lanes with the largest maxima hold kk keys at least that large, so
// every selected key is among those candidates, which are then ranked exactly.
// Writes the selected positions (ascending) and their values to sp / sv and
// returns false, having written nothing, when more than 64 candidates qualify.
template <int NPL>
__device__ __forceinline__ bool warp_top_few(const uint32_t (&key)[NPL], int kk, const float* row, uint32_t* ck,
                                             int* cpos, int* sp, float* sv) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t lm = 0;
#pragma unroll
  for (int i = 0; i < NPL; ++i) lm = key[i] > lm ? key[i] : lm;
  int rk = 0;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const uint32_t o = __shfl_sync(0xffffffffu, lm, j);
    rk += (o > lm) || (o == lm && j < lane);
  }
  const uint32_t bk = __ballot_sync(0xffffffffu, rk == kk - 1);  // one lane: ranks are distinct
  const uint32_t thr = __shfl_sync(0xffffffffu, lm, __ffs(bk) - 1);
  int n = 0;
#pragma unroll
  for (int i = 0; i < NPL; ++i) {  // candidates in ascending position
    const bool c = key[i] >= thr;
    const uint32_t b = __ballot_sync(0xffffffffu, c);
    const int j = n + __popc(b & lt);
    if (c && j < 64) {
      ck[j] = key[i];
      cpos[j] = lane + 32 * i;
    }
    n += __popc(b);
  }
  if (n > 64) return false;
  __syncwarp();
  bool sel[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = lane + 32 * h;
    int r = 0;
    if (j < n) {
      const uint32_t kj = ck[j];
      for (int m = 0; m < n; ++m) r += ck[m] > kj || (ck[m] == kj && m < j);  // m < j: lower position
    }
    sel[h] = j < n && r < kk;
  }
  const uint32_t b0 = __ballot_sync(0xffffffffu, sel[0]), b1 = __ballot_sync(0xffffffffu, sel[1]);
  int pos0 = 0, pos1 = 0;
  if (sel[0]) pos0 = cpos[lane];
  if (sel[1]) pos1 = cpos[lane + 32];
  __syncwarp();
  if (sel[0]) {
    const int o = __popc(b0 & lt);
    sp[o] = pos0;
    sv[o] = row[pos0];
  }
  if (sel[1]) {
    const int o = __popc(b0) + __popc(b1 & lt);
    sp[o] = pos1;
    sv[o] = row[pos1];
  }
  return true;
}

// The kk highest per-contingency maxima of one (topology, timestep) row (one
// warp): their values and positions in ov / op, by descending loading with
// ties to the lower position.  ck, cq, sp, sv: 64-entry scratch of the warp.
template <int NPL>
__device__ __forceinline__ void select_cases(const float* __restrict__ row, int C, int kk, uint32_t* ck, int* cq,
                                             int* sp, float* sv, float* ov, int* op) {
  const int lane = threadIdx.x & 31;
  uint32_t key[NPL];
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const int p = lane + 32 * i;
    key[i] = p < C ? float_key(row[p]) : 0u;
  }
  if (kk < 1 || kk > 32 || !warp_top_few<NPL>(key, kk, row, ck, cq, sp, sv)) {  // warp-uniform
    bool sel[NPL];
    uint32_t thr;
    warp_top_k<NPL>(key, kk, sel, thr);
    int off = 0;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {  // the selected cases in ascending position
      const uint32_t b = __ballot_sync(0xffffffffu, sel[i]);
      if (sel[i]) {
        const int j = off + __popc(b & ((1u << lane) - 1u));
        sp[j] = lane + 32 * i;
        sv[j] = row[lane + 32 * i];
      }
      off += __popc(b);
    }
  }
  __syncwarp();
  for (int j = lane; j < kk; j += 32) {  // descending loading, ties to the lower position
    const float v = sv[j];
    const int p = sp[j];
    int rank = 0;
    for (int m = 0; m < kk; ++m) rank += sv[m] > v || (sv[m] == v && sp[m] < p);
    ov[rank] = v;
    op[rank] = p;
  }
  __syncwarp();
}

// 7 resident blocks per SM (72 registers, a few bytes spilled in the select):
// the column pass waits on its loads, and more warps in flight hide them better
// than 5 blocks with no spill (measured 2.04 against 2.64 ms on the 500-bus study)
template <class Real, int RMAX, int NPL>
__global__ __launch_bounds__(128, 7) void k_topcases(Args a, const float* __restrict__ cmax,
                                                   const int* __restrict__ cont_inv, const Real* __restrict__ PhiCM,
                                                   int k) {
  __shared__ float sv_[4][64];
  __shared__ int sp_[4][64];
  __shared__ Real vts[4][8][RMAX];  // Vt columns of the 8 cases of a pass, per warp
  __shared__ float ov_[4][64];
  __shared__ int op_[4][64];
  const int q = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.y * 4 + w;
  const QInfo qi = a.qi[q];
  const int T = a.T, M = a.M, C = a.C, Mp = a.Mpad, tau = qi.tau;
  if (t >= T) return;
  const dcflow_results& o = a.out;
  const size_t ob = ((size_t)tau * T + t) * k;
  if (qi.status != ST_OK) {
    for (int j = lane; j < k; j += 32) {
      o.top_cont[ob + j] = -1;
      o.top_mon[ob + j] = -1;
      o.top_loading[ob + j] = 0.f;
    }
    return;
  }
  const int kk = k < C ? k : C;
  __shared__ uint32_t ck_[4][64];
  __shared__ int cq_[4][64];
  select_cases<NPL>(cmax + ((size_t)tau * T + t) * C, C, kk, ck_[w], cq_[w], sp_[w], sv_[w], ov_[w], op_[w]);
  const Real* Zs = static_cast<const Real*>(a.Zs) + (size_t)q * kRMax * Mp;
  const Real* ptil = static_cast<const Real*>(a.ptil) + (size_t)q * T * Mp;
  const Real* meta = static_cast<const Real*>(a.diagv) + (size_t)q * 4 * Mp;
  const Real* VtR = static_cast<const Real*>(a.VtR) + (size_t)q * kRMax * C;
  const Real* sv = static_cast<const Real*>(a.s) + (size_t)q * T * C;
  // the most loaded monitored branch of every case: the columns recomputed as in
  // the N-1 kernel, 8 cases per pass over the rows (the row operands are shared)
  constexpr int KG = 8;
  for (int j0 = 0; j0 < k; j0 += KG) {
    int cj[KG];
    Real stj[KG], vr[KG];
    int arg[KG];
#pragma unroll
    for (int g = 0; g < KG; ++g) {
      const int j = j0 + g;
      const bool valid = j < kk && ov_[w][j] >= 0.f;
      cj[g] = valid ? cont_inv[op_[w][j]] : -1;
      stj[g] = cj[g] >= 0 ? sv[(size_t)t * C + cj[g]] : (Real)0;
      vr[g] = (Real)-1;
      arg[g] = 0x7fffffff;
    }
    __syncwarp();
    for (int p = lane; p < KG * RMAX; p += 32) {
      const int g = p / RMAX, jj = p % RMAX;
      vts[w][g][jj] = cj[g] >= 0 ? VtR[(size_t)jj * C + cj[g]] : (Real)0;
    }
    __syncwarp();
    for (int l = lane; l < M; l += 32) {
      Real zr[RMAX];
#pragma unroll
      for (int jj = 0; jj < RMAX; ++jj) zr[jj] = Zs[(size_t)jj * Mp + l];
      const Real pt = ptil[(size_t)t * Mp + l], rm = meta[Mp + l], dg = meta[l];
      const int cp = a.cpos[l];
#pragma unroll
      for (int g = 0; g < KG; ++g) {
        if (cj[g] < 0) continue;
        const Real ph = phi_entry<Real, RMAX>(PhiCM[(size_t)cj[g] * Mp + l], zr, vts[w][g], rm, cp, cj[g], dg);
        const Real x = fabs(fma(ph, stj[g], pt));
        if (x > vr[g]) {
          vr[g] = x;
          arg[g] = l;
        }
      }
    }
#pragma unroll
    for (int g = 0; g < KG; ++g) {
      Real v = vr[g];  // compared in the working precision
      int ar = arg[g];
      for (int off2 = 16; off2; off2 >>= 1) {
        const Real v2 = __shfl_xor_sync(0xffffffffu, v, off2);
        const int a2 = __shfl_xor_sync(0xffffffffu, ar, off2);
        if (v2 > v || (v2 == v && a2 < ar)) {
          v = v2;
          ar = a2;
        }
      }
      const int j = j0 + g;
      if (lane == 0 && j < k) {
        const bool valid = cj[g] >= 0;
        o.top_cont[ob + j] = valid ? op_[w][j] : -1;
        o.top_mon[ob + j] = valid ? ar : -1;
        o.top_loading[ob + j] = valid ? ov_[w][j] : 0.f;
      }
    }
  }
}


// The same per topology (one block of 8 warps): the top k of every timestep
// (one warp per timestep), then the distinct selected contingencies' Phi_f
// columns, up to `cbm` at a time, into shared memory ([column][monitored row],
// the N-1 kernels' arithmetic), and every case of those contingencies against
// them (the cases in turn over the warps: the most loaded monitored branch,
// the lowest on ties).  The k cases of the timesteps of a topology share few
// contingencies, so the column builds fall from one per case to one per
// distinct contingency.  Timesteps in chunks of 32.
template <class Real, int RMAX, int NPL>
__global__ __launch_bounds__(256) void k_topcols(Args a, const float* __restrict__ cmax,
                                                 const int* __restrict__ cont_inv, const Real* __restrict__ PhiCM,
                                                 int k, int cbm) {
  constexpr int NW = 8, TCH = 32, CBX = 16;
  __shared__ float sv_[NW][64];
  __shared__ int sp_[NW][64];
  __shared__ uint32_t ck_[NW][64];
  __shared__ int cq_[NW][64];
  __shared__ float ov_[NW][64];
  __shared__ int op_[NW][64];
  __shared__ int16_t cc_s[TCH * 64];  // internal contingency of case (timestep of the chunk, rank), or -1
  __shared__ int16_t rk_s[TCH * 64];  // its position among the chunk's distinct contingencies
  __shared__ int16_t dl_s[2048];      // the chunk's distinct contingencies, ascending
  __shared__ uint32_t cmask[64];      // at most 2048 contingencies
  __shared__ int wpre[64];            // distinct contingencies below each mask word
  __shared__ Real vt_s[CBX][RMAX];
  __shared__ int nd_s;
  extern __shared__ __align__(16) unsigned char tc_dyn[];
  Real* s_col = reinterpret_cast<Real*>(tc_dyn);  // [cbm][M]
  const int q = blockIdx.x, tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const QInfo qi = a.qi[q];
  const int T = a.T, M = a.M, C = a.C, Mp = a.Mpad, tau = qi.tau;
  const dcflow_results& o = a.out;
  if (qi.status != ST_OK) {
    for (size_t i = tid; i < (size_t)T * k; i += blockDim.x) {
      o.top_cont[(size_t)tau * T * k + i] = -1;
      o.top_mon[(size_t)tau * T * k + i] = -1;
      o.top_loading[(size_t)tau * T * k + i] = 0.f;
    }
    return;
  }
  const int kk = k < C ? k : C;
  const Real* Zs = static_cast<const Real*>(a.Zs) + (size_t)q * kRMax * Mp;
  const Real* ptil = static_cast<const Real*>(a.ptil) + (size_t)q * T * Mp;
  const Real* meta = static_cast<const Real*>(a.diagv) + (size_t)q * 4 * Mp;
  const Real* VtR = static_cast<const Real*>(a.VtR) + (size_t)q * kRMax * C;
  const Real* sv = static_cast<const Real*>(a.s) + (size_t)q * T * C;
  for (int t0 = 0; t0 < T; t0 += TCH) {
    const int tn = min(TCH, T - t0), ne = tn * k;
    __syncthreads();  // the previous chunk's lists and columns are consumed
    if (tid < 64) cmask[tid] = 0u;
    __syncthreads();
    for (int tl = w; tl < tn; tl += NW) {
      const int t = t0 + tl;
      select_cases<NPL>(cmax + ((size_t)tau * T + t) * C, C, kk, ck_[w], cq_[w], sp_[w], sv_[w], ov_[w], op_[w]);
      const size_t ob = ((size_t)tau * T + t) * k;
      for (int j = lane; j < k; j += 32) {
        const bool valid = j < kk && ov_[w][j] >= 0.f;
        const int c = valid ? cont_inv[op_[w][j]] : -1;
        cc_s[tl * 64 + j] = (int16_t)c;
        o.top_cont[ob + j] = valid ? op_[w][j] : -1;
        o.top_loading[ob + j] = valid ? ov_[w][j] : 0.f;
        if (!valid) o.top_mon[ob + j] = -1;
        if (c >= 0) atomicOr(&cmask[c >> 5], 1u << (c & 31));
      }
      __syncwarp();  // the next timestep's selection rewrites the warp's lists
    }
    __syncthreads();
    if (w == 0) {  // the distinct contingencies in ascending order
      int base = 0;
      for (int w0 = 0; w0 < 64; w0 += 32) {
        const uint32_t m = cmask[w0 + lane];
        const int cnt = __popc(m);
        int inc = cnt;
        for (int off = 1; off < 32; off <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, inc, off);
          if (lane >= off) inc += y;
        }
        int pos = base + inc - cnt;
        wpre[w0 + lane] = pos;
        for (uint32_t b = m; b; b &= b - 1u) dl_s[pos++] = (int16_t)((w0 + lane) * 32 + __ffs(b) - 1);
        base += __shfl_sync(0xffffffffu, inc, 31);
      }
      if (lane == 0) nd_s = base;
    }
    __syncthreads();
    for (int e = tid; e < ne; e += blockDim.x) {
      const int c = cc_s[(e / k) * 64 + e % k];
      rk_s[e] = (int16_t)(c < 0 ? -1 : wpre[c >> 5] + __popc(cmask[c >> 5] & ((1u << (c & 31)) - 1u)));
    }
    const int nd = nd_s;
    for (int d0 = 0; d0 < nd; d0 += cbm) {
      const int dn = min(cbm, nd - d0);
      __syncthreads();  // the previous batch's cases are evaluated (and the ranks written)
      for (int i = tid; i < dn * RMAX; i += blockDim.x)
        vt_s[i / RMAX][i % RMAX] = VtR[(size_t)(i % RMAX) * C + dl_s[d0 + i / RMAX]];
      __syncthreads();
      for (int i = tid; i < dn * M; i += blockDim.x) {
        const int dd = i / M, l = i % M, c = dl_s[d0 + dd];
        Real zr[RMAX];
#pragma unroll
        for (int j = 0; j < RMAX; ++j) zr[j] = Zs[(size_t)j * Mp + l];
        s_col[i] = phi_entry<Real, RMAX>(PhiCM[(size_t)c * Mp + l], zr, vt_s[dd], meta[Mp + l], a.cpos[l], c, meta[l]);
      }
      __syncthreads();
      int nm = 0;  // matches so far (warp-uniform): match i goes to warp i % NW
      for (int e0 = 0; e0 < ne; e0 += 32) {
        const int e = e0 + lane;
        const int rk = e < ne ? rk_s[e] : -1;
        const uint32_t bal = __ballot_sync(0xffffffffu, rk >= d0 && rk < d0 + dn);
        for (uint32_t b = bal; b; b &= b - 1u, ++nm) {
          if (nm % NW != w) continue;
          const int ec = e0 + __ffs(b) - 1, tl = ec / k, j = ec % k, t = t0 + tl;
          const int c = cc_s[tl * 64 + j];
          const Real* col = s_col + (size_t)(rk_s[ec] - d0) * M;
          const Real st = sv[(size_t)t * C + c];
          Real v = (Real)-1;
          int arg = 0x7fffffff;
          for (int l = lane; l < M; l += 32) {
            const Real x = fabs(fma(col[l], st, ptil[(size_t)t * Mp + l]));
            if (x > v) {
              v = x;
              arg = l;
            }
          }
          for (int off = 16; off; off >>= 1) {
            const Real v2 = __shfl_xor_sync(0xffffffffu, v, off);
            const int a2 = __shfl_xor_sync(0xffffffffu, arg, off);
            if (v2 > v || (v2 == v && a2 < arg)) {
              v = v2;
              arg = a2;
            }
          }
          if (lane == 0) o.top_mon[((size_t)tau * T + t) * k + j] = arg;
        }
      }
    }
  }
}

// The top-k pass after the tracking N-1 pass (one warp per timestep, as
// k_topcases): each case's maximum lies in the 16-row tile that pass recorded,
// so its most loaded monitored branch comes from those 16 rows (half a warp
// per case, two cases at a time; the lowest row on ties).  A case of the short
// contingency remainder (no N-1 block, no tile) rebuilds its whole column.
template <class Real, int RMAX, int NPL>
__global__ __launch_bounds__(128) void k_topcases_tile(Args a, const float* __restrict__ cmax,
                                                       const int* __restrict__ cont_inv,
                                                       const Real* __restrict__ PhiCM, int k) {
  __shared__ float sv_[4][64];
  __shared__ int sp_[4][64];
  __shared__ uint32_t ck_[4][64];
  __shared__ int cq_[4][64];
  __shared__ float ov_[4][64];
  __shared__ int op_[4][64];
  const int q = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.y * 4 + w;
  const QInfo qi = a.qi[q];
  const int T = a.T, M = a.M, C = a.C, Mp = a.Mpad, tau = qi.tau;
  if (t >= T) return;
  const dcflow_results& o = a.out;
  const size_t ob = ((size_t)tau * T + t) * k;
  if (qi.status != ST_OK) {
    for (int j = lane; j < k; j += 32) {
      o.top_cont[ob + j] = -1;
      o.top_mon[ob + j] = -1;
      o.top_loading[ob + j] = 0.f;
    }
    return;
  }
  const int kk = k < C ? k : C;
  select_cases<NPL>(cmax + ((size_t)tau * T + t) * C, C, kk, ck_[w], cq_[w], sp_[w], sv_[w], ov_[w], op_[w]);
  const Real* Zs = static_cast<const Real*>(a.Zs) + (size_t)q * kRMax * Mp;
  const Real* ptil = static_cast<const Real*>(a.ptil) + (size_t)q * T * Mp + (size_t)t * Mp;
  const Real* meta = static_cast<const Real*>(a.diagv) + (size_t)q * 4 * Mp;
  const Real* VtR = static_cast<const Real*>(a.VtR) + (size_t)q * kRMax * C;
  const Real* sv = static_cast<const Real*>(a.s) + (size_t)q * T * C + (size_t)t * C;
  const uint16_t* tile = a.tile + ((size_t)q * T + t) * C;
  const int h = lane >> 4, r16 = lane & 15;
  bool rem = false;  // some case lies in the remainder (warp-uniform after the ballot below)
  for (int j0 = 0; j0 < k; j0 += 2) {
    const int j = j0 + h;
    const bool valid = j < kk && ov_[w][j] >= 0.f;
    const int c = valid ? cont_inv[op_[w][j]] : -1;
    const bool tiled = c >= 0 && c < a.c_rem;
    rem |= c >= a.c_rem;
    Real v = (Real)-1;
    int arg = 0x7fffffff;
    if (tiled) {
      const int l = 16 * (int)tile[c] + r16;
      if (l < M) {
        Real vt[RMAX], zr[RMAX];
#pragma unroll
        for (int jj = 0; jj < RMAX; ++jj) {
          vt[jj] = VtR[(size_t)jj * C + c];
          zr[jj] = Zs[(size_t)jj * Mp + l];
        }
        const Real ph = phi_entry<Real, RMAX>(PhiCM[(size_t)c * Mp + l], zr, vt, meta[Mp + l], a.cpos[l], c, meta[l]);
        v = fabs(fma(ph, sv[c], ptil[l]));
        arg = l;
      }
    }
    for (int off = 8; off; off >>= 1) {  // within the half warp
      const Real v2 = __shfl_xor_sync(0xffffffffu, v, off);
      const int a2 = __shfl_xor_sync(0xffffffffu, arg, off);
      if (v2 > v || (v2 == v && a2 < arg)) {
        v = v2;
        arg = a2;
      }
    }
    if (r16 == 0 && j < k) {
      o.top_cont[ob + j] = valid ? op_[w][j] : -1;
      o.top_mon[ob + j] = tiled ? arg : -1;
      o.top_loading[ob + j] = valid ? ov_[w][j] : 0.f;
    }
  }
  if (!__any_sync(0xffffffffu, rem)) return;
  __syncwarp();  // the half-warps' writes above come first
  for (int j = 0; j < kk; ++j) {  // the remainder's cases: the whole column
    if (ov_[w][j] < 0.f) continue;
    const int c = cont_inv[op_[w][j]];
    if (c < a.c_rem) continue;
    Real vt[RMAX];
#pragma unroll
    for (int jj = 0; jj < RMAX; ++jj) vt[jj] = VtR[(size_t)jj * C + c];
    Real v = (Real)-1;
    int arg = 0x7fffffff;
    for (int l = lane; l < M; l += 32) {
      Real zr[RMAX];
#pragma unroll
      for (int jj = 0; jj < RMAX; ++jj) zr[jj] = Zs[(size_t)jj * Mp + l];
      const Real ph = phi_entry<Real, RMAX>(PhiCM[(size_t)c * Mp + l], zr, vt, meta[Mp + l], a.cpos[l], c, meta[l]);
      const Real x = fabs(fma(ph, sv[c], ptil[l]));
      if (x > v) {
        v = x;
        arg = l;
      }
    }
    for (int off = 16; off; off >>= 1) {
      const Real v2 = __shfl_xor_sync(0xffffffffu, v, off);
      const int a2 = __shfl_xor_sync(0xffffffffu, arg, off);
      if (v2 > v || (v2 == v && a2 < arg)) {
        v = v2;
        arg = a2;
      }
    }
    if (lane == 0) o.top_mon[ob + j] = arg;
  }
}

// Output-first candidates (Sec. III-A's injection module): the winner's top-k
// cases, computed for every (timestep, candidate) in the loop, copied to the
// outputs once Eq. (8) has chosen it.  One thread per (topology slot,
// timestep, case); a topology without a choice gets -1 / -1 / 0.
__global__ void k_top_gather(Args a, int U, int k, const int* __restrict__ ctop, const int* __restrict__ mtop,
                             const float* __restrict__ ltop) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int T = a.T;
  if (i >= (size_t)a.nq * T * k) return;
  const int q = (int)(i / ((size_t)T * k)), t = (int)((i / k) % T), j = (int)(i % k);
  const int tau = a.qi[q].tau;
  const int u = a.qi[q].status == ST_OK ? a.best_u[(size_t)q * T + t] : -1;
  const size_t o = ((size_t)tau * T + t) * k + j;
  if (u < 0) {
    a.out.top_cont[o] = -1;
    a.out.top_mon[o] = -1;
    a.out.top_loading[o] = 0.f;
    return;
  }
  const size_t src = (((size_t)tau * T + t) * U + u) * k + j;
  a.out.top_cont[o] = ctop[src];
  a.out.top_mon[o] = mtop[src];
  a.out.top_loading[o] = ltop[src];
}

__global__ void k_fill_f(float* __restrict__ p, size_t n, float v) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// ---------------------------------------------------------------------------
// generator-failure N-1 (the "N-1 generator" case of Sec. III-A): generator g
// at bus b with output P_g[t] fails, the slack takes it up, and the flows
// become p_f - P_g PTDF_f[:, b].  The topology's PTDF column follows from the
// same rank-r update as p_f from p0 (Eq. (3)):
//   PTDF_f[l, b] = PTDF[l, b] - Z[l, :] K^{-1} Sigma^T PTDF[:, b]
// One warp per (topology, timestep): max over generators and monitored
// branches of |flow| / limit, the generator reaching it (lowest on ties), and
// the overload sum.
// ---------------------------------------------------------------------------
// PTDF[mon, gen_bus] / limit, one row per generator, row stride ld (once per solve)
template <class Real>
__global__ void k_gen_cols(int G, int M, int ld, int V, const int* __restrict__ gen_bus, const int* __restrict__ monN,
                           const double* __restrict__ PtdfN, const double* __restrict__ inv_lim, Real* __restrict__ PG) {
  const int g = blockIdx.y;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < M; l += gridDim.x * blockDim.x)
    PG[(size_t)g * ld + l] = (Real)(PtdfN[(size_t)monN[l] * V + gen_bus[g]] * inv_lim[l]);
}

// One block per topology; thread i owns monitored rows i, i + 128, ...: per
// row its p_f over TT timesteps and its Z row are loaded once, and each
// generator's column entry (independent of t) is formed once and applied to
// every timestep; per-timestep (max, generator, overload) accumulators live in
// registers until one block reduction per timestep.
template <class Real, int RMAX, int TT>
__global__ __launch_bounds__(128) void k_gen_n1(Args a, int G, const int* __restrict__ gen_bus,
                                                 const double* __restrict__ gen_p, const double* __restrict__ PtdfN,
                                                 int V, const Real* __restrict__ PG, int t0) {
  __shared__ EntSmem S;
  __shared__ Real beta_s[64][RMAX];  // K^{-1} Sigma^T PTDF[:, bus_g], up to 64 generators per round
  __shared__ Real pg_s[TT][64];      // their outputs over this pass's timesteps
  __shared__ Real rv[4];  // maxima compared in the working precision
  __shared__ double ro[4];
  __shared__ int ra[4];
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const QInfo qi = a.qi[q];
  const int T = a.T, M = a.M, Mp = a.Mpad, tau = qi.tau;
  const dcflow_results& o = a.out;
  if (qi.status != ST_OK) {
    for (int t = t0 + tid; t < T && t < t0 + TT; t += blockDim.x) {
      o.gen_max_loading[(size_t)tau * T + t] = 0.0;
      o.worst_gen[(size_t)tau * T + t] = -1;
      o.gen_overload_sum[(size_t)tau * T + t] = 0.0;
    }
    return;
  }
  const int r = qi.r;
  load_entries(S, a, q, r);  // block-wide (contains a barrier)
  const double* Kinv = a.Kinv + (size_t)q * kRMax * kRMax;
  const Real* Zs = static_cast<const Real*>(a.Zs) + (size_t)q * kRMax * Mp;
  const Real* ptil = static_cast<const Real*>(a.ptil) + (size_t)q * T * Mp;
  const Real* meta = static_cast<const Real*>(a.diagv) + (size_t)q * 4 * Mp;
  Real mx[TT], ov[TT];  // working precision per entry (FP32 form: overload via the saturating FMA, x 2^-20)
  int ag[TT];
#pragma unroll
  for (int j = 0; j < TT; ++j) {
    mx[j] = (Real)-1;
    ov[j] = (Real)0;
    ag[j] = 0x7fffffff;
  }
  for (int g0 = 0; g0 < G; g0 += 64) {
    const int gn = min(64, G - g0);
    __syncthreads();
    for (int p = tid; p < gn * RMAX; p += blockDim.x) {  // beta of generator g0 + p / RMAX, component p % RMAX
      const int g = p / RMAX, j = p % RMAX, b = gen_bus[g0 + g];
      double x = 0.0;
      for (int i = 0; i < r; ++i) {
        double sv = 0.0;
        for (int e = S.mp[i]; e < S.mp[i + 1]; ++e) sv = fma(S.esd[e], PtdfN[(size_t)S.en[e] * V + b], sv);
        x = fma(Kinv[j * kRMax + i], sv, x);
      }
      beta_s[g][j] = (Real)x;
    }
    for (int p = tid; p < TT * 64; p += blockDim.x) {
      const int j = p / 64, g = p % 64;
      pg_s[j][g] = (g < gn && t0 + j < T) ? (Real)gen_p[(size_t)(t0 + j) * G + g0 + g] : (Real)0;
    }
    __syncthreads();
    for (int l = tid; l < M; l += blockDim.x) {
      Real zr[RMAX], pt[TT];
#pragma unroll
      for (int j = 0; j < RMAX; ++j) zr[j] = Zs[(size_t)j * Mp + l];
#pragma unroll
      for (int j = 0; j < TT; ++j) pt[j] = (t0 + j < T) ? ptil[(size_t)(t0 + j) * Mp + l] : (Real)0;
      const Real rm = meta[Mp + l];  // an outaged monitored branch carries nothing
      for (int g = 0; g < gn; ++g) {
        Real col = PG[(size_t)(g0 + g) * Mp + l];
#pragma unroll
        for (int j = 0; j < RMAX; ++j) col = fma(-zr[j], beta_s[g][j], col);
        col *= rm;
#pragma unroll
        for (int j = 0; j < TT; ++j) {
          const Real v = fma(-pg_s[j][g], col, pt[j]);
          if (fabs(v) > mx[j]) {
            mx[j] = fabs(v);
            ag[j] = g0 + g;
          }
          Real dummy = (Real)0;
          Acc<Real>::add(dummy, ov[j], v);
        }
      }
    }
  }
  // per timestep: block reduction (max, lowest generator on ties; overload sum)
#pragma unroll
  for (int j = 0; j < TT; ++j) {
    if (t0 + j >= T) break;  // uniform over the block
    Real v = mx[j];
    double s2 = (double)ov[j] * Acc<Real>::ovl_scale();
    int g = ag[j];
    for (int off = 16; off; off >>= 1) {
      const Real v2 = __shfl_xor_sync(0xffffffffu, v, off);
      const int g2 = __shfl_xor_sync(0xffffffffu, g, off);
      s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      if (v2 > v || (v2 == v && g2 < g)) {
        v = v2;
        g = g2;
      }
    }
    if (lane == 0) {
      rv[w] = v;
      ra[w] = g;
      ro[w] = s2;
    }
    __syncthreads();
    if (tid == 0) {
      Real bv = rv[0];
      double bo = ro[0];
      int bg = ra[0];
      for (int k = 1; k < 4; ++k) {
        bo += ro[k];
        if (rv[k] > bv || (rv[k] == bv && ra[k] < bg)) {
          bv = rv[k];
          bg = ra[k];
        }
      }
      const size_t k2 = (size_t)tau * T + t0 + j;
      o.gen_max_loading[k2] = G ? (double)bv : 0.0;
      o.worst_gen[k2] = G ? bg : -1;
      o.gen_overload_sum[k2] = bo;
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------------------
// multi-outage N-1 (Def. 4, MODF): a set O of up to 4 branches fails at once,
//   p_n1 = p_f + Phi_f[:, O] (I - Phi_f[O, O])^{-1} p_f[O],
// with Phi_f[:, o] = Phi[:, o] - Z K^{-1} (Sigma^T Phi[:, o] - s_o) as for the
// single contingencies; the natural-order LU pivots of I - Phi_f[O, O] are the
// sequential LODF denominators, so a pivot at or below the threshold means the
// set islands the topology.
// k_multi_prep (one warp per topology and set, FP64 for the small systems):
//   vt [q][set][4][kRMax]  K^{-1} (Sigma^T Phi[:, o_a] - s_{o_a})  (Real)
//   w  [q][set][T][4]      (I - Phi_f[O, O])^{-1} p_f[O, t]        (Real)
//   flag [q][set]          0 evaluated, 1 islands the topology, 2 a member is
//                          already out in the topology (skipped, not counted)
// k_multi_rows (one block per topology): every monitored row against every set.
// ---------------------------------------------------------------------------
template <class Real>
__global__ __launch_bounds__(128) void k_multi_prep(Args a, int n_multi, const int* __restrict__ mptr,
                                                    const int* __restrict__ mN, Real* __restrict__ mvt,
                                                    Real* __restrict__ mw, int* __restrict__ mflag,
                                                    const float* __restrict__ p0f) {
  extern __shared__ unsigned char dyn_mp[];
  Real* alph_s = reinterpret_cast<Real*>(dyn_mp);  // [r][T] alpha in the working precision
  __shared__ EntSmem S;
  __shared__ int outN[kRMax];
  __shared__ double bv_s[4][4][kRMax], z_s[4][4][kRMax], vt_s[4][4][kRMax];
  __shared__ Real zr_s[4][4][kRMax];
  __shared__ double A_s[4][4][4];
  __shared__ int flag_s[4];
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const QInfo qi = a.qi[q];
  if (qi.status != ST_OK) return;
  const int r = qi.r, ks = qi.ks, nout = qi.r - qi.ks, T = a.T, NN = a.NN;
  load_entries(S, a, q, r);  // block-wide (contains a barrier)
  for (int i = tid; i < nout; i += blockDim.x) outN[i] = S.en[S.mp[ks + i]];
  for (int p = tid; p < r * T; p += blockDim.x) alph_s[p] = (Real)a.alpha[(size_t)q * kRMax * T + p];
  __syncthreads();
  const int m = blockIdx.y * 4 + wp;
  if (m >= n_multi) return;  // warp-uniform; no block barrier follows
  const int e0 = mptr[m], n = mptr[m + 1] - e0;
  const size_t qm = (size_t)q * n_multi + m;
  bool lost = false;  // a member the topology already lost
  for (int p = lane; p < n * nout; p += 32) lost |= outN[p % nout] == mN[e0 + p / nout];
  if (__any_sync(0xffffffffu, lost)) {
    if (lane == 0) mflag[qm] = 2;
    return;
  }
  const double* Kinv = a.Kinv + (size_t)q * kRMax * kRMax;
  // the (member, modification) items packed to the topology's rank: n r <= 64 items
  // over the warp's lanes (B300's FP64 pipe issues a whole warp for any active lane)
  for (int p = lane; p < n * r; p += 32) {  // Sigma^T Phi[:, o] - s_o and the Z row of member o
    const int a2 = p / r, i = p % r;
    double acc = 0.0;
    const int oN = mN[e0 + a2];
    for (int e = S.mp[i]; e < S.mp[i + 1]; ++e) {
      const int mm = S.en[e];
      acc = fma(S.esd[e], a.PhiN[(size_t)mm * NN + oN], acc);
      if (i < ks && mm == oN) acc -= S.esd[e];
    }
    const double z = z_entry_col(S, a.PhiN, NN, a.bN, oN, i);
    bv_s[wp][a2][i] = acc;
    z_s[wp][a2][i] = z;
    zr_s[wp][a2][i] = (Real)z;  // the working-precision copy for the weights below
  }
  __syncwarp();
  Real* vt = mvt + qm * 4 * kRMax;
  for (int p = lane; p < 4 * kRMax; p += 32) vt[p] = (Real)0;  // rows past the rank and absent members
  __syncwarp();
  for (int p = lane; p < n * r; p += 32) {  // K^{-1} is zero outside r x r
    const int a2 = p / r, j = p % r;
    double x = 0.0;
    for (int i = 0; i < r; ++i) x = fma(Kinv[j * kRMax + i], bv_s[wp][a2][i], x);
    vt_s[wp][a2][j] = x;
    vt[a2 * kRMax + j] = (Real)x;
  }
  __syncwarp();
  if (lane < n * n) {  // A = I - Phi_f[O, O]
    const int a2 = lane / n, b2 = lane % n;
    double phi = a.PhiN[(size_t)mN[e0 + a2] * NN + mN[e0 + b2]];
    for (int j = 0; j < r; ++j) phi = fma(-z_s[wp][a2][j], vt_s[wp][b2][j], phi);
    A_s[wp][a2][b2] = (a2 == b2 ? 1.0 : 0.0) - phi;
  }
  __syncwarp();
  {  // natural-order LU, lane i owning row i (the same operations per entry as a row loop)
    int f = 0;
    for (int k = 0; k < n; ++k) {
      const double piv = A_s[wp][k][k];  // warp-uniform
      if (!(piv > a.tol)) {
        f = 1;
        break;
      }
      if (lane > k && lane < n) {
        const double fct = A_s[wp][lane][k] / piv;
        A_s[wp][lane][k] = fct;
        for (int j = k + 1; j < n; ++j) A_s[wp][lane][j] = fma(-fct, A_s[wp][k][j], A_s[wp][lane][j]);
      }
      __syncwarp();
    }
    if (lane == 0) {
      flag_s[wp] = f;
      mflag[qm] = f;
    }
  }
  __syncwarp();
  if (flag_s[wp]) return;
  __shared__ Real Lr_s[4][4][4];  // the LU factors in the working precision, converted once per warp
  if (lane < 16) {
    const int i = lane >> 2, k = lane & 3;
    Lr_s[wp][i][k] = (i < n && k < n) ? (Real)A_s[wp][i][k] : (Real)(i == k);
  }
  __syncwarp();
  Real L[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) L[i][k] = Lr_s[wp][i][k];
  Real* w = mw + qm * T * 4;
  for (int t = lane; t < T; t += 32) {  // p_f[O, t] as the row operands do, then the two triangular solves
    Real y[4];
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) {
      Real pf = (Real)0;
      if (a2 < n) {
        if constexpr (sizeof(Real) == 4) pf = p0f[(size_t)mN[e0 + a2] * T + t];
        else pf = a.p0[(size_t)mN[e0 + a2] * T + t];
        for (int j = 0; j < r; ++j) pf = fma(-zr_s[wp][a2][j], alph_s[j * T + t], pf);
      }
      y[a2] = pf;
    }
#pragma unroll
    for (int i = 1; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < i; ++k) y[i] = fma(-L[i][k], y[k], y[i]);
#pragma unroll
    for (int i = 3; i >= 0; --i) {
#pragma unroll
      for (int k = i + 1; k < 4; ++k) y[i] = fma(-L[i][k], y[k], y[i]);
      y[i] /= L[i][i];
    }
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) w[t * 4 + a2] = y[a2];
  }
}

// one set's N members at one monitored row, TT timesteps: the N-1 loading and
// its running maximum (lowest set on ties) and overload sum
template <class Real, int N, int TT>
__device__ __forceinline__ void multi_apply(const Real (&col)[4], const Real* __restrict__ w, const Real (&pt)[TT],
                                            Real (&mx)[TT], int (&ag)[TT], Real (&ov)[TT], int m) {
#pragma unroll
  for (int jt = 0; jt < TT; ++jt) {
    Real v = pt[jt];
#pragma unroll
    for (int a2 = 0; a2 < N; ++a2) v = fma(col[a2], w[jt * 4 + a2], v);
    if (fabs(v) > mx[jt]) {
      mx[jt] = fabs(v);
      ag[jt] = m;
    }
    Real dummy = (Real)0;
    Acc<Real>::add(dummy, ov[jt], v);
  }
}

template <class Real, int RMAX, int TT, int SG>
__global__ __launch_bounds__(128) void k_multi_rows(Args a, int n_multi, const int* __restrict__ mptr,
                                                    const int* __restrict__ mmpos, const Real* __restrict__ PhiMO,
                                                    const Real* __restrict__ mvt, const Real* __restrict__ mw,
                                                    const int* __restrict__ mflag) {
  __shared__ __align__(16) Real vt_s[SG][4][RMAX];
  __shared__ __align__(16) Real w_s[SG][TT][4];
  __shared__ int fl_s[SG], e0_s[SG], mp_s[SG][4];
  __shared__ int nisl_s;
  __shared__ Real rv_s[TT][4];  // maxima compared in the working precision
  __shared__ double ro_s[TT][4];
  __shared__ int ra_s[TT][4];
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const QInfo qi = a.qi[q];
  const int T = a.T, M = a.M, Mp = a.Mpad, tau = qi.tau;
  const dcflow_results& o = a.out;
  if (qi.status != ST_OK) {
    for (int t = tid; t < T; t += blockDim.x) {
      o.multi_max_loading[(size_t)tau * T + t] = 0.0;
      o.worst_multi[(size_t)tau * T + t] = -1;
      o.multi_overload_sum[(size_t)tau * T + t] = 0.0;
    }
    if (tid == 0) o.n_island_multi[tau] = 0;
    return;
  }
  const Real* Zs = static_cast<const Real*>(a.Zs) + (size_t)q * kRMax * Mp;
  const Real* ptil = static_cast<const Real*>(a.ptil) + (size_t)q * T * Mp;
  const Real* meta = static_cast<const Real*>(a.diagv) + (size_t)q * 4 * Mp;
  const size_t qS = (size_t)q * n_multi;
  if (tid == 0) nisl_s = 0;
  for (int t0 = 0; t0 < T; t0 += TT) {
    Real mx[TT], ov[TT];
    int ag[TT];
#pragma unroll
    for (int j = 0; j < TT; ++j) {
      mx[j] = (Real)-1;
      ov[j] = (Real)0;
      ag[j] = 0x7fffffff;
    }
    for (int g0 = 0; g0 < n_multi; g0 += SG) {
      const int ng = min(SG, n_multi - g0);
      __syncthreads();  // the previous group's shared values are consumed
      for (int s = tid; s < SG; s += blockDim.x) {
        const int m = g0 + s;
        const int f = s < ng ? mflag[qS + m] : 3;
        fl_s[s] = f;
        if (s < ng) {
          const int e0 = mptr[m], n = mptr[m + 1] - e0;
          e0_s[s] = e0;
          for (int k = 0; k < 4; ++k) mp_s[s][k] = k < n ? mmpos[e0 + k] : -2;
          if (t0 == 0 && f == 1) atomicAdd(&nisl_s, 1);
        }
      }
      for (int p = tid; p < ng * 4 * RMAX; p += blockDim.x) {
        const int s = p / (4 * RMAX), a2 = (p / RMAX) % 4, j = p % RMAX;
        vt_s[s][a2][j] = mvt[(qS + g0 + s) * 4 * kRMax + a2 * kRMax + j];
      }
      for (int p = tid; p < ng * TT * 4; p += blockDim.x) {
        const int s = p / (TT * 4), jt = (p / 4) % TT, a2 = p % 4;
        const int t = t0 + jt < T ? t0 + jt : T - 1;  // a tail pass repeats the last timestep, never written
        w_s[s][jt][a2] = mflag[qS + g0 + s] == 0 ? mw[((qS + g0 + s) * T + t) * 4 + a2] : (Real)0;
      }
      __syncthreads();
      for (int l = tid; l < M; l += blockDim.x) {
        Real zr[RMAX], pt[TT];
#pragma unroll
        for (int j = 0; j < RMAX; ++j) zr[j] = Zs[(size_t)j * Mp + l];
#pragma unroll
        for (int jt = 0; jt < TT; ++jt) pt[jt] = ptil[(size_t)(t0 + jt < T ? t0 + jt : T - 1) * Mp + l];
        const Real rm = meta[Mp + l];  // an outaged monitored branch carries nothing
        for (int s = 0; s < ng; ++s) {
          if (fl_s[s]) continue;  // uniform
          const int e0 = e0_s[s];
          Real col[4];
          bool in_set = false;  // a member itself carries nothing (the MODF rows of O are -I)
          int n = 0;
#pragma unroll
          for (int a2 = 0; a2 < 4; ++a2) {
            const int mp = mp_s[s][a2];
            Real c = (Real)0;
            if (mp != -2) {
              c = PhiMO[(size_t)(e0 + a2) * Mp + l];
#pragma unroll
              for (int j = 0; j < RMAX; ++j) c = fma(-zr[j], vt_s[s][a2][j], c);
              ++n;
            }
            col[a2] = c * rm;
            in_set |= mp == l;
          }
          const int m = g0 + s;
          if (in_set) {  // rare: loading 0 at every timestep
#pragma unroll
            for (int jt = 0; jt < TT; ++jt)
              if ((Real)0 > mx[jt]) {
                mx[jt] = (Real)0;
                ag[jt] = m;
              }
          } else {  // n is the same for the whole block
            const Real* w = &w_s[s][0][0];
            if (n == 1) multi_apply<Real, 1, TT>(col, w, pt, mx, ag, ov, m);
            else if (n == 2) multi_apply<Real, 2, TT>(col, w, pt, mx, ag, ov, m);
            else if (n == 3) multi_apply<Real, 3, TT>(col, w, pt, mx, ag, ov, m);
            else multi_apply<Real, 4, TT>(col, w, pt, mx, ag, ov, m);
          }
        }
      }
    }
#pragma unroll
    for (int jt = 0; jt < TT; ++jt) {
      Real v = mx[jt];
      double s2 = (double)ov[jt] * Acc<Real>::ovl_scale();
      int g = ag[jt];
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        const Real v2 = __shfl_xor_sync(0xffffffffu, v, off);
        const int g2 = __shfl_xor_sync(0xffffffffu, g, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
        if (v2 > v || (v2 == v && g2 < g)) {
          v = v2;
          g = g2;
        }
      }
      if (lane == 0) {
        rv_s[jt][wp] = v;
        ra_s[jt][wp] = g;
        ro_s[jt][wp] = s2;
      }
    }
    __syncthreads();
    if (tid < TT && t0 + tid < T) {
      Real bv = rv_s[tid][0];
      double bo = ro_s[tid][0];
      int bg = ra_s[tid][0];
      for (int k = 1; k < 4; ++k) {
        bo += ro_s[tid][k];
        if (rv_s[tid][k] > bv || (rv_s[tid][k] == bv && ra_s[tid][k] < bg)) {
          bv = rv_s[tid][k];
          bg = ra_s[tid][k];
        }
      }
      const size_t k2 = (size_t)tau * T + t0 + tid;
      const bool any = bg != 0x7fffffff;
      o.multi_max_loading[k2] = any ? (double)bv : 0.0;
      o.worst_multi[k2] = any ? bg : -1;
      o.multi_overload_sum[k2] = bo;
    }
  }
  __syncthreads();
  if (tid == 0) o.n_island_multi[tau] = nisl_s;
}

}  // namespace dcf

#include "n1_launch.cuh"
#include "sec_tile.cuh"

using namespace dcf;

namespace {

struct Plan {
  int TT, RMAX, LT;
};

int pick_tt(int T, bool fp64) {
  const int opts32[] = {1, 4, 8, 16, 24, 32};
  const int opts64[] = {1, 4, 8, 12, 24};
  const int* o = fp64 ? opts64 : opts32;
  const int n = fp64 ? 5 : 6;
  for (int i = 0; i < n; ++i)
    if (T <= o[i]) return o[i];
  return o[n - 1];
}

template <class Real, int TT, int RMAX>
void launch_n1_t(const Args& a, dim3 grid, cudaStream_t st, int t0) {
  constexpr int LT = sizeof(Real) == 8 ? 8 : 16;
  k_n1<Real, TT, RMAX, LT><<<grid, 64, 0, st>>>(a, t0);
}

template <class Real, int RMAX>
int launch_n1_r(const Args& a, int TT, dim3 grid, cudaStream_t st, int t0) {
  switch (TT) {
    case 1: launch_n1_t<Real, 1, RMAX>(a, grid, st, t0); break;
    case 4: launch_n1_t<Real, 4, RMAX>(a, grid, st, t0); break;
    case 8: launch_n1_t<Real, 8, RMAX>(a, grid, st, t0); break;
    default:
      if constexpr (sizeof(Real) == 4) {
        if (TT == 16) launch_n1_t<Real, 16, RMAX>(a, grid, st, t0);
        else if (TT == 24) launch_n1_t<Real, 24, RMAX>(a, grid, st, t0);
        else launch_n1_t<Real, 32, RMAX>(a, grid, st, t0);
      } else {
        if (TT == 12) launch_n1_t<Real, 12, RMAX>(a, grid, st, t0);
        else if (TT == 24) launch_n1_t<Real, 24, RMAX>(a, grid, st, t0);
        else return DCFLOW_ERR_INVALID_ARG;
      }
  }
  return 0;
}

template <class Real>
int launch_n1(const Args& a, int RMAX, int TT, dim3 grid, cudaStream_t st, int t0) {
  if (RMAX == 4) return launch_n1_r<Real, 4>(a, TT, grid, st, t0);
  if (RMAX == 8) return launch_n1_r<Real, 8>(a, TT, grid, st, t0);
  return launch_n1_r<Real, 16>(a, TT, grid, st, t0);
}

template <class Real>
int launch_final(const Args& a, int RMAX, cudaStream_t st, const void* phicm, const int* nsel = nullptr) {
  const Real* pc = static_cast<const Real*>(phicm);
  // shared memory: the remainder columns' Phi_f entries (at most 4 x M), then one
  // column for the worst monitored branches when it fits
  const size_t rem = nsel ? 0 : (size_t)(a.C_eff - a.c_rem) * a.M * sizeof(Real);
  const size_t big = 200 * 1024;
  if (rem > big) return DCFLOW_ERR_INVALID_ARG;
  const int col_room = rem + (size_t)a.M * sizeof(Real) <= big ? 1 : 0;
  const size_t dyn = rem + (col_room ? (size_t)a.M * sizeof(Real) : 0);
  static uint64_t attr[3] = {0, 0, 0};
  if (RMAX == 4) {
    if (dyn > 48 * 1024 && smem_attr_once(k_final<Real, 4>, (int)big, attr[0]) != cudaSuccess) return DCFLOW_ERR_CUDA;
    k_final<Real, 4><<<a.nq, 128, dyn, st>>>(a, nsel, pc, col_room);
  } else if (RMAX == 8) {
    if (dyn > 48 * 1024 && smem_attr_once(k_final<Real, 8>, (int)big, attr[1]) != cudaSuccess) return DCFLOW_ERR_CUDA;
    k_final<Real, 8><<<a.nq, 128, dyn, st>>>(a, nsel, pc, col_room);
  } else {
    if (dyn > 48 * 1024 && smem_attr_once(k_final<Real, 16>, (int)big, attr[2]) != cudaSuccess) return DCFLOW_ERR_CUDA;
    k_final<Real, 16><<<a.nq, 128, dyn, st>>>(a, nsel, pc, col_room);
  }
  return 0;
}

template <class Real, int RMAX>
int launch_topcases_r(const Args& a, const float* cmax, const int* cinv, const void* phicm, int k, cudaStream_t st) {
  const Real* pc = static_cast<const Real*>(phicm);
  if (a.tile) {  // after the tracking N-1 pass: 16 rows per case
    const dim3 g(a.nq, (a.T + 3) / 4);
    if (a.C <= 256) k_topcases_tile<Real, RMAX, 8><<<g, 128, 0, st>>>(a, cmax, cinv, pc, k);
    else if (a.C <= 512) k_topcases_tile<Real, RMAX, 16><<<g, 128, 0, st>>>(a, cmax, cinv, pc, k);
    else if (a.C <= 768) k_topcases_tile<Real, RMAX, 24><<<g, 128, 0, st>>>(a, cmax, cinv, pc, k);
    else if (a.C <= 1024) k_topcases_tile<Real, RMAX, 32><<<g, 128, 0, st>>>(a, cmax, cinv, pc, k);
    else k_topcases_tile<Real, RMAX, 64><<<g, 128, 0, st>>>(a, cmax, cinv, pc, k);
    return 0;
  }
  // distinct columns per build phase: as many as 40 KB of shared memory hold (at most 16),
  // at least one (up to 150 KB for the largest studies)
  const size_t colb = (size_t)std::max(a.M, 1) * sizeof(Real);
  const int cbm = (int)std::max<size_t>(1, std::min<size_t>(16, (40 * 1024) / colb));
  const size_t dyn = (size_t)cbm * colb;
  if (dyn <= 150 * 1024) {  // each distinct selected contingency's column built once per topology
    static uint64_t attr[5] = {0, 0, 0, 0, 0};
    auto go = [&](auto kern, int i) -> int {
      if (smem_attr_once(kern, 150 * 1024, attr[i]) != cudaSuccess) return DCFLOW_ERR_CUDA;
      kern<<<a.nq, 256, dyn, st>>>(a, cmax, cinv, pc, k, cbm);
      return 0;
    };
    if (a.C <= 256) return go(k_topcols<Real, RMAX, 8>, 0);
    if (a.C <= 512) return go(k_topcols<Real, RMAX, 16>, 1);
    if (a.C <= 768) return go(k_topcols<Real, RMAX, 24>, 2);
    if (a.C <= 1024) return go(k_topcols<Real, RMAX, 32>, 3);
    return go(k_topcols<Real, RMAX, 64>, 4);
  }
  const dim3 grid(a.nq, (a.T + 3) / 4);
  if (a.C <= 256) k_topcases<Real, RMAX, 8><<<grid, 128, 0, st>>>(a, cmax, cinv, pc, k);
  else if (a.C <= 512) k_topcases<Real, RMAX, 16><<<grid, 128, 0, st>>>(a, cmax, cinv, pc, k);
  else if (a.C <= 1024) k_topcases<Real, RMAX, 32><<<grid, 128, 0, st>>>(a, cmax, cinv, pc, k);
  else k_topcases<Real, RMAX, 64><<<grid, 128, 0, st>>>(a, cmax, cinv, pc, k);
  return 0;
}
template <class Real>
int launch_topcases(const Args& a, int RMAX, const float* cmax, const int* cinv, const void* phicm, int k,
                    cudaStream_t st) {
  if (RMAX == 4) return launch_topcases_r<Real, 4>(a, cmax, cinv, phicm, k, st);
  if (RMAX == 8) return launch_topcases_r<Real, 8>(a, cmax, cinv, phicm, k, st);
  return launch_topcases_r<Real, 16>(a, cmax, cinv, phicm, k, st);
}

template <class Real>
void launch_ti_expand(const Args& ap, int RMAX, int T, int U, const dcflow_batch* bt, ChunkBufs& B, int nq,
                      cudaStream_t st) {
  const dim3 grid(T, nq);
#define DCF_TI_EXPAND(R_)                                                                                    \
  k_ti_expand<Real, R_><<<grid, 256, 0, st>>>(ap, T, U, bt->ti_ptr, bt->ti_mask, bt->inj_p, bt->n_inj,      \
                                              B.tiel.as<int>(), B.tirow.as<int>(), B.nel.as<int>(),         \
                                              B.zcd.as<Real>(), B.ptv.as<Real>(), B.svv.as<Real>())
  if (RMAX == 4) DCF_TI_EXPAND(4);
  else if (RMAX == 8) DCF_TI_EXPAND(8);
  else DCF_TI_EXPAND(16);
#undef DCF_TI_EXPAND
}

// timesteps per pass of the register-tiled FP32 kernels (8 TR): the fewest passes
inline int sec_tr(int T) { return T > 16 ? 3 : (T > 8 ? 2 : 1); }

// FP64: one thread per monitored row, passes of 8 timesteps; FP32: the
// TMA-fed kernel, every pass in one launch (grid y).  Returns the launches, or
// minus an error code.
template <class Real, int RMAX>
int launch_gen_r(const Args& a, int G, const int* gen_bus, const double* gen_p, const double* ptdf, int V,
                 const Real* P, cudaStream_t st) {
  if constexpr (sizeof(Real) == 4) {
    const int tr = sec_tr(a.T), TT = 8 * tr;
    const dim3 grid(a.nq, (a.T + TT - 1) / TT);
    const uint64_t M = (uint64_t)a.M, Mp = (uint64_t)a.Mpad, nq = (uint64_t)a.nq;
    GenMaps maps;
    const uint64_t d_pg[2] = {M, (uint64_t)G}, s_pg[1] = {Mp * 4};
    const uint32_t b_pg[2] = {32, 16};
    const uint64_t d_zt[3] = {M, (uint64_t)kRMax, nq}, s_zt[2] = {Mp * 4, Mp * kRMax * 4};
    const uint32_t b_zt[3] = {32, (uint32_t)RMAX, 1};
    const uint64_t d_me[3] = {M, 4, nq}, s_me[2] = {Mp * 4, Mp * 16};
    const uint32_t b_me[3] = {32, 4, 1};
    const uint64_t d_pt[3] = {M, (uint64_t)a.T, nq}, s_pt[2] = {Mp * 4, Mp * a.T * 4};
    const uint32_t b_pt[3] = {GenTmaLayout<1, RMAX>::PL, (uint32_t)TT, 1};  // 36-float lines
    int rc = encode_map(&maps.pg, P, 2, d_pg, s_pg, b_pg, true);  // 128-byte swizzled
    if (!rc) rc = encode_map(&maps.zt, a.Zs, 3, d_zt, s_zt, b_zt);
    if (!rc) rc = encode_map(&maps.meta, a.diagv, 3, d_me, s_me, b_me);
    if (!rc) rc = encode_map(&maps.pt, a.ptil, 3, d_pt, s_pt, b_pt);
    if (rc) return -rc;
    static uint64_t attr[3] = {0, 0, 0};
    auto go = [&](auto kern, int bytes, int i) -> int {
      if (smem_attr_once(kern, bytes, attr[i]) != cudaSuccess) {
        set_error("dcflow_solve_batch: generator pass shared memory");
        return -DCFLOW_ERR_CUDA;
      }
      kern<<<grid, 128, bytes, st>>>(maps, a, G, gen_bus, gen_p, ptdf, V);
      return 1;
    };
    if (tr == 3) return go(k_gen_tma<RMAX, 3>, GenTmaLayout<3, RMAX>::kBytes, 0);
    if (tr == 2) return go(k_gen_tma<RMAX, 2>, GenTmaLayout<2, RMAX>::kBytes, 1);
    return go(k_gen_tma<RMAX, 1>, GenTmaLayout<1, RMAX>::kBytes, 2);
  } else {
    constexpr int TT = 8;
    int n = 0;
    for (int t0 = 0; t0 < a.T; t0 += TT, ++n)
      k_gen_n1<Real, RMAX, TT><<<a.nq, 128, 0, st>>>(a, G, gen_bus, gen_p, ptdf, V, P, t0);
    return n;
  }
}
template <class Real>
int launch_gen(const Args& a, int RMAX, int G, const int* gen_bus, const double* gen_p, const double* ptdf, int V,
               const void* pg, cudaStream_t st) {
  const Real* P = static_cast<const Real*>(pg);
  if (RMAX == 4) return launch_gen_r<Real, 4>(a, G, gen_bus, gen_p, ptdf, V, P, st);
  if (RMAX == 8) return launch_gen_r<Real, 8>(a, G, gen_bus, gen_p, ptdf, V, P, st);
  return launch_gen_r<Real, 16>(a, G, gen_bus, gen_p, ptdf, V, P, st);
}

template <class Real>
void launch_multi_prep(const Args& a, int n_multi, const int* mptr, const int* mN, ChunkBufs& B, const float* p0f,
                       cudaStream_t st) {
  const size_t dyn = (size_t)kRMax * a.T * sizeof(Real);
  k_multi_prep<Real><<<dim3(a.nq, (n_multi + 3) / 4), 128, dyn, st>>>(a, n_multi, mptr, mN, B.mvt.as<Real>(),
                                                                      B.mw.as<Real>(), B.mflag.as<int>(), p0f);
}

template <class Real>
int launch_multi_rows(const Args& a, int RMAX, int n_multi, int n_ent, const int* mptr, const int* mmpos,
                      const void* phimo, ChunkBufs& B, cudaStream_t st) {
  const Real* P = static_cast<const Real*>(phimo);
  const Real *vt = B.mvt.as<Real>(), *w = B.mw.as<Real>();
  const int* f = B.mflag.as<int>();
  if constexpr (sizeof(Real) == 4) {  // TMA-fed, every timestep pass in one launch (grid y)
    const int tr = sec_tr(a.T), TT = 8 * tr;
    const dim3 grid(a.nq, (a.T + TT - 1) / TT);
    const uint64_t M = (uint64_t)a.M, Mp = (uint64_t)a.Mpad, nq = (uint64_t)a.nq;
    MultiMaps maps;
    const uint64_t d_ph[2] = {M, (uint64_t)n_ent}, s_ph[1] = {Mp * 4};
    const uint32_t b_ph[2] = {32, 128};
    const uint64_t d_zt[3] = {M, (uint64_t)kRMax, nq}, s_zt[2] = {Mp * 4, Mp * kRMax * 4};
    const uint32_t b_zt[3] = {32, (uint32_t)RMAX, 1};
    const uint64_t d_me[3] = {M, 4, nq}, s_me[2] = {Mp * 4, Mp * 16};
    const uint32_t b_me[3] = {32, 4, 1};
    const uint64_t d_pt[3] = {M, (uint64_t)a.T, nq}, s_pt[2] = {Mp * 4, Mp * a.T * 4};
    const uint32_t b_pt[3] = {MultiTmaLayout<1, 4>::PL, (uint32_t)TT, 1};  // 36-float lines
    int rc = encode_map(&maps.phi, P, 2, d_ph, s_ph, b_ph, true);  // 128-byte swizzled
    if (!rc) rc = encode_map(&maps.zt, a.Zs, 3, d_zt, s_zt, b_zt);
    if (!rc) rc = encode_map(&maps.meta, a.diagv, 3, d_me, s_me, b_me);
    if (!rc) rc = encode_map(&maps.pt, a.ptil, 3, d_pt, s_pt, b_pt);
    if (rc) return rc;
    static uint64_t attr[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    auto go = [&](auto kern, int bytes, int i) -> int {
      if (smem_attr_once(kern, bytes, attr[i]) != cudaSuccess) {
        set_error("dcflow_solve_batch: multi-outage pass shared memory");
        return DCFLOW_ERR_CUDA;
      }
      kern<<<grid, 256, bytes, st>>>(maps, a, n_multi, mptr, mmpos, vt, w, f);
      return 0;
    };
#define DCF_MULTI_TMA(R_, TR_, I_) go(k_multi_tma<R_, TR_>, MultiTmaLayout<TR_, R_>::kBytes, I_)
    const int ri = RMAX == 4 ? 0 : (RMAX == 8 ? 1 : 2);
    if (ri == 0) return tr == 3 ? DCF_MULTI_TMA(4, 3, 0) : (tr == 2 ? DCF_MULTI_TMA(4, 2, 1) : DCF_MULTI_TMA(4, 1, 2));
    if (ri == 1) return tr == 3 ? DCF_MULTI_TMA(8, 3, 3) : (tr == 2 ? DCF_MULTI_TMA(8, 2, 4) : DCF_MULTI_TMA(8, 1, 5));
    return tr == 3 ? DCF_MULTI_TMA(16, 3, 6) : (tr == 2 ? DCF_MULTI_TMA(16, 2, 7) : DCF_MULTI_TMA(16, 1, 8));
#undef DCF_MULTI_TMA
  } else {
    constexpr int TT = 12, SG = 32;
    (void)n_ent;
    if (RMAX == 4) k_multi_rows<Real, 4, TT, SG><<<a.nq, 128, 0, st>>>(a, n_multi, mptr, mmpos, P, vt, w, f);
    else if (RMAX == 8) k_multi_rows<Real, 8, TT, SG><<<a.nq, 128, 0, st>>>(a, n_multi, mptr, mmpos, P, vt, w, f);
    else k_multi_rows<Real, 16, TT, SG><<<a.nq, 128, 0, st>>>(a, n_multi, mptr, mmpos, P, vt, w, f);
    return 0;
  }
}

// per-topology r x r systems and row operands of one chunk
template <class Real>
void launch_prep(const Args& a, int RMAX, int nq, size_t dyn, cudaStream_t st, void* zcd, const float* p0f,
                 const float* PhiNf, const float* bNf) {
  Real* zc = static_cast<Real*>(zcd);
  if (RMAX == 4) {
    k_small<Real, 4><<<nq, 128, 0, st>>>(a);
    k_rows<Real, 4><<<nq, 128, dyn, st>>>(a, zc, p0f, PhiNf, bNf);
  } else if (RMAX == 8) {
    k_small<Real, 8><<<nq, 128, 0, st>>>(a);
    k_rows<Real, 8><<<nq, 128, dyn, st>>>(a, zc, p0f, PhiNf, bNf);
  } else {
    k_small<Real, 16><<<nq, 128, 0, st>>>(a);
    k_rows<Real, 16><<<nq, 128, dyn, st>>>(a, zc, p0f, PhiNf, bNf);
  }
}

}  // namespace

namespace {

// What a call of the per-batch path produces besides (or instead of) the
// N-1 results: the screener's feature rows only, or the screened N-1.
enum : int { kModeFull = 0, kModeFeatures = 1, kModeScreened = 2 };
struct ScreenCall {
  int mode = kModeFull;
  dcflow_screen* scr = nullptr;
  int top_k = 64;
  float fallback_logit = 0.f;
  float min_logit = 0.f;  // every score above it is evaluated too (INFINITY: none)
  const dcflow_screen_report* rep = nullptr;
  void* X = nullptr;  // features mode: rows tau * T + t, pitch ldx
  int64_t ldx = 0;
  uint8_t* status = nullptr;
};

template <class Real, int TT, int RMAX>
void launch_sel_t(const Args& a, const void* phicm, const ChunkBufs& B, int grid, cudaStream_t st, int t0) {
  constexpr int LT = sizeof(Real) == 8 ? 8 : 16;
  k_n1_sel<Real, TT, RMAX, LT><<<grid, 64, 0, st>>>(a, static_cast<const Real*>(phicm), B.csel.as<int>(),
                                                      B.nsel.as<int>(), B.work.as<int>(), B.nwork.as<int>(), t0);
}

template <class Real, int RMAX>
int launch_sel_r(const Args& a, const void* phicm, const ChunkBufs& B, int TT, int grid, cudaStream_t st, int t0) {
  switch (TT) {
    case 1: launch_sel_t<Real, 1, RMAX>(a, phicm, B, grid, st, t0); break;
    case 4: launch_sel_t<Real, 4, RMAX>(a, phicm, B, grid, st, t0); break;
    case 8: launch_sel_t<Real, 8, RMAX>(a, phicm, B, grid, st, t0); break;
    default:
      if constexpr (sizeof(Real) == 4) {
        if (TT == 16) launch_sel_t<Real, 16, RMAX>(a, phicm, B, grid, st, t0);
        else if (TT == 24) launch_sel_t<Real, 24, RMAX>(a, phicm, B, grid, st, t0);
        else launch_sel_t<Real, 32, RMAX>(a, phicm, B, grid, st, t0);
      } else {
        if (TT == 12) launch_sel_t<Real, 12, RMAX>(a, phicm, B, grid, st, t0);
        else if (TT == 24) launch_sel_t<Real, 24, RMAX>(a, phicm, B, grid, st, t0);
        else return DCFLOW_ERR_INVALID_ARG;
      }
  }
  return 0;
}

template <class Real>
int launch_sel(const Args& a, const void* phicm, const ChunkBufs& B, int RMAX, int TT, int grid, cudaStream_t st,
               int t0) {
  if (RMAX == 4) return launch_sel_r<Real, 4>(a, phicm, B, TT, grid, st, t0);
  if (RMAX == 8) return launch_sel_r<Real, 8>(a, phicm, B, TT, grid, st, t0);
  return launch_sel_r<Real, 16>(a, phicm, B, TT, grid, st, t0);
}

int launch_select(const Args& a, int T, int C, const float* Z, int ldz, int k, uint32_t fb_key, uint32_t min_key,
                  const ChunkBufs& B,
                  int W, int32_t* pred, cudaStream_t st) {
  const int64_t rows = (int64_t)a.nq * T;
  const unsigned grid = (unsigned)((rows * 32 + 255) / 256);
  uint32_t* mk = B.selmask.as<uint32_t>();
  uint8_t* fb = B.sfb.as<uint8_t>();
  if (C <= 256) k_select<8><<<grid, 256, 0, st>>>(a.qi, a.nq, T, C, Z, ldz, k, fb_key, min_key, mk, W, fb, pred);
  else if (C <= 512) k_select<16><<<grid, 256, 0, st>>>(a.qi, a.nq, T, C, Z, ldz, k, fb_key, min_key, mk, W, fb, pred);
  else if (C <= 1024) k_select<32><<<grid, 256, 0, st>>>(a.qi, a.nq, T, C, Z, ldz, k, fb_key, min_key, mk, W, fb, pred);
  else k_select<64><<<grid, 256, 0, st>>>(a.qi, a.nq, T, C, Z, ldz, k, fb_key, min_key, mk, W, fb, pred);
  return 0;
}

uint32_t host_float_key(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

}  // namespace

static int autotune_impl(dcflow_ctx* ctx, const dcflow_batch* bt, const dcflow_results* res, void* stream,
                         std::vector<dcflow_schedule>* tried, dcf::SchedPlan* pick, float* pick_ms);

static dcflow_schedule to_schedule(const dcf::SchedPlan& P, float ms) {
  dcflow_schedule o{};
  o.budget_mb = P.budget_mb;
  for (int i = 0; i < 3; ++i) o.rank_bounds[i] = P.bounds[i];
  o.compact_n1 = P.compact;
  o.remainder = P.remainder;
  o.ms = ms;
  return o;
}

static int solve_impl(dcflow_ctx* ctx, const dcflow_batch* bt, const dcflow_results* res, void* stream,
                      const ScreenCall* sc) {
  const int mode = sc ? sc->mode : kModeFull;
  dcflow_results none{};
  if (mode == kModeFeatures) res = &none;
  if (!ctx || !bt || !res) {
    set_error("dcflow_solve_batch: null argument");
    return DCFLOW_ERR_INVALID_ARG;
  }
  if (!ctx->has_study) {
    set_error("dcflow_solve_batch: no study bound (dcflow_set_study)");
    return DCFLOW_ERR_NO_STUDY;
  }
  DeviceGuard dg(ctx->dev);  // the context's device for this call
  if (dg.err != cudaSuccess) {
    set_error(std::string("dcflow_solve_batch: cudaSetDevice: ") + cudaGetErrorString(dg.err));
    return DCFLOW_ERR_CUDA;
  }
  const int N = bt->n_topo, T = bt->n_time;
  if (N < 0 || T < 1 || T > 256 || bt->n_var < 0) {
    set_error("dcflow_solve_batch: need n_topo >= 0, 1 <= n_time <= 256, n_var >= 0");
    return DCFLOW_ERR_INVALID_ARG;
  }
  ctx->launches = 0;
  if (N == 0) return DCFLOW_OK;
  if (!bt->split_ptr || !bt->out_ptr || !bt->inj ||
      (mode != kModeFeatures && (!res->n1_max_loading || !res->overload_sum || !res->worst_cont ||
                                 !res->island_flag || !res->n_island_cont))) {
    set_error("dcflow_solve_batch: missing required pointer");
    return DCFLOW_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool fp64 = ctx->opt.precision == DCFLOW_FP64;
  const bool tc = ctx->opt.precision == DCFLOW_BF16X3;  // the N-1 tiles' Phi_f on the tensor cores
  const size_t rs = fp64 ? sizeof(double) : sizeof(float);
  const int M = ctx->M, C = ctx->C, NN = ctx->NN;
  // injection candidates T_i (Eq. (8)): read the small CSR to the host, validate
  // it, and map every entry to a pool bus (a column of the extended base flows)
  const int U = bt->n_var;
  // injection topologies t_i: the per-topology candidate counts come to the
  // host (one int per topology) to size the candidate pipeline
  const bool TI = bt->ti_ptr != nullptr;
  int UI = 0;
  if (TI) {
    if (mode != kModeFull || U > 0 || bt->n_inj < 0 || (bt->n_inj > 0 && (!bt->inj_bus || !bt->inj_p))) {
      set_error("dcflow_solve_batch: injection topologies need inj_bus and inj_p (n_inj >= 0), without "
                "injection candidates or the screener");
      return DCFLOW_ERR_INVALID_ARG;
    }
    std::vector<int> tp(N + 1), ib(std::max(bt->n_inj, 1));
    DCF_CUDA(cudaMemcpyAsync(tp.data(), bt->ti_ptr, sizeof(int) * (N + 1), cudaMemcpyDeviceToHost, st));
    if (bt->n_inj)
      DCF_CUDA(cudaMemcpyAsync(ib.data(), bt->inj_bus, sizeof(int) * bt->n_inj, cudaMemcpyDeviceToHost, st));
    DCF_CUDA(cudaStreamSynchronize(st));
    bool ok = tp[0] == 0;
    for (int i = 0; i < N && ok; ++i) {
      ok = tp[i + 1] >= tp[i];
      UI = std::max(UI, tp[i + 1] - tp[i]);
    }
    for (int e = 0; e < bt->n_inj && ok; ++e) ok = ib[e] >= 0 && ib[e] < ctx->V;
    if (!ok || (tp[N] > 0 && !bt->ti_mask)) {
      set_error("dcflow_solve_batch: ti_ptr must start at 0 and not decrease, ti_mask must be given, "
                "inj_bus in range");
      return DCFLOW_ERR_INVALID_ARG;
    }
    UI = std::max(UI, 1);  // every topology without candidates is invalid; keep the pipeline shape
    if ((int64_t)T * UI > (1 << 20)) {
      set_error("dcflow_solve_batch: n_time * max |T_i| > 2^20");
      return DCFLOW_ERR_INVALID_ARG;
    }
  }
  const int Uc = U > 0 ? U : UI;  // candidates per (topology, timestep) of either form
  const int top_k = mode == kModeFeatures ? 0 : res->top_k;
  if (top_k != 0 && (top_k < 1 || top_k > 64 || !res->top_cont || !res->top_mon || !res->top_loading ||
                     mode != kModeFull || ctx->C > 2048)) {
    set_error("dcflow_solve_batch: top_k in [1, 64] with its three arrays, at most 2048 contingencies, "
              "not with the screened solve");
    return DCFLOW_ERR_INVALID_ARG;
  }
  const bool want_multi = mode == kModeFull && res->multi_max_loading;
  if ((res->multi_max_loading || res->worst_multi || res->multi_overload_sum || res->n_island_multi) &&
      (!res->multi_max_loading || !res->worst_multi || !res->multi_overload_sum || !res->n_island_multi ||
       mode != kModeFull || Uc > 0 || ctx->n_multi == 0)) {
    set_error("dcflow_solve_batch: multi-outage outputs need all four arrays and a study with multi-outage sets, "
              "without injection candidates or the screener");
    return DCFLOW_ERR_INVALID_ARG;
  }
  const int G = mode == kModeFull ? bt->n_gen : 0;
  if (bt->n_gen < 0 || (bt->n_gen > 0 && (mode != kModeFull || Uc > 0 || !bt->gen_bus || !bt->gen_p ||
                                          !res->gen_max_loading || !res->worst_gen || !res->gen_overload_sum))) {
    set_error("dcflow_solve_batch: generator failures need gen_bus, gen_p and the three generator outputs, "
              "without injection candidates or the screener");
    return DCFLOW_ERR_INVALID_ARG;
  }
  if (mode != kModeFull && Uc > 0) {
    set_error("dcflow_solve_batch: the screener runs without injection candidates");
    return DCFLOW_ERR_INVALID_ARG;
  }
  // the schedule: forced while tuning, fixed by the caller, tuned for this batch shape, or the defaults
  SchedPlan plan;
  plan.compact = ctx->opt.compact_n1 ? 1 : 0;
  {
    ShapeKey key;
    key.T = T;
    key.U = Uc;
    key.ti = TI;
    key.top_k = top_k;
    key.gen = G;
    key.multi = want_multi;
    key.mode = mode;
    bool found = false;
    if (ctx->tuning) {
      plan = ctx->tune_plan;
      found = true;
    } else if (ctx->sched_fixed) {
      plan = ctx->sched;
      found = true;
    } else {
      for (const auto& kv : ctx->tuned)
        if (kv.first == key) {
          plan = kv.second;
          found = true;
        }
    }
    if (!found && ctx->opt.autotune && mode == kModeFull) {
      // tune on a prefix of this batch (the CSR prefixes are the first topologies' lists)
      dcflow_batch pre = *bt;
      pre.n_topo = std::min(N, std::max(1, ctx->opt.autotune_sample));
      SchedPlan pk;
      float ms = 0.f;
      const int rc = autotune_impl(ctx, &pre, res, stream, nullptr, &pk, &ms);
      if (rc) return rc;
      plan = pk;  // autotune_impl stored it under this key
    }
  }
  ctx->last_plan = plan;
  ctx->last_uc = Uc;
  ctx->launches = 0;
  int R = 0;
  if (U > 0) {
    if (!bt->var_ptr || !bt->var_bus || !bt->var_delta || (int64_t)T * U > (1 << 20)) {
      set_error("dcflow_solve_batch: candidate arrays missing or n_time * n_var > 2^20");
      return DCFLOW_ERR_INVALID_ARG;
    }
    std::vector<int> vp(U + 1);
    DCF_CUDA(cudaMemcpyAsync(vp.data(), bt->var_ptr, sizeof(int) * (U + 1), cudaMemcpyDeviceToHost, st));
    DCF_CUDA(cudaStreamSynchronize(st));
    if (vp[0] != 0) {
      set_error("dcflow_solve_batch: var_ptr[0] must be 0");
      return DCFLOW_ERR_INVALID_ARG;
    }
    for (int u = 0; u < U; ++u)
      if (vp[u + 1] < vp[u]) {
        set_error("dcflow_solve_batch: var_ptr must be non-decreasing");
        return DCFLOW_ERR_INVALID_ARG;
      }
    const int nnz = vp[U];
    std::vector<int> vb(std::max(nnz, 1));
    if (nnz) {
      DCF_CUDA(cudaMemcpyAsync(vb.data(), bt->var_bus, sizeof(int) * nnz, cudaMemcpyDeviceToHost, st));
      DCF_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<int> pool;
    for (int k = 0; k < nnz; ++k) {
      if (vb[k] < 0 || vb[k] >= ctx->V) {
        set_error("dcflow_solve_batch: var_bus out of range");
        return DCFLOW_ERR_INVALID_ARG;
      }
      pool.push_back(vb[k]);
    }
    std::sort(pool.begin(), pool.end());
    pool.erase(std::unique(pool.begin(), pool.end()), pool.end());
    R = (int)pool.size();
    std::vector<int> vk(std::max(nnz, 1));
    for (int k = 0; k < nnz; ++k) vk[k] = (int)(std::lower_bound(pool.begin(), pool.end(), vb[k]) - pool.begin());
    if (ctx->pool.ensure(sizeof(int) * std::max(R, 1)) || ctx->var_k.ensure(sizeof(int) * std::max(nnz, 1)))
      return DCFLOW_ERR_OOM;
    if (R) DCF_CUDA(cudaMemcpyAsync(ctx->pool.p, pool.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
    if (nnz) DCF_CUDA(cudaMemcpyAsync(ctx->var_k.p, vk.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, st));
  }
  const int Text = T + R;  // timesteps plus pool columns through the preparation
  // p0 = PTDF[N, :] inj^T (and the pool columns)
  if (ctx->p0.ensure((size_t)NN * Text * sizeof(double))) return DCFLOW_ERR_OOM;
  k_p0<<<(NN * 32 + 255) / 256, 256, 0, st>>>(NN, ctx->V, T, Text, ctx->PtdfN.as<double>(), bt->inj,
                                               ctx->p0.as<double>());
  if (R > 0) {
    k_p0_pool<<<(NN + 127) / 128, 128, 0, st>>>(NN, ctx->V, T, R, Text, ctx->pool.as<int>(), ctx->PtdfN.as<double>(),
                                                ctx->p0.as<double>());
    ++ctx->launches;
  }
  if (!fp64) {  // the FP32 form's row operands read a float copy
    if (ctx->p0f.ensure((size_t)NN * Text * sizeof(float))) return DCFLOW_ERR_OOM;
    k_to_float<<<(unsigned)std::min<size_t>(((size_t)NN * Text + 255) / 256, 148 * 64), 256, 0, st>>>(
        ctx->p0.as<double>(), ctx->p0f.as<float>(), (size_t)NN * Text);
    ++ctx->launches;
  }
  ++ctx->launches;
  DCF_CHECK_LAUNCH();
  GridDev g{ctx->f.as<int>(), ctx->t.as<int>(), ctx->b.as<double>(), ctx->inc_ptr.as<int>(), ctx->inc_list.as<int>(),
            ctx->nidx.as<int>(), ctx->split_ok.as<uint8_t>(), ctx->out_ok.as<uint8_t>(), ctx->V, ctx->E};
  BatchDev in{bt->split_ptr, bt->split_sub, bt->split_mask, bt->out_ptr, bt->out_branch};
  // rank of every topology -> group by rank class (no dummy padding of uneven k)
  if (ctx->rank.ensure(N)) return DCFLOW_ERR_OOM;
  k_rank<<<(N + 127) / 128, 128, 0, st>>>(g, in, N, ctx->rank.as<int8_t>());
  ++ctx->launches;
  DCF_CHECK_LAUNCH();
  std::vector<int8_t> hr(N);
  int herr = 0;
  if (ctx->err.ensure(sizeof(int))) return DCFLOW_ERR_OOM;
  DCF_CUDA(cudaMemcpyAsync(hr.data(), ctx->rank.p, N, cudaMemcpyDeviceToHost, st));
  DCF_CUDA(cudaMemcpyAsync(&herr, ctx->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  DCF_CUDA(cudaStreamSynchronize(st));
  if (herr) {  // a kernel of an earlier call gave up: bounded wait expired (1) or misaligned staging (2)
    DCF_CUDA(cudaMemsetAsync(ctx->err.p, 0, sizeof(int), st));
    set_error(herr == 1 ? "dcflow_solve_batch: a bounded device wait of an earlier call expired"
                        : "dcflow_solve_batch: an earlier call found its shared staging buffer misaligned");
    return herr == 1 ? DCFLOW_ERR_TIMEOUT : DCFLOW_ERR_CUDA;
  }
  std::vector<int> perm;
  perm.reserve(N);
  // rank classes of the schedule (ascending bounds, the last 16): a topology of rank r
  // goes to the first class whose bound is at least r
  int classes[3] = {16, 16, 16};
  int ncls = 0;
  for (int i = 0; i < 3; ++i)
    if (plan.bounds[i] > 0) classes[ncls++] = plan.bounds[i];
  std::vector<int> cls_start(ncls + 1, 0);
  auto class_of = [&](int r) {
    for (int ci = 0; ci < ncls; ++ci)
      if (r <= classes[ci]) return ci;
    return ncls - 1;
  };
  for (int ci = 0; ci < ncls; ++ci) {
    cls_start[ci] = (int)perm.size();
    for (int i = 0; i < N; ++i) {
      const int r = hr[i] < 0 ? 0 : hr[i];
      if (class_of(r) == ci) perm.push_back(i);
    }
  }
  cls_start[ncls] = N;
  if (ctx->perm.ensure(sizeof(int) * N)) return DCFLOW_ERR_OOM;
  DCF_CUDA(cudaMemcpyAsync(ctx->perm.p, perm.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  // chunk capacity from a scratch budget per buffer set (two sets alternate);
  // large chunks keep the N-1 launches wide (measured better than many small
  // overlapping chunks: the N-1 kernel fills the SMs' registers and shared
  // memory, so preparation kernels of the next chunk only run in its tail)
  const int C_eff = ctx->C_eff;       // contingencies that can be valid (base-grid bridges excluded)
  // FP32 full solve on request: the N-1 kernel runs over each topology's compacted valid contingencies
  const bool cmp = !fp64 && mode == kModeFull && C_eff > 0 && plan.compact;
  // top-k cases after the dense FFMA-build N-1: its tracking variant records each maximum's
  // 16-row tile, and the top-k pass evaluates only that tile per case
  // output-first candidates: the top-k cases of every (timestep, candidate) in the loop
  const bool of = ctx->opt.output_first && Uc > 0 && top_k > 0 && mode == kModeFull;
  const bool use_tile = top_k > 0 && !fp64 && !tc && !cmp && mode == kModeFull && C_eff > 0 &&
                        pick_tt(T, false) >= 4 && !of;
  // a remainder of at most kRemCols contingencies beyond the last full block of 64
  // goes to the final pass (a column each over the monitored rows) instead of an
  // N-1 block that would compute 64 columns for it (plain full solves only)
  constexpr int kRemCols = 4;
  const bool use_rem = plan.remainder && mode == kModeFull && Uc == 0 && !cmp && C_eff > 64 && C_eff % 64 > 0 &&
                       C_eff % 64 <= kRemCols && (size_t)(C_eff % 64) * M * rs <= 200 * 1024;
  const int ncb = use_rem ? C_eff / 64 : (C_eff + 63) / 64;  // 64-contingency blocks of the N-1 kernels
  const int Mp = (int)round_up(M, 16);
  const int TV = T * Uc;  // virtual timesteps: (timestep, candidate) pairs
  if (R > 64) {
    set_error("dcflow_solve_batch: at most 64 distinct candidate buses");
    return DCFLOW_ERR_INVALID_ARG;
  }
  size_t per_slot = (size_t)kEntMax * (sizeof(int) + sizeof(double) + 1) + (kRMax + 1) * 2 + sizeof(QInfo) +
                    (size_t)kRMax * kRMax * 8 + (size_t)kRMax * Text * 8 + (size_t)kRMax * C * (8 + rs) +
                    (size_t)Mp * (kRMax + Text + 4) * rs + (size_t)Text * C * rs + C + 4 +
                    (size_t)T * ncb * (rs + 4 + 8) + 64;
  if (TI) per_slot += (size_t)kRMax * C * rs + 64 * 8 + 4;
  if (tc) per_slot += (size_t)Mp * 16 * 4;  // BF16 hi / lo Z rows
  if (mode == kModeFull) per_slot += (size_t)T * C * rs + (size_t)T * ncb * rs;  // the tie band's maxima
  if (cmp) per_slot += (size_t)C * 4 + 4;
  if (Uc > 0)
    per_slot += (size_t)TV * (Mp + C) * rs + (size_t)TV * ncb * (rs + 4 + 8) + (size_t)T * 4 + (size_t)T * (Mp + C) * rs;
  const size_t SM_ = want_multi ? (size_t)ctx->n_multi : 0;
  per_slot += SM_ * ((4 * kRMax + 4 * (size_t)T) * rs + 4);
  int64_t cap = ctx->opt.chunk_topo > 0 ? ctx->opt.chunk_topo
                                         : (int64_t)(((size_t)std::max(plan.budget_mb, 1)) << 20) / (int64_t)per_slot;
  cap = std::max<int64_t>(1, std::min<int64_t>({cap, 8192, (int64_t)N}));
  for (int bi = 0; bi < 2; ++bi) {
    const size_t c = (size_t)cap;
    ChunkBufs& B = ctx->bufs[bi];
    if (B.q_info.ensure(c * sizeof(QInfo)) || B.ent_n.ensure(c * kEntMax * sizeof(int)) ||
        B.ent_s.ensure(c * kEntMax) || B.ent_w.ensure(c * kEntMax * sizeof(double)) ||
        B.mod_ptr.ensure(c * (kRMax + 1) * sizeof(int16_t)) || B.Kinv.ensure(c * kRMax * kRMax * 8) ||
        B.alpha.ensure(c * kRMax * Text * 8) || B.Vt64.ensure(c * kRMax * std::max(C, 1) * 8) ||
        (!fp64 && B.VtR.ensure(c * kRMax * std::max(C, 1) * rs)) || B.Zs.ensure(c * Mp * kRMax * rs) ||
        B.ptil.ensure(c * Mp * Text * rs) || B.meta.ensure(c * 4 * Mp * rs) ||
        B.s.ensure(c * Text * std::max(C, 1) * rs) || B.valid.ensure(c * std::max(C, 1)) ||
        B.nisl.ensure(c * sizeof(int)) || B.pmax.ensure(c * T * std::max(ncb, 1) * rs) ||
        B.parg.ensure(c * T * std::max(ncb, 1) * sizeof(int)) ||
        B.povl.ensure(c * T * std::max(ncb, 1) * sizeof(double)))
      return DCFLOW_ERR_OOM;
    if (cmp && (B.csel.ensure(c * std::max(C, 1) * sizeof(int)) || B.nsel.ensure(c * sizeof(int))))
      return DCFLOW_ERR_OOM;
    if (tc && B.Zbf.ensure(c * Mp * 16 * 4)) return DCFLOW_ERR_OOM;
    if (mode == kModeFull && (B.cmr.ensure(c * T * std::max(C, 1) * rs) ||
                              B.p2max.ensure(c * T * std::max(ncb, 1) * rs)))
      return DCFLOW_ERR_OOM;
    if (use_tile && B.tile.ensure(c * T * std::max(C, 1) * sizeof(uint16_t))) return DCFLOW_ERR_OOM;
    if (TI && (B.zcd.ensure(c * kRMax * std::max(C, 1) * rs) || B.tiel.ensure(c * 64 * sizeof(int)) ||
               B.tirow.ensure(c * 64 * sizeof(int)) || B.nel.ensure(c * sizeof(int))))
      return DCFLOW_ERR_OOM;
    if (Uc > 0 && (B.ptv.ensure(c * TV * Mp * rs) || B.svv.ensure(c * TV * std::max(C, 1) * rs) ||
                  B.pmaxv.ensure(c * TV * std::max(ncb, 1) * rs) ||
                  B.pargv.ensure(c * TV * std::max(ncb, 1) * sizeof(int)) ||
                  B.povlv.ensure(c * TV * std::max(ncb, 1) * sizeof(double)) || B.bestu.ensure(c * T * sizeof(int)) ||
                  B.ptb.ensure(c * T * Mp * rs) || B.sb.ensure(c * T * std::max(C, 1) * rs)))
      return DCFLOW_ERR_OOM;
    if (SM_ > 0 && (B.mvt.ensure(c * SM_ * 4 * kRMax * rs) || B.mw.ensure(c * SM_ * T * 4 * rs) ||
                    B.mflag.ensure(c * SM_ * sizeof(int))))
      return DCFLOW_ERR_OOM;
  }
  dcflow_screen* scr = sc ? sc->scr : nullptr;
  const int W = (C + 31) / 32;
  const int64_t srows = round_up((int64_t)cap * T, 128);  // feature rows of a chunk
  if (mode == kModeScreened) {
    if (ctx->bufs[0].selmask.ensure((size_t)cap * std::max(W, 1) * 4) || ctx->bufs[0].sfb.ensure((size_t)cap) ||
        ctx->bufs[0].csel.ensure((size_t)cap * std::max(C, 1) * 4) || ctx->bufs[0].nsel.ensure((size_t)cap * 4) ||
        ctx->bufs[0].work.ensure((size_t)cap * std::max(ncb, 1) * 4) || ctx->bufs[0].nwork.ensure(4) ||
        scr->iX.ensure((size_t)srows * scr->Fp * 2) || scr->iH1.ensure((size_t)srows * scr->H * 2) ||
        scr->iH2.ensure((size_t)srows * scr->H * 2) || scr->iZ.ensure((size_t)srows * scr->Cp * 4))
      return DCFLOW_ERR_OOM;
  }
  if (!ctx->phicm_ready) {  // transposed factors: contiguous contingency columns (final pass, screened N-1)
    if (ctx->PhiCM.ensure((size_t)std::max(C, 1) * Mp * rs)) return DCFLOW_ERR_OOM;
    const dim3 blk(32, 8), grd((Mp + 31) / 32, (std::max(C, 1) + 31) / 32);
    if (fp64)
      k_phi_cm<double><<<grd, blk, 0, st>>>(ctx->PhiMC.as<double>(), M, C, ctx->ldc, Mp, ctx->PhiCM.as<double>());
    else
      k_phi_cm<float><<<grd, blk, 0, st>>>(ctx->PhiMC.as<float>(), M, C, ctx->ldc, Mp, ctx->PhiCM.as<float>());
    DCF_CHECK_LAUNCH();
    ++ctx->launches;
    ctx->phicm_ready = true;
  }
  if (G > 0) {  // generator buses in range; base PTDF columns of the monitored rows, scaled by 1 / limit
    std::vector<int> gb(G);
    DCF_CUDA(cudaMemcpyAsync(gb.data(), bt->gen_bus, sizeof(int) * G, cudaMemcpyDeviceToHost, st));
    DCF_CUDA(cudaStreamSynchronize(st));
    for (int g = 0; g < G; ++g)
      if (gb[g] < 0 || gb[g] >= ctx->V) {
        set_error("dcflow_solve_batch: gen_bus out of range");
        return DCFLOW_ERR_INVALID_ARG;
      }
    if (ctx->gen_cols.ensure((size_t)G * Mp * rs)) return DCFLOW_ERR_OOM;  // rows of Mp: 16-byte pitch (TMA)
    const dim3 grd((M + 255) / 256, G);
    if (fp64)
      k_gen_cols<double><<<grd, 256, 0, st>>>(G, M, Mp, ctx->V, bt->gen_bus, ctx->monN.as<int>(),
                                              ctx->PtdfN.as<double>(), ctx->inv_lim.as<double>(),
                                              ctx->gen_cols.as<double>());
    else
      k_gen_cols<float><<<grd, 256, 0, st>>>(G, M, Mp, ctx->V, bt->gen_bus, ctx->monN.as<int>(),
                                             ctx->PtdfN.as<double>(), ctx->inv_lim.as<double>(),
                                             ctx->gen_cols.as<float>());
    DCF_CHECK_LAUNCH();
    ++ctx->launches;
  }
  ctx->chunk_cap = cap;
  if (!ctx->side) {
    DCF_CUDA(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
    cudaEvent_t* evs[] = {&ctx->ev_ready, &ctx->ev_prep[0], &ctx->ev_prep[1], &ctx->ev_free[0], &ctx->ev_free[1]};
    for (cudaEvent_t* e : evs) DCF_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  Args base{};
  base.M = M;
  base.C = C;
  base.NN = NN;
  base.T = T;
  base.U = Uc;
  base.monN = ctx->monN.as<int>();
  base.contN = ctx->contN.as<int>();
  base.cpos = ctx->cpos_of_mon.as<int>();
  base.mpos = ctx->mpos_of_cont.as<int>();
  base.inv_lim = ctx->inv_lim.as<double>();
  base.PhiN = ctx->PhiN.as<double>();
  base.bN = ctx->bN.as<double>();
  base.PhiMC = ctx->PhiMC.p;
  base.p0 = ctx->p0.as<double>();
  base.tol = ctx->opt.island_tol;
  base.ncb = ncb;
  base.C_eff = C_eff;
  base.c_rem = use_rem ? ncb * 64 : C_eff;
  // tie band of the reported indices: the form's tolerance unless the option sets one (negative: none)
  base.tie_eps = ctx->opt.tie_band < 0 ? 0.0 : (ctx->opt.tie_band > 0 ? ctx->opt.tie_band : (fp64 ? 1e-10 : 1e-4));
  base.cont_inv = ctx->cont_inv.as<int>();
  base.tile = nullptr;
  base.cont_pos = ctx->cont_pos.as<int>();
  base.Mpad = Mp;
  base.ldc = ctx->ldc;
  base.err = ctx->err.as<int>();
  base.best_u = nullptr;
  base.out = *res;
  if (top_k > 0 && !res->n1_cont_max) {  // the top-k pass reads the per-contingency maxima
    if (ctx->cm_scratch.ensure((size_t)N * T * std::max(C, 1) * sizeof(float))) return DCFLOW_ERR_OOM;
    base.out.n1_cont_max = ctx->cm_scratch.as<float>();
  }
  const size_t of_n = of ? (size_t)N * T * Uc : 0;  // (topology, timestep, candidate) triples
  if (of) {
    const size_t ncm = of_n * std::max(C, 1);
    if (ctx->of_cmax.ensure(ncm * sizeof(float)) || ctx->of_top.ensure(of_n * top_k * 12)) {
      set_error("dcflow_solve_batch: output-first scratch (n_topo * n_time * candidates * n_cont floats)");
      return DCFLOW_ERR_OOM;
    }
    k_fill_f<<<4 * 148, 256, 0, st>>>(ctx->of_cmax.as<float>(), ncm, -1.f);  // bridges and skipped topologies
    ++ctx->launches;
    DCF_CHECK_LAUNCH();
  }
  auto chunk_args = [&](int bi) {
    Args a = base;
    ChunkBufs& B = ctx->bufs[bi];
    a.qi = B.q_info.as<QInfo>();
    a.ent_n = B.ent_n.as<int>();
    a.ent_s = B.ent_s.as<int8_t>();
    a.ent_w = B.ent_w.as<double>();
    a.mod_ptr = B.mod_ptr.as<int16_t>();
    a.Kinv = B.Kinv.as<double>();
    a.alpha = B.alpha.as<double>();
    a.Vt64 = B.Vt64.as<double>();
    a.VtR = fp64 ? B.Vt64.p : B.VtR.p;
    a.Zs = B.Zs.p;
    a.Zbf = tc ? B.Zbf.as<uint32_t>() : nullptr;
    a.ptil = B.ptil.p;
    a.rowmul = nullptr;
    a.diagv = B.meta.p;
    a.s = B.s.p;
    a.valid = B.valid.as<uint8_t>();
    a.nisl = B.nisl.as<int>();
    a.pmax = B.pmax.p;
    a.parg = B.parg.as<int>();
    a.povl = B.povl.as<double>();
    a.cmr = mode == kModeFull ? B.cmr.p : nullptr;
    a.p2max = mode == kModeFull ? B.p2max.p : nullptr;
    return a;
  };
  const int TT = pick_tt(T, fp64);
  const size_t dyn = (size_t)kRMax * Text * rs;
  // N-1 passes over Tn (virtual) timesteps whose operands are a.ptil / a.s;
  // ovl = false screens the maximum only (FP32 form)
  auto encode_maps = [&](const Args& a, int RMAX, int Tn, int TTn, N1Maps& maps) -> int {
    const bool tc = ctx->opt.precision == DCFLOW_BF16X3 && TTn >= 4;  // one-timestep passes: FFMA build
    {
      const uint64_t d_phi[2] = {(uint64_t)C, (uint64_t)M}, s_phi[1] = {(uint64_t)ctx->ldc * 4};
      // the tensor-core build reads a 68-column tile (its pitch spreads the fragment loads over the banks)
      const uint32_t b_phi[2] = {tc ? (uint32_t)kPhW : (uint32_t)kCB, kLT};
      const uint64_t d_me[3] = {(uint64_t)M, 4, (uint64_t)cap};
      const uint64_t s_me[2] = {(uint64_t)Mp * 4, (uint64_t)Mp * 16};
      const uint32_t b_me[3] = {kLT, 4, 1};
      const uint64_t d_zt[3] = {(uint64_t)M, (uint64_t)kRMax, (uint64_t)cap};
      const uint64_t s_zt[2] = {(uint64_t)Mp * 4, (uint64_t)Mp * kRMax * 4};
      const uint32_t b_zt[3] = {kLT, (uint32_t)RMAX, 1};
      const uint64_t d_pt[3] = {(uint64_t)M, (uint64_t)Tn, (uint64_t)cap};
      const uint64_t s_pt[2] = {(uint64_t)Mp * 4, (uint64_t)Mp * Tn * 4};
      const uint32_t b_pt[3] = {kLT, (uint32_t)TTn, 1};
      int rc = encode_map(&maps.phi, ctx->PhiMC.p, 2, d_phi, s_phi, b_phi);
      if (!rc) rc = encode_map(&maps.meta, a.diagv, 3, d_me, s_me, b_me);
      if (!rc && !tc) rc = encode_map(&maps.zt, a.Zs, 3, d_zt, s_zt, b_zt);
      if (!rc && tc) {  // BF16 hi / lo Z rows [slot][Mpad][KB words]
        const uint64_t KB = RMAX <= 8 ? 8 : 16;
        const uint64_t d_zb[3] = {KB, (uint64_t)M, (uint64_t)cap};
        const uint64_t s_zb[2] = {KB * 4, (uint64_t)Mp * KB * 4};
        const uint32_t b_zb[3] = {(uint32_t)KB, kLT, 1};
        rc = encode_map(&maps.zt, a.Zbf, 3, d_zb, s_zb, b_zb);
      }
      if (!rc) rc = encode_map(&maps.pt, a.ptil, 3, d_pt, s_pt, b_pt);
      return rc;
    }
  };
  // cmp: the chunk's compacted valid-contingency lists (FP32, TT >= 4), or null
  auto run_n1 = [&](const Args& a, int RMAX, int Tn, bool ovl, const ChunkBufs* cmp) -> int {
    const int TTn = ovl ? pick_tt(Tn, fp64) : (fp64 ? 8 : 32);
    if (TTn < 4) cmp = nullptr;
    N1Maps maps;
    if (!fp64) {
      int rc = encode_maps(a, RMAX, Tn, TTn, maps);
      if (rc) return rc;
    }
    // one launch per 65,535 passes: grid z runs the passes over TTn timesteps each
    // (no tail between passes)
    const int npass = (Tn + TTn - 1) / TTn;
    for (int z0 = 0; z0 < npass; z0 += 65535) {
      const int t0 = z0 * TTn;
      const dim3 grid(ncb, a.nq, std::min(65535, npass - z0));
      const int pe = ctx->prof_begin(st);  // screening and full passes alike
      int rc;
      if (fp64) rc = launch_n1<double>(a, RMAX, TTn, grid, st, t0);
      else if (cmp)
        rc = launch_reg_cmp(maps, a, SelArgs{ctx->PhiCM.as<float>(), Mp, cmp->csel.as<int>(), cmp->nsel.as<int>(), nullptr},
                            RMAX, TTn, ovl, grid, st, t0, tc);
      else rc = ovl ? launch_tma(maps, a, RMAX, TTn, grid, st, t0, tc)
                    : launch_tma_screen(maps, a, RMAX, grid, st, t0, tc);
      if (rc) return rc;
      ++ctx->launches;
      DCF_CHECK_LAUNCH();
      ctx->prof_end(pe, DCFLOW_PROF_N1, st);
    }
    return 0;
  };
  (void)TT;
  // chunk plan: rank class by rank class
  struct Chunk {
    int cls, c0, nq;
  };
  std::vector<Chunk> chunks;
  for (int ci = 0; ci < ncls; ++ci)
    for (int c0 = cls_start[ci]; c0 < cls_start[ci + 1]; c0 += (int)cap)
      chunks.push_back({ci, c0, std::min<int>((int)cap, cls_start[ci + 1] - c0)});
  // two-stream pipeline: preparation of chunk i (decode, r x r systems, row
  // operands; FP64-heavy) on the side stream overlaps the N-1 and final
  // kernels of chunk i-1 (FP32) on the caller's stream
  cudaStream_t side = ctx->side;
  DCF_CUDA(cudaEventRecord(ctx->ev_ready, st));
  DCF_CUDA(cudaStreamWaitEvent(side, ctx->ev_ready, 0));
  for (size_t i = 0; i < chunks.size(); ++i) {
    const Chunk& ch = chunks[i];
    const int bi = (int)(i & 1);
    ChunkBufs& B = ctx->bufs[bi];
    Args a = chunk_args(bi);
    a.nq = ch.nq;
    const int RMAX = classes[ch.cls];
    // preparation: with candidates it carries the pool columns (Text) and leaves
    // the N-0 outputs to the gather of the chosen candidate
    Args ap = a;
    ap.T = Text;
    if (Uc > 0) {
      ap.out.n0_flow = nullptr;
      ap.out.n0_max_loading = nullptr;
    }
    if (i >= 2) DCF_CUDA(cudaStreamWaitEvent(side, ctx->ev_free[bi], 0));
    const int* dperm = ctx->perm.as<int>() + ch.c0;
    k_decode<<<(ch.nq + 127) / 128, 128, 0, side>>>(g, in, dperm, ap);
    if (TI) {
      k_ti_decode<<<ch.nq, 128, 0, side>>>(g, in, ap, bt->n_inj, bt->inj_bus, bt->ti_ptr, bt->ti_mask,
                                            B.tiel.as<int>(), B.tirow.as<int>(), B.nel.as<int>());
      ++ctx->launches;
    }
    if (fp64) launch_prep<double>(ap, RMAX, ch.nq, dyn, side, TI ? B.zcd.p : nullptr, nullptr, nullptr, nullptr);
    else
      launch_prep<float>(ap, RMAX, ch.nq, dyn, side, TI ? B.zcd.p : nullptr, ctx->p0f.as<float>(),
                         ctx->PhiNf.as<float>(), ctx->bNf.as<float>());
    ctx->launches += 3;
    DCF_CHECK_LAUNCH();
    if (cmp) {  // the valid contingencies of every topology (after the denominators)
      k_valid_compact<<<(ch.nq * 32 + 127) / 128, 128, 0, side>>>(a, B.csel.as<int>(), B.nsel.as<int>());
      ++ctx->launches;
      DCF_CHECK_LAUNCH();
    }
    if (want_multi) {  // the multi-outage small systems ride with the FP64 preparation
      const int pe = ctx->prof_begin(side);
      if (fp64)
        launch_multi_prep<double>(ap, ctx->n_multi, ctx->multi_ptr.as<int>(), ctx->multiN.as<int>(), B, nullptr, side);
      else
        launch_multi_prep<float>(ap, ctx->n_multi, ctx->multi_ptr.as<int>(), ctx->multiN.as<int>(), B,
                                 ctx->p0f.as<float>(), side);
      ++ctx->launches;
      DCF_CHECK_LAUNCH();
      ctx->prof_end(pe, DCFLOW_PROF_MULTI_PREP, side);
    }
    DCF_CUDA(cudaEventRecord(ctx->ev_prep[bi], side));
    DCF_CUDA(cudaStreamWaitEvent(st, ctx->ev_prep[bi], 0));
    Args af = a;  // final stage: T real timesteps
    if (Uc > 0) {
      // expand, screen (metric-first: maximum only), select, gather
      const int pex = ctx->prof_begin(st);
      if (TI) {
        if (fp64)
          launch_ti_expand<double>(ap, RMAX, T, Uc, bt, B, ch.nq, st);
        else
          launch_ti_expand<float>(ap, RMAX, T, Uc, bt, B, ch.nq, st);
      } else if (fp64) {
        k_var_expand<double><<<dim3(TV, ch.nq), 128, 0, st>>>(ap, T, U, bt->var_ptr, ctx->var_k.as<int>(),
                                                               bt->var_delta, B.ptv.as<double>(), B.svv.as<double>());
      } else {
        k_var_expand<float><<<dim3(TV, ch.nq), 128, 0, st>>>(ap, T, U, bt->var_ptr, ctx->var_k.as<int>(),
                                                              bt->var_delta, B.ptv.as<float>(), B.svv.as<float>());
      }
      ++ctx->launches;
      DCF_CHECK_LAUNCH();
      ctx->prof_end(pex, DCFLOW_PROF_EXPAND, st);
      Args av = a;
      av.T = TV;
      av.out.n1_cont_max = of ? ctx->of_cmax.as<float>() : nullptr;
      av.cmr = nullptr;  // the screening pass keeps no per-contingency maxima
      av.p2max = nullptr;
      av.ptil = B.ptv.p;
      av.s = B.svv.p;
      av.pmax = B.pmaxv.p;
      av.parg = B.pargv.as<int>();
      av.povl = B.povlv.as<double>();
      if (C_eff > 0) {
        int rc = run_n1(av, RMAX, TV, false, cmp ? &B : nullptr);
        if (rc) return rc;
      } else {
        DCF_CUDA(cudaMemsetAsync(B.pargv.p, 0xff, (size_t)ch.nq * TV * sizeof(int), st));
      }
      int* of_c = ctx->of_top.as<int>();
      int* of_m = of_c + of_n * top_k;
      float* of_l = reinterpret_cast<float*>(of_m + of_n * top_k);
      if (of) {  // output-first: agg_i of every (timestep, candidate), inside the candidate loop
        Args at = av;
        at.tile = nullptr;
        at.out.top_cont = of_c;
        at.out.top_mon = of_m;
        at.out.top_loading = of_l;
        const int pet = ctx->prof_begin(st);
        const int rct = fp64 ? launch_topcases<double>(at, RMAX, at.out.n1_cont_max, ctx->cont_inv.as<int>(),
                                                       ctx->PhiCM.p, top_k, st)
                             : launch_topcases<float>(at, RMAX, at.out.n1_cont_max, ctx->cont_inv.as<int>(),
                                                      ctx->PhiCM.p, top_k, st);
        if (rct) {
          set_error("dcflow_solve_batch: top-k pass shared memory");
          return rct;
        }
        ++ctx->launches;
        DCF_CHECK_LAUNCH();
        ctx->prof_end(pet, DCFLOW_PROF_TOPCASES, st);
      }
      const dim3 gs(ch.nq, (T + 7) / 8);
      if (fp64) k_var_select<double><<<gs, 256, 0, st>>>(av, T, Uc, B.bestu.as<int>());
      else k_var_select<float><<<gs, 256, 0, st>>>(av, T, Uc, B.bestu.as<int>());
      af.ptil = B.ptb.p;
      af.s = B.sb.p;
      af.best_u = B.bestu.as<int>();
      if (fp64) k_var_gather<double><<<dim3(T, ch.nq), 128, 0, st>>>(af, Uc, B.ptv.as<double>(), B.svv.as<double>());
      else k_var_gather<float><<<dim3(T, ch.nq), 128, 0, st>>>(af, Uc, B.ptv.as<float>(), B.svv.as<float>());
      ctx->launches += 2;
      DCF_CHECK_LAUNCH();
      if (of) {  // the chosen candidate's cases
        const size_t nt = (size_t)ch.nq * T * top_k;
        k_top_gather<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(af, Uc, top_k, of_c, of_m, of_l);
        ++ctx->launches;
        DCF_CHECK_LAUNCH();
      }
    }
    if (mode == kModeFeatures) {
      if (fp64)
        k_features<double><<<ch.nq, 256, 0, st>>>(a, g, in, scr->foff.as<int>(), scr->Fp,
                                                   static_cast<__nv_bfloat16*>(sc->X), sc->ldx, 1, sc->status);
      else
        k_features<float><<<ch.nq, 256, 0, st>>>(a, g, in, scr->foff.as<int>(), scr->Fp,
                                                  static_cast<__nv_bfloat16*>(sc->X), sc->ldx, 1, sc->status);
      ++ctx->launches;
      DCF_CHECK_LAUNCH();
      DCF_CUDA(cudaEventRecord(ctx->ev_free[bi], st));
      continue;
    }
    const int* nsel_dev = nullptr;
    if (mode == kModeScreened) {
      // features -> scores (tensor cores) -> top k per row -> union -> N-1 over the union
      const int rows = ch.nq * T, Br = (int)round_up(rows, 128), Fp = scr->Fp, H = scr->H, Cp = scr->Cp;
      if (fp64)
        k_features<double><<<ch.nq, 256, 0, st>>>(a, g, in, scr->foff.as<int>(), Fp, scr->iX.as<__nv_bfloat16>(),
                                                   Fp, 0, nullptr);
      else
        k_features<float><<<ch.nq, 256, 0, st>>>(a, g, in, scr->foff.as<int>(), Fp, scr->iX.as<__nv_bfloat16>(), Fp,
                                                  0, nullptr);
      DCF_CHECK_LAUNCH();
      int* gerr = ctx->err.as<int>();
      GemmSpec g1;
      g1.A = scr->iX.p; g1.lda = Fp; g1.B = scr->wb[0].p; g1.ldb = Fp; g1.M = Br; g1.N = H; g1.K = Fp;
      g1.bias = scr->prm[kB1].as<float>(); g1.relu = true; g1.D = scr->iH1.p; g1.ldd = H; g1.out_bf16 = true;
      GemmSpec g2;
      g2.A = scr->iH1.p; g2.lda = H; g2.B = scr->wb[1].p; g2.ldb = H; g2.M = Br; g2.N = H; g2.K = H;
      g2.bias = scr->prm[kB2].as<float>(); g2.relu = true; g2.D = scr->iH2.p; g2.ldd = H; g2.out_bf16 = true;
      GemmSpec g3;
      g3.A = scr->iH2.p; g3.lda = H; g3.B = scr->wb[2].p; g3.ldb = H; g3.M = Br; g3.N = Cp; g3.K = H;
      g3.bias = scr->prm[kB3].as<float>(); g3.D = scr->iZ.p; g3.ldd = Cp;
      int rc = gemm_run(g1, gerr, st);
      if (!rc) rc = gemm_run(g2, gerr, st);
      if (!rc) rc = gemm_run(g3, gerr, st);
      if (rc) return rc;
      const ChunkBufs& SB = ctx->bufs[0];
      DCF_CUDA(cudaMemsetAsync(SB.selmask.p, 0, (size_t)ch.nq * W * 4, st));
      DCF_CUDA(cudaMemsetAsync(SB.sfb.p, 0, (size_t)ch.nq, st));
      DCF_CUDA(cudaMemsetAsync(SB.nwork.p, 0, 4, st));
      const dcflow_screen_report* rep = sc->rep;
      launch_select(a, T, C, scr->iZ.as<float>(), Cp, sc->top_k, host_float_key(sc->fallback_logit),
                    host_float_key(sc->min_logit), SB, W,
                    rep ? rep->pred : nullptr, st);
      DCF_CHECK_LAUNCH();
      k_compact<<<(ch.nq * 32 + 255) / 256, 256, 0, st>>>(a.qi, ch.nq, C, C_eff, ctx->cont_inv.as<int>(), W,
                                                         SB.selmask.as<uint32_t>(),
                                                         SB.sfb.as<uint8_t>(), SB.csel.as<int>(), SB.nsel.as<int>(),
                                                         SB.work.as<int>(), SB.nwork.as<int>(),
                                                         rep ? rep->n_eval : nullptr, rep ? rep->fallback : nullptr, rep ? rep->evaluated : nullptr);
      DCF_CHECK_LAUNCH();
      ctx->launches += 6;
      const int TTs = pick_tt(T, fp64);
      const int sgrid = (int)std::min<int64_t>((int64_t)ch.nq * ncb, 148 * 16);
      const bool reg_sel = !fp64 && TTs >= 4;  // FP32: the register-tiled kernel over the work items
      int items = 0;
      N1Maps smaps;
      if (reg_sel) {
        DCF_CUDA(cudaMemcpyAsync(&items, SB.nwork.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        DCF_CUDA(cudaStreamSynchronize(st));
        if ((rc = encode_maps(af, RMAX, T, TTs, smaps))) return rc;
      }
      const SelArgs sargs{ctx->PhiCM.as<float>(), Mp, SB.csel.as<int>(), SB.nsel.as<int>(), SB.work.as<int>()};
      for (int t0 = 0; t0 < T; t0 += TTs) {
        const int pe = ctx->prof_begin(st);
        if (reg_sel) rc = items ? launch_reg_sel(smaps, af, sargs, RMAX, TTs, items, st, t0, tc) : 0;
        else rc = fp64 ? launch_sel<double>(af, ctx->PhiCM.p, SB, RMAX, TTs, sgrid, st, t0)
                       : launch_sel<float>(af, ctx->PhiCM.p, SB, RMAX, TTs, sgrid, st, t0);
        if (rc) return rc;
        ++ctx->launches;
        DCF_CHECK_LAUNCH();
        ctx->prof_end(pe, DCFLOW_PROF_N1, st);
      }
      nsel_dev = SB.nsel.as<int>();
    } else if (C_eff > 0) {
      if (use_tile) af.tile = B.tile.as<uint16_t>();
      int rc = run_n1(af, RMAX, T, true, cmp ? &B : nullptr);
      if (rc) return rc;
    }
    {
      const int rcf = fp64 ? launch_final<double>(af, RMAX, st, ctx->PhiCM.p, nsel_dev)
                           : launch_final<float>(af, RMAX, st, ctx->PhiCM.p, nsel_dev);
      if (rcf) {
        set_error("dcflow_solve_batch: final pass launch (remainder columns' shared memory)");
        return rcf;
      }
    }
    ++ctx->launches;
    DCF_CHECK_LAUNCH();
    if (want_multi) {
      const int pe = ctx->prof_begin(st);
      const int rcm = fp64 ? launch_multi_rows<double>(af, RMAX, ctx->n_multi, ctx->n_multi_ent, ctx->multi_ptr.as<int>(),
                                                       ctx->multi_mpos.as<int>(), ctx->PhiMO.p, B, st)
                           : launch_multi_rows<float>(af, RMAX, ctx->n_multi, ctx->n_multi_ent, ctx->multi_ptr.as<int>(),
                                                      ctx->multi_mpos.as<int>(), ctx->PhiMO.p, B, st);
      if (rcm) return rcm;
      ++ctx->launches;
      DCF_CHECK_LAUNCH();
      ctx->prof_end(pe, DCFLOW_PROF_MULTI, st);
    }
    if (G > 0) {
      const int pe = ctx->prof_begin(st);
      const int ng = fp64 ? launch_gen<double>(af, RMAX, G, bt->gen_bus, bt->gen_p, ctx->PtdfN.as<double>(), ctx->V,
                                               ctx->gen_cols.p, st)
                          : launch_gen<float>(af, RMAX, G, bt->gen_bus, bt->gen_p, ctx->PtdfN.as<double>(), ctx->V,
                                              ctx->gen_cols.p, st);
      if (ng < 0) return -ng;  // a tensor map the driver refused (the message is set)
      ctx->launches += ng;
      DCF_CHECK_LAUNCH();
      ctx->prof_end(pe, DCFLOW_PROF_GEN, st);
    }
    if (top_k > 0 && !of) {  // metric-first: the chosen candidate's cases only
      const int pe = ctx->prof_begin(st);
      const int rct = fp64 ? launch_topcases<double>(af, RMAX, af.out.n1_cont_max, ctx->cont_inv.as<int>(),
                                                     ctx->PhiCM.p, top_k, st)
                           : launch_topcases<float>(af, RMAX, af.out.n1_cont_max, ctx->cont_inv.as<int>(),
                                                    ctx->PhiCM.p, top_k, st);
      if (rct) {
        set_error("dcflow_solve_batch: top-k pass shared memory");
        return rct;
      }
      ++ctx->launches;
      DCF_CHECK_LAUNCH();
      ctx->prof_end(pe, DCFLOW_PROF_TOPCASES, st);
    }
    DCF_CUDA(cudaEventRecord(ctx->ev_free[bi], st));
  }
  return DCFLOW_OK;
}

extern "C" int dcflow_solve_batch(dcflow_ctx* ctx, const dcflow_batch* bt, const dcflow_results* res, void* stream) {
  return solve_impl(ctx, bt, res, stream, nullptr);
}

// ---------------------------------------------------------------------------
// autotuner: coordinate descent over the schedule, each candidate timed on the
// sample with CUDA events (a warm-up solve, then the best of two)
// ---------------------------------------------------------------------------
static int autotune_impl(dcflow_ctx* ctx, const dcflow_batch* bt, const dcflow_results* res, void* stream,
                         std::vector<dcflow_schedule>* tried, SchedPlan* pick, float* pick_ms) {
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  DCF_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    set_error("dcflow_autotune: cudaEventCreate failed");
    return DCFLOW_ERR_CUDA;
  }
  const bool prof = ctx->prof_on;
  ctx->prof_on = false;  // tuning solves stay out of the kernel timers
  const bool fp64 = ctx->opt.precision == DCFLOW_FP64;
  int rc = 0;
  auto time_plan = [&](const SchedPlan& P, float* ms) -> int {
    ctx->tuning = true;
    ctx->tune_plan = P;
    int r = solve_impl(ctx, bt, res, stream, nullptr);  // warm-up: first-use allocations
    float best = 3.4e38f;
    for (int k = 0; k < 2 && !r; ++k) {
      if (cudaEventRecord(e0, st) != cudaSuccess) r = DCFLOW_ERR_CUDA;
      if (!r) r = solve_impl(ctx, bt, res, stream, nullptr);
      if (!r && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
        r = DCFLOW_ERR_CUDA;
      float t = 0.f;
      if (!r && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) r = DCFLOW_ERR_CUDA;
      if (!r) best = std::min(best, t);
    }
    ctx->tuning = false;
    *ms = best;
    if (!r && tried) tried->push_back(to_schedule(P, best));
    return r;
  };
  SchedPlan cur;
  cur.compact = ctx->opt.compact_n1 ? 1 : 0;
  float tcur = 0.f;
  rc = time_plan(cur, &tcur);
  // a candidate replaces the current schedule only when it is faster by more than 1 %
  auto consider = [&](const SchedPlan& P) -> int {
    if (P == cur) return 0;
    float t = 0.f;
    const int r = time_plan(P, &t);
    if (!r && t < 0.99f * tcur) {
      cur = P;
      tcur = t;
    }
    return r;
  };
  // 1. scratch budget (chunk size): bounded by a third of the free device memory per set
  size_t free_b = 0, total_b = 0;
  if (!rc && cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) rc = DCFLOW_ERR_CUDA;
  const int budgets[] = {2048, 32768};
  for (int b : budgets) {
    if (rc) break;
    if (((size_t)b << 20) * 3 > free_b) continue;
    SchedPlan P = cur;
    P.budget_mb = b;
    rc = consider(P);
  }
  // 2. rank classes
  const int bounds[][3] = {{8, 16, 0}, {4, 16, 0}, {16, 0, 0}};
  for (const auto& bd : bounds) {
    if (rc) break;
    SchedPlan P = cur;
    for (int i = 0; i < 3; ++i) P.bounds[i] = bd[i];
    rc = consider(P);
  }
  // 3. dense or compacted N-1 (FP32 forms)
  if (!rc && !fp64) {
    SchedPlan P = cur;
    P.compact = 1 - cur.compact;
    rc = consider(P);
  }
  // 4. the contingency remainder in the final pass or in a block of its own (when there is one)
  if (!rc && ctx->C_eff > 64 && ctx->C_eff % 64 > 0 && ctx->C_eff % 64 <= 4) {
    SchedPlan P = cur;
    P.remainder = 1 - cur.remainder;
    rc = consider(P);
  }
  ctx->prof_on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  ShapeKey key;
  key.T = bt->n_time;
  key.U = bt->n_var;
  key.ti = bt->ti_ptr != nullptr;
  if (key.ti) key.U = ctx->last_uc;
  key.top_k = res->top_k;
  key.gen = bt->n_gen;
  key.multi = res->multi_max_loading != nullptr;
  key.mode = 0;
  bool stored = false;
  for (auto& kv : ctx->tuned)
    if (kv.first == key) {
      kv.second = cur;
      stored = true;
    }
  if (!stored) ctx->tuned.push_back({key, cur});
  if (pick) *pick = cur;
  if (pick_ms) *pick_ms = tcur;
  return DCFLOW_OK;
}

extern "C" int dcflow_autotune(dcflow_ctx* ctx, const dcflow_batch* sample, const dcflow_results* res, void* stream,
                               dcflow_schedule* tried, int32_t max_tried, int32_t* n_tried, dcflow_schedule* pick) {
  if (!ctx || !sample || !res || sample->n_topo < 1 || (tried && max_tried < 0)) {
    set_error("dcflow_autotune: null argument or empty sample");
    return DCFLOW_ERR_INVALID_ARG;
  }
  if (ctx->tuning) {
    set_error("dcflow_autotune: already tuning");
    return DCFLOW_ERR_INVALID_ARG;
  }
  std::vector<dcflow_schedule> all;
  SchedPlan pk;
  float ms = 0.f;
  const int rc = autotune_impl(ctx, sample, res, stream, &all, &pk, &ms);
  if (rc) return rc;
  if (n_tried) *n_tried = (int32_t)all.size();
  if (tried)
    for (int i = 0; i < (int)all.size() && i < max_tried; ++i) tried[i] = all[i];
  if (pick) *pick = to_schedule(pk, ms);
  return DCFLOW_OK;
}

extern "C" int dcflow_set_schedule(dcflow_ctx* ctx, const dcflow_schedule* s) {
  if (!ctx) {
    set_error("dcflow_set_schedule: null context");
    return DCFLOW_ERR_INVALID_ARG;
  }
  if (!s) {
    ctx->sched_fixed = false;
    return DCFLOW_OK;
  }
  // bounds: ascending, from {4, 8, 16}, the last 16, then zeros
  int prev = 0, last = 0;
  bool ok = s->budget_mb > 0;
  for (int i = 0; i < 3 && ok; ++i) {
    const int b = s->rank_bounds[i];
    if (b == 0) {
      for (int j = i; j < 3; ++j) ok = ok && s->rank_bounds[j] == 0;
      break;
    }
    ok = (b == 4 || b == 8 || b == 16) && b > prev;
    prev = last = b;
  }
  if (!ok || last != 16) {
    set_error("dcflow_set_schedule: budget_mb > 0 and rank_bounds ascending from {4, 8, 16} ending with 16");
    return DCFLOW_ERR_INVALID_ARG;
  }
  SchedPlan P;
  P.budget_mb = s->budget_mb;
  for (int i = 0; i < 3; ++i) P.bounds[i] = s->rank_bounds[i];
  P.compact = s->compact_n1 ? 1 : 0;
  P.remainder = s->remainder ? 1 : 0;
  ctx->sched = P;
  ctx->sched_fixed = true;
  return DCFLOW_OK;
}

extern "C" int dcflow_last_schedule(const dcflow_ctx* ctx, dcflow_schedule* out) {
  if (!ctx || !out) {
    set_error("dcflow_last_schedule: null argument");
    return DCFLOW_ERR_INVALID_ARG;
  }
  *out = to_schedule(ctx->last_plan, 0.f);
  return DCFLOW_OK;
}

static int screen_matches(const dcflow_ctx* ctx, const dcflow_screen* s, const char* who) {
  if (!ctx || !s) {
    set_error(std::string(who) + ": null context or screener");
    return DCFLOW_ERR_INVALID_ARG;
  }
  if (s->ctx != ctx || s->M != ctx->M || s->C != ctx->C || s->V != ctx->V) {
    set_error(std::string(who) + ": the screener was created for another context or study");
    return DCFLOW_ERR_INVALID_ARG;
  }
  return 0;
}

extern "C" int dcflow_screen_features(dcflow_ctx* ctx, const dcflow_screen* s, const dcflow_batch* bt, void* X,
                                      int64_t ldx, uint8_t* status, void* stream) {
  int rc = screen_matches(ctx, s, "dcflow_screen_features");
  if (rc) return rc;
  if (!X || ldx < s->Fp || ldx % 8) {
    set_error("dcflow_screen_features: need X with ldx >= F_pad, ldx % 8 == 0");
    return DCFLOW_ERR_INVALID_ARG;
  }
  ScreenCall sc;
  sc.mode = kModeFeatures;
  sc.scr = const_cast<dcflow_screen*>(s);
  sc.X = X;
  sc.ldx = ldx;
  sc.status = status;
  return solve_impl(ctx, bt, nullptr, stream, &sc);
}

extern "C" int dcflow_solve_batch_screened(dcflow_ctx* ctx, const dcflow_batch* bt, const dcflow_results* res,
                                           dcflow_screen* s, const dcflow_screen_options* opt,
                                           const dcflow_screen_report* rep, void* stream) {
  int rc = screen_matches(ctx, s, "dcflow_solve_batch_screened");
  if (rc) return rc;
  if (!opt || opt->top_k < 1) {
    set_error("dcflow_solve_batch_screened: need options with top_k >= 1");
    return DCFLOW_ERR_INVALID_ARG;
  }
  ScreenCall sc;
  sc.mode = kModeScreened;
  sc.scr = s;
  sc.top_k = opt->top_k;
  sc.fallback_logit = opt->fallback_logit;
  // probability threshold -> logit threshold (0 or out of (0, 1): no additions)
  sc.min_logit = (opt->min_prob > 0.f && opt->min_prob < 1.f) ? std::log(opt->min_prob / (1.f - opt->min_prob))
                                                                : INFINITY;
  sc.rep = rep;
  return solve_impl(ctx, bt, res, stream, &sc);
}

extern "C" int dcflow_profile(dcflow_ctx* ctx, int32_t enable) {
  if (!ctx) return DCFLOW_ERR_INVALID_ARG;
  ctx->prof_on = enable != 0;
  ctx->prof_used = 0;
  return DCFLOW_OK;
}

extern "C" int dcflow_profile_read_kind(dcflow_ctx* ctx, int32_t kind, double* ms_out, int64_t* launches) {
  if (!ctx || !ms_out || !launches) return DCFLOW_ERR_INVALID_ARG;
  double ms = 0.0;
  int64_t n = 0;
  for (size_t i = 0; i + 1 < ctx->prof_used; i += 2) {
    if (ctx->prof_kind[i / 2] != kind) continue;
    DCF_CUDA(cudaEventSynchronize(ctx->prof_ev[i + 1]));
    float x = 0.f;
    DCF_CUDA(cudaEventElapsedTime(&x, ctx->prof_ev[i], ctx->prof_ev[i + 1]));
    ms += x;
    ++n;
  }
  *ms_out = ms;
  *launches = n;
  return DCFLOW_OK;
}

extern "C" int dcflow_profile_read(dcflow_ctx* ctx, double* n1_ms, int64_t* n1_launches) {
  return dcflow_profile_read_kind(ctx, DCFLOW_PROF_N1, n1_ms, n1_launches);
}
