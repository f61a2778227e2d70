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
#include "internal.cuh"

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
    if (c < 0 || c >= g.E || g.nidx[c] < 0) return ST_INVALID;
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
  int8_t es[kEntMax];
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
    S.es[e] = a.ent_s[(size_t)q * kEntMax + e];
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
      acc = fma((double)S.es[e], z_entry(S, a.PhiN + (size_t)m * a.NN, m, j), acc);
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
        for (int e = S.mp[i]; e < S.mp[i + 1]; ++e) acc = fma((double)S.es[e], a.p0[(size_t)S.en[e] * T + t], acc);
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
  // Vt[j][c]
  const int C = a.C;
  Real* VtR = static_cast<Real*>(a.VtR);
  for (int c = tid; c < C; c += blockDim.x) {
    const int nc = a.contN[c];
    double v[RMAX];
#pragma unroll
    for (int i = 0; i < RMAX; ++i) {
      double acc = 0.0;
      if (i < r)
        for (int e = S.mp[i]; e < S.mp[i + 1]; ++e) {
          const int m = S.en[e];
          acc = fma((double)S.es[e], a.PhiN[(size_t)m * a.NN + nc], acc);
          if (i < ks && m == nc) acc -= (double)S.es[e];
        }
      v[i] = acc;
    }
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
      double x = 0.0;
#pragma unroll
      for (int i = 0; i < RMAX; ++i) x = fma(Ki[j][i], v[i], x);  // Ki is zero outside r x r
      const size_t o = ((size_t)q * kRMax + j) * C + c;
      a.Vt64[o] = x;
      VtR[o] = (Real)x;
    }
  }
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
__global__ __launch_bounds__(128) void k_rows(Args a) {
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
    for (int j = 0; j < RMAX; ++j) z[j] = (j < r) ? z_entry_col_r<Real>(S, a.PhiN, NN, a.bN, nl, j) : (Real)0;
    const Real il = (Real)a.inv_lim[l];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) Zs[(size_t)j * Mp + l] = outd ? (Real)0 : z[j] * il;
    meta[l] = (Real)0;
    meta[Mp + l] = outd ? (Real)0 : (Real)1;
    if (sizeof(Real) == 4) {
      reinterpret_cast<int*>(meta)[2 * Mp + l] = a.cpos[l];
    } else {
      meta[2 * Mp + l] = (Real)a.cpos[l];
    }
    meta[3 * Mp + l] = (Real)0;
    for (int t = 0; t < T; ++t) {
      Real pf = (Real)a.p0[(size_t)nl * T + t];
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
    for (int t = 0; t < T; ++t) {
      Real pf = (Real)a.p0[(size_t)nc * T + t];
#pragma unroll
      for (int j = 0; j < RMAX; ++j) pf = fma(-(Real)z[j], alph[j * T + t], pf);
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
      double m = 0.0;
      for (int l = lane; l < M; l += 32) m = fmax(m, fabs((double)ptil[(size_t)t * Mp + l]));
      for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) a.out.n0_max_loading[(size_t)tau * T + t] = m;
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
  static __device__ __forceinline__ void add(double& mx, double& ov, double v) {
    const double av = fabs(v);
    mx = fmax(mx, av);
    ov += fmax(av - 1.0, 0.0);
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

template <class Real, int TT, int RMAX, int LT>
__global__ __launch_bounds__(64) void k_n1(Args a, int t0) {
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
      phi[i] = phi_entry<Real, RMAX>(base, zs[i], vt, rm[i], cp[i], c, dg[i]);
    }
#pragma unroll
    for (int t = 0; t < TT; ++t) {
      const Real st = s[t];
#pragma unroll
      for (int i = 0; i < LT; ++i) Acc<Real>::add(mx[t], ov[t], fma(phi[i], st, pt[i][t]));
    }
  }
  // reduce the 64 contingencies of this block: max (ties: lowest c) and overload sum
  const bool ok = cin && a.valid[(size_t)q * C + c];
  if (a.out.n1_cont_max && cin) {
#pragma unroll
    for (int t = 0; t < TT; ++t)
      if (t0 + t < T) a.out.n1_cont_max[((size_t)qi.tau * T + t0 + t) * C + c] = ok ? (float)mx[t] : -1.f;
  }
  __shared__ double rv[2], ro[2];
  __shared__ int ra[2];
  const int lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int t = 0; t < TT; ++t) {
    if (t0 + t < T) {  // uniform over the block
      double v = ok ? (double)mx[t] : -1.0;
      int arg = ok ? c : 0x7fffffff;
      double o = ok ? (double)ov[t] * Acc<Real>::ovl_scale() : 0.0;
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, off);
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
        double bv = rv[0];
        int ba = ra[0];
        if (rv[1] > bv || (rv[1] == bv && ra[1] < ba)) {
          bv = rv[1];
          ba = ra[1];
        }
        const size_t o2 = ((size_t)q * T + t0 + t) * a.ncb + blockIdx.x;
        static_cast<Real*>(a.pmax)[o2] = (Real)bv;
        a.parg[o2] = (bv < 0.0) ? -1 : ba;
        a.povl[o2] = ro[0] + ro[1];
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
__global__ __launch_bounds__(128) void k_final(Args a) {
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
  const Real* PhiMC = static_cast<const Real*>(a.PhiMC);
  const Real* Zs = static_cast<const Real*>(a.Zs) + (size_t)q * kRMax * Mp;
  const Real* ptil = static_cast<const Real*>(a.ptil) + (size_t)q * T * Mp;
  const Real* meta = static_cast<const Real*>(a.diagv) + (size_t)q * 4 * Mp;
  const Real* VtR = static_cast<const Real*>(a.VtR) + (size_t)q * kRMax * C;
  const Real* sv = static_cast<const Real*>(a.s) + (size_t)q * T * C;
  for (int t = tid >> 5; t < T; t += nw) {
    double bv = -1.0, ovl = 0.0;
    int ba = 0x7fffffff;
    for (int b = lane; b < a.ncb; b += 32) {
      const size_t k = ((size_t)q * T + t) * a.ncb + b;
      const double v = (double)static_cast<const Real*>(a.pmax)[k];
      const int ar = a.parg[k];
      if (ar >= 0 && (v > bv || (v == bv && ar < ba))) {
        bv = v;
        ba = ar;
      }
      ovl += a.povl[k];
    }
    for (int off = 16; off; off >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, bv, off);
      const int a2 = __shfl_xor_sync(0xffffffffu, ba, off);
      ovl += __shfl_xor_sync(0xffffffffu, ovl, off);
      if (v2 > bv || (v2 == bv && a2 < ba)) {
        bv = v2;
        ba = a2;
      }
    }
    const int c = (ba == 0x7fffffff) ? -1 : ba;
    if (lane == 0) {
      const size_t k = (size_t)tau * T + t;
      o.n1_max_loading[k] = c >= 0 ? bv : 0.0;
      o.overload_sum[k] = ovl;
      o.worst_cont[k] = c;
      if (o.best_var) o.best_var[k] = a.best_u ? a.best_u[(size_t)q * T + t] : -1;
    }
    if (o.worst_mon) {
      double v = -1.0;
      int arg = 0x7fffffff;
      if (c >= 0) {
        Real vt[RMAX];
#pragma unroll
        for (int j = 0; j < RMAX; ++j) vt[j] = VtR[(size_t)j * C + c];
        const Real st = sv[(size_t)t * C + c];
        for (int l = lane; l < M; l += 32) {
          Real zr[RMAX];
#pragma unroll
          for (int j = 0; j < RMAX; ++j) zr[j] = Zs[(size_t)j * Mp + l];
          const Real ph = phi_entry<Real, RMAX>(PhiMC[(size_t)l * a.ldc + c], zr, vt, meta[Mp + l], a.cpos[l], c, meta[l]);
          const double x = (double)fabs(fma(ph, st, ptil[(size_t)t * Mp + l]));
          if (x > v) {
            v = x;
            arg = l;
          }
        }
      }
      for (int off = 16; off; off >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, off);
        const int a2 = __shfl_xor_sync(0xffffffffu, arg, off);
        if (v2 > v || (v2 == v && a2 < arg)) {
          v = v2;
          arg = a2;
        }
      }
      if (lane == 0) o.worst_mon[(size_t)tau * T + t] = (c >= 0) ? arg : -1;
    }
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
  for (int l = threadIdx.x; l < M; l += blockDim.x) {
    Real v = pt[(size_t)t * Mp + l];
    for (int k = k0; k < k1; ++k) v = fma((Real)var_delta[k], pt[(size_t)(T + var_k[k]) * Mp + l], v);
    po[l] = v;
  }
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    Real v = sv[(size_t)t * C + c];
    for (int k = k0; k < k1; ++k) v = fma((Real)var_delta[k], sv[(size_t)(T + var_k[k]) * C + c], v);
    so[c] = v;
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
  double bv = 1e300;
  int bu = 0x7fffffff;
  for (int u = lane; u < U; u += 32) {
    double v = -1.0;
    for (int b = 0; b < av.ncb; ++b) {
      const size_t k = ((size_t)q * TV + (size_t)t * U + u) * av.ncb + b;
      if (av.parg[k] >= 0) v = fmax(v, (double)static_cast<const Real*>(av.pmax)[k]);
    }
    if (v < 0.0) v = 0.0;  // no valid contingency: loading 0
    if (v < bv || (v == bv && u < bu)) {
      bv = v;
      bu = u;
    }
  }
  for (int off = 16; off; off >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, bv, off);
    const int u2 = __shfl_xor_sync(0xffffffffu, bu, off);
    if (v2 < bv || (v2 == bv && u2 < bu)) {
      bv = v2;
      bu = u2;
    }
  }
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
  double m = 0.0;
  for (int l = threadIdx.x; l < M; l += blockDim.x) {
    const Real v = pi[l];
    po[l] = v;
    m = fmax(m, fabs((double)v));
    if (af.out.n0_flow) af.out.n0_flow[((size_t)qi.tau * T + t) * M + l] = (double)v / af.inv_lim[l];
  }
  for (int c = threadIdx.x; c < C; c += blockDim.x) so[c] = si[c];
  if (af.out.n0_max_loading) {
    __shared__ double red[32];
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      double x = red[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) x = fmax(x, red[w]);
      af.out.n0_max_loading[(size_t)qi.tau * T + t] = x;
    }
  }
}

}  // namespace dcf

#include "n1_tma.cuh"

using namespace dcf;

namespace {

struct Plan {
  int TT, RMAX, LT;
};

int pick_tt(int T, bool fp64) {
  const int opts32[] = {1, 4, 8, 16, 24, 32};
  const int opts64[] = {1, 4, 8};
  const int* o = fp64 ? opts64 : opts32;
  const int n = fp64 ? 3 : 6;
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
        return DCFLOW_ERR_INVALID_ARG;
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
void launch_final(const Args& a, int RMAX, cudaStream_t st) {
  if (RMAX == 4) k_final<Real, 4><<<a.nq, 128, 0, st>>>(a);
  else if (RMAX == 8) k_final<Real, 8><<<a.nq, 128, 0, st>>>(a);
  else k_final<Real, 16><<<a.nq, 128, 0, st>>>(a);
}

int rank_class(int r) { return r <= 4 ? 4 : (r <= 8 ? 8 : 16); }

// per-topology r x r systems and row operands of one chunk
template <class Real>
void launch_prep(const Args& a, int RMAX, int nq, size_t dyn, cudaStream_t st) {
  if (RMAX == 4) {
    k_small<Real, 4><<<nq, 128, 0, st>>>(a);
    k_rows<Real, 4><<<nq, 128, dyn, st>>>(a);
  } else if (RMAX == 8) {
    k_small<Real, 8><<<nq, 128, 0, st>>>(a);
    k_rows<Real, 8><<<nq, 128, dyn, st>>>(a);
  } else {
    k_small<Real, 16><<<nq, 128, 0, st>>>(a);
    k_rows<Real, 16><<<nq, 128, dyn, st>>>(a);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
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

// Row-major FP32 tensor of `rank` dims (innermost first); strides in bytes for dims 1..rank-1.
int encode_map(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
               const uint32_t* box) {
  auto fn = tensor_map_encoder();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return DCFLOW_ERR_CUDA;
  }
  cuuint64_t d[5], s[4];
  cuuint32_t b[5], e[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    e[i] = 1;
    if (i + 1 < rank) s[i] = strides[i];
  }
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<void*>(base), d, s, b, e,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return DCFLOW_ERR_CUDA;
  }
  return 0;
}

template <int TT, int RMAX, bool OVL = true>
int launch_tma_t(const N1Maps& maps, const Args& a, dim3 grid, cudaStream_t st, int t0) {
  using L = TmaLayout<TT, RMAX>;
  constexpr int NTH = TT >= 16 ? 2 : 1;  // threads per contingency
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_n1_tma<TT, RMAX, NTH, OVL>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes) !=
        cudaSuccess)
      return DCFLOW_ERR_CUDA;
    attr = true;
  }
  k_n1_tma<TT, RMAX, NTH, OVL><<<grid, kCB * NTH, L::kBytes, st>>>(maps, a, t0);
  return 0;
}

// max-only pass over 32 virtual timesteps (injection candidates)
int launch_tma_screen(const N1Maps& maps, const Args& a, int RMAX, dim3 grid, cudaStream_t st, int t0) {
  if (RMAX == 4) return launch_tma_t<32, 4, false>(maps, a, grid, st, t0);
  if (RMAX == 8) return launch_tma_t<32, 8, false>(maps, a, grid, st, t0);
  return launch_tma_t<32, 16, false>(maps, a, grid, st, t0);
}

template <int RMAX>
int launch_tma_r(const N1Maps& maps, const Args& a, int TT, dim3 grid, cudaStream_t st, int t0) {
  switch (TT) {
    case 1: return launch_tma_t<1, RMAX>(maps, a, grid, st, t0);
    case 4: return launch_tma_t<4, RMAX>(maps, a, grid, st, t0);
    case 8: return launch_tma_t<8, RMAX>(maps, a, grid, st, t0);
    case 16: return launch_tma_t<16, RMAX>(maps, a, grid, st, t0);
    case 24: return launch_tma_t<24, RMAX>(maps, a, grid, st, t0);
    default: return launch_tma_t<32, RMAX>(maps, a, grid, st, t0);
  }
}

int launch_tma(const N1Maps& maps, const Args& a, int RMAX, int TT, dim3 grid, cudaStream_t st, int t0) {
  if (RMAX == 4) return launch_tma_r<4>(maps, a, TT, grid, st, t0);
  if (RMAX == 8) return launch_tma_r<8>(maps, a, TT, grid, st, t0);
  return launch_tma_r<16>(maps, a, TT, grid, st, t0);
}

}  // namespace

extern "C" int dcflow_solve_batch(dcflow_ctx* ctx, const dcflow_batch* bt, const dcflow_results* res, void* stream) {
  if (!ctx || !bt || !res) {
    set_error("dcflow_solve_batch: null argument");
    return DCFLOW_ERR_INVALID_ARG;
  }
  if (!ctx->has_study) {
    set_error("dcflow_solve_batch: no study bound (dcflow_set_study)");
    return DCFLOW_ERR_NO_STUDY;
  }
  const int N = bt->n_topo, T = bt->n_time;
  if (N < 0 || T < 1 || T > 256 || bt->n_var < 0) {
    set_error("dcflow_solve_batch: need n_topo >= 0, 1 <= n_time <= 256, n_var >= 0");
    return DCFLOW_ERR_INVALID_ARG;
  }
  ctx->launches = 0;
  if (N == 0) return DCFLOW_OK;
  if (!bt->split_ptr || !bt->out_ptr || !bt->inj || !res->n1_max_loading || !res->overload_sum ||
      !res->worst_cont || !res->island_flag || !res->n_island_cont) {
    set_error("dcflow_solve_batch: missing required pointer");
    return DCFLOW_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool fp64 = ctx->opt.precision == DCFLOW_FP64;
  const size_t rs = fp64 ? sizeof(double) : sizeof(float);
  const int M = ctx->M, C = ctx->C, NN = ctx->NN;
  // injection candidates T_i (Eq. (8)): read the small CSR to the host, validate
  // it, and map every entry to a pool bus (a column of the extended base flows)
  const int U = bt->n_var;
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
  ++ctx->launches;
  DCF_CHECK_LAUNCH();
  GridDev g{ctx->f.as<int>(), ctx->t.as<int>(), ctx->b.as<double>(), ctx->inc_ptr.as<int>(), ctx->inc_list.as<int>(),
            ctx->nidx.as<int>(), ctx->split_ok.as<uint8_t>(), ctx->V, ctx->E};
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
  std::vector<int> cls_start(4, 0);
  const int classes[3] = {4, 8, 16};
  for (int ci = 0; ci < 3; ++ci) {
    cls_start[ci] = (int)perm.size();
    for (int i = 0; i < N; ++i) {
      const int r = hr[i] < 0 ? 0 : hr[i];
      if (rank_class(r) == classes[ci]) perm.push_back(i);
    }
  }
  cls_start[3] = N;
  if (ctx->perm.ensure(sizeof(int) * N)) return DCFLOW_ERR_OOM;
  DCF_CUDA(cudaMemcpyAsync(ctx->perm.p, perm.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  // chunk capacity from a scratch budget per buffer set (two sets alternate);
  // large chunks keep the N-1 launches wide (measured better than many small
  // overlapping chunks: the N-1 kernel fills the SMs' registers and shared
  // memory, so preparation kernels of the next chunk only run in its tail)
  const int ncb = (C + 63) / 64;
  const int Mp = (int)round_up(M, 16);
  const int TV = T * U;  // virtual timesteps: (timestep, candidate) pairs
  if (R > 64) {
    set_error("dcflow_solve_batch: at most 64 distinct candidate buses");
    return DCFLOW_ERR_INVALID_ARG;
  }
  size_t per_slot = (size_t)kEntMax * (sizeof(int) + sizeof(double) + 1) + (kRMax + 1) * 2 + sizeof(QInfo) +
                    (size_t)kRMax * kRMax * 8 + (size_t)kRMax * Text * 8 + (size_t)kRMax * C * (8 + rs) +
                    (size_t)Mp * (kRMax + Text + 4) * rs + (size_t)Text * C * rs + C + 4 +
                    (size_t)T * ncb * (rs + 4 + 8) + 64;
  if (U > 0)
    per_slot += (size_t)TV * (Mp + C) * rs + (size_t)TV * ncb * (rs + 4 + 8) + (size_t)T * 4 + (size_t)T * (Mp + C) * rs;
  int64_t cap = ctx->opt.chunk_topo > 0 ? ctx->opt.chunk_topo : (int64_t)((size_t)2 << 30) / (int64_t)per_slot;
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
    if (U > 0 && (B.ptv.ensure(c * TV * Mp * rs) || B.svv.ensure(c * TV * std::max(C, 1) * rs) ||
                  B.pmaxv.ensure(c * TV * std::max(ncb, 1) * rs) ||
                  B.pargv.ensure(c * TV * std::max(ncb, 1) * sizeof(int)) ||
                  B.povlv.ensure(c * TV * std::max(ncb, 1) * sizeof(double)) || B.bestu.ensure(c * T * sizeof(int)) ||
                  B.ptb.ensure(c * T * Mp * rs) || B.sb.ensure(c * T * std::max(C, 1) * rs)))
      return DCFLOW_ERR_OOM;
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
  base.U = U;
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
  base.Mpad = Mp;
  base.ldc = ctx->ldc;
  base.err = ctx->err.as<int>();
  base.best_u = nullptr;
  base.out = *res;
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
    a.ptil = B.ptil.p;
    a.rowmul = nullptr;
    a.diagv = B.meta.p;
    a.s = B.s.p;
    a.valid = B.valid.as<uint8_t>();
    a.nisl = B.nisl.as<int>();
    a.pmax = B.pmax.p;
    a.parg = B.parg.as<int>();
    a.povl = B.povl.as<double>();
    return a;
  };
  const int TT = pick_tt(T, fp64);
  const size_t dyn = (size_t)kRMax * Text * rs;
  // N-1 passes over Tn (virtual) timesteps whose operands are a.ptil / a.s;
  // ovl = false screens the maximum only (FP32 form)
  auto run_n1 = [&](const Args& a, int RMAX, int Tn, bool ovl) -> int {
    const int TTn = ovl ? pick_tt(Tn, fp64) : (fp64 ? 8 : 32);
    N1Maps maps;
    if (!fp64) {
      const uint64_t d_phi[2] = {(uint64_t)C, (uint64_t)M}, s_phi[1] = {(uint64_t)ctx->ldc * 4};
      const uint32_t b_phi[2] = {kCB, kLT};
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
      if (!rc) rc = encode_map(&maps.zt, a.Zs, 3, d_zt, s_zt, b_zt);
      if (!rc) rc = encode_map(&maps.pt, a.ptil, 3, d_pt, s_pt, b_pt);
      if (rc) return rc;
    }
    for (int t0 = 0; t0 < Tn; t0 += TTn) {
      const dim3 grid(ncb, a.nq);
      const bool prof = ctx->prof_on;  // screening and full passes alike
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (prof) {
        while (ctx->prof_ev.size() < ctx->prof_used + 2) {
          cudaEvent_t e;
          DCF_CUDA(cudaEventCreate(&e));
          ctx->prof_ev.push_back(e);
        }
        e0 = ctx->prof_ev[ctx->prof_used];
        e1 = ctx->prof_ev[ctx->prof_used + 1];
        ctx->prof_used += 2;
        DCF_CUDA(cudaEventRecord(e0, st));
      }
      int rc;
      if (fp64) rc = launch_n1<double>(a, RMAX, TTn, grid, st, t0);
      else rc = ovl ? launch_tma(maps, a, RMAX, TTn, grid, st, t0) : launch_tma_screen(maps, a, RMAX, grid, st, t0);
      if (rc) return rc;
      ++ctx->launches;
      DCF_CHECK_LAUNCH();
      if (prof) DCF_CUDA(cudaEventRecord(e1, st));
    }
    return 0;
  };
  (void)TT;
  // chunk plan: rank class by rank class
  struct Chunk {
    int cls, c0, nq;
  };
  std::vector<Chunk> plan;
  for (int ci = 0; ci < 3; ++ci)
    for (int c0 = cls_start[ci]; c0 < cls_start[ci + 1]; c0 += (int)cap)
      plan.push_back({ci, c0, std::min<int>((int)cap, cls_start[ci + 1] - c0)});
  // two-stream pipeline: preparation of chunk i (decode, r x r systems, row
  // operands; FP64-heavy) on the side stream overlaps the N-1 and final
  // kernels of chunk i-1 (FP32) on the caller's stream
  cudaStream_t side = ctx->side;
  DCF_CUDA(cudaEventRecord(ctx->ev_ready, st));
  DCF_CUDA(cudaStreamWaitEvent(side, ctx->ev_ready, 0));
  for (size_t i = 0; i < plan.size(); ++i) {
    const Chunk& ch = plan[i];
    const int bi = (int)(i & 1);
    ChunkBufs& B = ctx->bufs[bi];
    Args a = chunk_args(bi);
    a.nq = ch.nq;
    const int RMAX = classes[ch.cls];
    // preparation: with candidates it carries the pool columns (Text) and leaves
    // the N-0 outputs to the gather of the chosen candidate
    Args ap = a;
    ap.T = Text;
    if (U > 0) {
      ap.out.n0_flow = nullptr;
      ap.out.n0_max_loading = nullptr;
    }
    if (i >= 2) DCF_CUDA(cudaStreamWaitEvent(side, ctx->ev_free[bi], 0));
    const int* dperm = ctx->perm.as<int>() + ch.c0;
    k_decode<<<(ch.nq + 127) / 128, 128, 0, side>>>(g, in, dperm, ap);
    if (fp64) launch_prep<double>(ap, RMAX, ch.nq, dyn, side);
    else launch_prep<float>(ap, RMAX, ch.nq, dyn, side);
    ctx->launches += 3;
    DCF_CHECK_LAUNCH();
    DCF_CUDA(cudaEventRecord(ctx->ev_prep[bi], side));
    DCF_CUDA(cudaStreamWaitEvent(st, ctx->ev_prep[bi], 0));
    Args af = a;  // final stage: T real timesteps
    if (U > 0) {
      // expand, screen (metric-first: maximum only), select, gather
      if (fp64)
        k_var_expand<double><<<dim3(TV, ch.nq), 128, 0, st>>>(ap, T, U, bt->var_ptr, ctx->var_k.as<int>(),
                                                               bt->var_delta, B.ptv.as<double>(), B.svv.as<double>());
      else
        k_var_expand<float><<<dim3(TV, ch.nq), 128, 0, st>>>(ap, T, U, bt->var_ptr, ctx->var_k.as<int>(),
                                                              bt->var_delta, B.ptv.as<float>(), B.svv.as<float>());
      ++ctx->launches;
      DCF_CHECK_LAUNCH();
      Args av = a;
      av.T = TV;
      av.out.n1_cont_max = nullptr;
      av.ptil = B.ptv.p;
      av.s = B.svv.p;
      av.pmax = B.pmaxv.p;
      av.parg = B.pargv.as<int>();
      av.povl = B.povlv.as<double>();
      if (C > 0) {
        int rc = run_n1(av, RMAX, TV, false);
        if (rc) return rc;
      } else {
        DCF_CUDA(cudaMemsetAsync(B.pargv.p, 0xff, (size_t)ch.nq * TV * sizeof(int), st));
      }
      const dim3 gs(ch.nq, (T + 7) / 8);
      if (fp64) k_var_select<double><<<gs, 256, 0, st>>>(av, T, U, B.bestu.as<int>());
      else k_var_select<float><<<gs, 256, 0, st>>>(av, T, U, B.bestu.as<int>());
      af.ptil = B.ptb.p;
      af.s = B.sb.p;
      af.best_u = B.bestu.as<int>();
      if (fp64) k_var_gather<double><<<dim3(T, ch.nq), 128, 0, st>>>(af, U, B.ptv.as<double>(), B.svv.as<double>());
      else k_var_gather<float><<<dim3(T, ch.nq), 128, 0, st>>>(af, U, B.ptv.as<float>(), B.svv.as<float>());
      ctx->launches += 2;
      DCF_CHECK_LAUNCH();
    }
    if (C > 0) {
      int rc = run_n1(af, RMAX, T, true);
      if (rc) return rc;
    }
    if (fp64) launch_final<double>(af, RMAX, st);
    else launch_final<float>(af, RMAX, st);
    ++ctx->launches;
    DCF_CHECK_LAUNCH();
    DCF_CUDA(cudaEventRecord(ctx->ev_free[bi], st));
  }
  return DCFLOW_OK;
}

extern "C" int dcflow_profile(dcflow_ctx* ctx, int32_t enable) {
  if (!ctx) return DCFLOW_ERR_INVALID_ARG;
  ctx->prof_on = enable != 0;
  ctx->prof_used = 0;
  return DCFLOW_OK;
}

extern "C" int dcflow_profile_read(dcflow_ctx* ctx, double* n1_ms, int64_t* n1_launches) {
  if (!ctx || !n1_ms || !n1_launches) return DCFLOW_ERR_INVALID_ARG;
  double ms = 0.0;
  for (size_t i = 0; i + 1 < ctx->prof_used; i += 2) {
    DCF_CUDA(cudaEventSynchronize(ctx->prof_ev[i + 1]));
    float x = 0.f;
    DCF_CUDA(cudaEventElapsedTime(&x, ctx->prof_ev[i], ctx->prof_ev[i + 1]));
    ms += x;
  }
  *n1_ms = ms;
  *n1_launches = (int64_t)(ctx->prof_used / 2);
  return DCFLOW_OK;
}
