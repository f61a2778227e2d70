// TMA-fed FP32 kernels of the generator-failure N-1 (Sec. III-A) and the
// multi-outage N-1 (Def. 4, MODF).  Both evaluate, per topology, a set of
// cases (a generator, a set of branches) against every monitored row and
// timestep; like the fused N-1 kernel they keep one running |max| per
// (case, timestep) cell in registers, fold two rows per packed multiply-add,
// form a cell's overload sum only over the row tiles where its maximum exceeds
// 1, and take the arg-max over the cases once at the end (the lowest case on
// ties).  Included by solve.cu after the per-chunk argument block.
#pragma once

#include "args.cuh"
#include "n1_tma.cuh"

namespace dcf {

__device__ __forceinline__ float sec_max3abs(float a, float b, float c) {
  float r;
  asm("max.abs.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// overload term of one entry, x 2^-20: sat((|v| - 1) 2^-20) = max(0, |v| - 1) 2^-20
__device__ __forceinline__ float sec_ovl(float v) { return __saturatef(fmaf(fabsf(v), 0x1p-20f, -0x1p-20f)); }

// ---------------------------------------------------------------------------
// generator failures: generator g at bus b with output P_g[t] fails, the slack
// takes it up, and the flows become p_f - P_g PTDF_f[:, b] with
//   PTDF_f[l, b] = PTDF[l, b] - Z[l, :] K^{-1} Sigma^T PTDF[:, b]   (Eq. (3)).
// Block = one topology and one pass of TT = 8 TR timesteps (grid y), the
// generators in groups of 16, fed like the fused N-1 kernel: a 2-stage TMA ring
// of 32-row tiles holding the 16 generators' rows PTDF[l, b_g] / limit_l
// [16][32], Z / limit [RMAX][32], the metadata rows [4][32] and p_f / limit
// [TT][32], the last with 128-byte swizzling so that the compute threads read
// its row pairs without bank conflicts and without a transposition.  Per tile
// thread (g, tb) builds rows 4 tb .. 4 tb + 3 of generator g's column; thread
// (g, tg) owns the cells of generator g at timesteps TR tg + j.  The column
// entries and flows are the multiply-adds of the one-thread-per-row FP64 form.
// Waits are bounded (error flag 1).
struct GenMaps {
  CUtensorMap pg, zt, meta, pt;
};
template <int TR, int RMAX>
struct GenTmaLayout {
  static constexpr int TT = 8 * TR, RT = 32, GG = 16;
  static constexpr int a1k(int x) { return (x + 1023) / 1024 * 1024; }
  static constexpr int kPt = TT * RT * 4;           // swizzled, first in the stage (1024-aligned)
  static constexpr int kOffPg = kPt;
  static constexpr int kOffZt = kOffPg + GG * RT * 4;
  static constexpr int kOffMeta = kOffZt + RMAX * RT * 4;
  static constexpr int kTx = kOffMeta + 4 * RT * 4;  // bytes landing per stage
  static constexpr int kStage = a1k(kTx);
  static constexpr int kCP = GG + 1;                 // float2 pitch of a column row pair
  static constexpr int kOffCol = 2 * kStage;         // float2 [RT / 2][kCP]
  static constexpr int kOffBar = kOffCol + (RT / 2) * kCP * 8;
  static constexpr int kBytes = kOffBar + 64 + 1024;  // + alignment slack of the dynamic base
};

template <int RMAX, int TR>
__global__ __launch_bounds__(128) void k_gen_tma(const __grid_constant__ GenMaps maps, Args a, int G,
                                                 const int* __restrict__ gen_bus, const double* __restrict__ gen_p,
                                                 const double* __restrict__ PtdfN, int V) {
  using L = GenTmaLayout<TR, RMAX>;
  constexpr int TT = L::TT, RT = L::RT, GG = L::GG, CP = L::kCP;
  extern __shared__ unsigned char gen_dyn[];
  __shared__ double sv_s[kRMax][GG];
  __shared__ float beta_s[GG][RMAX];
  __shared__ float mx_s[TT][GG + 1], ov_s[TT][GG + 1];
  __shared__ int mp_s[kRMax + 1];
  __shared__ float bv_s[TT];
  __shared__ int bg_s[TT];
  __shared__ double bo_s[TT];
  const int q = blockIdx.x, tid = threadIdx.x;
  const int t0 = blockIdx.y * TT;
  const QInfo qi = a.qi[q];
  const int T = a.T, M = a.M, tau = qi.tau;
  const dcflow_results& o = a.out;
  if (qi.status != ST_OK) {
    for (int t = t0 + tid; t < T && t < t0 + TT; t += blockDim.x) {
      o.gen_max_loading[(size_t)tau * T + t] = 0.0;
      o.worst_gen[(size_t)tau * T + t] = -1;
      o.gen_overload_sum[(size_t)tau * T + t] = 0.0;
    }
    return;
  }
  const uint32_t raw = smem_u32(gen_dyn);
  unsigned char* sm = gen_dyn + (((raw + 1023u) & ~1023u) - raw);  // 1024-aligned (the swizzled tiles)
  float2* s_col = reinterpret_cast<float2*>(sm + L::kOffCol);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::kOffBar);
  const int r = qi.r;
  for (int i = tid; i <= r; i += blockDim.x) mp_s[i] = a.mod_ptr[(size_t)q * (kRMax + 1) + i];
  for (int t = tid; t < TT; t += blockDim.x) {
    bv_s[t] = -1.f;
    bg_s[t] = -1;
    bo_s[t] = 0.0;
  }
  if (tid == 0) {
    for (int st = 0; st < 2; ++st) mbar_init(smem_u32(&bars[st]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const double* Kinv = a.Kinv + (size_t)q * kRMax * kRMax;
  const int* en = a.ent_n + (size_t)q * kEntMax;
  const int8_t* es = a.ent_s + (size_t)q * kEntMax;
  const int cg = tid & 15, tg = tid >> 4;  // compute role; build role: generator cg, rows 4 tg .. 4 tg + 3
  const int ntile = (M + RT - 1) / RT;
  int seq = 0;  // tiles issued so far over the generator groups (the ring's phase)
  bool failed = false;
  int fsq = 0;  // the tile whose wait expired (the only one in flight then)
  for (int g0 = 0; g0 < G && !failed; g0 += GG) {
    const int gn = min(GG, G - g0);
    __syncthreads();  // mp_s and the barriers ready; the previous group's maxima consumed
    for (int p = tid; p < r * GG; p += blockDim.x) {  // Sigma^T PTDF[:, b_g] per modification (FP64)
      const int i = p / GG, g = p % GG;
      double x = 0.0;
      if (g < gn) {
        const int b = gen_bus[g0 + g];
        for (int e = mp_s[i]; e < mp_s[i + 1]; ++e) x = fma((double)es[e], PtdfN[(size_t)en[e] * V + b], x);
      }
      sv_s[i][g] = x;
    }
    __syncthreads();
    for (int p = tid; p < GG * RMAX; p += blockDim.x) {  // K^{-1} times it
      const int g = p / RMAX, j = p % RMAX;
      double x = 0.0;
      for (int i = 0; i < r; ++i) x = fma(Kinv[j * kRMax + i], sv_s[i][g], x);
      beta_s[g][j] = (float)x;
    }
    float2 s2[TR];  // -P_g[t] of the thread's cells, duplicated for the row pairs
    float mx[TR], ov[TR];
    int tx[TR];  // the cells' timesteps within the pass: line index of the swizzled p_f tile
#pragma unroll
    for (int j = 0; j < TR; ++j) {
      const int t = tg * TR + j;
      const float pv = (cg < gn && t0 + t < T) ? (float)gen_p[(size_t)(t0 + t) * G + g0 + cg] : 0.f;
      s2[j] = make_float2(-pv, -pv);
      mx[j] = 0.f;
      ov[j] = 0.f;
      tx[j] = t;
    }
    auto issue = [&](int k, int sq) {
      const int st = sq & 1;
      unsigned char* base = sm + st * L::kStage;
      const uint32_t bar = smem_u32(&bars[st]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar, L::kTx);
      tma_load_3d(smem_u32(base), &maps.pt, k * RT, t0, q, bar);
      tma_load_2d(smem_u32(base + L::kOffPg), &maps.pg, k * RT, g0, bar);
      tma_load_3d(smem_u32(base + L::kOffZt), &maps.zt, k * RT, 0, q, bar);
      tma_load_3d(smem_u32(base + L::kOffMeta), &maps.meta, k * RT, 0, q, bar);
    };
    __syncthreads();  // beta ready; every thread is past the previous group's last tile
    if (tid == 0 && ntile > 0) issue(0, seq);
    for (int k = 0; k < ntile; ++k) {
      const int sq = seq + k, st = sq & 1;
      const bool got = mbar_wait(smem_u32(&bars[st]), (uint32_t)((sq >> 1) & 1));
      if (__syncthreads_or(!got)) {  // also: every thread is done with tile k - 1 (s_col, the other stage)
        failed = true;
        fsq = sq;
        break;
      }
      if (tid == 0 && k + 1 < ntile) issue(k + 1, sq + 1);
      const unsigned char* base = sm + st * L::kStage;
      const float* pg_t = reinterpret_cast<const float*>(base + L::kOffPg);
      const float* zt_t = reinterpret_cast<const float*>(base + L::kOffZt);
      const float* rm_t = reinterpret_cast<const float*>(base + L::kOffMeta) + RT;  // metadata row 1
      {  // build rows 4 tg .. 4 tg + 3 of generator cg's column
        const int r0 = 4 * tg;
        const float4 pg4 = *reinterpret_cast<const float4*>(&pg_t[cg * RT + r0]);
        float c[4] = {pg4.x, pg4.y, pg4.z, pg4.w};
#pragma unroll
        for (int j = 0; j < RMAX; ++j) {
          const float4 z = *reinterpret_cast<const float4*>(&zt_t[j * RT + r0]);
          const float b = beta_s[cg][j];
          c[0] = fmaf(-z.x, b, c[0]);
          c[1] = fmaf(-z.y, b, c[1]);
          c[2] = fmaf(-z.z, b, c[2]);
          c[3] = fmaf(-z.w, b, c[3]);
        }
        const float4 rm = *reinterpret_cast<const float4*>(&rm_t[r0]);
        s_col[(2 * tg) * CP + cg] = make_float2(c[0] * rm.x, c[1] * rm.y);
        s_col[(2 * tg + 1) * CP + cg] = make_float2(c[2] * rm.z, c[3] * rm.w);
      }
      __syncthreads();
      float mt[TR];
#pragma unroll
      for (int rp = 0; rp < RT / 2; ++rp) {
        const float2 ph = s_col[rp * CP + cg];
#pragma unroll
        for (int j = 0; j < TR; ++j) {
          // rows 2 rp, 2 rp + 1 of timestep tx[j]: 16-byte chunk rp / 2 of line tx[j], swizzled
          const float2 pt = *reinterpret_cast<const float2*>(
              base + tx[j] * 128 + ((((rp >> 1) ^ tx[j]) & 7) << 4) + ((rp & 1) << 3));
          const float2 v = __ffma2_rn(ph, s2[j], pt);
          mt[j] = rp == 0 ? sec_max3abs(v.x, v.y, v.y) : sec_max3abs(mt[j], v.x, v.y);
        }
      }
#pragma unroll
      for (int j = 0; j < TR; ++j) {
        mx[j] = fmaxf(mx[j], mt[j]);
        if (mt[j] > 1.f) {  // the overload terms of this cell over the tile
          float sum = 0.f;
          for (int rp = 0; rp < RT / 2; ++rp) {
            const float2 pt = *reinterpret_cast<const float2*>(
                base + tx[j] * 128 + ((((rp >> 1) ^ tx[j]) & 7) << 4) + ((rp & 1) << 3));
            const float2 v = __ffma2_rn(s_col[rp * CP + cg], s2[j], pt);
            sum += sec_ovl(v.x) + sec_ovl(v.y);
          }
          ov[j] += sum;
        }
      }
    }
    seq += ntile;
    if (failed) break;
#pragma unroll
    for (int j = 0; j < TR; ++j) {
      mx_s[tg * TR + j][cg] = mx[j];
      ov_s[tg * TR + j][cg] = ov[j];
    }
    __syncthreads();
    for (int t = tid; t < TT; t += blockDim.x) {  // over the generators, the lowest on ties
      if (t0 + t >= T) continue;
      float bv = bv_s[t];
      int bg = bg_s[t];
      double bo = bo_s[t];
      for (int g = 0; g < gn; ++g) {
        bo += (double)ov_s[t][g] * 1048576.0;
        if (mx_s[t][g] > bv) {
          bv = mx_s[t][g];
          bg = g0 + g;
        }
      }
      bv_s[t] = bv;
      bg_s[t] = bg;
      bo_s[t] = bo;
    }
  }
  if (failed) {  // the tile in flight lands (bounded wait) before the block exits
    if (tid == 0) {
      mbar_wait(smem_u32(&bars[fsq & 1]), (uint32_t)((fsq >> 1) & 1));
      atomicExch(a.err, 1);
    }
    return;
  }
  __syncthreads();
  for (int t = tid; t < TT; t += blockDim.x) {
    if (t0 + t >= T) continue;
    const size_t k2 = (size_t)tau * T + t0 + t;
    o.gen_max_loading[k2] = G ? (double)bv_s[t] : 0.0;
    o.worst_gen[k2] = G ? bg_s[t] : -1;
    o.gen_overload_sum[k2] = bo_s[t];
  }
}

// ---------------------------------------------------------------------------
// multi-outage sets: p_n1 = p_f + Phi_f[:, O] w_t with w_t = (I - Phi_f[O, O])^{-1}
// p_f[O, t] from the set preparation.  Block = one topology and one pass of
// TT = 8 TR timesteps (grid y), 256 threads, sets in groups of 32, fed by a
// 2-stage TMA ring of 32-row tiles: p_f / limit [TT][32] (128-byte swizzled),
// the group's member rows Phi[mon, o] / limit [128][32] (the sets of a group
// own consecutive entries, so one box covers them), Z / limit [RMAX][32] and
// the metadata rows [4][32].  Per tile thread (set, member, half) builds 16
// rows of its member column Phi_f[:, o_a] / limit into the column tile (absent
// members are zero columns); thread (warp w, lane) owns set 4 w + lane / 8 at
// timesteps TR (lane % 8) + j: per row pair four packed multiply-adds (members
// in order, as the one-thread-per-row FP64 form) and one three-input |max|
// per timestep.  A member's own monitored row carries nothing: its column entry
// there becomes Phi_f[o, o] / limit - 1 / limit, which makes the row's flow
// cancel to (rounding) zero, the convention LODF[c, c] = -1 of the single
// contingencies.  Waits are bounded (error flag 1).
// ---------------------------------------------------------------------------
struct MultiMaps {
  CUtensorMap phi, zt, meta, pt;
};
template <int TR, int RMAX>
struct MultiTmaLayout {
  static constexpr int TT = 8 * TR, SG = 32, RT = 32, NE = 4 * SG;
  static constexpr int a1k(int x) { return (x + 1023) / 1024 * 1024; }
  static constexpr int kOffPhi = TT * RT * 4;  // after the swizzled p_f box
  static constexpr int kOffZt = kOffPhi + NE * RT * 4;
  static constexpr int kOffMeta = kOffZt + RMAX * RT * 4;
  static constexpr int kTx = kOffMeta + 4 * RT * 4;
  static constexpr int kStage = a1k(kTx);
  static constexpr int kOffCol = 2 * kStage;  // float2 [RT / 2][NE]: [row pair][set][member]
  static constexpr int kOffBar = kOffCol + (RT / 2) * NE * 8;
  static constexpr int kBytes = kOffBar + 64 + 1024;  // + alignment slack of the dynamic base
};

template <int RMAX, int TR>
__global__ __launch_bounds__(256, 3) void k_multi_tma(const __grid_constant__ MultiMaps maps, Args a, int n_multi,
                                                   const int* __restrict__ mptr, const int* __restrict__ mmpos,
                                                   const float* __restrict__ mvt, const float* __restrict__ mw,
                                                   const int* __restrict__ mflag) {
  using L = MultiTmaLayout<TR, RMAX>;
  constexpr int TT = L::TT, SG = L::SG, RT = L::RT, NE = L::NE;
  extern __shared__ unsigned char mt_dyn[];
  __shared__ float mx_s[SG][TT + 1];
  __shared__ float ov_s[SG][TT + 1];
  __shared__ int fl_s[SG];
  __shared__ float bv_s[TT];
  __shared__ int bg_s[TT];
  __shared__ double bo_s[TT];
  __shared__ int nisl_s;
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int t0 = blockIdx.y * TT;
  const QInfo qi = a.qi[q];
  const int T = a.T, M = a.M, tau = qi.tau;
  const dcflow_results& o = a.out;
  if (qi.status != ST_OK) {
    for (int t = t0 + tid; t < T && t < t0 + TT; t += blockDim.x) {
      o.multi_max_loading[(size_t)tau * T + t] = 0.0;
      o.worst_multi[(size_t)tau * T + t] = -1;
      o.multi_overload_sum[(size_t)tau * T + t] = 0.0;
    }
    if (tid == 0 && blockIdx.y == 0) o.n_island_multi[tau] = 0;
    return;
  }
  const uint32_t raw = smem_u32(mt_dyn);
  unsigned char* sm = mt_dyn + (((raw + 1023u) & ~1023u) - raw);  // 1024-aligned (the swizzled tiles)
  float2* col_s = reinterpret_cast<float2*>(sm + L::kOffCol);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::kOffBar);
  const size_t qS = (size_t)q * n_multi;
  if (tid == 0) {
    nisl_s = 0;
    for (int st = 0; st < 2; ++st) mbar_init(smem_u32(&bars[st]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int t = tid; t < TT; t += blockDim.x) {
    bv_s[t] = -1.f;
    bg_s[t] = 0x7fffffff;
    bo_s[t] = 0.0;
  }
  // builder role: column (set bs, member ba), rows [16 bh, 16 bh + 16) of each tile
  const int bs = tid >> 3, ba = (tid >> 1) & 3, bh = tid & 1;
  // compute role: set cs, timesteps TR ct + j
  const int cs = 4 * w + (lane >> 3), ct = lane & 7;
  const int ntile = (M + RT - 1) / RT;
  int seq = 0;  // tiles issued so far over the set groups (the ring's phase)
  bool failed = false;
  int fsq = 0;  // the tile whose wait expired (the only one in flight then)
  for (int g0 = 0; g0 < n_multi && !failed; g0 += SG) {
    const int ng = min(SG, n_multi - g0);
    __syncthreads();  // barriers ready; the previous group's maxima, flags and tiles consumed
    const int ebase = mptr[g0];  // the group's first entry: the Phi box's row coordinate
    // the builder's member: its K^{-1}-weighted factors, its monitored row
    float vb[RMAX];
    int brow = -1, eloc = -1;
    if (bs < ng) {
      const int m = g0 + bs, e0 = mptr[m], n = mptr[m + 1] - e0;
      if (ba < n) {
        eloc = e0 + ba - ebase;
        brow = mmpos[e0 + ba];
      }
    }
#pragma unroll
    for (int j = 0; j < RMAX; ++j) vb[j] = eloc >= 0 ? mvt[(qS + g0 + bs) * 4 * kRMax + ba * kRMax + j] : 0.f;
    const float bil = brow >= 0 ? (float)a.inv_lim[brow] : 0.f;
    // the compute thread's set: its weights w_t (zero for absent members and sets not evaluated)
    float2 w2[TR][4];
    {
      int cflag = 3, n = 0;
      if (cs < ng) {
        cflag = mflag[qS + g0 + cs];
        n = mptr[g0 + cs + 1] - mptr[g0 + cs];
      }
#pragma unroll
      for (int j = 0; j < TR; ++j) {
        const int t = t0 + ct * TR + j;
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2) {
          const float x = (cflag == 0 && a2 < n && t < T) ? mw[((qS + g0 + cs) * T + t) * 4 + a2] : 0.f;
          w2[j][a2] = make_float2(x, x);
        }
      }
    }
    if (tid < SG) {
      const int f = tid < ng ? mflag[qS + g0 + tid] : 3;
      fl_s[tid] = f;
      if (t0 == 0 && f == 1) atomicAdd(&nisl_s, 1);
    }
    float mx[TR], ov[TR];
#pragma unroll
    for (int j = 0; j < TR; ++j) {
      mx[j] = 0.f;
      ov[j] = 0.f;
    }
    auto issue = [&](int k, int sq) {
      unsigned char* base = sm + (sq & 1) * L::kStage;
      const uint32_t bar = smem_u32(&bars[sq & 1]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar, L::kTx);
      tma_load_3d(smem_u32(base), &maps.pt, k * RT, t0, q, bar);
      tma_load_2d(smem_u32(base + L::kOffPhi), &maps.phi, k * RT, ebase, bar);
      tma_load_3d(smem_u32(base + L::kOffZt), &maps.zt, k * RT, 0, q, bar);
      tma_load_3d(smem_u32(base + L::kOffMeta), &maps.meta, k * RT, 0, q, bar);
    };
    if (tid == 0 && ntile > 0) issue(0, seq);
    for (int k = 0; k < ntile; ++k) {
      const int sq = seq + k;
      const bool got = mbar_wait(smem_u32(&bars[sq & 1]), (uint32_t)((sq >> 1) & 1));
      if (__syncthreads_or(!got)) {  // also: every thread is done with tile k - 1 (the column tile, the other stage)
        failed = true;
        fsq = sq;
        break;
      }
      if (tid == 0 && k + 1 < ntile) issue(k + 1, sq + 1);
      const unsigned char* base = sm + (sq & 1) * L::kStage;
      const float* phi_t = reinterpret_cast<const float*>(base + L::kOffPhi);
      const float* zt_t = reinterpret_cast<const float*>(base + L::kOffZt);
      const float* rm_t = reinterpret_cast<const float*>(base + L::kOffMeta) + RT;  // metadata row 1
      {  // rows [16 bh, 16 bh + 16) of column (bs, ba): Phi_f[l, o] / limit_l
        const int r0 = 16 * bh;
        float c[16];
#pragma unroll
        for (int i4 = 0; i4 < 4; ++i4) {
          const float4 p4 = eloc >= 0 ? *reinterpret_cast<const float4*>(&phi_t[eloc * RT + r0 + 4 * i4])
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
          c[4 * i4] = p4.x;
          c[4 * i4 + 1] = p4.y;
          c[4 * i4 + 2] = p4.z;
          c[4 * i4 + 3] = p4.w;
        }
#pragma unroll
        for (int j = 0; j < RMAX; ++j)
#pragma unroll
          for (int i4 = 0; i4 < 4; ++i4) {
            const float4 z = *reinterpret_cast<const float4*>(&zt_t[j * RT + r0 + 4 * i4]);
            c[4 * i4] = fmaf(-z.x, vb[j], c[4 * i4]);
            c[4 * i4 + 1] = fmaf(-z.y, vb[j], c[4 * i4 + 1]);
            c[4 * i4 + 2] = fmaf(-z.z, vb[j], c[4 * i4 + 2]);
            c[4 * i4 + 3] = fmaf(-z.w, vb[j], c[4 * i4 + 3]);
          }
#pragma unroll
        for (int i4 = 0; i4 < 4; ++i4) {
          const float4 rm = *reinterpret_cast<const float4*>(&rm_t[r0 + 4 * i4]);
          c[4 * i4] *= rm.x;
          c[4 * i4 + 1] *= rm.y;
          c[4 * i4 + 2] *= rm.z;
          c[4 * i4 + 3] *= rm.w;
        }
#pragma unroll
        for (int i2 = 0; i2 < 8; ++i2) col_s[(8 * bh + i2) * NE + bs * 4 + ba] = make_float2(c[2 * i2], c[2 * i2 + 1]);
        const int dr = brow - k * RT - r0;  // the member's own row: its flow cancels (same thread wrote it)
        if ((unsigned)dr < 16u) reinterpret_cast<float*>(&col_s[(8 * bh + dr / 2) * NE + bs * 4 + ba])[dr & 1] -= bil;
      }
      __syncthreads();
      float mt[TR];
#pragma unroll
      for (int j = 0; j < TR; ++j) mt[j] = 0.f;
#pragma unroll 2
      for (int rp = 0; rp < RT / 2; ++rp) {
        const float4 u0 = *reinterpret_cast<const float4*>(&col_s[rp * NE + cs * 4]);
        const float4 u1 = *reinterpret_cast<const float4*>(&col_s[rp * NE + cs * 4 + 2]);
        const float2 cc[4] = {make_float2(u0.x, u0.y), make_float2(u0.z, u0.w), make_float2(u1.x, u1.y),
                              make_float2(u1.z, u1.w)};
#pragma unroll
        for (int j = 0; j < TR; ++j) {
          const int t = ct * TR + j;  // rows 2 rp, 2 rp + 1 of line t: chunk rp / 2, swizzled
          float2 v = *reinterpret_cast<const float2*>(base + t * 128 + ((((rp >> 1) ^ t) & 7) << 4) + ((rp & 1) << 3));
#pragma unroll
          for (int a2 = 0; a2 < 4; ++a2) v = __ffma2_rn(cc[a2], w2[j][a2], v);
          mt[j] = sec_max3abs(mt[j], v.x, v.y);
        }
      }
#pragma unroll
      for (int j = 0; j < TR; ++j) {
        mx[j] = fmaxf(mx[j], mt[j]);
        if (mt[j] > 1.f) {  // the overload terms of this cell over the tile
          const int t = ct * TR + j;
          float sum = 0.f;
          for (int rp = 0; rp < RT / 2; ++rp) {
            float2 v = *reinterpret_cast<const float2*>(base + t * 128 + ((((rp >> 1) ^ t) & 7) << 4) + ((rp & 1) << 3));
#pragma unroll
            for (int a2 = 0; a2 < 4; ++a2) v = __ffma2_rn(col_s[rp * NE + cs * 4 + a2], w2[j][a2], v);
            sum += sec_ovl(v.x) + sec_ovl(v.y);
          }
          ov[j] += sum;
        }
      }
    }
    seq += ntile;
    if (failed) break;
#pragma unroll
    for (int j = 0; j < TR; ++j) {
      mx_s[cs][ct * TR + j] = mx[j];
      ov_s[cs][ct * TR + j] = ov[j];
    }
    __syncthreads();
    for (int t = tid; t < TT; t += blockDim.x) {  // over the sets in order: the lowest on ties
      if (t0 + t >= T) continue;
      float bv = bv_s[t];
      int bg = bg_s[t];
      double bo = bo_s[t];
      for (int s2 = 0; s2 < ng; ++s2) {
        if (fl_s[s2]) continue;
        bo += (double)ov_s[s2][t] * 1048576.0;
        if (mx_s[s2][t] > bv) {
          bv = mx_s[s2][t];
          bg = g0 + s2;
        }
      }
      bv_s[t] = bv;
      bg_s[t] = bg;
      bo_s[t] = bo;
    }
  }
  if (failed) {  // the tile in flight lands (bounded wait) before the block exits
    if (tid == 0) {
      mbar_wait(smem_u32(&bars[fsq & 1]), (uint32_t)((fsq >> 1) & 1));
      atomicExch(a.err, 1);
    }
    return;
  }
  __syncthreads();
  for (int t = tid; t < TT; t += blockDim.x) {
    if (t0 + t >= T) continue;
    const size_t k2 = (size_t)tau * T + t0 + t;
    const bool any = bg_s[t] != 0x7fffffff;
    o.multi_max_loading[k2] = any ? (double)bv_s[t] : 0.0;
    o.worst_multi[k2] = any ? bg_s[t] : -1;
    o.multi_overload_sum[k2] = bo_s[t];
  }
  if (tid == 0 && blockIdx.y == 0) o.n_island_multi[tau] = nisl_s;
}

}  // namespace dcf
