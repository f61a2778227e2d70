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
// generators in groups of 16, fed by a 3-stage TMA ring of 32-row tiles: the
// 16 generators' rows PTDF[l, b_g] / limit_l [16][32], Z / limit [RMAX][32],
// the metadata rows [4][32] and p_f / limit [TT][36] (36-float lines: rows 32
// to 35 belong to the next tile and are not read; with that pitch the eight
// timestep lines a warp reads at one row pair fall on distinct banks).  Thread
// (h, gp, tg) owns generators 2 gp, 2 gp + 1 at timesteps tg + 8 j over the 16
// rows of tile half h: one p_f pair load serves both generators.  Warp w reads
// the columns of generators 8 (w & 1) .. + 7 over half w >> 1 and builds
// exactly those (4 entries a lane), so one block barrier per tile suffices (the
// stage and column reuse).  The halves' maxima and overload sums meet once per
// group.  The column entries and
// flows are the multiply-adds of the one-thread-per-row FP64 form.  Waits are
// bounded (error flag 1).
struct GenMaps {
  CUtensorMap pg, zt, meta, pt;
};
template <int TR, int RMAX>
struct GenTmaLayout {
  static constexpr int TT = 8 * TR, RT = 32, GG = 16, NS = 3, PL = RT + 4;
  static constexpr int a1k(int x) { return (x + 1023) / 1024 * 1024; }
  // PTDF[l, b_g] / limit_l first (1024-aligned, 128-byte swizzled: chunk c of generator g's
  // row at c ^ (g & 7), so the builders' reads of 8 generators spread over every bank)
  static constexpr int kOffPt = GG * RT * 4;
  static constexpr int kOffZt = kOffPt + TT * PL * 4;  // TT PL 4 is a multiple of 1152 = 9 x 128
  static constexpr int kOffMeta = kOffZt + RMAX * RT * 4;
  static constexpr int kTx = kOffMeta + 4 * RT * 4;  // bytes landing per stage
  static constexpr int kStage = a1k(kTx);
  static constexpr int kOffCol = NS * kStage;       // float2 [RT / 2][GG]: [row pair][generator]
  static constexpr int kOffBar = kOffCol + (RT / 2) * GG * 8;
  static constexpr int kBytes = kOffBar + 64 + 1024;  // + alignment slack of the dynamic base
  // the halves' maxima and overload sums [2][TT][GG + 1] reuse stage 0 at the group's end
  static_assert(2 * 2 * TT * (GG + 1) * 4 <= kStage, "group reduction does not fit a stage");
};

template <int RMAX, int TR>
__global__ __launch_bounds__(128, 7) void k_gen_tma(const __grid_constant__ GenMaps maps, Args a, int G,
                                                 const int* __restrict__ gen_bus, const double* __restrict__ gen_p,
                                                 const double* __restrict__ PtdfN, int V) {
  using L = GenTmaLayout<TR, RMAX>;
  constexpr int TT = L::TT, RT = L::RT, GG = L::GG, NS = L::NS, PL = L::PL;
  extern __shared__ unsigned char gen_dyn[];
  __shared__ double sv_s[kRMax][GG];
  __shared__ float beta_s[GG][RMAX];
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
  unsigned char* sm = gen_dyn + (((raw + 1023u) & ~1023u) - raw);  // 1024-aligned stages (the swizzled tile)
  float2* s_col = reinterpret_cast<float2*>(sm + L::kOffCol);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::kOffBar);
  float(*mx_s)[TT][GG + 1] = reinterpret_cast<float(*)[TT][GG + 1]>(sm);  // [2][TT][GG + 1], group end only
  float(*ov_s)[TT][GG + 1] = reinterpret_cast<float(*)[TT][GG + 1]>(sm + 2 * TT * (GG + 1) * 4);
  const int r = qi.r;
  for (int i = tid; i <= r; i += blockDim.x) mp_s[i] = a.mod_ptr[(size_t)q * (kRMax + 1) + i];
  for (int t = tid; t < TT; t += blockDim.x) {
    bv_s[t] = -1.f;
    bg_s[t] = -1;
    bo_s[t] = 0.0;
  }
  if (tid == 0) {
    for (int st = 0; st < NS; ++st) mbar_init(smem_u32(&bars[st]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const double* Kinv = a.Kinv + (size_t)q * kRMax * kRMax;
  const int* en = a.ent_n + (size_t)q * kEntMax;
  const int8_t* es = a.ent_s + (size_t)q * kEntMax;
  // build role: generator bg, rows br0 .. br0 + 3 (the columns the thread's warp reads)
  const int bg = 8 * ((tid >> 5) & 1) + (tid & 7), br0 = 16 * (tid >> 6) + 4 * ((tid >> 3) & 3);
  const int h = tid >> 6, gp = (tid >> 3) & 7, tg = tid & 7;  // compute role
  const int ntile = (M + RT - 1) / RT;
  int seq = 0;  // tiles issued so far over the generator groups (the ring's position)
  bool failed = false;
  int fbase = 0, fk = 0, fiss = 0;  // on failure: its group's first tile, the tile whose wait expired, the
                                    // tiles issued in that group
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
    float2 s2[2][TR];  // -P_g[t] of the thread's cells, duplicated for the row pairs
    float mx[2][TR], ov[2][TR];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int j = 0; j < TR; ++j) {
        const int t = tg + 8 * j, g = 2 * gp + u;
        const float pv = (g < gn && t0 + t < T) ? (float)gen_p[(size_t)(t0 + t) * G + g0 + g] : 0.f;
        s2[u][j] = make_float2(-pv, -pv);
        mx[u][j] = 0.f;
        ov[u][j] = 0.f;
      }
    auto issue = [&](int k, int sq) {
      const int st = sq % NS;
      unsigned char* base = sm + st * L::kStage;
      const uint32_t bar = smem_u32(&bars[st]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar, L::kTx);
      tma_load_2d(smem_u32(base), &maps.pg, k * RT, g0, bar);
      tma_load_3d(smem_u32(base + L::kOffPt), &maps.pt, k * RT, t0, q, bar);
      tma_load_3d(smem_u32(base + L::kOffZt), &maps.zt, k * RT, 0, q, bar);
      tma_load_3d(smem_u32(base + L::kOffMeta), &maps.meta, k * RT, 0, q, bar);
    };
    __syncthreads();  // beta ready; every thread is past the previous group's last tile
    int iss = min(ntile, NS - 1);  // tiles of this group issued (the same count in every thread)
    if (tid == 0)
      for (int k = 0; k < iss; ++k) issue(k, seq + k);
    for (int k = 0; k < ntile; ++k) {
      const int sq = seq + k, st = sq % NS;
      const bool got = mbar_wait(smem_u32(&bars[st]), (uint32_t)((sq / NS) & 1));
      if (__syncthreads_or(!got)) {  // also: every thread is done with tile k - 1 (its stage)
        failed = true;
        fbase = seq;
        fk = k;
        fiss = iss;
        break;
      }
      if (k + NS - 1 < ntile) {
        if (tid == 0) issue(k + NS - 1, sq + NS - 1);
        ++iss;
      }
      const unsigned char* base = sm + st * L::kStage;
      const float* zt_t = reinterpret_cast<const float*>(base + L::kOffZt);
      const float* rm_t = reinterpret_cast<const float*>(base + L::kOffMeta) + RT;  // metadata row 1
      {  // build rows br0 .. br0 + 3 of generator bg's column (the warp is done with the previous tile's)
        const int r0 = br0;
        const float4 pg4 = *reinterpret_cast<const float4*>(base + bg * 128 + ((((r0 >> 2) ^ bg) & 7) << 4));
        float c[4] = {pg4.x, pg4.y, pg4.z, pg4.w};
#pragma unroll
        for (int j = 0; j < RMAX; ++j) {
          const float4 z = *reinterpret_cast<const float4*>(&zt_t[j * RT + r0]);
          const float b = beta_s[bg][j];
          c[0] = fmaf(-z.x, b, c[0]);
          c[1] = fmaf(-z.y, b, c[1]);
          c[2] = fmaf(-z.z, b, c[2]);
          c[3] = fmaf(-z.w, b, c[3]);
        }
        const float4 rm = *reinterpret_cast<const float4*>(&rm_t[r0]);
        s_col[(r0 / 2) * GG + bg] = make_float2(c[0] * rm.x, c[1] * rm.y);
        s_col[(r0 / 2 + 1) * GG + bg] = make_float2(c[2] * rm.z, c[3] * rm.w);
      }
      __syncwarp();
      // rows 16 h + 2 i, 16 h + 2 i + 1 of line tg + 8 j
      const float* pt_h = reinterpret_cast<const float*>(base + L::kOffPt) + tg * PL + 16 * h;
      const float4* col_h = reinterpret_cast<const float4*>(s_col) + (8 * h) * (GG / 2) + gp;
      float mt[2][TR];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int j = 0; j < TR; ++j) mt[u][j] = 0.f;
#pragma unroll 4
      for (int i = 0; i < 8; ++i) {
        const float4 c4 = col_h[i * (GG / 2)];
        const float2 c0 = make_float2(c4.x, c4.y), c1 = make_float2(c4.z, c4.w);
#pragma unroll
        for (int j = 0; j < TR; ++j) {
          const float2 pt = *reinterpret_cast<const float2*>(pt_h + 8 * j * PL + 2 * i);
          const float2 v0 = __ffma2_rn(c0, s2[0][j], pt);
          const float2 v1 = __ffma2_rn(c1, s2[1][j], pt);
          mt[0][j] = sec_max3abs(mt[0][j], v0.x, v0.y);
          mt[1][j] = sec_max3abs(mt[1][j], v1.x, v1.y);
        }
      }
#pragma unroll
      for (int j = 0; j < TR; ++j) {
        mx[0][j] = fmaxf(mx[0][j], mt[0][j]);
        mx[1][j] = fmaxf(mx[1][j], mt[1][j]);
        if (mt[0][j] > 1.f || mt[1][j] > 1.f) {  // the overload terms of both cells at this timestep
          float s0 = 0.f, s1 = 0.f;  // (a cell whose maximum is at most 1 adds exact zeros)
          for (int i = 0; i < 8; ++i) {
            const float2 pt = *reinterpret_cast<const float2*>(pt_h + 8 * j * PL + 2 * i);
            const float4 c4 = col_h[i * (GG / 2)];
            const float2 v0 = __ffma2_rn(make_float2(c4.x, c4.y), s2[0][j], pt);
            const float2 v1 = __ffma2_rn(make_float2(c4.z, c4.w), s2[1][j], pt);
            s0 += sec_ovl(v0.x) + sec_ovl(v0.y);
            s1 += sec_ovl(v1.x) + sec_ovl(v1.y);
          }
          ov[0][j] += s0;
          ov[1][j] += s1;
        }
      }
    }
    seq += ntile;
    if (failed) break;
    __syncthreads();  // every thread is done with the last tile: the reduction reuses stage 0
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int j = 0; j < TR; ++j) {
        mx_s[h][tg + 8 * j][2 * gp + u] = mx[u][j];
        ov_s[h][tg + 8 * j][2 * gp + u] = ov[u][j];
      }
    __syncthreads();
    for (int t = tid; t < TT; t += blockDim.x) {  // over the generators, the lowest on ties
      if (t0 + t >= T) continue;
      float bv = bv_s[t];
      int bgi = bg_s[t];
      float of = 0.f;  // the group's overload sums in FP32, one FP64 add (B300's FP64 rate)
      for (int g = 0; g < gn; ++g) {
        of += ov_s[0][t][g] + ov_s[1][t][g];
        const float m = fmaxf(mx_s[0][t][g], mx_s[1][t][g]);
        if (m > bv) {
          bv = m;
          bgi = g0 + g;
        }
      }
      bv_s[t] = bv;
      bg_s[t] = bgi;
      bo_s[t] += (double)(of * 1048576.f);
    }
  }
  if (failed) {  // the tiles in flight land (bounded waits) before the block exits
    if (tid == 0) {
      for (int k = fk; k < fiss; ++k)
        mbar_wait(smem_u32(&bars[(fbase + k) % NS]), (uint32_t)(((fbase + k) / NS) & 1));
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
// 2-stage TMA ring of 32-row tiles: p_f / limit [TT][36] (36-float lines, the
// last 4 rows not read: the eight timestep lines a warp reads at one row pair
// fall on distinct banks), the group's member rows Phi[mon, o] / limit
// [128][32] (the sets of a group own consecutive entries, so one box covers
// them), Z / limit [RMAX][32] and the metadata rows [4][32].  Thread (h, sp,
// ct) owns sets 2 sp, 2 sp + 1 at timesteps ct + 8 j over the 16 rows of tile
// half h: one p_f pair load serves both sets, and per row pair and set four
// packed multiply-adds (members in order, as the one-thread-per-row FP64 form)
// and one three-input |max|.  Warp w reads the columns of sets 8 (w & 3) .. + 7
// over half w >> 2 and builds exactly those: lane (set, member) the 16 rows of
// Phi_f[:, o_a] / limit (absent members are zero columns; row pairs in packed
// multiply-adds), so one block barrier per tile suffices (the stage and column
// reuse).  The halves' maxima and overload sums meet once per group.  A member's own
// monitored row carries nothing: its column entry there becomes Phi_f[o, o] /
// limit - 1 / limit, which makes the row's flow cancel to (rounding) zero, the
// convention LODF[c, c] = -1 of the single contingencies.  Waits are bounded
// (error flag 1).
struct MultiMaps {
  CUtensorMap phi, zt, meta, pt;
};
template <int TR, int RMAX>
struct MultiTmaLayout {
  static constexpr int TT = 8 * TR, SG = 32, RT = 32, NE = 4 * SG, PL = RT + 4;
  static constexpr int a1k(int x) { return (x + 1023) / 1024 * 1024; }
  // the member rows first (1024-aligned, 128-byte swizzled: chunk c of entry e's row at
  // c ^ (e & 7), so the builders' reads of 8 consecutive entries spread over every bank)
  static constexpr int kOffPt = NE * RT * 4;
  static constexpr int kOffZt = kOffPt + TT * PL * 4;  // TT PL 4 is a multiple of 1152 = 9 x 128
  static constexpr int kOffMeta = kOffZt + RMAX * RT * 4;
  static constexpr int kTx = kOffMeta + 4 * RT * 4;
  static constexpr int kStage = a1k(kTx);
  // column tile: per row pair 16 set pairs of 80 bytes (4 members x 2 sets as
  // float2, 16 bytes of padding: the 4 set pairs a warp reads fall on distinct banks)
  static constexpr int kSP = 80, kRP = 16 * kSP;
  static constexpr int kOffCol = 2 * kStage;
  static constexpr int kColBytes = (RT / 2) * kRP;
  // the halves' maxima and overload sums [2][SG][TT + 1] reuse the column tile at the group's end
  static_assert(2 * 2 * SG * (TT + 1) * 4 <= kColBytes, "group reduction does not fit the column tile");
  static constexpr int kOffBar = kOffCol + kColBytes;
  static constexpr int kBytes = kOffBar + 64 + 1024;  // + alignment slack of the dynamic base
};

template <int RMAX, int TR>
__global__ __launch_bounds__(256, 3) void k_multi_tma(const __grid_constant__ MultiMaps maps, Args a, int n_multi,
                                                   const int* __restrict__ mptr, const int* __restrict__ mmpos,
                                                   const float* __restrict__ mvt, const float* __restrict__ mw,
                                                   const int* __restrict__ mflag) {
  using L = MultiTmaLayout<TR, RMAX>;
  constexpr int TT = L::TT, SG = L::SG, RT = L::RT, PL = L::PL;
  extern __shared__ unsigned char mt_dyn[];
  __shared__ int fl_s[SG];
  __shared__ float bv_s[TT];
  __shared__ int bg_s[TT];
  __shared__ double bo_s[TT];
  __shared__ int nisl_s;
  const int q = blockIdx.x, tid = threadIdx.x;
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
  unsigned char* sm = mt_dyn + (((raw + 1023u) & ~1023u) - raw);  // 1024-aligned stages (the swizzled tile)
  unsigned char* col_b = sm + L::kOffCol;
  float(*mx_s)[SG][TT + 1] = reinterpret_cast<float(*)[SG][TT + 1]>(col_b);  // [2][SG][TT + 1], group end only
  float(*ov_s)[SG][TT + 1] = reinterpret_cast<float(*)[SG][TT + 1]>(col_b + 2 * SG * (TT + 1) * 4);
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
  // builder role: column (set bs, member ba), row pairs [8 bh, 8 bh + 8) of each tile (what the warp reads)
  const int bs = 8 * ((tid >> 5) & 3) + ((tid & 31) >> 2), ba = tid & 3, bh = tid >> 7;
  // compute role: tile half h, sets 2 sp + u, timesteps ct + 8 j
  const int h = tid >> 7, sp = (tid >> 3) & 15, ct = tid & 7;
  const int ntile = (M + RT - 1) / RT;
  int seq = 0;  // tiles issued so far over the set groups (the ring's phase)
  bool failed = false;
  int fsq = 0;  // the tile whose wait expired (the only one in flight then)
  for (int g0 = 0; g0 < n_multi && !failed; g0 += SG) {
    const int ng = min(SG, n_multi - g0);
    __syncthreads();  // barriers ready; the previous group's maxima, flags and tiles consumed
    const int ebase = mptr[g0];  // the group's first entry: the Phi box's row coordinate
    // the builder's member: its K^{-1}-weighted factors, its monitored row
    float2 vb[RMAX];
    int brow = -1, eloc = -1;
    if (bs < ng) {
      const int m = g0 + bs, e0 = mptr[m], n = mptr[m + 1] - e0;
      if (ba < n) {
        eloc = e0 + ba - ebase;
        brow = mmpos[e0 + ba];
      }
    }
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
      const float x = eloc >= 0 ? -mvt[(qS + g0 + bs) * 4 * kRMax + ba * kRMax + j] : 0.f;
      vb[j] = make_float2(x, x);
    }
    const float bil = brow >= 0 ? (float)a.inv_lim[brow] : 0.f;
    // the compute thread's sets: their weights w_t (zero for absent members and sets not evaluated)
    float2 w2[2][TR][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int cs = 2 * sp + u;
      int cflag = 3, n = 0;
      if (cs < ng) {
        cflag = mflag[qS + g0 + cs];
        n = mptr[g0 + cs + 1] - mptr[g0 + cs];
      }
#pragma unroll
      for (int j = 0; j < TR; ++j) {
        const int t = t0 + ct + 8 * j;
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2) {
          const float x = (cflag == 0 && a2 < n && t < T) ? mw[((qS + g0 + cs) * T + t) * 4 + a2] : 0.f;
          w2[u][j][a2] = make_float2(x, x);
        }
      }
    }
    if (tid < SG) {
      const int f = tid < ng ? mflag[qS + g0 + tid] : 3;
      fl_s[tid] = f;
      if (t0 == 0 && f == 1) atomicAdd(&nisl_s, 1);
    }
    float mx[2][TR], ov[2][TR];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int j = 0; j < TR; ++j) {
        mx[u][j] = 0.f;
        ov[u][j] = 0.f;
      }
    auto issue = [&](int k, int sq) {
      unsigned char* base = sm + (sq & 1) * L::kStage;
      const uint32_t bar = smem_u32(&bars[sq & 1]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar, L::kTx);
      tma_load_2d(smem_u32(base), &maps.phi, k * RT, ebase, bar);
      tma_load_3d(smem_u32(base + L::kOffPt), &maps.pt, k * RT, t0, q, bar);
      tma_load_3d(smem_u32(base + L::kOffZt), &maps.zt, k * RT, 0, q, bar);
      tma_load_3d(smem_u32(base + L::kOffMeta), &maps.meta, k * RT, 0, q, bar);
    };
    if (tid == 0 && ntile > 0) issue(0, seq);
    for (int k = 0; k < ntile; ++k) {
      const int sq = seq + k;
      const bool got = mbar_wait(smem_u32(&bars[sq & 1]), (uint32_t)((sq >> 1) & 1));
      if (__syncthreads_or(!got)) {  // also: every thread is done with tile k - 1 (the other stage)
        failed = true;
        fsq = sq;
        break;
      }
      if (tid == 0 && k + 1 < ntile) issue(k + 1, sq + 1);
      const unsigned char* base = sm + (sq & 1) * L::kStage;
      const float* zt_t = reinterpret_cast<const float*>(base + L::kOffZt);
      const float* rm_t = reinterpret_cast<const float*>(base + L::kOffMeta) + RT;  // metadata row 1
      {  // rows [16 bh, 16 bh + 16) of column (bs, ba): Phi_f[l, o] / limit_l, row pairs packed
        const int r0 = 16 * bh;
        float2 c[8];
#pragma unroll
        for (int i4 = 0; i4 < 4; ++i4) {
          const float4 p4 = eloc >= 0 ? *reinterpret_cast<const float4*>(
                                            base + eloc * 128 + (((((r0 >> 2) + i4) ^ eloc) & 7) << 4))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
          c[2 * i4] = make_float2(p4.x, p4.y);
          c[2 * i4 + 1] = make_float2(p4.z, p4.w);
        }
#pragma unroll
        for (int j = 0; j < RMAX; ++j)
#pragma unroll
          for (int i4 = 0; i4 < 4; ++i4) {
            const float4 z = *reinterpret_cast<const float4*>(&zt_t[j * RT + r0 + 4 * i4]);
            c[2 * i4] = __ffma2_rn(make_float2(z.x, z.y), vb[j], c[2 * i4]);
            c[2 * i4 + 1] = __ffma2_rn(make_float2(z.z, z.w), vb[j], c[2 * i4 + 1]);
          }
        unsigned char* dst = col_b + (8 * bh) * L::kRP + (bs >> 1) * L::kSP + (bs & 1) * 32 + ba * 8;
#pragma unroll
        for (int i4 = 0; i4 < 4; ++i4) {
          const float4 rm = *reinterpret_cast<const float4*>(&rm_t[r0 + 4 * i4]);
          c[2 * i4] = __fmul2_rn(c[2 * i4], make_float2(rm.x, rm.y));
          c[2 * i4 + 1] = __fmul2_rn(c[2 * i4 + 1], make_float2(rm.z, rm.w));
        }
#pragma unroll
        for (int i2 = 0; i2 < 8; ++i2) *reinterpret_cast<float2*>(dst + i2 * L::kRP) = c[i2];
        const int dr = brow - k * RT - r0;  // the member's own row: its flow cancels (same thread wrote it)
        if ((unsigned)dr < 16u) reinterpret_cast<float*>(dst + (dr >> 1) * L::kRP)[dr & 1] -= bil;
      }
      __syncwarp();
      // rows 16 h + 2 i, 16 h + 2 i + 1 of line ct + 8 j; the column pairs of sets 2 sp, 2 sp + 1
      const float* pt_h = reinterpret_cast<const float*>(base + L::kOffPt) + ct * PL + 16 * h;
      const unsigned char* col_h = col_b + (8 * h) * L::kRP + sp * L::kSP;
      float mt[2][TR];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int j = 0; j < TR; ++j) mt[u][j] = 0.f;
#pragma unroll 2
      for (int i = 0; i < 8; ++i) {
        float2 cc[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int a4 = 0; a4 < 2; ++a4) {
            const float4 x = *reinterpret_cast<const float4*>(col_h + i * L::kRP + u * 32 + a4 * 16);
            cc[u][2 * a4] = make_float2(x.x, x.y);
            cc[u][2 * a4 + 1] = make_float2(x.z, x.w);
          }
#pragma unroll
        for (int j = 0; j < TR; ++j) {
          const float2 p = *reinterpret_cast<const float2*>(pt_h + 8 * j * PL + 2 * i);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            float2 v = p;
#pragma unroll
            for (int a2 = 0; a2 < 4; ++a2) v = __ffma2_rn(cc[u][a2], w2[u][j][a2], v);
            mt[u][j] = sec_max3abs(mt[u][j], v.x, v.y);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int j = 0; j < TR; ++j) {
          mx[u][j] = fmaxf(mx[u][j], mt[u][j]);
          if (mt[u][j] > 1.f) {  // the overload terms of this cell over the tile half
            float sum = 0.f;
            for (int i = 0; i < 8; ++i) {
              float2 v = *reinterpret_cast<const float2*>(pt_h + 8 * j * PL + 2 * i);
              const float2* cp = reinterpret_cast<const float2*>(col_h + i * L::kRP + u * 32);
#pragma unroll
              for (int a2 = 0; a2 < 4; ++a2) v = __ffma2_rn(cp[a2], w2[u][j][a2], v);
              sum += sec_ovl(v.x) + sec_ovl(v.y);
            }
            ov[u][j] += sum;
          }
        }
    }
    seq += ntile;
    if (failed) break;
    __syncthreads();  // every thread is done with the last column tile: the reduction reuses it
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int j = 0; j < TR; ++j) {
        mx_s[h][2 * sp + u][ct + 8 * j] = mx[u][j];
        ov_s[h][2 * sp + u][ct + 8 * j] = ov[u][j];
      }
    __syncthreads();
    for (int t = tid; t < TT; t += blockDim.x) {  // over the sets in order: the lowest on ties
      if (t0 + t >= T) continue;
      float bv = bv_s[t];
      int bg = bg_s[t];
      float of = 0.f;  // the group's overload sums in FP32, one FP64 add (B300's FP64 rate)
      for (int s2 = 0; s2 < ng; ++s2) {
        if (fl_s[s2]) continue;
        of += ov_s[0][s2][t] + ov_s[1][s2][t];
        const float m = fmaxf(mx_s[0][s2][t], mx_s[1][s2][t]);
        if (m > bv) {
          bv = m;
          bg = g0 + s2;
        }
      }
      bv_s[t] = bv;
      bg_s[t] = bg;
      bo_s[t] += (double)(of * 1048576.f);
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

