// FP32 fused N-1 kernel, register-tiled (Def. 3 / Eq. (5), agg_m of Sec. III-A).
//
// One block = one topology x 64 contingencies x TT timesteps.  The operand
// tiles arrive as in k_n1_tma (a TMA ring, here 2 stages, mbarrier completion,
// bounded waits): per 16 monitored rows Phi/limit [16][64], Z^T/limit
// [RMAX][16], p_f^T/limit [TT][16] and the metadata rows.  Per tile:
//   build   every thread builds RB rows of one contingency's Phi_f column
//           (FFMA2 over row pairs) into s_ph[row pair][contingency] and the
//           block transposes p_f into s_pt[row pair][timestep] (float2 pairs);
//   compute thread (cg, tg) owns contingencies cg + 16 i (i < 4) and
//           timesteps TR tg .. TR tg + TR - 1: per row pair four LDS.64 of
//           Phi_f pairs and the p_f pairs of its timesteps feed 4 TR packed
//           FFMA2 (two rows each) and 4 TR three-input |max| (folding both
//           rows), i.e. one FP32 issue slot per N-1 entry;
//   overload the (contingency, timestep) items whose tile maximum exceeds 1
//           are queued per warp, one ballot per item class (so the lanes of
//           a serving round read consecutive contingencies: no bank
//           conflicts), and their 16 entries recomputed with the
//           saturating-FMA overload term (a bit mask per thread with a warp
//           prefix sum to place the items measured slower: its queue order
//           groups a lane's items, and the serving reads then conflict).
// SEL (a per-topology contingency list): block (cb, q) takes the cb-th 64
// contingencies of topology q's list, either from a work list (the learned
// screener's selection: one work item per block) or from the grid itself
// (every valid contingency of the topology, compacted: the contingencies that
// island the topology are never computed; a block past the end of its list
// writes an empty partial result).  The Phi tile is gathered from the
// transposed factors [cont][Mpad]: each contingency's 16 rows are one 64-byte
// run, copied with cp.async into a contingency-major tile (pitch 20 floats:
// the builders' reads spread over all banks); the other operands arrive by TMA.
//
// TC (the split-BF16x3 form): the Phi_f tile is built on the tensor cores
// instead of the FFMA2 builders.  Per tile and warp, mma.sync m16n8k16 (k8 for
// rank classes 4 and 8) computes D[c, l] = Phi[l, c] / limit + sum_j
// (-Vt[j, c]) Z[l, j] / limit for 16 contingencies x 8 rows, with each operand
// split as x = hi + lo in BF16 and three products hi.hi + hi.lo + lo.hi
// accumulated in FP32 (the lo.lo term, below 2^-16 of the product, is
// dropped).  -Vt^T is the A operand, held in registers for the block; Z rows
// arrive by TMA already split (BF16 hi and lo per row, written by the row
// preparation); Phi initialises the accumulator.  The D fragment of a thread
// holds the row pair (2 q, 2 q + 1) of contingencies g and g + 8: exactly the
// row-pair layout of s_ph, written with one 8-byte store each.  The tile of Phi
// is TMA'd 68 columns wide and s_ph has a pitch of 68 pairs, which spreads
// both the accumulator loads and the stores over all banks.  The shape
// (16 rows x 64 contingencies, K = the rank class) is below the smallest
// tcgen05 tile, so the warp-level MMA is the tensor-core instruction here.
#pragma once

#include <cuda.h>

#include "bf16x3.cuh"
#include "n1_tma.cuh"

namespace dcf {

constexpr int kRegStages = 2;  // TMA ring depth of this kernel (shared memory sets its occupancy)

// D += A B, m16n8k16 / m16n8k8, BF16 operands, FP32 accumulators
__device__ __forceinline__ void mma_bf16_k16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_bf16_k8(float (&d)[4], const uint32_t (&a)[4], uint32_t b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5}, {%6}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(b0));
}

template <int TT>
struct RegTile {
  static constexpr int NTH = TT >= 24 ? 2 : 1;  // 64 NTH threads
  static constexpr int NT = kCB * NTH;
  static constexpr int CR = 4;  // contingencies per thread (2 measured slower at 24 and 8 timesteps)
  static constexpr int CG = kCB / CR;           // contingency groups
  static constexpr int TG = NT / CG;            // timestep groups
  static constexpr int TR = TT / TG;            // timesteps per thread
  static constexpr int RB = kLT / NTH;          // tile rows built per thread
  static_assert(TR * TG == TT && TR >= 1, "timestep split");
  static_assert(RB % 4 == 0, "build split");
};

template <int TT, int RMAX, bool SEL = false, bool TC = false>
struct RegLayout {
  using R = RegTile<TT>;
  static constexpr int a128(int x) { return (x + 127) / 128 * 128; }
  static constexpr int kPW = TC ? kPhW : kCB;  // columns of a TMA'd Phi tile row; pairs per s_ph row
  static constexpr int kPhi = SEL ? kCB * kPP * 4 : kLT * kPW * 4;
  static constexpr int kZt = TC ? kLT * TcK<RMAX>::KB * 4 : RMAX * kLT * 4;  // TC: [16 rows][hi KB | lo KB] bf16
  static constexpr int kPt = TT * kLT * 4;
  static constexpr int kMeta = 4 * kLT * 4;
  static constexpr int kTx = (SEL ? 0 : kPhi) + kZt + kPt + kMeta;  // bytes landing by TMA
  static constexpr int kOffZt = a128(kPhi);
  static constexpr int kOffPt = kOffZt + a128(kZt);
  static constexpr int kOffMeta = kOffPt + a128(kPt);
  static constexpr int kStage = kOffMeta + a128(kMeta);
  static constexpr int kTP = TT + 2;   // row pitch (float2) of the transposed p_f: spreads the banks
  static constexpr int kSP = kCB + 1;  // row pitch (float) of the per-timestep arrays: spreads the banks
  static constexpr int kOffPh = kRegStages * kStage;              // float2 [kLT/2][kPW]
  static constexpr int kOffPtT = kOffPh + a128(kLT / 2 * kPW * 8); // float2 [kLT/2][kTP]
  static constexpr int kOffOv = kOffPtT + a128(kLT / 2 * kTP * 8); // float [TT][kSP]
  // the per-timestep maxima of the final scan reuse the (then idle) stages
  static_assert(TT * kSP * 4 <= kRegStages * kStage, "final scan fits the stages");
  static constexpr int kOffVt = kOffOv + a128(TT * kSP * 4);      // float [RMAX][kCB]: -Vt (not with TC)
  static constexpr int kOffBar = kOffVt + (TC ? 0 : a128(RMAX * kCB * 4));  // uint64 [kRegStages]
  static constexpr int kOffOk = kOffBar + 64;                     // uint8 [kCB]
  static constexpr int kOffCi = kOffOk + 128;                     // int [kCB]: contingency of each column
  static constexpr int kOffQ = kOffCi + kCB * 4;                  // uint16 [warps][32 CR TR]
  static constexpr int kBytes = kOffQ + (R::NT / 32) * 32 * R::CR * R::TR * 2;
};

template <int TT, int RMAX, bool OVL, bool SEL = false, bool TC = false, bool TRK = false>
__global__ __launch_bounds__(RegTile<TT>::NT, (TC && TT == 24) ? 7 : 0) void k_n1_reg(const __grid_constant__ N1Maps maps, Args a, int t0_base,
                                                            const SelArgs sel) {
  const int t0 = t0_base + (int)blockIdx.z * TT;  // grid z: the passes over TT timesteps each
  using L = RegLayout<TT, RMAX, SEL, TC>;
  constexpr int PH = L::kPW;  // pitch (pairs) of s_ph
  using R = RegTile<TT>;
  constexpr int CR = R::CR, TR = R::TR, RB = R::RB;
  int q = blockIdx.y, cb = blockIdx.x;  // topology slot and 64-contingency block
  if constexpr (SEL) {
    if (sel.work) {
      const int item = sel.work[blockIdx.x];
      q = item >> 6;
      cb = item & 63;
    }
  }
  const QInfo qi = a.qi[q];
  if (qi.status != ST_OK) return;  // whole block: before any barrier
  if constexpr (SEL) {
    if (!sel.work && cb * kCB >= sel.nsel[q]) {  // past the end of the list: an empty partial result
      for (int t = threadIdx.x; t < TT; t += blockDim.x)
        if (t0 + t < a.T) {
          const size_t o2 = ((size_t)q * a.T + t0 + t) * a.ncb + cb;
          static_cast<float*>(a.pmax)[o2] = 0.f;
          a.parg[o2] = -1;
          a.povl[o2] = 0.0;
          if (a.p2max) static_cast<float*>(a.p2max)[o2] = -1.f;
        }
      return;
    }
  }
  extern __shared__ __align__(128) unsigned char sm[];
  if (smem_u32(sm) & 127u) {  // the TMA destinations need the alignment: refuse, never fault
    if (threadIdx.x == 0) atomicExch(a.err, 2);
    return;
  }
  float2* s_ph = reinterpret_cast<float2*>(sm + L::kOffPh);
  float2* s_pt = reinterpret_cast<float2*>(sm + L::kOffPtT);
  float* s_s = reinterpret_cast<float*>(sm);  // after the tile loop: per-timestep maxima (stage memory)
  float* s_ov = reinterpret_cast<float*>(sm + L::kOffOv);
  float* s_vt = reinterpret_cast<float*>(sm + L::kOffVt);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::kOffBar);
  const int tid = threadIdx.x;
  const int M = a.M, C = a.C, T = a.T;
  const int c0 = cb * kCB;  // first column: a contingency, or a position in the selected list
  int* s_ci = reinterpret_cast<int*>(sm + L::kOffCi);
  if constexpr (SEL) {
    const int ns = sel.nsel[q];
    for (int i = tid; i < kCB; i += R::NT) s_ci[i] = c0 + i < ns ? sel.csel[(size_t)q * C + c0 + i] : -1;
  } else {
    for (int i = tid; i < kCB; i += R::NT) s_ci[i] = c0 + i < C ? c0 + i : -1;
  }
  __syncthreads();
  const float* VtR = static_cast<const float*>(a.VtR) + (size_t)q * kRMax * C;
  const float* sv = static_cast<const float*>(a.s) + (size_t)q * T * C;
  // builder role: contingency bl, rows [bth RB, bth RB + RB)
  const int bl = tid % kCB, bth = tid / kCB;
  const int bc = s_ci[bl];
  const int bdrow = bc >= 0 ? a.mpos[bc] : -1;  // monitored row of its own branch (LODF[c, c] = -1)
  // compute role: contingencies c0 + cg + 16 i, timesteps TR tg + j
  constexpr int TP = L::kTP, SP = L::kSP;
  const int cg = tid % R::CG, tg = tid / R::CG;
  if constexpr (!TC) {
    for (int i = tid; i < RMAX * kCB; i += R::NT) {
      const int j = i / kCB, c = s_ci[i % kCB];
      s_vt[i] = c >= 0 ? -VtR[(size_t)j * C + c] : 0.f;
    }
  }
  for (int i = tid; i < TT * kCB; i += R::NT) s_ov[(i / kCB) * SP + i % kCB] = 0.f;  // overload sums, x 2^-20
  if (tid == 0) {
    for (int st = 0; st < kRegStages; ++st) mbar_init(smem_u32(&bars[st]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  float2 s2[CR][TR];  // N-1 weights s[c, t], duplicated for the row pairs
#pragma unroll
  for (int i = 0; i < CR; ++i)
#pragma unroll
    for (int j = 0; j < TR; ++j) {
      const int c = s_ci[cg + R::CG * i], t = tg * TR + j;
      const float v = (c >= 0 && t0 + t < T) ? sv[(size_t)(t0 + t) * C + c] : 0.f;
      s2[i][j] = make_float2(v, v);
    }
  const int ntiles = (M + kLT - 1) / kLT;
  auto issue = [&](int k) {
    const int st = k % kRegStages;
    unsigned char* base = sm + st * L::kStage;
    const uint32_t bar = smem_u32(&bars[st]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, L::kTx);
    if constexpr (!SEL) tma_load_2d(smem_u32(base), &maps.phi, c0, k * kLT, bar);
    if constexpr (TC) tma_load_3d(smem_u32(base + L::kOffZt), &maps.zt, 0, k * kLT, q, bar);
    else tma_load_3d(smem_u32(base + L::kOffZt), &maps.zt, k * kLT, 0, q, bar);
    tma_load_3d(smem_u32(base + L::kOffPt), &maps.pt, k * kLT, t0, q, bar);
    tma_load_3d(smem_u32(base + L::kOffMeta), &maps.meta, k * kLT, 0, q, bar);
  };
  // SEL: every builder of rows 0.. copies its contingency's 16 rows of tile k
  // (one cp.async group per thread and tile, possibly empty)
  auto issue_phi = [&](int k) {
    if constexpr (SEL) {
      float* dst = reinterpret_cast<float*>(sm + (k % kRegStages) * L::kStage) + bl * kPP;
      if (bth == 0) {
        if (bc >= 0) {
          const float* src = sel.phicm + (size_t)bc * sel.mp + (size_t)k * kLT;
#pragma unroll
          for (int i = 0; i < 4; ++i)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst + 4 * i)), "l"(src + 4 * i)
                         : "memory");
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) *reinterpret_cast<float4*>(dst + 4 * i) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  };
  for (int k = 0; k < kRegStages - 1 && k < ntiles; ++k) {
    if (tid == 0) issue(k);
    issue_phi(k);
  }
  float mx[CR][TR];
  int tk[TRK ? CR : 1][TRK ? TR : 1];  // TRK: the tile of each maximum (the first on ties)
#pragma unroll
  for (int i = 0; i < CR; ++i)
#pragma unroll
    for (int j = 0; j < TR; ++j) {
      mx[i][j] = 0.f;
      if constexpr (TRK) tk[i][j] = 0;
    }
  // the builder's K^{-1}-weighted factors of its contingency, fixed for the block
  constexpr bool kVtReg = RMAX <= 8 && !TC;
  float vb[kVtReg ? RMAX : 1];
  if constexpr (kVtReg) {
#pragma unroll
    for (int j = 0; j < RMAX; ++j) vb[j] = s_vt[j * kCB + bl];
  }
  // TC: the MMA A operand -Vt^T, split into BF16 hi / lo, for the warp's m-blocks
  // (16 contingencies each): lane (g, qd) holds contingencies 16 mb + g and
  // 16 mb + g + 8 at depths 2 qd, 2 qd + 1 (and 2 qd + 8, 2 qd + 9 for K = 16)
  constexpr int KB = TcK<RMAX>::KB;
  constexpr int NW = R::NT / 32, MB = TC ? (kCB / 16) / NW : 1;
  const int lane_g = (tid & 31) >> 2, lane_q = tid & 3, warp = tid >> 5;
  uint32_t ah[MB][4], al[MB][4];
  int drow[MB][2];  // monitored row of each held contingency's own branch, or -1
  if constexpr (TC) {
#pragma unroll
    for (int m = 0; m < MB; ++m) {
      const int mb = warp + NW * m;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = s_ci[16 * mb + lane_g + 8 * h];
        drow[m][h] = c >= 0 ? a.mpos[c] : -1;
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 2 * lane_q + (e & 1) + 8 * (e >> 1);
          v[e] = (c >= 0 && j < RMAX && (e < 2 || KB == 16)) ? -VtR[(size_t)j * C + c] : 0.f;
        }
        // fragment registers: a0 (row g, k 2qd..), a1 (row g + 8, k 2qd..), a2 / a3 the same at k + 8
        bf16_split2(v[0], v[1], ah[m][h], al[m][h]);
        bf16_split2(v[2], v[3], ah[m][2 + h], al[m][2 + h]);
      }
    }
  }
  bool failed = false;
  for (int k = 0; k < ntiles; ++k) {
    const int st = k % kRegStages;
    if constexpr (SEL) asm volatile("cp.async.wait_group 0;" ::: "memory");  // this thread's copies of tile k
    const bool got = mbar_wait(smem_u32(&bars[st]), (uint32_t)((k / kRegStages) & 1));
    // one barrier: the block-uniform failure decision, and proof that every
    // thread is done with tile k-1 (its stage is refilled next, s_ph / s_pt rebuilt)
    if (__syncthreads_or(!got)) {
      failed = true;
      const int last = min(ntiles - 1, k + kRegStages - 2);
      for (int k2 = k; k2 <= last; ++k2) mbar_wait(smem_u32(&bars[k2 % kRegStages]), (uint32_t)((k2 / kRegStages) & 1));
      break;
    }
    if (k + kRegStages - 1 < ntiles) {
      if (tid == 0) issue(k + kRegStages - 1);
      issue_phi(k + kRegStages - 1);
    }
    const unsigned char* base = sm + st * L::kStage;
    const float* phi_t = reinterpret_cast<const float*>(base);
    const float* zt_t = reinterpret_cast<const float*>(base + L::kOffZt);
    const float* pt_t = reinterpret_cast<const float*>(base + L::kOffPt);
    const float* meta_t = reinterpret_cast<const float*>(base + L::kOffMeta);
    if constexpr (TC) {  // Phi_f tile on the tensor cores: warp x (m-blocks of 16 contingencies) x 2 row blocks
      const uint32_t* zb = reinterpret_cast<const uint32_t*>(zt_t);  // row l: KB / 2 words hi, then KB / 2 lo
#pragma unroll
      for (int nb = 0; nb < 2; ++nb) {
        const uint32_t* zr = zb + (8 * nb + lane_g) * KB;
        const uint32_t bh0 = zr[lane_q], bl0 = zr[KB / 2 + lane_q];
        uint32_t bh1 = 0, bl1 = 0;
        if constexpr (KB == 16) {
          bh1 = zr[4 + lane_q];
          bl1 = zr[8 + 4 + lane_q];
        }
        const int l0 = 8 * nb + 2 * lane_q;  // rows l0, l0 + 1 of the tile
        const float2 rm = *reinterpret_cast<const float2*>(&meta_t[1 * kLT + l0]);
        const float2 dg = *reinterpret_cast<const float2*>(&meta_t[l0]);
#pragma unroll
        for (int m = 0; m < MB; ++m) {
          const int cl = 16 * (warp + NW * m) + lane_g;  // contingencies cl and cl + 8 of the block
          float d[4];
          if constexpr (SEL) {
            const float2 u = *reinterpret_cast<const float2*>(&phi_t[cl * kPP + l0]);
            const float2 w = *reinterpret_cast<const float2*>(&phi_t[(cl + 8) * kPP + l0]);
            d[0] = u.x; d[1] = u.y; d[2] = w.x; d[3] = w.y;
          } else {
            d[0] = phi_t[l0 * kPhW + cl];
            d[1] = phi_t[(l0 + 1) * kPhW + cl];
            d[2] = phi_t[l0 * kPhW + cl + 8];
            d[3] = phi_t[(l0 + 1) * kPhW + cl + 8];
          }
          if constexpr (KB == 16) {
            mma_bf16_k16(d, ah[m], bh0, bh1);
            mma_bf16_k16(d, ah[m], bl0, bl1);
            mma_bf16_k16(d, al[m], bh0, bh1);
          } else {
            mma_bf16_k8(d, ah[m], bh0);
            mma_bf16_k8(d, ah[m], bl0);
            mma_bf16_k8(d, al[m], bh0);
          }
          float2 lo = make_float2(d[0] * rm.x, d[1] * rm.y), hi = make_float2(d[2] * rm.x, d[3] * rm.y);
          const int r0 = k * kLT + l0;  // LODF[c, c] = -1: Phi_f entry := -den_c / limit
          if (drow[m][0] == r0) lo.x = dg.x;
          if (drow[m][0] == r0 + 1) lo.y = dg.y;
          if (drow[m][1] == r0) hi.x = dg.x;
          if (drow[m][1] == r0 + 1) hi.y = dg.y;
          s_ph[(l0 / 2) * PH + cl] = lo;
          s_ph[(l0 / 2) * PH + cl + 8] = hi;
        }
      }
    } else {  // build rows [bth RB, bth RB + RB) of Phi_f / limit for contingency bl
      const int r0 = bth * RB;
      float2 p[RB / 2];
#pragma unroll
      for (int i2 = 0; i2 < RB / 2; ++i2) {
        if constexpr (SEL) p[i2] = *reinterpret_cast<const float2*>(&phi_t[bl * kPP + r0 + 2 * i2]);
        else p[i2] = make_float2(phi_t[(r0 + 2 * i2) * kCB + bl], phi_t[(r0 + 2 * i2 + 1) * kCB + bl]);
      }
#pragma unroll
      for (int j = 0; j < RMAX; ++j) {
        float v;
        if constexpr (kVtReg) v = vb[j];
        else v = s_vt[j * kCB + bl];
        const float2 v2 = make_float2(v, v);
#pragma unroll
        for (int i4 = 0; i4 < RB / 4; ++i4) {
          const float4 z = *reinterpret_cast<const float4*>(&zt_t[j * kLT + r0 + 4 * i4]);
          p[2 * i4] = __ffma2_rn(make_float2(z.x, z.y), v2, p[2 * i4]);
          p[2 * i4 + 1] = __ffma2_rn(make_float2(z.z, z.w), v2, p[2 * i4 + 1]);
        }
      }
#pragma unroll
      for (int i4 = 0; i4 < RB / 4; ++i4) {
        const float4 rm = *reinterpret_cast<const float4*>(&meta_t[1 * kLT + r0 + 4 * i4]);
        p[2 * i4] = __fmul2_rn(p[2 * i4], make_float2(rm.x, rm.y));
        p[2 * i4 + 1] = __fmul2_rn(p[2 * i4 + 1], make_float2(rm.z, rm.w));
      }
      const int dr = bdrow - k * kLT - r0;
      if ((unsigned)dr < (unsigned)RB) {  // LODF[c, c] = -1: Phi_f entry := -den_c / limit
        const float dg = meta_t[r0 + dr];
#pragma unroll
        for (int i2 = 0; i2 < RB / 2; ++i2) {
          if (2 * i2 == dr) p[i2].x = dg;
          if (2 * i2 + 1 == dr) p[i2].y = dg;
        }
      }
#pragma unroll
      for (int i2 = 0; i2 < RB / 2; ++i2) s_ph[(r0 / 2 + i2) * PH + bl] = p[i2];
    }
    // p_f / limit as row pairs per timestep: s_pt[rp][t] = (pt[t][2 rp], pt[t][2 rp + 1])
    for (int i = tid; i < (kLT / 2) * TT; i += R::NT) {
      const int rp = i % (kLT / 2), t = i / (kLT / 2);
      s_pt[rp * TP + t] = *reinterpret_cast<const float2*>(&pt_t[t * kLT + 2 * rp]);
    }
    __syncthreads();
    float mt[CR][TR];  // maxima over this tile (the overload test), folded into mx
#pragma unroll
    for (int rp = 0; rp < kLT / 2; ++rp) {
      float2 ph[CR];
#pragma unroll
      for (int i = 0; i < CR; ++i) ph[i] = s_ph[rp * PH + cg + R::CG * i];
      float2 pt[TR];
      if constexpr (TR % 2 == 0) {
#pragma unroll
        for (int j2 = 0; j2 < TR / 2; ++j2) {
          const float4 u = *reinterpret_cast<const float4*>(&s_pt[rp * TP + tg * TR + 2 * j2]);
          pt[2 * j2] = make_float2(u.x, u.y);
          pt[2 * j2 + 1] = make_float2(u.z, u.w);
        }
      } else {
#pragma unroll
        for (int j = 0; j < TR; ++j) pt[j] = s_pt[rp * TP + tg * TR + j];
      }
#pragma unroll
      for (int i = 0; i < CR; ++i)
#pragma unroll
        for (int j = 0; j < TR; ++j) {
          const float2 v = __ffma2_rn(ph[i], s2[i][j], pt[j]);  // rows 2 rp and 2 rp + 1
          if (OVL) mt[i][j] = rp == 0 ? max3abs(v.x, v.y, v.y) : max3abs(mt[i][j], v.x, v.y);
          else mx[i][j] = max3abs(mx[i][j], v.x, v.y);
        }
    }
    if (OVL) {
#pragma unroll
      for (int i = 0; i < CR; ++i)
#pragma unroll
        for (int j = 0; j < TR; ++j) {
          if constexpr (TRK) {
            const bool up = mt[i][j] > mx[i][j];
            mx[i][j] = up ? mt[i][j] : mx[i][j];
            tk[i][j] = up ? k : tk[i][j];
          } else {
            mx[i][j] = fmaxf(mx[i][j], mt[i][j]);
          }
        }
      // overload sum only for the (contingency, timestep) items whose tile
      // maximum exceeds 1: the warp queues them and serves the queue with all
      // lanes (items of one tile are distinct (t, c) pairs: no write conflicts)
      const int lane = tid & 31;
      uint16_t* queue = reinterpret_cast<uint16_t*>(sm + L::kOffQ) + (tid >> 5) * 32 * CR * TR;
      const uint32_t lt = (1u << lane) - 1u;
      int n = 0;
#pragma unroll
      for (int i = 0; i < CR; ++i)
#pragma unroll
        for (int j = 0; j < TR; ++j) {
          const bool hit = mt[i][j] > 1.0f;
          const uint32_t m = __ballot_sync(0xffffffffu, hit);
          if (hit) queue[n + __popc(m & lt)] = (uint16_t)((lane << 8) | (i * TR + j));
          n += __popc(m);
        }
      if (n) {
        __syncwarp();
        for (int jq = lane; jq < n; jq += 32) {
          const int item = queue[jq];
          const int src = (tid & ~31) | (item >> 8), b = item & 255;
          const int cl = src % R::CG + R::CG * (b / TR), t = (src / R::CG) * TR + b % TR;
          const int cs = s_ci[cl];
          const float stv = (cs >= 0 && t0 + t < T) ? sv[(size_t)(t0 + t) * C + cs] : 0.f;
          const float2 s22 = make_float2(stv, stv);
          float2 o2 = make_float2(0.f, 0.f);
#pragma unroll
          for (int rp = 0; rp < kLT / 2; ++rp) {
            const float2 v = __ffma2_rn(s_ph[rp * PH + cl], s22, s_pt[rp * TP + t]);
            o2 = __fadd2_rn(o2, make_float2(__saturatef(fmaf(fabsf(v.x), 0x1p-20f, -0x1p-20f)),
                                            __saturatef(fmaf(fabsf(v.y), 0x1p-20f, -0x1p-20f))));
          }
          s_ov[t * SP + cl] += o2.x + o2.y;
        }
        __syncwarp();
      }
    }
  }
  if (failed) {
    if constexpr (SEL) asm volatile("cp.async.wait_all;" ::: "memory");
    if (tid == 0) atomicExch(a.err, 1);
    return;
  }
  // per-timestep maxima to shared memory (s is held in registers), then one
  // thread per timestep scans the 64 contingencies in order: max with the
  // lowest contingency on ties, and the overload sum in a fixed order
  __syncthreads();
  uint8_t* okc = sm + L::kOffOk;
#pragma unroll
  for (int i = 0; i < CR; ++i)
#pragma unroll
    for (int j = 0; j < TR; ++j) s_s[(tg * TR + j) * SP + cg + R::CG * i] = mx[i][j];
  if (tid < kCB) okc[tid] = (s_ci[tid] >= 0) && a.valid[(size_t)q * C + s_ci[tid]];
  __syncthreads();
  if (a.out.n1_cont_max) {  // per-contingency maxima (screener labels)
    for (int i = tid; i < TT * kCB; i += R::NT) {
      const int t = t0 + i / kCB, cl = i % kCB, c = s_ci[cl];
      if (t < T && c >= 0)
        a.out.n1_cont_max[((size_t)qi.tau * T + t) * C + a.cont_pos[c]] = okc[cl] ? s_s[(i / kCB) * SP + cl] : -1.f;
    }
  }
  if constexpr (TRK) {  // the tile of every maximum (internal order), through the idle stages
    static_assert(TT * SP * 4 + TT * SP * 2 <= kRegStages * L::kStage, "tiles fit the stages");
    uint16_t* s_tk = reinterpret_cast<uint16_t*>(sm + TT * SP * 4);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < CR; ++i)
#pragma unroll
      for (int j = 0; j < TR; ++j) s_tk[(tg * TR + j) * SP + cg + R::CG * i] = (uint16_t)tk[i][j];
    __syncthreads();
    for (int i = tid; i < TT * kCB; i += R::NT) {
      const int t = t0 + i / kCB, cl = i % kCB, c = s_ci[cl];
      if (t < T && c >= 0) a.tile[((size_t)q * T + t) * C + c] = s_tk[(i / kCB) * SP + cl];
    }
  }
  if (a.cmr) {  // the same in internal order for the final pass's tie band
    for (int i = tid; i < TT * kCB; i += R::NT) {
      const int t = t0 + i / kCB, cl = i % kCB, c = s_ci[cl];
      if (t < T && c >= 0)
        static_cast<float*>(a.cmr)[((size_t)q * T + t) * C + c] = okc[cl] ? s_s[(i / kCB) * SP + cl] : -1.f;
    }
  }
  for (int t = tid; t < TT; t += R::NT) {
    if (t0 + t >= T) continue;
    float bv = -1.f, b2 = -1.f;  // the largest (lowest contingency on ties) and the second largest
    int ba = -1;
    // the overload sums of 8 consecutive contingencies in FP32, then one FP64
    // add: the B300's FP64 pipe would otherwise hold the block's slot for a
    // conversion and an add per contingency
    double o = 0.0;
    float o8 = 0.f;
    for (int k2 = 0; k2 < kCB; ++k2) {
      if (okc[k2]) {
        const float v = s_s[t * SP + k2];
        if (v > bv) {
          b2 = bv;
          bv = v;
          ba = s_ci[k2];
        } else if (v > b2) {
          b2 = v;
        }
        o8 += s_ov[t * SP + k2];
      }
      if ((k2 & 7) == 7) {
        o += (double)(o8 * 1048576.f);
        o8 = 0.f;
      }
    }
    const size_t o2 = ((size_t)q * T + t0 + t) * a.ncb + cb;
    static_cast<float*>(a.pmax)[o2] = bv;
    a.parg[o2] = ba;
    a.povl[o2] = o;
    if (a.p2max) static_cast<float*>(a.p2max)[o2] = b2;
  }
}

}  // namespace dcf
