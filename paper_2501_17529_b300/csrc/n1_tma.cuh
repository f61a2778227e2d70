// FP32 fused N-1 kernel with TMA-staged tiles (Def. 3 / Eq. (5), agg_m of Sec. III-A).
//
// One block = one topology x 64 contingencies (one per thread).  The block
// streams the monitored rows in tiles of 16; a 2-stage ring in shared memory
// is filled by the tensor-memory accelerator (cp.async.bulk.tensor, completion
// on an mbarrier) with, per tile:
//   phi  [16 rows][64 cont]  Phi[mon, cont] / limit          (per study, 2-D map)
//   zt   [RMAX][16 rows]     Z / limit, transposed            (per topology, 3-D map)
//   pt   [TT][16 rows]       p_f / limit, transposed          (per topology, 3-D map)
//   meta [4][16 rows]        diagonal override, row mask, contingency position
// Rows beyond the last monitored branch and columns beyond the last
// contingency are zero-filled by the TMA unit.  Per thread and tile:
//   Phi_f[l, c] = Phi[l, c] - Z[l, :] . Vt[:, c]   (FFMA2 over row pairs)
//   per timestep: v = Phi_f[l, c] s[c, t] + p_f[l, t]  (FFMA2), |v| max via the
//   3-input max.abs, and the overload sum only when the tile's max exceeds 1.
#pragma once

#include <cuda.h>

#include "n1_types.cuh"

namespace dcf {

constexpr int kStages = 3;  // TMA ring depth

template <int TT, int RMAX>
struct TmaLayout {
  static constexpr int a128(int x) { return (x + 127) / 128 * 128; }
  static constexpr int kPhi = kLT * kCB * 4;
  static constexpr int kZt = RMAX * kLT * 4;
  static constexpr int kPt = TT * kLT * 4;
  static constexpr int kMeta = 4 * kLT * 4;
  static constexpr int kTx = kPhi + kZt + kPt + kMeta;  // bytes landing per stage
  static constexpr int kOffZt = a128(kPhi);
  static constexpr int kOffPt = kOffZt + a128(kZt);
  static constexpr int kOffMeta = kOffPt + a128(kPt);
  static constexpr int kStage = kOffMeta + a128(kMeta);
  static constexpr int kOffPh = kStages * kStage;             // float2 ph[kLT/2][kCB]: the built Phi_f tile
  static constexpr int kOffS = kOffPh + kLT * kCB * 4;        // float s[TT][kCB]
  static constexpr int kOffOv = kOffS + a128(TT * kCB * 4);   // float ov[TT][kCB]
  static constexpr int kOffBar = kOffOv + a128(TT * kCB * 4); // uint64 bar[kStages]
  static constexpr int kOffOk = kOffBar + 64;                 // uint8 ok[kCB]
  static constexpr int kOffQ = kOffOk + 128;                  // uint16 queue[warps][32 * TT]
  static constexpr int kBytes = kOffQ + (kCB / 32) * 2 * 32 * TT * 2;  // one queue per warp (up to 4 warps)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait on an mbarrier phase; false if the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float max3abs(float a, float b, float c) {
  float r;
  asm("max.abs.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}


// NTH threads per contingency, each owning TT / NTH timesteps; the block
// builds each tile's Phi_f [16 rows x 64 contingencies] once into shared memory
// (thread group th builds rows th*16/NTH ...), then every thread reads its
// contingency's 16 values back.
// OVL = false drops the overload sum (metric-first screening of injection
// candidates needs only the maximum loading).
template <int TT, int RMAX, int NTH, bool OVL>
__global__ __launch_bounds__(kCB * NTH) void k_n1_tma(const __grid_constant__ N1Maps maps, Args a, int t0_base) {
  const int t0 = t0_base + (int)blockIdx.z * TT;  // grid z: the passes over TT timesteps each
  using L = TmaLayout<TT, RMAX>;
  constexpr int TH = TT / NTH;    // timesteps per thread
  constexpr int RB = kLT / NTH;   // tile rows built per thread
  static_assert(TT % NTH == 0 && RB % 4 == 0, "tile split");
  const int q = blockIdx.y;
  const QInfo qi = a.qi[q];
  if (qi.status != ST_OK) return;  // whole block: before any barrier
  // the dynamic shared block starts 128-byte aligned (no static shared memory in
  // this kernel); indexing it directly keeps every access in the shared space
  extern __shared__ __align__(128) unsigned char sm[];
  if (smem_u32(sm) & 127u) {  // the TMA destinations need the alignment: refuse, never fault
    if (threadIdx.x == 0) atomicExch(a.err, 2);
    return;
  }
  float2* s_ph = reinterpret_cast<float2*>(sm + L::kOffPh);
  float* s_s = reinterpret_cast<float*>(sm + L::kOffS);
  float* s_ov = reinterpret_cast<float*>(sm + L::kOffOv);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::kOffBar);
  const int tid = threadIdx.x, cl = tid % kCB, th = tid / kCB;
  const int M = a.M, C = a.C, T = a.T;
  const int c0 = blockIdx.x * kCB, c = c0 + cl;
  const bool cin = c < C;
  const int cc = cin ? c : C - 1;
  const float* VtR = static_cast<const float*>(a.VtR) + (size_t)q * kRMax * C;
  const float* sv = static_cast<const float*>(a.s) + (size_t)q * T * C;
  // monitored row of this contingency's own branch (LODF[c, c] = -1 override), or -1
  const int drow = cin ? a.mpos[c] : -1;
  float2 nvt[RMAX];
#pragma unroll
  for (int j = 0; j < RMAX; ++j) {
    const float v = -VtR[(size_t)j * C + cc];
    nvt[j] = make_float2(v, v);
  }
#pragma unroll
  for (int tt = 0; tt < TH; ++tt) {
    const int t = th * TH + tt;
    s_s[t * kCB + cl] = (cin && t0 + t < T) ? sv[(size_t)(t0 + t) * C + cc] : 0.f;
    s_ov[t * kCB + cl] = 0.f;  // overload partial sums, scaled by 2^-20
  }
  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(smem_u32(&bars[st]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int ntiles = (M + kLT - 1) / kLT;
  auto issue = [&](int k) {
    const int st = k % kStages;
    unsigned char* base = sm + st * L::kStage;
    const uint32_t bar = smem_u32(&bars[st]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, L::kTx);
    tma_load_2d(smem_u32(base), &maps.phi, c0, k * kLT, bar);
    tma_load_3d(smem_u32(base + L::kOffZt), &maps.zt, k * kLT, 0, q, bar);
    tma_load_3d(smem_u32(base + L::kOffPt), &maps.pt, k * kLT, t0, q, bar);
    tma_load_3d(smem_u32(base + L::kOffMeta), &maps.meta, k * kLT, 0, q, bar);
  };
  if (tid == 0)
    for (int k = 0; k < kStages - 1 && k < ntiles; ++k) issue(k);
  float mx[TH];
#pragma unroll
  for (int tt = 0; tt < TH; ++tt) mx[tt] = 0.f;
  bool failed = false;
  for (int k = 0; k < ntiles; ++k) {
    const int st = k % kStages;
    const bool got = mbar_wait(smem_u32(&bars[st]), (uint32_t)((k / kStages) & 1));
    // one barrier: the block-uniform failure decision, and proof that every
    // thread is done with tile k-1 (its stage is refilled next, its Phi_f rebuilt)
    if (__syncthreads_or(!got)) {
      failed = true;
      const int last = min(ntiles - 1, k + kStages - 2);
      for (int k2 = k; k2 <= last; ++k2) mbar_wait(smem_u32(&bars[k2 % kStages]), (uint32_t)((k2 / kStages) & 1));
      break;
    }
    if (tid == 0 && k + kStages - 1 < ntiles) issue(k + kStages - 1);
    const unsigned char* base = sm + st * L::kStage;
    const float* phi_t = reinterpret_cast<const float*>(base);
    const float* zt_t = reinterpret_cast<const float*>(base + L::kOffZt);
    const float* pt_t = reinterpret_cast<const float*>(base + L::kOffPt);
    const float* meta_t = reinterpret_cast<const float*>(base + L::kOffMeta);
    {  // build rows [th*RB, th*RB + RB) of Phi_f / limit for contingency cl
      const int r0 = th * RB;
      float2 p[RB / 2];
#pragma unroll
      for (int i2 = 0; i2 < RB / 2; ++i2)
        p[i2] = make_float2(phi_t[(r0 + 2 * i2) * kCB + cl], phi_t[(r0 + 2 * i2 + 1) * kCB + cl]);
#pragma unroll
      for (int j = 0; j < RMAX; ++j) {
#pragma unroll
        for (int i4 = 0; i4 < RB / 4; ++i4) {
          const float4 z = *reinterpret_cast<const float4*>(&zt_t[j * kLT + r0 + 4 * i4]);
          p[2 * i4] = __ffma2_rn(make_float2(z.x, z.y), nvt[j], p[2 * i4]);
          p[2 * i4 + 1] = __ffma2_rn(make_float2(z.z, z.w), nvt[j], p[2 * i4 + 1]);
        }
      }
#pragma unroll
      for (int i4 = 0; i4 < RB / 4; ++i4) {
        const float4 rm = *reinterpret_cast<const float4*>(&meta_t[1 * kLT + r0 + 4 * i4]);
        p[2 * i4] = __fmul2_rn(p[2 * i4], make_float2(rm.x, rm.y));
        p[2 * i4 + 1] = __fmul2_rn(p[2 * i4 + 1], make_float2(rm.z, rm.w));
      }
      const int dr = drow - k * kLT - r0;
      if ((unsigned)dr < (unsigned)RB) {  // LODF[c, c] = -1: Phi_f entry := -den_c / limit
        const float dg = meta_t[r0 + dr];
#pragma unroll
        for (int i2 = 0; i2 < RB / 2; ++i2) {
          if (2 * i2 == dr) p[i2].x = dg;
          if (2 * i2 + 1 == dr) p[i2].y = dg;
        }
      }
#pragma unroll
      for (int i2 = 0; i2 < RB / 2; ++i2) s_ph[(r0 / 2 + i2) * kCB + cl] = p[i2];
    }
    __syncthreads();
    float2 ph[kLT / 2];
#pragma unroll
    for (int i2 = 0; i2 < kLT / 2; ++i2) ph[i2] = s_ph[i2 * kCB + cl];
    float mt[TH];
#pragma unroll
    for (int tt = 0; tt < TH; ++tt) {
      const int t = th * TH + tt;
      const float stv = s_s[t * kCB + cl];
      const float2 s2 = make_float2(stv, stv);
      float2 v[kLT / 2];
#pragma unroll
      for (int i4 = 0; i4 < kLT / 4; ++i4) {
        const float4 p4 = *reinterpret_cast<const float4*>(&pt_t[t * kLT + 4 * i4]);
        v[2 * i4] = __ffma2_rn(ph[2 * i4], s2, make_float2(p4.x, p4.y));
        v[2 * i4 + 1] = __ffma2_rn(ph[2 * i4 + 1], s2, make_float2(p4.z, p4.w));
      }
      const float m0 = max3abs(v[0].x, v[0].y, v[1].x);
      const float m1 = max3abs(v[1].y, v[2].x, v[2].y);
      const float m2 = max3abs(v[3].x, v[3].y, v[4].x);
      const float m3 = max3abs(v[4].y, v[5].x, v[5].y);
      const float m4 = max3abs(v[6].x, v[6].y, v[7].x);
      const float m = fmaxf(fmaxf(fmaxf(m0, m1), fmaxf(m2, m3)), max3abs(m4, v[7].y, v[7].y));
      mt[tt] = m;
      mx[tt] = fmaxf(mx[tt], m);
    }
    // overload sum only for (tile, timestep, contingency) items whose tile max
    // exceeds 1 (a few percent): the warp queues them timestep by timestep
    // (one ballot per timestep) and serves the queue with all lanes; items of
    // one timestep read the same p_f row (broadcast) and the built tile in s_ph
    if (OVL) {
      const int lane = tid & 31, cb = (tid & (kCB - 1)) & ~31;  // first contingency of this warp
      uint16_t* queue = reinterpret_cast<uint16_t*>(sm + L::kOffQ) + (tid >> 5) * 32 * TT;
      const uint32_t lt = (1u << lane) - 1u;
      int n = 0;
#pragma unroll
      for (int tt = 0; tt < TH; ++tt) {
        const bool hit = mt[tt] > 1.0f;
        const uint32_t msk = __ballot_sync(0xffffffffu, hit);
        if (hit) queue[n + __popc(msk & lt)] = (uint16_t)(tt * 32 + lane);
        n += __popc(msk);
      }
      if (n) {
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
          const int item = queue[j];
          const int t = th * TH + (item >> 5), cj = cb + (item & 31);
          const float stv = s_s[t * kCB + cj];
          const float2 s2 = make_float2(stv, stv);
          float2 o2 = make_float2(0.f, 0.f);
#pragma unroll
          for (int i4 = 0; i4 < kLT / 4; ++i4) {
            const float4 p4 = *reinterpret_cast<const float4*>(&pt_t[t * kLT + 4 * i4]);
            const float2 va = __ffma2_rn(s_ph[(2 * i4) * kCB + cj], s2, make_float2(p4.x, p4.y));
            const float2 vb = __ffma2_rn(s_ph[(2 * i4 + 1) * kCB + cj], s2, make_float2(p4.z, p4.w));
            o2 = __fadd2_rn(o2, make_float2(__saturatef(fmaf(fabsf(va.x), 0x1p-20f, -0x1p-20f)),
                                            __saturatef(fmaf(fabsf(va.y), 0x1p-20f, -0x1p-20f))));
            o2 = __fadd2_rn(o2, make_float2(__saturatef(fmaf(fabsf(vb.x), 0x1p-20f, -0x1p-20f)),
                                            __saturatef(fmaf(fabsf(vb.y), 0x1p-20f, -0x1p-20f))));
          }
          s_ov[t * kCB + cj] += o2.x + o2.y;  // items of one tile are distinct (t, contingency) pairs
        }
        __syncwarp();
      }
    }
  }
  if (failed) {
    if (tid == 0) atomicExch(a.err, 1);
    return;
  }
  // per-timestep maxima to shared memory (the s array is no longer needed), then
  // one thread per timestep scans the 64 contingencies in order: max with the
  // lowest contingency on ties, and the overload sum in a fixed order
  __syncthreads();
#pragma unroll
  for (int tt = 0; tt < TH; ++tt) s_s[(th * TH + tt) * kCB + cl] = mx[tt];
  uint8_t* okc = sm + L::kOffOk;
  const bool okv = cin && a.valid[(size_t)q * C + c];
  if (th == 0) okc[cl] = okv;
  if (a.out.n1_cont_max && cin) {  // per-contingency maxima (screener labels)
#pragma unroll
    for (int tt = 0; tt < TH; ++tt) {
      const int t = t0 + th * TH + tt;
      if (t < T) a.out.n1_cont_max[((size_t)qi.tau * T + t) * C + a.cont_pos[c]] = okv ? mx[tt] : -1.f;
    }
  }
  if (a.cmr && cin) {  // the same for the final pass's tie band (internal order)
#pragma unroll
    for (int tt = 0; tt < TH; ++tt) {
      const int t = t0 + th * TH + tt;
      if (t < T) static_cast<float*>(a.cmr)[((size_t)q * T + t) * C + c] = okv ? mx[tt] : -1.f;
    }
  }
  __syncthreads();
  for (int t = tid; t < TT; t += kCB * NTH) {
    if (t0 + t >= T) continue;
    float bv = -1.f, b2 = -1.f;  // the largest (lowest contingency on ties) and the second largest
    int ba = -1;
    double o = 0.0;  // 8 contingencies' overload sums in FP32, then one FP64 add (B300's FP64 rate)
    float o8 = 0.f;
    for (int k2 = 0; k2 < kCB; ++k2) {
      if (okc[k2]) {
        const float v = s_s[t * kCB + k2];
        if (v > bv) {
          b2 = bv;
          bv = v;
          ba = c0 + k2;
        } else if (v > b2) {
          b2 = v;
        }
        o8 += s_ov[t * kCB + k2];
      }
      if ((k2 & 7) == 7) {
        o += (double)(o8 * 1048576.f);
        o8 = 0.f;
      }
    }
    const size_t o2 = ((size_t)q * T + t0 + t) * a.ncb + blockIdx.x;
    static_cast<float*>(a.pmax)[o2] = bv;
    a.parg[o2] = ba;
    a.povl[o2] = o;
    if (a.p2max) static_cast<float*>(a.p2max)[o2] = b2;
  }
}

}  // namespace dcf
