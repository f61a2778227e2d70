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

namespace dcf {

constexpr int kLT = 16;     // monitored rows per tile
constexpr int kCB = 64;     // contingencies per block
constexpr int kStages = 2;  // TMA ring depth
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: bounded mbarrier wait

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
  static constexpr int kOffS = kStages * kStage;             // float s[TT][kCB]
  static constexpr int kOffOv = kOffS + a128(TT * kCB * 4);   // float ov[TT][kCB]
  static constexpr int kOffBar = kOffOv + a128(TT * kCB * 4); // uint64 bar[kStages]
  static constexpr int kBytes = kOffBar + 64 + 128;           // + alignment slack
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

struct N1Maps {
  CUtensorMap phi, zt, pt, meta;
};

template <int TT, int RMAX>
__global__ __launch_bounds__(kCB) void k_n1_tma(const __grid_constant__ N1Maps maps, Args a, int t0) {
  using L = TmaLayout<TT, RMAX>;
  const int q = blockIdx.y;
  const QInfo qi = a.qi[q];
  if (qi.status != ST_OK) return;  // whole block: before any barrier
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~uintptr_t(127));
  float* s_s = reinterpret_cast<float*>(sm + L::kOffS);
  float* s_ov = reinterpret_cast<float*>(sm + L::kOffOv);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::kOffBar);
  const int tid = threadIdx.x, M = a.M, C = a.C, T = a.T;
  const int c0 = blockIdx.x * kCB, c = c0 + tid;
  const bool cin = c < C;
  const int cc = cin ? c : C - 1;
  const float* VtR = static_cast<const float*>(a.VtR) + (size_t)q * kRMax * C;
  const float* sv = static_cast<const float*>(a.s) + (size_t)q * T * C;
  float2 nvt[RMAX];
#pragma unroll
  for (int j = 0; j < RMAX; ++j) {
    const float v = -VtR[(size_t)j * C + cc];
    nvt[j] = make_float2(v, v);
  }
#pragma unroll
  for (int t = 0; t < TT; ++t) {
    s_s[t * kCB + tid] = (cin && t0 + t < T) ? sv[(size_t)(t0 + t) * C + cc] : 0.f;
    s_ov[t * kCB + tid] = 0.f;
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
  float mx[TT];
#pragma unroll
  for (int t = 0; t < TT; ++t) mx[t] = 0.f;
  bool failed = false;
  for (int k = 0; k < ntiles; ++k) {
    if (tid == 0 && k + kStages - 1 < ntiles) issue(k + kStages - 1);
    const int st = k % kStages;
    const bool got = mbar_wait(smem_u32(&bars[st]), (uint32_t)((k / kStages) & 1));
    if (__syncthreads_or(!got)) {  // block-uniform decision
      failed = true;
      // wait (bounded) for this block's copies still in flight before leaving
      const int last = min(ntiles - 1, k + kStages - 1);
      for (int k2 = k; k2 <= last; ++k2) mbar_wait(smem_u32(&bars[k2 % kStages]), (uint32_t)((k2 / kStages) & 1));
      break;
    }
    const unsigned char* base = sm + st * L::kStage;
    const float* phi_t = reinterpret_cast<const float*>(base);
    const float* zt_t = reinterpret_cast<const float*>(base + L::kOffZt);
    const float* pt_t = reinterpret_cast<const float*>(base + L::kOffPt);
    const float* meta_t = reinterpret_cast<const float*>(base + L::kOffMeta);
    // Phi_f / limit for this thread's contingency and the tile's 16 rows
    float2 ph[kLT / 2];
#pragma unroll
    for (int i2 = 0; i2 < kLT / 2; ++i2) {
      float2 p = make_float2(phi_t[(2 * i2) * kCB + tid], phi_t[(2 * i2 + 1) * kCB + tid]);
#pragma unroll
      for (int j = 0; j < RMAX; ++j) {
        const float2 z = *reinterpret_cast<const float2*>(&zt_t[j * kLT + 2 * i2]);
        p = __ffma2_rn(z, nvt[j], p);
      }
      const float2 rm = *reinterpret_cast<const float2*>(&meta_t[1 * kLT + 2 * i2]);
      p = __fmul2_rn(p, rm);
      const float2 dg = *reinterpret_cast<const float2*>(&meta_t[0 * kLT + 2 * i2]);
      const int2 cp = *reinterpret_cast<const int2*>(&meta_t[2 * kLT + 2 * i2]);
      if (cp.x == c) p.x = dg.x;
      if (cp.y == c) p.y = dg.y;
      ph[i2] = p;
    }
#pragma unroll
    for (int t = 0; t < TT; ++t) {
      const float s = s_s[t * kCB + tid];
      const float2 s2 = make_float2(s, s);
      float2 v[kLT / 2];
#pragma unroll
      for (int i4 = 0; i4 < kLT / 4; ++i4) {
        const float4 p4 = *reinterpret_cast<const float4*>(&pt_t[t * kLT + 4 * i4]);
        v[2 * i4] = __ffma2_rn(ph[2 * i4], s2, make_float2(p4.x, p4.y));
        v[2 * i4 + 1] = __ffma2_rn(ph[2 * i4 + 1], s2, make_float2(p4.z, p4.w));
      }
      float m = max3abs(v[0].x, v[0].y, v[1].x);
      m = max3abs(m, v[1].y, v[2].x);
      m = max3abs(m, v[2].y, v[3].x);
      m = max3abs(m, v[3].y, v[4].x);
      m = max3abs(m, v[4].y, v[5].x);
      m = max3abs(m, v[5].y, v[6].x);
      m = max3abs(m, v[6].y, v[7].x);
      m = max3abs(m, v[7].y, v[7].y);
      mx[t] = fmaxf(mx[t], m);
      if (m > 1.0f) {
        float o = 0.f;
#pragma unroll
        for (int i2 = 0; i2 < kLT / 2; ++i2) {
          o += __saturatef(fmaf(fabsf(v[i2].x), 0x1p-20f, -0x1p-20f));
          o += __saturatef(fmaf(fabsf(v[i2].y), 0x1p-20f, -0x1p-20f));
        }
        s_ov[t * kCB + tid] += o;
      }
    }
    __syncthreads();  // every thread is done with this stage before it is refilled
  }
  if (failed) {
    if (tid == 0) atomicExch(a.err, 1);
    return;
  }
  // reduce the 64 contingencies of this block: max (ties: lowest c) and overload sum
  const bool ok = cin && a.valid[(size_t)q * C + c];
  __shared__ double rv[2], ro[2];
  __shared__ int ra[2];
  const int lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int t = 0; t < TT; ++t) {
    if (t0 + t < T) {
      double v = ok ? (double)mx[t] : -1.0;
      int arg = ok ? c : 0x7fffffff;
      double o = ok ? (double)s_ov[t * kCB + tid] * 1048576.0 : 0.0;
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
        static_cast<float*>(a.pmax)[o2] = (float)bv;
        a.parg[o2] = (bv < 0.0) ? -1 : ba;
        a.povl[o2] = ro[0] + ro[1];
      }
      __syncthreads();
    }
  }
}

}  // namespace dcf
