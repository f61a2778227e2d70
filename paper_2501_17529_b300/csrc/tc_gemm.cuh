// BF16 GEMM on the 5th-generation tensor cores (tcgen05) with FP32 accumulation
// in tensor memory: D[M x N] = A[M x K] * B[N x K]^T (+ bias[N], optional ReLU),
// both operands K-major bf16, D row-major in FP32 or BF16.
//
// One CTA per 128 x 128 output tile, 128 threads, a 6-stage shared-memory
// ring with two single-thread roles: warp 0 lane 0 is the TMA producer (waits
// for a stage to be free on its "empty" mbarrier, then loads 128 x 64 bf16
// boxes of A and B with 128-byte swizzle, completion on the stage's "full"
// mbarrier); warp 1 lane 0 issues the MMAs (waits for "full", four
// tcgen05.mma.kind::f16 with K = 16 into a 128 x 128 FP32 accumulator in
// tensor memory, then tcgen05.commit frees the stage on "empty").  Neither
// role waits for the other's latest step, so loads run STAGES - 1 k-tiles
// ahead of the tensor pipe.  After the last k-tile a commit signals the
// epilogue: each warp reads its 32 accumulator lanes (rows) with
// tcgen05.ld.32x32b.
// Epilogue options: bias[N], ReLU, a ReLU-derivative mask (D := 0 where a
// bf16 tensor of D's shape is <= 0), FP32 or BF16 output, an optional second
// BF16 store of D transposed, and split-K: gridDim.z CTAs share the K range of
// a tile and each stores its FP32 partial at D + z * split_stride.
// Every mbarrier wait is bounded; on expiry the CTA records an error, waits
// (bounded) for its outstanding copies and MMAs, frees its tensor memory and
// returns.  Shapes: M, N multiples of 128, K a multiple of 64 * gridDim.z.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace dcf {
namespace tc {

constexpr int BM = 128, BK = 64;
// Output tile 128 x BN (BN = 128 or 256): an N = 256 MMA reads 12 KB of
// operands from shared memory per 1 MFLOP, an N = 128 one 8 KB per 0.5 MFLOP,
// so the wide tile leaves the shared-memory port headroom.
template <int BN>
struct Cfg {
  static constexpr int STAGES = BN == 256 ? 4 : 6;
  static constexpr int kTileA = BM * BK * 2;                  // 16 KB
  static constexpr int kTileB = BN * BK * 2;                  // 16 or 32 KB
  static constexpr int kStageBytes = kTileA + kTileB;
  static constexpr int kSmemBytes = 1024 /*align*/ + STAGES * kStageBytes + 256 /*barriers, tmem slot*/;
};
constexpr long long kWait = 4000000000LL;        // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_expect(uint32_t b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(b), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWait) return false;
  }
}
__device__ __forceinline__ void tma2d(uint32_t dst, const CUtensorMap* m, int x, int y, uint32_t b) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(m), "r"(x), "r"(y), "r"(b)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);         // start address
  d |= (uint64_t)(16 >> 4) << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                         // descriptor version of this architecture
  d |= (uint64_t)2 << 61;                         // layout: 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

struct GemmArgs {
  int M, N, K;
  const float* bias;             // [N] or null
  int relu;
  const __nv_bfloat16* mask;     // [M x ldm] or null: D := 0 where mask <= 0
  int ldm;
  void* D;                       // row-major [M x ldd] or null
  int ldd;
  int out_bf16;
  __nv_bfloat16* Dt;             // [N x lddt] transposed BF16 copy of D, or null
  int lddt;
  long long split_stride;        // elements between the FP32 partials of split-K
  int* err;
};

template <int BN>
__global__ __launch_bounds__(128) void k_gemm_bf16(const __grid_constant__ CUtensorMap mA,
                                                   const __grid_constant__ CUtensorMap mB, GemmArgs g) {
  constexpr int STAGES = Cfg<BN>::STAGES, kStageBytes = Cfg<BN>::kStageBytes, kTileBytes = Cfg<BN>::kTileA;
  extern __shared__ __align__(1024) unsigned char smem[];
  const uint32_t raw = su32(smem);
  const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned tile area
  const uint32_t bars = base + STAGES * kStageBytes;  // full[S], empty[S], done
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (STAGES + s); };
  const uint32_t done = bars + 8u * (2 * STAGES);
  const uint32_t tslot = done + 8u;  // tensor-memory address written by tcgen05.alloc
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tiles in groups of 8 M-rows: a wave of CTAs covers a compact block of the
  // output, so the A rows and B columns it streams are shared through L2
  int tm, tn;
  {
    const int gx = gridDim.x, gy = gridDim.y, lin = blockIdx.y * gx + blockIdx.x;
    const int G = 8, grp = lin / (G * gx), first = grp * G, rows = min(G, gy - first);
    const int r = lin - grp * G * gx;
    tm = first + r % rows;
    tn = r / rows;
  }
  const int m0 = tm * BM, n0 = tn * BN;
  const int KT = g.K / BK / (int)gridDim.z;  // k-tiles of this CTA's share
  const int kt0 = (int)blockIdx.z * KT;
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      bar_init(full(s), 1);
      bar_init(empty(s), 1);
    }
    bar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tslot), "r"(BN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  uint32_t tmem;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(tmem) : "r"(tslot) : "memory");
  __shared__ int failed;    // a role gave up on a bounded wait
  __shared__ int consumed;  // k-tiles whose MMAs were issued
  __shared__ int issued;    // k-tiles whose loads were issued
  if (tid == 0) {
    failed = 0;
    consumed = 0;
    issued = 0;
  }
  __syncthreads();
  volatile int* vfailed = &failed;
  volatile int* vconsumed = &consumed;
  if (tid == 0) {  // TMA producer
    int kt = 0;
    for (; kt < KT; ++kt) {
      const int s = kt % STAGES;
      if (kt >= STAGES && !bar_wait(empty(s), (uint32_t)((kt / STAGES - 1) & 1))) {
        *vfailed = 1;
        break;
      }
      if (*vfailed) break;
      const uint32_t a = base + s * kStageBytes, b = a + kTileBytes;
      bar_expect(full(s), (uint32_t)kStageBytes);
      tma2d(a, &mA, (kt0 + kt) * BK, m0, full(s));
      tma2d(b, &mB, (kt0 + kt) * BK, n0, full(s));
      issued = kt + 1;
    }
  } else if (tid == 32) {  // MMA issuer
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % STAGES;
      if (*vfailed || !bar_wait(full(s), (uint32_t)((kt / STAGES) & 1))) {
        *vfailed = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a = base + s * kStageBytes, b = a + kTileBytes;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)  // 16 bf16 = 32 bytes per K step inside the swizzle atom
        mma_bf16(tmem, sw128_desc(a + 32 * kk), sw128_desc(b + 32 * kk), idesc, (kt | kk) != 0);
      mma_commit(empty(s));
      *vconsumed = kt + 1;
    }
    mma_commit(done);
  }
  __syncthreads();
  if (failed && tid == 0)  // loads issued but never consumed: bounded waits on phases not yet waited for
    for (int k = consumed; k < issued; ++k) bar_wait(full(k % STAGES), (uint32_t)((k / STAGES) & 1));
  const bool fin = bar_wait(done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (failed || !fin) {
    if (tid == 0) atomicExch(g.err, 1);
  } else {
    // epilogue: warp w owns accumulator lanes (rows) 32w .. 32w + 31
    const int row = m0 + warp * 32 + lane;  // < M: M is a multiple of 128
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float x = __uint_as_float(r[j]);
        if (g.bias) x += g.bias[n0 + c0 + j];
        if (g.relu) x = fmaxf(x, 0.f);
        v[j] = x;
      }
      if (g.mask) {
        const __nv_bfloat16* mk = g.mask + (size_t)row * g.ldm + n0 + c0;
#pragma unroll
        for (int j = 0; j < 16; j += 8) {
          const uint4 u = *reinterpret_cast<const uint4*>(mk + j);
          const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (!(__bfloat162float(h[e]) > 0.f)) v[j + e] = 0.f;
        }
      }
      if (g.D) {
        if (g.out_bf16) {
          __nv_bfloat16* d = static_cast<__nv_bfloat16*>(g.D) + (size_t)row * g.ldd + n0 + c0;
#pragma unroll
          for (int j = 0; j < 16; j += 2)
            *reinterpret_cast<__nv_bfloat162*>(d + j) = __floats2bfloat162_rn(v[j], v[j + 1]);
        } else {
          float* d = static_cast<float*>(g.D) + (size_t)blockIdx.z * g.split_stride + (size_t)row * g.ldd + n0 + c0;
#pragma unroll
          for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4*>(d + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
      }
      if (g.Dt) {  // lanes hold consecutive rows: each column is a 64-byte run
#pragma unroll
        for (int j = 0; j < 16; ++j) g.Dt[(size_t)(n0 + c0 + j) * g.lddt + row] = __float2bfloat16_rn(v[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

}  // namespace tc
}  // namespace dcf
