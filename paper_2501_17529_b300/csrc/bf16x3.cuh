// Split of an FP32 value into two BF16 parts for the three-product (BF16x3)
// tensor-core contractions: x = hi + lo with hi = bf16(x) and lo = bf16(x - hi),
// so that |x - hi - lo| <= 2^-16 |x| and a product x y is carried by
// hi_x hi_y + hi_x lo_y + lo_x hi_y up to about 2^-16 of |x y|.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace dcf {

// (x0, x1) -> packed BF16 pairs (x0 in the low half, the MMA operand order)
__device__ __forceinline__ void bf16_split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// depth of the BF16 Z rows for a rank class (the MMA K: 8 or 16)
template <int RMAX>
struct TcK {
  static constexpr int KB = RMAX <= 8 ? 8 : 16;
};

}  // namespace dcf
