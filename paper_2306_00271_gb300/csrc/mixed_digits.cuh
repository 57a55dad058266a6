// Fixed-point digit arithmetic shared by the mixed-precision kernels (integrate_mixed.cu for
// N <= 64, integrate_mixed_wide.cu for 64 < N <= 128): error-free float transformations for the
// double-float state, power-of-two scales, and the four signed 8-bit digits whose products the
// tensor cores accumulate without rounding.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace trh {
namespace mixed {

constexpr int NDIG = 4;                          // fixed-point digits per operand
constexpr long long kWaitCycles = 4000000000LL;  // bounded waits: about 2 s at 2 GHz
constexpr float kMagic = 12582912.0f;            // 1.5 * 2^23: x + M - M rounds x to an integer

// Error-free transformations. The explicit _rn intrinsics are never contracted into FMAs: a
// contraction would make the rounded sum differ from the one the error term assumes.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ float rint_magic(float x) {  // |x| < 2^22, round to nearest even
  return __fsub_rn(__fadd_rn(x, kMagic), kMagic);
}

// Smallest power of two >= x (x > 0 finite); 1 for x == 0.
__device__ __forceinline__ float pow2_ceil(float x) {
  if (!(x > 0.0f)) return 1.0f;
  const uint32_t b = __float_as_uint(x);
  uint32_t e = b & 0x7F800000u;
  if (b & 0x007FFFFFu) e += 0x00800000u;
  return __uint_as_float(e);
}
// 1 / g for a normal power of two g, from its exponent bits.
__device__ __forceinline__ float pow2_inv(float g) {
  return __uint_as_float((254u << 23) - (__float_as_uint(g) & 0x7F800000u));
}

// Fixed-point digits of v = x / scale (|v| <= 1): BF16 bit patterns of d0..d3. The remainders
// are exact in FP32 (power-of-two scalings and differences of nearby values).
__device__ __forceinline__ void digits4(float x, float inv_scale, uint16_t (&b)[NDIG]) {
  float v = __fmul_rn(__fmul_rn(x, inv_scale), 128.0f);
#pragma unroll
  for (int i = 0; i < NDIG; ++i) {
    const float d = rint_magic(v);
    // integers of magnitude <= 256 have zero low halves: the BF16 pattern is the top 16 bits
    b[i] = (uint16_t)(__float_as_uint(d) >> 16);
    v = __fmul_rn(__fsub_rn(v, d), 256.0f);
  }
}

}  // namespace mixed
}  // namespace trh
