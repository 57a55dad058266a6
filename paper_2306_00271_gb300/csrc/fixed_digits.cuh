// Fixed-point digits of binary64 operands by integer arithmetic, for tensor-core products whose
// inputs arrive in binary64 (the reverse sweep's contraction): no binary64 instruction is needed
// to scale, round or cut an entry, only its bit pattern.
//
// For a row (or column) whose largest |entry| is at most 2^E, an entry x becomes the integer
//   V = round(x 2^(31 - E)),  |V| <= 2^31,  |x 2^-E - V 2^-31| <= 2^-32,
// written in balanced base 256 as V = d0 2^24 + d1 2^16 + d2 2^8 + d3 with |d_i| <= 128, so that
//   x ~ 2^E (d0 + d1 / 2^8 + d2 / 2^16 + d3 / 2^24) / 2^7,
// the four-digit format of mixed_digits.cuh: every digit is exact in BF16, every digit product is
// an integer below 2^14 in magnitude, and the products of one order summed over K <= 128 stay
// below 2^24. Host and device compile the same code (the host form serves the CPU tests).
#pragma once
#include <climits>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace trh {
namespace fixed {

__host__ __device__ __forceinline__ unsigned long long bits_of(double x) {
#if defined(__CUDA_ARCH__)
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, sizeof(b));
  return b;
#endif
}

__host__ __device__ __forceinline__ float float_of_bits(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float f;
  std::memcpy(&f, &b, sizeof(f));
  return f;
#endif
}

__host__ __device__ __forceinline__ uint32_t bits_of_float(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  uint32_t b;
  std::memcpy(&b, &f, sizeof(b));
  return b;
#endif
}

// Exponent of the smallest power of two >= |x|; INT_MIN for x = 0 (subnormals, far below every
// scale in use, count as 2^-1022).
__host__ __device__ __forceinline__ int ceil_exp(double x) {
  const unsigned long long b = bits_of(x) & 0x7FFFFFFFFFFFFFFFull;
  if (b == 0) return INT_MIN;
  const int ex = (int)(b >> 52);
  if (ex == 0) return -1022;
  return ex - 1023 + ((b & 0xFFFFFFFFFFFFFull) != 0 ? 1 : 0);
}

// 2^e as an FP32 value, -126 <= e <= 127.
__host__ __device__ __forceinline__ float pow2f(int e) {
  return float_of_bits((uint32_t)(e + 127) << 23);
}

// V = x 2^(31 - E) rounded to the nearest integer (ties away from zero); requires |x| <= 2^E.
// Subnormal x gives 0.
__host__ __device__ __forceinline__ long long fixed31(double x, int E) {
  const unsigned long long b = bits_of(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;
  const long long mant = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));  // x = mant 2^(ex-1075)
  const int k = 1044 + E - ex;  // x 2^(31-E) = mant 2^-k, and |x| <= 2^E gives k >= 21
  const long long v = (k >= 60) ? 0 : (((mant >> (k - 1)) + 1) >> 1);
  return (b >> 63) ? -v : v;
}

// BF16 bit pattern of an integer |d| <= 256 (exact): 1.5 * 2^23 + d as an FP32 bit pattern,
// minus 1.5 * 2^23.
__host__ __device__ __forceinline__ uint16_t bf16_of_int(int d) {
  const float f = float_of_bits(0x4B400000u + (uint32_t)d) - 12582912.0f;
  return (uint16_t)(bits_of_float(f) >> 16);
}

// Balanced base-256 digits of V (|V| <= 2^31) as BF16 bit patterns: b[0] the leading digit.
__host__ __device__ __forceinline__ void digits_of(long long V, uint16_t (&b)[4]) {
#pragma unroll
  for (int i = 3; i >= 1; --i) {
    const int r = (int)((V + 128) & 255) - 128;
    b[i] = bf16_of_int(r);
    V = (V - r) >> 8;
  }
  b[0] = bf16_of_int((int)V);
}

}  // namespace fixed
}  // namespace trh
