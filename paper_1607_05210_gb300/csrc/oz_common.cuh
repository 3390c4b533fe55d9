// Digit extraction shared by the digit-slice kernels (oz_split.cu, modes_oz.cu):
// x = sign(x) 2^E sum_{t=1..7} d_t 2^(-7t) up to the truncated tail (< 2^(E-49)),
// d_1 in [0, 128], d_2..d_7 in [-64, 63], for |x| < 2^E (Ozaki et al. 2012
// error-free splitting, fixed-point form).
#pragma once

#include <stdint.h>

#include "hapod_internal.cuh"

namespace hapod {

// 64 in each of the six lower base-128 digit positions: adding it makes every lower
// digit non-negative (balanced -> offset digits), the carry lands in d_1.
constexpr uint64_t kOzBalance = 64ull * (1ull + (1ull << 7) + (1ull << 14) + (1ull << 21) + (1ull << 28) + (1ull << 35));

// bf16 bit pattern of the digit v = code - bias (|v| <= 128): the float built from the
// integer code by the 2^23 exponent trick is exact, and so is its upper half.
__device__ __forceinline__ uint32_t digit_bf16(uint32_t code, float bias, uint32_t sign) {
  const float f = __uint_as_float(0x4B000000u | code) - bias;
  return (__float_as_uint(f) >> 16) ^ sign;
}

// The 7 digits of x (bf16 bit patterns in the low halves).
__device__ __forceinline__ void oz_digits(double x, int E, uint32_t (&d)[kOzDigits]) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 63) << 15;
  const int eb = (int)((b >> 52) & 0x7FF);
  uint64_t mant = b & 0x000FFFFFFFFFFFFFull;
  if (eb) mant |= 1ull << 52;
  // |x| = mant 2^(max(eb,1) - 1075); A = floor(|x| 2^(49 - E)) = mant >> sh
  const int sh = E + 1026 - (eb ? eb : 1);
  const uint64_t A = (sh < 64 ? (mant >> sh) : 0ull) + kOzBalance;
  d[0] = digit_bf16((uint32_t)(A >> 42), 8388608.f, sign);
#pragma unroll
  for (int t = 1; t < kOzDigits; ++t)
    d[t] = digit_bf16((uint32_t)(A >> (7 * (6 - t))) & 127u, 8388672.f, sign);  // 2^23 + 64
}

}  // namespace hapod
