// Digit extraction shared by the digit-slice kernels (oz_split.cu, gram_oz.cu,
// modes_oz.cu): for |x| < 2^E,
//   A = floor(|x| 2^(55 - E)) < 2^55 = d_1 2^48 + d_2 2^40 + ... + d_7   (balanced base 256)
//   d_1 in [0, 128], d_2..d_7 in [-128, 127],
// so x = sign(x) 2^(E+1) sum_{t=1..7} d_t 2^(-8t) up to the truncated tail (< 2^(E-55)):
// the error-free splitting of Ozaki, Ogita, Oishi and Rump (2012) in fixed-point form.
// Every digit is an integer of magnitude <= 128, exact in bf16, and every product of
// two digits is at most 2^14 in magnitude.
#pragma once

#include <stdint.h>

#include "hapod_internal.cuh"

namespace hapod {

// 128 in each of the six lower base-256 digit positions: adding it turns the
// balanced digits into bytes (offset digits); the carry lands in d_1.
constexpr uint32_t kOzBalanceLo = 0x80808080u;  // positions 0..3
constexpr uint32_t kOzBalanceHi = 0x8080u;      // positions 4..5

// A + balance as (hi, lo) 32-bit words for |x| < 2^E.
__device__ __forceinline__ void oz_fixed(double x, int E, uint32_t& ahi, uint32_t& alo) {
  const uint32_t h = (uint32_t)(__double_as_longlong(x) >> 32);
  const uint32_t l = (uint32_t)__double_as_longlong(x);
  const int eb = (int)((h >> 20) & 0x7FF);
  const uint32_t mh = (h & 0xFFFFFu) | (eb ? 0x100000u : 0u);  // mantissa = mh:l (53 bits)
  // |x| = mantissa 2^(max(eb,1) - 1075); A = mantissa >> sh (a left shift for sh < 0; sh >= -2)
  const int sh = E + 1020 - (eb ? eb : 1);
  uint32_t hi, lo;
  if (sh < 0) {
    hi = __funnelshift_l(l, mh, -sh);
    lo = l << -sh;
  } else if (sh < 32) {
    lo = __funnelshift_r(l, mh, sh);
    hi = mh >> sh;
  } else {
    lo = sh < 64 ? (mh >> (sh - 32)) : 0u;
    hi = 0u;
  }
  // + balance (64-bit add)
  alo = lo + kOzBalanceLo;
  ahi = hi + kOzBalanceHi + (alo < lo ? 1u : 0u);
}

// Float bit patterns of the 7 digits of x (bf16 pattern = upper half), sign applied
// by the caller.  The float built from a digit code c by the 2^23 exponent trick,
// minus the bias, is exact.
__device__ __forceinline__ void oz_digit_floats(uint32_t ahi, uint32_t alo, uint32_t (&f)[kOzDigits]) {
  f[0] = __float_as_uint(__uint_as_float(0x4B000000u | (ahi >> 16)) - 8388608.f);
  f[1] = __float_as_uint(__uint_as_float(__byte_perm(ahi, 0x4B000000u, 0x7441)) - 8388736.f);  // 2^23 + 128
  f[2] = __float_as_uint(__uint_as_float(__byte_perm(ahi, 0x4B000000u, 0x7440)) - 8388736.f);
  f[3] = __float_as_uint(__uint_as_float(__byte_perm(alo, 0x4B000000u, 0x7443)) - 8388736.f);
  f[4] = __float_as_uint(__uint_as_float(__byte_perm(alo, 0x4B000000u, 0x7442)) - 8388736.f);
  f[5] = __float_as_uint(__uint_as_float(__byte_perm(alo, 0x4B000000u, 0x7441)) - 8388736.f);
  f[6] = __float_as_uint(__uint_as_float(__byte_perm(alo, 0x4B000000u, 0x7440)) - 8388736.f);
}

// The 7 digits of x as bf16 bit patterns in the low halves.
__device__ __forceinline__ void oz_digits(double x, int E, uint32_t (&d)[kOzDigits]) {
  uint32_t ahi, alo, f[kOzDigits];
  oz_fixed(x, E, ahi, alo);
  oz_digit_floats(ahi, alo, f);
  const uint32_t sign = (uint32_t)((uint64_t)__double_as_longlong(x) >> 63) << 15;
#pragma unroll
  for (int t = 0; t < kOzDigits; ++t) d[t] = (f[t] >> 16) ^ sign;
}

// The 7 digits of two values of one column (same E), packed bf16x2 per digit plane:
// x0 in the low half, x1 in the high half.
__device__ __forceinline__ void oz_digits2(double x0, double x1, int E, uint32_t (&w)[kOzDigits]) {
  uint32_t h0, l0, h1, l1, f0[kOzDigits], f1[kOzDigits];
  oz_fixed(x0, E, h0, l0);
  oz_fixed(x1, E, h1, l1);
  oz_digit_floats(h0, l0, f0);
  oz_digit_floats(h1, l1, f1);
  const uint32_t smask = (((uint32_t)((uint64_t)__double_as_longlong(x0) >> 63)) << 15) |
                         (((uint32_t)((uint64_t)__double_as_longlong(x1) >> 63)) << 31);
#pragma unroll
  for (int t = 0; t < kOzDigits; ++t) w[t] = __byte_perm(f0[t], f1[t], 0x7632) ^ smask;
}

// Exact level sums of one flush, combined into the two int64 fixed-point sums
// (units 2^-32 and 2^-64 of 2^(E_i + E_j + 2)): level s = lv + 2 carries 2^(-8 s).
//   hi += L_2 2^16 + L_3 2^8 + L_4,   lo += L_5 2^24 + L_6 2^16 + L_7 2^8 + L_8.
__device__ __forceinline__ long long oz_level_weight(int lv) {
  return lv < 3 ? (1ll << (8 * (2 - lv))) : (1ll << (8 * (6 - lv)));
}

// value = 2^(shift) (hi 2^32 + lo), rounded once to FP64
__device__ __forceinline__ double oz_combine(long long hi, long long lo, int shift) {
  return scalbn((double)hi * 4294967296.0 + (double)lo, shift);
}

}  // namespace hapod
