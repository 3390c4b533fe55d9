// Digit extraction shared by the digit-slice kernels (oz_split.cu, gram_oz.cu,
// modes_oz.cu): for |x| < 2^E,
//   A = floor(|x| 2^(55 - E)) < 2^55 = d_1 2^48 + d_2 2^40 + ... + d_7   (balanced base 256)
//   d_1 in [0, 128], d_2..d_7 in [-128, 127],
// so x = sign(x) 2^(E+1) sum_{t=1..7} d_t 2^(-8t) up to the truncated tail (< 2^(E-55)):
// the error-free splitting of Ozaki, Ogita, Oishi and Rump (2012) in fixed-point form.
// Every digit is an integer of magnitude <= 128, exact in fp16, and every product of
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
  // (branch-free: the elements of one warp take different shifts)
  const int sh = E + 1020 - (eb ? eb : 1);
  const uint64_t mant = ((uint64_t)mh << 32) | l;
  const uint64_t left = mant << (sh < 0 ? -sh : 0);
  const uint64_t A = sh < 0 ? left : (sh < 64 ? (mant >> (sh & 63)) : 0ull);
  const uint64_t Ab = A + (((uint64_t)kOzBalanceHi << 32) | kOzBalanceLo);
  ahi = (uint32_t)(Ab >> 32);
  alo = (uint32_t)Ab;
}

// Digit codes (bytes of A + balance): code t of plane t sits in byte kOzByte[t] of
// (t == 0 ? ahi : t < 3 ? ahi : alo); the value is code - 128 (code for the top digit).
// fp16 patterns of two digits of one plane, two elements at once: the bytes are placed
// under the exponent pattern 0x64 (1024 + code, exact in fp16) and one signed fused
// multiply-add gives sign * (code - bias), exact.
__device__ __forceinline__ uint32_t oz_pair(uint32_t a, uint32_t b, uint32_t sel, uint32_t sgn2, uint32_t nb2) {
  const uint32_t t = (__byte_perm(a, b, sel) & 0x00FF00FFu) | 0x64006400u;
  uint32_t r;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(t), "r"(sgn2), "r"(nb2));
  return r;
}

// The 7 digit planes of two values of one column (same E), packed f16x2 per plane:
// x0 in the low half, x1 in the high half.
__device__ __forceinline__ void oz_digits2(double x0, double x1, int E, uint32_t (&w)[kOzDigits]) {
  uint32_t h0, l0, h1, l1;
  oz_fixed(x0, E, h0, l0);
  oz_fixed(x1, E, h1, l1);
  // +-1 per half, and -bias * sign for the top digit (1024) and the others (1152)
  const uint32_t sgn2 = 0x3C003C00u | ((uint32_t)((uint64_t)__double_as_longlong(x0) >> 63) << 15) |
                        ((uint32_t)((uint64_t)__double_as_longlong(x1) >> 63) << 31);
  uint32_t nb_top, nb_low;
  asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(nb_top) : "r"(sgn2), "r"(0xE400E400u));  // -1024
  asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(nb_low) : "r"(sgn2), "r"(0xE480E480u));  // -1152
  w[0] = oz_pair(h0, h1, 0x6622u, sgn2, nb_top);
  w[1] = oz_pair(h0, h1, 0x5511u, sgn2, nb_low);
  w[2] = oz_pair(h0, h1, 0x4400u, sgn2, nb_low);
  w[3] = oz_pair(l0, l1, 0x7733u, sgn2, nb_low);
  w[4] = oz_pair(l0, l1, 0x6622u, sgn2, nb_low);
  w[5] = oz_pair(l0, l1, 0x5511u, sgn2, nb_low);
  w[6] = oz_pair(l0, l1, 0x4400u, sgn2, nb_low);
}

// The 7 digits of x as fp16 bit patterns in the low halves.
__device__ __forceinline__ void oz_digits(double x, int E, uint32_t (&d)[kOzDigits]) {
  uint32_t w[kOzDigits];
  oz_digits2(x, 0.0, E, w);
#pragma unroll
  for (int t = 0; t < kOzDigits; ++t) d[t] = w[t] & 0xFFFFu;
}

// Exact level sums of one flush, combined into the two int64 fixed-point sums
// (units 2^-32 and 2^-64 of 2^(E_i + E_j + 2)): level s = lv + 2 carries 2^(-8 s).
//   hi += L_2 2^16 + L_3 2^8 + L_4,   lo += L_5 2^24 + L_6 2^16 + L_7 2^8 + L_8.
__device__ __forceinline__ long long oz_level_weight(int lv) {
  return lv < 3 ? (1ll << (8 * (2 - lv))) : (1ll << (8 * (6 - lv)));
}

// value = 2^(shift) (hi 2^32 + lo), rounded once to FP64 (to nearest, ties to even),
// with integer arithmetic: the FP64 pipe of this part is a small fraction of its
// integer rate.  Results outside the normal range take the FP64 route.
__device__ __forceinline__ double oz_combine(long long hi, long long lo, int shift) {
  // T = hi 2^32 + lo as a signed 128-bit integer
  const __int128 T = ((__int128)hi << 32) + (__int128)lo;
  if (T == 0) return 0.0;
  const bool neg = T < 0;
  const unsigned __int128 M = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
  const uint64_t mh = (uint64_t)(M >> 64), ml = (uint64_t)M;
  const int z = mh ? __clzll((long long)mh) : 64 + __clzll((long long)ml);  // leading zeros of M
  const unsigned __int128 N = M << z;                                       // top bit at 127
  const uint64_t w = (uint64_t)(N >> 64), rest = (uint64_t)N;
  uint64_t mant = w >> 11;  // 53 bits, leading one at bit 52
  const uint64_t half = (w >> 10) & 1u;
  const bool sticky = (w & 0x3FFu) != 0 || rest != 0;
  int be = (127 - z) + shift + 1023;  // biased exponent of the leading bit
  mant += half & ((sticky ? 1u : 0u) | (mant & 1u));
  if (mant >> 53) {
    mant >>= 1;
    ++be;
  }
  if (be < 1 || be > 2046) {
    const double v = (double)hi * 4294967296.0 + (double)lo;
    return scalbn(v, shift);
  }
  const uint64_t bits = ((uint64_t)neg << 63) | ((uint64_t)be << 52) | (mant & 0x000FFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

}  // namespace hapod
