// K1, fixed-point mixed form: Gramian G = X^T X (Sec. 2, Remark
// def:method_of_snapshots) of FP32 snapshots on the 5th-generation tensor cores
// (tcgen05, kind::f16, fp16 digit operands) with exact accumulation.
//
// The squared condition number of the Gram matrix (footnote of the method-of-
// snapshots remark) puts the discarded tail sums of a node at 1e-9..1e-10 of its
// trace for eps = 1e-4..1e-5 rel; the tensor core's FP32 accumulator truncates at
// every step, unevenly across entries, which leaves noise of that very size on the
// small eigenvalues.  This form therefore adds nothing inexactly until the very end:
//
// Digits: every column j has the exponent E_j with max_r |x_rj| < 2^E_j over the
// whole node (a one-read pass before the launch, shared with the X V of the node),
// and every value becomes the 32-bit integer A = rint(x 2^(31-E)) written as four
// balanced base-256 digits A = d1 2^24 + d2 2^16 + d3 2^8 + d4, |d_t| <= 128 (round
// to nearest at each step, so the pieces are unbiased).  The representation error is
// at most 2^(E-32): every FP32 value within 2^8 of its column maximum is exact.
// Products: x_i x_j = 2^(E_i+E_j-62) sum_{t,u} d_t d_u 2^(8(8-t-u)); the levels
// s = t + u = 2..6 are kept (thirteen digit pairs; the dropped ones weigh less than
// 2^(E_i+E_j-38.9) per row).  Levels 2..5 are summed on the tensor cores as integers
// over a group of 128 rows, L_s <= 128 * 4 * 2^14 = 2^23, which the FP32 accumulator
// holds exactly; the three level-6 pairs enter the level-5 accumulator through B
// digit planes scaled by 2^-8 (exact in fp16), so L'_5 = L_5 + 2^-8 L_6 carries a
// fraction whose FP32 rounding is below 2^-24 |L'_5| per step.  (Dropping level 6
// instead leaves a random error of 2^(E_i+E_j-33.6) per row, which at n ~ 2^10..2^18
// rows reaches the tail sums of eps = 1e-5 rel.)
// Flush: after each group, v = L_2 2^28 + L_3 2^20 + L_4 2^12 + rint(16 L'_5) (exact,
// |v| < 2^49.1: level 2 is a single pair) is added into an int64 sum per entry whose
// unit is 2^(E_i+E_j-42) -- every group has the same scales, so the sums are plain
// additions; a row split holds at most 2^20 rows, so the sum stays below 2^62.1.  The
// item writes ldexp(sum, E_i + E_j - 42) in FP64 -- one rounding -- and row splits
// are summed in FP64 in a fixed order.  Columns holding Inf or NaN give NaN rows and
// columns of G.
//
// Work item = one 128 x 64 tile (A columns 128 I.., B columns 64 J.., J >= 2 I) of
// one node's G over one row split; items are ordered by split first.  One CTA per
// item, 18 warps:
//   warp 0        TMA producer: FP32 blocks of 32 rows x 128 A columns (and 64 B
//                 columns when they are not inside the A panel), 128-byte swizzled,
//                 6 (A only) or 4 stages deep
//   warp 1        TMEM owner and single-thread MMA issuer: per 16 rows four MMAs,
//                 digit t of A against the B digits 1 .. 5 - t (consecutive planes,
//                 N = 64 (5 - t)) into the adjacent level accumulators L_{t+1} .. L_5,
//                 and three (N = 64) of the A digits 2, 3, 4 against the scaled B
//                 digits 4, 3, 2 into L_5; two accumulator sets (2 x 256 TMEM columns)
//                 alternate between 128-row groups
//   warps 2..9    converters: digits (K-major 8 x 8 core matrices, no swizzle) with
//                 the column scales held in shared memory, 2 stages deep
//   warps 10..17  flushers: int64 sums of 32 entries per thread
// Every mbarrier wait is bounded: a timeout raises the error flag, the CTA drains
// its copies and MMAs and frees TMEM.
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "hapod_internal.cuh"
#include "tc_common.cuh"

namespace hapod {
namespace {

constexpr int kRows = 32;                              // rows per stage (K of two MMAs)
constexpr int kGroupStages = 4;                        // stages per accumulator flush (128 rows)
constexpr int kACols = 128;
constexpr int kBCols = 64;
constexpr int kStA = kRows * kACols * 4;               // FP32 staging of the A panel, 16 KB
constexpr int kStB = kRows * kBCols * 4;               // 8 KB
constexpr int kStSlot = kStA + kStB;
constexpr int kStRegion = 96 * 1024;                   // staging ring: two blocks in flight
constexpr int kStSlotsMax = kStRegion / kStA;          // 6 (B inside A) or kStRegion / kStSlot = 4
constexpr int kPlaneA = kRows * kACols * 2;            // one digit plane of A, 8 KB
constexpr int kPlaneB = kRows * kBCols * 2;            // 4 KB
constexpr int kDigits = 4;
constexpr int kScaled = 3;                             // B digits 2..4 scaled by 2^-8 (level 6 into L_5)
constexpr int kOpSlot = kDigits * (kPlaneA + kPlaneB) + kScaled * kPlaneB;  // 60 KB
constexpr int kOpSlots = 2;
constexpr int kSmemBytes = kStRegion + kOpSlots * kOpSlot + 1024;
constexpr int kThreads = 576;
constexpr int kConvThreads = 256;
constexpr int kFirstFlushWarp = 10;
constexpr uint32_t kLbo = 128;                         // next core matrix along K (8 rows)
constexpr uint32_t kSbo = (kRows / 8) * 128;           // next core matrix along M / N (8 columns)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kSetCols = 256;                     // one set of L2 | L3 | L4 | L5
constexpr int kExpZero = kFxExpZero;                   // exponent of an all-zero column block
constexpr int kExpBad = kFxExpBad;                     // exponent marking Inf / NaN
static_assert(kSmemBytes + 2048 <= 227 * 1024, "shared memory");
constexpr int64_t kMaxSplitRows = (int64_t)1 << 20;   // keeps the int64 sums below 2^62.1

struct Bars {
  uint64_t full[kStSlotsMax];     // TMA -> converters
  uint64_t st_free[kStSlotsMax];  // converters -> TMA
  uint64_t op_full[kOpSlots];     // converters -> issuer
  uint64_t op_free[kOpSlots];     // issuer (MMA completion) -> converters
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t mma_done;
};

struct Shared {
  Bars bars;
  float2 sc[kACols + kBCols];  // scale factors s1 s2 = 2^(31 - E): A columns, then B columns
  int ex[kACols + kBCols];     // column exponents E (kExpZero zero column, kExpBad Inf / NaN)
  uint32_t tmem_base;
  int abort_flag;
};

// Four balanced base-256 digits of rint(x 2^(31 - E)) (as floats holding integers in
// [-128, 128]): each digit is a round to nearest by adding and subtracting 1.5 2^23
// (whose FP32 ulp is 1) after a power-of-two scaling; the remainders are exact.
__device__ __forceinline__ void digits4(float x, float s1, float s2, float (&d)[4]) {
  const float C = 12582912.0f;                        // 1.5 2^23 (ulp 1): (y + C) - C = rint(y), |y| < 2^22
  const float a = (x * s1) * s2;                      // |a| < 2^31, exact (power-of-two scaling)
  d[0] = __fadd_rn(__fmaf_rn(a, 1.0f / 16777216.0f, C), -C);  // rint(a 2^-24), |d1| <= 128
  const float r1 = __fmaf_rn(d[0], -16777216.0f, a);  // |r1| <= 2^23, exact
  d[1] = __fadd_rn(__fmaf_rn(r1, 1.0f / 65536.0f, C), -C);
  const float r2 = __fmaf_rn(d[1], -65536.0f, r1);    // |r2| <= 2^15, exact
  d[2] = __fadd_rn(__fmaf_rn(r2, 1.0f / 256.0f, C), -C);
  const float r3 = __fmaf_rn(d[2], -256.0f, r2);      // |r3| <= 2^7, exact
  d[3] = __fadd_rn(__fadd_rn(r3, C), -C);
}

__device__ __forceinline__ uint32_t h2bits(float lo, float hi) {
  const __half2 v = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Scale factors s1 s2 = 2^(31 - E) (two factors so that both stay in range).
__device__ __forceinline__ void scales(int E, float& s1, float& s2) {
  if (E <= kExpZero || E >= kExpBad) {
    s1 = 0.f;
    s2 = 0.f;
    return;
  }
  const int e = 31 - E;  // in [-97, 180]
  const int e1 = max(-126, min(127, e));
  s1 = ldexpf(1.0f, e1);
  s2 = ldexpf(1.0f, e - e1);
}

// Convert the unit (column c of the staged panel, row octet g) of one stage: 8 values
// from the 128-byte-swizzled staging, four fp16 digit planes out at column dc (B
// planes, planes_are_b, are followed by the three scaled planes of digits 2..4), and
// with `dup` again at column dc2 of the B plane set `planes2` (digits and scaled).
template <bool planes_are_b, bool dup>
__device__ __forceinline__ void convert_unit(const uint8_t* __restrict__ st, int c, uint8_t* __restrict__ planes,
                                             uint32_t plane_bytes, int dc, uint8_t* __restrict__ planes2, int dc2,
                                             int g, float s1, float s2) {
  const float4 v0 = *reinterpret_cast<const float4*>(st + c * 128 + (((2 * g) ^ (c & 7)) << 4));
  const float4 v1 = *reinterpret_cast<const float4*>(st + c * 128 + (((2 * g + 1) ^ (c & 7)) << 4));
  const float x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
  uint32_t w[kDigits][4], ws[kScaled][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float da[kDigits], db[kDigits];
    digits4(x[2 * i], s1, s2, da);
    digits4(x[2 * i + 1], s1, s2, db);
#pragma unroll
    for (int t = 0; t < kDigits; ++t) w[t][i] = h2bits(da[t], db[t]);
    if (planes_are_b || dup) {
#pragma unroll
      for (int t = 0; t < kScaled; ++t)  // d 2^-8, |d| <= 128: exact in fp16
        ws[t][i] = h2bits(da[t + 1] * 0.00390625f, db[t + 1] * 0.00390625f);
    }
  }
  const uint32_t off = (uint32_t)(dc >> 3) * kSbo + (uint32_t)g * kLbo + (uint32_t)(dc & 7) * 16;
#pragma unroll
  for (int t = 0; t < kDigits; ++t)
    *reinterpret_cast<uint4*>(planes + t * plane_bytes + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
  if constexpr (planes_are_b) {
#pragma unroll
    for (int t = 0; t < kScaled; ++t)
      *reinterpret_cast<uint4*>(planes + (kDigits + t) * plane_bytes + off) =
          make_uint4(ws[t][0], ws[t][1], ws[t][2], ws[t][3]);
  }
  if constexpr (dup) {
    const uint32_t off2 = (uint32_t)(dc2 >> 3) * kSbo + (uint32_t)g * kLbo + (uint32_t)(dc2 & 7) * 16;
#pragma unroll
    for (int t = 0; t < kDigits; ++t)
      *reinterpret_cast<uint4*>(planes2 + t * kPlaneB + off2) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
#pragma unroll
    for (int t = 0; t < kScaled; ++t)
      *reinterpret_cast<uint4*>(planes2 + (kDigits + t) * kPlaneB + off2) =
          make_uint4(ws[t][0], ws[t][1], ws[t][2], ws[t][3]);
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    gram_fx3_kernel(const GramJob* __restrict__ jobs, const CUtensorMap* __restrict__ maps,
                    const int4* __restrict__ items, double* __restrict__ partials, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ Shared sh;
  Bars& bars = sh.bars;
  volatile int* abort_flag = &sh.abort_flag;

  const int4 it = items[blockIdx.x];
  const GramJob J = jobs[it.x];
  const CUtensorMap* mapA = maps + 2 * it.x;
  const CUtensorMap* mapB = maps + 2 * it.x + 1;
  const int I = it.y, Jt = it.z, sp = it.w;
  const int a0 = kACols * I, b0 = kBCols * Jt;
  const bool b_in_a = b0 >= a0 && b0 < a0 + kACols;  // B columns inside the A panel
  const int64_t r0 = (int64_t)sp * J.rows_per_split;
  const int64_t r1 = min(J.n, r0 + J.rows_per_split);
  const int nst = r1 > r0 ? (int)((r1 - r0 + kRows - 1) / kRows) : 0;
  const int ngroups = (nst + kGroupStages - 1) / kGroupStages;
  // a tile whose B columns lie inside its A panel stages only the A panel (16 KB per
  // stage, 6 slots); otherwise A and B (24 KB per stage, 4 slots).
  const int kStSlots = b_in_a ? kStRegion / kStA : kStRegion / kStSlot;
  const int st_bytes = b_in_a ? kStA : kStSlot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const tc::WaitBudget wb = tc::wait_budget(err);
  auto st_a = [&](int s) -> uint8_t* { return smem + (size_t)s * st_bytes; };
  auto st_b = [&](int s) -> uint8_t* { return smem + (size_t)s * st_bytes + kStA; };
  uint8_t* op_ring = smem + (size_t)kStRegion;
  auto op_a = [&](int t) -> uint8_t* { return op_ring + (size_t)t * kOpSlot; };
  auto op_b = [&](int t) -> uint8_t* { return op_ring + (size_t)t * kOpSlot + kDigits * kPlaneA; };

  if (tid == 0) {
    for (int s = 0; s < kStSlotsMax; ++s) {
      tc::mbar_init(&bars.full[s], 1);
      tc::mbar_init(&bars.st_free[s], 8);
    }
    for (int t = 0; t < kOpSlots; ++t) {
      tc::mbar_init(&bars.op_full[t], 8);
      tc::mbar_init(&bars.op_free[t], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bars.acc_full[b], 1);
      tc::mbar_init(&bars.acc_empty[b], 8);
    }
    tc::mbar_init(&bars.mma_done, 1);
    sh.abort_flag = 0;
    tc::mbar_fence_init();
  }
  // column exponents of the node (computed before the launch) and the scale factors
  for (int i = tid; i < kACols + kBCols; i += blockDim.x) {
    const int col = i < kACols ? a0 + i : b0 + (i - kACols);
    const int E = col < J.m ? J.col_exp[col] : kExpZero;
    float s1, s2;
    scales(E, s1, s2);
    sh.ex[i] = E;
    sh.sc[i] = make_float2(s1, s2);
  }
  if (warp == 1) tc::tmem_alloc(&sh.tmem_base, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = sh.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0 && nst > 0) {
      tc::tensormap_acquire(mapA);
      if (!b_in_a) tc::tensormap_acquire(mapB);
      const uint32_t bytes = (uint32_t)(kStA + (b_in_a ? 0 : kStB));
      int issued = 0;
      for (int k = 0; k < nst; ++k) {
        const int s = k % kStSlots;
        if (k >= kStSlots && !tc::mbar_wait(&bars.st_free[s], ((k / kStSlots) - 1) & 1, abort_flag, err, wb)) break;
        tc::mbar_expect_tx(&bars.full[s], bytes);
        const int row = (int)(r0 + (int64_t)k * kRows);
        tc::tma_load_2d(st_a(s), mapA, row, a0, &bars.full[s]);
        if (!b_in_a) tc::tma_load_2d(st_b(s), mapB, row, b0, &bars.full[s]);
        issued = k + 1;
      }
      if (*abort_flag) {
        for (int k = max(0, issued - kStSlots); k < issued; ++k) {
          const long long t0 = clock64();
          while (!tc::mbar_try(&bars.full[k % kStSlots], (k / kStSlots) & 1) && clock64() - t0 < tc::kWaitBudget) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t idn[kDigits];
#pragma unroll
      for (int t = 0; t < kDigits; ++t) idn[t] = tc::idesc_f16_f32_major(128, (uint32_t)(kBCols * (kDigits - t)), 0, 0);
      for (int k = 0; k < nst; ++k) {
        const int t = k % kOpSlots;
        const int grp = k / kGroupStages;
        const bool grp_first = (k % kGroupStages) == 0;
        const bool grp_last = (k % kGroupStages) == kGroupStages - 1 || k == nst - 1;
        const int set = grp & 1;
        if (grp_first && grp >= 2 &&
            !tc::mbar_wait(&bars.acc_empty[set], ((grp >> 1) - 1) & 1, abort_flag, err, wb))
          break;
        if (!tc::mbar_wait(&bars.op_full[t], (k / kOpSlots) & 1, abort_flag, err, wb)) break;
        tc::tc_fence_after();
        const uint32_t pa = tc::smem_u32(op_a(t)), pb = tc::smem_u32(op_b(t));
        const uint32_t d = tbase + (uint32_t)set * kSetCols;
#pragma unroll
        for (int kk = 0; kk < kRows / 16; ++kk) {
          const uint32_t ko = (uint32_t)kk * 2 * kLbo;
          // digit t of A against the B digits 1 .. 4 - t (consecutive planes, one
          // operand of N = 64 (4 - t)) into the level accumulators L_{t+1} .. L_5
#pragma unroll
          for (int tt = 0; tt < kDigits; ++tt)
            tc::umma_f16(d + (uint32_t)(kBCols * tt), tc::ns_desc(pa + (uint32_t)tt * kPlaneA + ko, kLbo, kSbo),
                         tc::ns_desc(pb + ko, kLbo, kSbo), idn[tt], (grp_first && kk == 0 && tt == 0) ? 0u : 1u);
          // level 6 into L_5: A digit 2, 3, 4 against the scaled B digit 4, 3, 2
#pragma unroll
          for (int tt = 1; tt < kDigits; ++tt)
            tc::umma_f16(d + (uint32_t)(kBCols * (kDigits - 1)),
                         tc::ns_desc(pa + (uint32_t)tt * kPlaneA + ko, kLbo, kSbo),
                         tc::ns_desc(pb + (uint32_t)(kDigits + kDigits - 1 - tt) * kPlaneB + ko, kLbo, kSbo),
                         idn[kDigits - 1], 1u);
        }
        tc::umma_commit(&bars.op_free[t]);
        if (grp_last) tc::umma_commit(&bars.acc_full[set]);
      }
      tc::umma_commit(&bars.mma_done);
      const long long t0 = clock64();
      while (!tc::mbar_try(&bars.mma_done, 0) && clock64() - t0 < tc::kWaitBudget) {
      }
    }
  } else if (warp < kFirstFlushWarp) {
    // ------------------------------------------------------------ converters
    const int ct = tid - 64;  // 0..255
    bool ok = true;
    for (int k = 0; k < nst && ok; ++k) {
      const int s = k % kStSlots, t = k % kOpSlots;
      ok = tc::mbar_wait_warp(&bars.full[s], (k / kStSlots) & 1, abort_flag, err, wb);
      if (ok && k >= kOpSlots) ok = tc::mbar_wait_warp(&bars.op_free[t], ((k / kOpSlots) - 1) & 1, abort_flag, err, wb);
      if (!ok) break;
      // A panel: 128 columns x 4 octets = 512 units, two per thread
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int u = ct + h * kConvThreads;
        const int c = u & (kACols - 1), g = u >> 7;
        const float2 sc = sh.sc[c];
        const bool dup = b_in_a && c >= b0 - a0 && c < b0 - a0 + kBCols;  // also a B column
        if (dup)
          convert_unit<false, true>(st_a(s), c, op_a(t), kPlaneA, c, op_b(t), c - (b0 - a0), g, sc.x, sc.y);
        else
          convert_unit<false, false>(st_a(s), c, op_a(t), kPlaneA, c, nullptr, 0, g, sc.x, sc.y);
      }
      if (!b_in_a) {  // B panel: 64 columns x 4 octets = 256 units, one per thread
        const int c = ct & (kBCols - 1), g = ct >> 6;
        const float2 sc = sh.sc[kACols + c];
        convert_unit<true, false>(st_b(s), c, op_b(t), kPlaneB, c, nullptr, 0, g, sc.x, sc.y);
      }
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&bars.st_free[s]);
        tc::mbar_arrive(&bars.op_full[t]);
      }
    }
  } else {
    // ------------------------------------------------------------ flushers + result
    const int fw = warp - kFirstFlushWarp;  // 0..7
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int h = fw >> 2;                  // column half: B columns 32 h .. 32 h + 31
    const int ai = 32 * q + lane;           // tile row (A column)
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    // rows a0 + 32 q .. of a tile whose B columns are inside its A panel may all lie
    // below the diagonal of G for this warp's columns: nothing of theirs is kept
    const bool below_diag = a0 + 32 * q > b0 + 32 * h + 31;
    long long acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0;
    bool ok = true;
    for (int grp = 0; grp < ngroups && ok; ++grp) {
      const int set = grp & 1;
      ok = tc::mbar_wait_warp(&bars.acc_full[set], (grp >> 1) & 1, abort_flag, err, wb);
      if (!ok) break;
      tc::tc_fence_after();
      if (!below_diag) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {  // 8 columns at a time
          const uint32_t col = (uint32_t)set * kSetCols + (uint32_t)(32 * h + 8 * g);
          uint32_t l2[8], l3[8], l4[8], l5[8];
          tc::tmem_ld8_raw(tbase + lanes + col, l2);
          tc::tmem_ld8_raw(tbase + lanes + col + kBCols, l3);
          tc::tmem_ld8_raw(tbase + lanes + col + 2 * kBCols, l4);
          tc::tmem_ld8_raw(tbase + lanes + col + 3 * kBCols, l5);
          tc::tmem_wait_ld();
          tc::reg_barrier8(l2);
          tc::reg_barrier8(l3);
          tc::reg_barrier8(l4);
          tc::reg_barrier8(l5);
#pragma unroll
          for (int i = 0; i < 8; ++i)  // every group carries the same column scales: plain sums
            acc[8 * g + i] += (long long)__float2int_rn(__uint_as_float(l2[i])) * 268435456LL +
                              (long long)__float2int_rn(__uint_as_float(l3[i])) * 1048576LL +
                              (long long)__float2int_rn(__uint_as_float(l4[i])) * 4096LL +
                              (long long)__float2int_rn(__uint_as_float(l5[i]) * 16.0f);
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars.acc_empty[set]);
    }
    if (__all_sync(0xffffffffu, ok && !*abort_flag) && !below_diag) {
      const int gi = a0 + ai;
      const int Ei = sh.ex[ai];
      const int jmax = (J.m + kBCols - 1) / kBCols;
      const int tile_idx = I * jmax - I * (I - 1) + (Jt - 2 * I);
      double* out = J.splits > 1 ? partials + ((size_t)J.item_base + (size_t)tile_idx * J.splits + sp) *
                                                  (size_t)(kACols * kBCols)
                                 : nullptr;
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const int bj = 32 * h + jj;  // column within the B panel
        const int gj = b0 + bj;
        const int Ej = b_in_a ? sh.ex[gj - a0] : sh.ex[kACols + bj];
        double v;
        if (Ei >= kExpBad || Ej >= kExpBad)
          v = __longlong_as_double(0x7FF8000000000000LL);
        else if (Ei <= kExpZero || Ej <= kExpZero)
          v = 0.0;
        else
          v = ldexp((double)acc[jj], Ei + Ej - 42);
        if (out) {
          out[(size_t)ai * kBCols + bj] = v;
        } else if (gi < J.m && gj < J.m && gj >= gi) {
          J.G[(size_t)gj * J.m + gi] = v;
          J.G[(size_t)gi * J.m + gj] = v;
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, kTmemCols);
}

// Sum the split partials of every reduce-list tile (job, I, J, first) in split order;
// entries i <= j of G and their mirror images.
__global__ void gram_fx3_reduce(const GramJob* __restrict__ jobs, const int4* __restrict__ reduce,
                                const double* __restrict__ partials) {
  const int4 r = reduce[blockIdx.y];
  const GramJob J = jobs[r.x];
  const int I = r.y, Jt = r.z;
  const int jmax = (J.m + kBCols - 1) / kBCols;
  const int tile_idx = I * jmax - I * (I - 1) + (Jt - 2 * I);
  const double* p = partials + ((size_t)J.item_base + (size_t)tile_idx * J.splits) * (size_t)(kACols * kBCols);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kACols * kBCols; e += gridDim.x * blockDim.x) {
    const int gi = kACols * I + e / kBCols, gj = kBCols * Jt + e % kBCols;
    if (gi >= J.m || gj >= J.m || gj < gi) continue;
    double s = 0.0;
    for (int sp = 0; sp < J.splits; ++sp) s += p[(size_t)sp * (kACols * kBCols) + e];
    J.G[(size_t)gj * J.m + gi] = s;
    J.G[(size_t)gi * J.m + gj] = s;
  }
}

}  // namespace

int gram_fx3_rows_per_stage() { return kRows; }
int gram_fx3_a_cols() { return kACols; }
int gram_fx3_b_cols() { return kBCols; }

void plan_gram_fx3(GramJob* jobs, int njobs, int target_items, std::vector<int4>& items, std::vector<int4>& reduce,
                   size_t* partial_bytes, int split_pct) {
  // tiles (I, J), J >= 2 I, of every job; one split count for the batch chosen as in
  // plan_gram: the fewest waves of `target_items` CTAs per unit of work
  int64_t total_tiles = 0, max_n = 1;
  for (int j = 0; j < njobs; ++j) {
    const int64_t imax = (jobs[j].m + kACols - 1) / kACols, jmax = (jobs[j].m + kBCols - 1) / kBCols;
    int64_t t = 0;
    for (int64_t I = 0; I < imax; ++I) t += std::max<int64_t>(0, jmax - 2 * I);
    jobs[j].tiles = (int32_t)t;
    total_tiles += t;
    max_n = std::max<int64_t>(max_n, jobs[j].n);
  }
  const int64_t min_rows = 4096;
  const int64_t s_cap = std::max<int64_t>(
      1, std::min<int64_t>(max_n / min_rows, total_tiles > 0 ? 8 * (int64_t)target_items / total_tiles + 1 : 1));
  int64_t splits = 1;
  double best = 1e300;
  for (int64_t s = 1; s <= s_cap && total_tiles > 0; ++s) {
    const double waves = (double)((total_tiles * s + target_items - 1) / target_items);
    if (waves / (double)s < best * (1.0 - 1e-9)) {
      best = waves / (double)s;
      splits = s;
    }
  }
  // an autotuned factor on the split count (hapod_autotune), 100 = the rule above
  if (split_pct != 100) splits = std::max<int64_t>(1, splits * split_pct / 100);
  int64_t slot = 0;
  items.clear();
  reduce.clear();
  for (int j = 0; j < njobs; ++j) {
    GramJob& J = jobs[j];
    int64_t s = std::max<int64_t>(1, std::min(splits, std::max<int64_t>(1, J.n / min_rows)));
    s = std::max<int64_t>(s, (J.n + kMaxSplitRows - 1) / kMaxSplitRows);
    int64_t rps = (J.n + s - 1) / s;
    rps = (rps + 63) / 64 * 64;  // whole 64-row exponent blocks
    s = std::max<int64_t>(1, (J.n + rps - 1) / rps);
    J.splits = (int32_t)s;
    J.rows_per_split = rps;
    J.item_base = slot;
    const int imax = (J.m + kACols - 1) / kACols, jmax = (J.m + kBCols - 1) / kBCols;
    for (int I = 0; I < imax; ++I)
      for (int Jt = 2 * I; Jt < jmax; ++Jt) {
        if (s > 1) reduce.push_back(make_int4(j, I, Jt, 0));
        for (int sp = 0; sp < s; ++sp) items.push_back(make_int4(j, I, Jt, sp));
      }
    slot += (int64_t)J.tiles * s;
  }
  std::stable_sort(items.begin(), items.end(), [](const int4& a, const int4& b) { return a.w < b.w; });
  *partial_bytes = reduce.empty() ? 0 : (size_t)slot * kACols * kBCols * sizeof(double);
}

cudaError_t launch_gram_fx3(const GramJob* jobs_dev, const CUtensorMap* maps_dev, const int4* items_dev,
                            int num_items, const int4* reduce_dev, int num_reduce, double* partials, int* err_flag,
                            cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gram_fx3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (num_items > 0)
    gram_fx3_kernel<<<num_items, kThreads, kSmemBytes, s>>>(jobs_dev, maps_dev, items_dev, partials, err_flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || num_reduce <= 0) return e;
  gram_fx3_reduce<<<dim3(8, num_reduce), 256, 0, s>>>(jobs_dev, reduce_dev, partials);
  return cudaGetLastError();
}

}  // namespace hapod
