// K4, fixed-point mixed form: Y = X V_k diag(scale) (Sec. 2, Remark
// def:method_of_snapshots: sigma_k phi_k = X psi_k, or phi_k with scale = 1/sigma)
// of FP32 snapshots on the 5th-generation tensor cores (tcgen05, kind::f16, fp16
// digit operands) with exact accumulation.
//
// With E_j the exponent of column j's largest |x| (2^(E_j-1) <= max < 2^E_j, recorded
// by the Gram kernel) and F_c that of max_j 2^E_j |V_jc|, every x_rj is the integer
// A_rj = rint(x_rj 2^(30-E_j)) (|A| <= 2^30) and every V_jc the integer
// B_jc = rint(V_jc 2^(E_j+31-F_c)) (|B| < 2^31), each written as four base-256 digits,
// so that
//   Y_rc = sum_j x_rj V_jc = 2^(F_c-61) sum_j A_rj B_jc   (the column scales cancel),
// sum_j A_rj B_jc = sum_{t,u} 2^(8(8-t-u)) L_{t+u} with L_s the level sums of digit
// products.  The digits of A are the bytes of A + 0x80808080 less 128 (in [-128, 127];
// the sum reproduces A exactly because |A| <= 2^30), those of B balanced (rounded to
// nearest at each step, |b| <= 128).  Levels 2..5 (ten digit pairs) are kept; over a
// chunk of 256 columns every L_s <= 4 * 256 * 2^14 = 2^24 is an exact integer in the
// FP32 accumulator; the chunks are added exactly into int64 sums (unit 2^(F_c-37)) and
// rounded once to FP32 at the end.  Columns holding Inf or NaN give NaN columns of Y.
//
// Persistent: one CTA per SM walks a contiguous range of the items (node, 128-row
// tile, 64-mode tile), the mode tiles of a row tile adjacent so that the second read of
// X comes from L2; the stage ring and the two accumulator sets run on across items.  18 warps:
//   warp 0        loader: TMA box of X (128 rows x 16 columns FP32) and a bulk copy
//                 of the 16-column chunk of V digits (8 KB), 6 stages deep
//   warp 1        TMEM owner and single-thread MMA issuer: per 16 columns four MMAs,
//                 X digit t against the V digits 1 .. 5 - t (N = 64 (5 - t)) into
//                 the level accumulators L_{t+1} .. L_5; two accumulator sets
//                 (2 x 256 TMEM columns) alternate between chunks
//   warps 2..9    converters: X -> four digit planes (K-major core matrices)
//   warps 10..17  output: int64 sums of 32 entries per thread, then Y
// Every mbarrier wait is bounded: a timeout raises the error flag, the CTA drains
// its copies and MMAs and frees TMEM.
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "hapod_internal.cuh"
#include "tc_common.cuh"

namespace hapod {
namespace {

constexpr int kDigits = 4;
constexpr int kRowsT = 128;                          // rows of X per item (M)
constexpr int kModesT = 64;                          // modes per item
constexpr int kK = 16;                               // columns of X per stage (one MMA K)
constexpr int kChunkStages = 16;                     // 256 columns between exact flushes
constexpr int kStX = kRowsT * kK * 4;                // FP32 staging of X, 8 KB
constexpr int kPlaneX = kRowsT * kK * 2;             // one digit plane of X, 4 KB
constexpr int kPlaneV = kModesT * kK * 2;            // one digit plane of V, 2 KB
constexpr int kOpX = kDigits * kPlaneX;              // 16 KB
constexpr int kOpV = kDigits * kPlaneV;              // 8 KB
constexpr int kStages = 6;
constexpr int kSmemBytes = kStages * (kStX + kOpX + kOpV) + 1024;
constexpr int kConvWarps = 8;
constexpr int kFirstConvWarp = 2;
constexpr int kFirstOutWarp = kFirstConvWarp + kConvWarps;
constexpr int kOutWarps = 8;
constexpr int kThreads = (kFirstOutWarp + kOutWarps) * 32;
constexpr uint32_t kLbo = 128;                       // next core matrix along K
constexpr uint32_t kSbo = (kK / 8) * 128;            // next core matrix along M / N
constexpr uint32_t kSetCols = 256;                   // L2 | L3 | L4 | L5 of 64 modes
constexpr uint32_t kTmemCols = 512;
constexpr int kExpZero = kFxExpZero;
constexpr int kExpBad = kFxExpBad;
static_assert(kSmemBytes <= 227 * 1024, "shared memory");

struct Bars {
  uint64_t full[kStages];    // loader: X (TMA) and V digits (bulk), transaction bytes
  uint64_t xfree[kStages];   // converters: X staging read
  uint64_t ofull[kStages];   // converters: X digits written
  uint64_t ofree[kStages];   // MMA completion: operands free
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t mma_done;
};

__device__ __forceinline__ int find_job(const FxModesJob* jobs, int njobs, int64_t item) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].item_base <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Item `it` of the launch: job, first row, mode tile, stages (16 columns each).
struct Item {
  int jb;
  int row0;
  int mt;
  int nst;
};
__device__ __forceinline__ Item item_of(const FxModesJob* jobs, int njobs, int64_t it) {
  Item r;
  r.jb = find_job(jobs, njobs, it);
  const FxModesJob& J = jobs[r.jb];
  const int64_t local = it - J.item_base;
  r.row0 = (int)((local / J.mode_tiles) * kRowsT);
  r.mt = (int)(local % J.mode_tiles);
  r.nst = (J.m + kK - 1) / kK;
  return r;
}

// FP32 value of an int64 in FP32 arithmetic only (a 64-bit conversion would run on
// the FP64 unit): |a| split into 32-bit halves, at most two roundings.
__device__ __forceinline__ float i64_to_f32(long long a) {
  const unsigned long long u = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
  const float f = fmaf(__uint2float_rn((unsigned)(u >> 32)), 4294967296.0f, __uint2float_rn((unsigned)u));
  return a < 0 ? -f : f;
}

// fp16 pair (lo, hi) = (byte b of u0 - 128, byte b of u1 - 128): the bytes are placed
// in the mantissas of 1024 (0x6400), and 1152 is subtracted, exactly.
__device__ __forceinline__ uint32_t digit_pair(uint32_t u0, uint32_t u1, uint32_t sel) {
  const uint32_t w = (__byte_perm(u0, u1, sel) & 0x00FF00FFu) | 0x64006400u;
  const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&w), __floats2half2_rn(1152.f, 1152.f));
  return *reinterpret_cast<const uint32_t*>(&h);
}

__global__ void __launch_bounds__(kThreads, 1)
    modes_fx_kernel(const FxModesJob* __restrict__ jobs, const CUtensorMap* __restrict__ maps, int njobs,
                    int64_t total_items, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ Bars bars;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const tc::WaitBudget wb = tc::wait_budget(err);
  // a contiguous range of items per CTA: the mode tiles of a row tile follow each
  // other, so the second read of the tile's X comes from L2
  const int64_t per_cta = (total_items + gridDim.x - 1) / gridDim.x;
  const int64_t it_begin = (int64_t)blockIdx.x * per_cta;
  const int64_t it_end = it_begin + per_cta < total_items ? it_begin + per_cta : total_items;
  auto st_x = [&](int s) -> uint8_t* { return smem + (size_t)s * kStX; };
  auto op_x = [&](int s) -> uint8_t* { return smem + (size_t)kStages * kStX + (size_t)s * (kOpX + kOpV); };
  auto op_v = [&](int s) -> uint8_t* { return op_x(s) + kOpX; };

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&bars.full[s], 1);
      tc::mbar_init(&bars.xfree[s], kConvWarps);
      tc::mbar_init(&bars.ofull[s], kConvWarps);
      tc::mbar_init(&bars.ofree[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bars.acc_full[b], 1);
      tc::mbar_init(&bars.acc_empty[b], kOutWarps);
    }
    tc::mbar_init(&bars.mma_done, 1);
    abort_flag = 0;
    tc::mbar_fence_init();
  }
  if (warp == 1) tc::tmem_alloc(&tmem_base, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ loader
    if (lane == 0) {
      int64_t g = 0;  // stages issued by this CTA
      int cur_jb = -1;
      bool ok = true;
      for (int64_t it = it_begin; it < it_end && ok; ++it) {
        const Item I = item_of(jobs, njobs, it);
        const FxModesJob& J = jobs[I.jb];
        const CUtensorMap* map = maps + I.jb;
        if (I.jb != cur_jb) {
          tc::tensormap_acquire(map);
          cur_jb = I.jb;
        }
        const uint8_t* vsrc = reinterpret_cast<const uint8_t*>(J.vdig) + (size_t)I.mt * I.nst * kOpV;
        for (int k = 0; k < I.nst; ++k, ++g) {
          const int s = (int)(g % kStages);
          const uint32_t use = (uint32_t)(g / kStages);
          // the slot's X staging and its operand area must both be free
          if (g >= kStages && (!tc::mbar_wait(&bars.xfree[s], (use - 1) & 1, &abort_flag, err, wb) ||
                               !tc::mbar_wait(&bars.ofree[s], (use - 1) & 1, &abort_flag, err, wb))) {
            ok = false;
            break;
          }
          tc::mbar_expect_tx(&bars.full[s], (uint32_t)(kStX + kOpV));
          tc::tma_load_2d(st_x(s), map, I.row0, k * kK, &bars.full[s]);
          tc::bulk_load(op_v(s), vsrc + (size_t)k * kOpV, (uint32_t)kOpV, &bars.full[s]);
        }
      }
      if (abort_flag) {  // wait (bounded) for the copies still in flight
        for (int64_t k = (g > kStages ? g - kStages : 0); k < g; ++k) {
          const long long t0 = clock64();
          while (!tc::mbar_try(&bars.full[k % kStages], (uint32_t)(k / kStages) & 1) &&
                 clock64() - t0 < tc::kWaitBudget) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t idn[kDigits];
#pragma unroll
      for (int t = 0; t < kDigits; ++t) idn[t] = tc::idesc_f16_f32_major(128, (uint32_t)(kModesT * (kDigits - t)), 0, 0);
      int64_t g = 0, ch = 0;
      bool ok = true;
      for (int64_t it = it_begin; it < it_end && ok; ++it) {
        const Item I = item_of(jobs, njobs, it);
        for (int k = 0; k < I.nst; ++k, ++g) {
          const int s = (int)(g % kStages);
          const uint32_t use = (uint32_t)(g / kStages);
          const bool first = (k % kChunkStages) == 0;
          const bool last = (k % kChunkStages) == kChunkStages - 1 || k == I.nst - 1;
          const int set = (int)(ch & 1);
          if (first && ch >= 2 &&
              !tc::mbar_wait(&bars.acc_empty[set], (uint32_t)((ch >> 1) - 1) & 1, &abort_flag, err, wb)) {
            ok = false;
            break;
          }
          if (!tc::mbar_wait(&bars.ofull[s], use & 1, &abort_flag, err, wb) ||
              !tc::mbar_wait(&bars.full[s], use & 1, &abort_flag, err, wb)) {  // the V digits landed
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t px = tc::smem_u32(op_x(s)), pv = tc::smem_u32(op_v(s));
          const uint32_t d = tbase + (uint32_t)set * kSetCols;
#pragma unroll
          for (int t = 0; t < kDigits; ++t)
            tc::umma_f16(d + (uint32_t)(kModesT * t), tc::ns_desc(px + (uint32_t)t * kPlaneX, kLbo, kSbo),
                         tc::ns_desc(pv, kLbo, kSbo), idn[t], (first && t == 0) ? 0u : 1u);
          tc::umma_commit(&bars.ofree[s]);
          if (last) {
            tc::umma_commit(&bars.acc_full[set]);
            ++ch;
          }
        }
      }
      tc::umma_commit(&bars.mma_done);
      const long long t0 = clock64();
      while (!tc::mbar_try(&bars.mma_done, 0) && clock64() - t0 < tc::kWaitBudget) {
      }
    }
  } else if (warp < kFirstOutWarp) {
    // ------------------------------------------------------------ converters
    // thread (r, g): row r of the tile, column octet g of the stage (a warp: 32
    // consecutive rows, every staging load 128 contiguous bytes); its 16-byte digit
    // stores fill core-matrix rows
    const int ct = tid - kFirstConvWarp * 32;  // 0..255
    const int r = ct & (kRowsT - 1), g8 = ct >> 7;
    const uint32_t off = (uint32_t)(r >> 3) * kSbo + (uint32_t)g8 * kLbo + (uint32_t)(r & 7) * 16;
    int64_t g = 0;
    bool ok = true;
    for (int64_t it = it_begin; it < it_end && ok; ++it) {
      const Item I = item_of(jobs, njobs, it);
      const float2* __restrict__ xsc = jobs[I.jb].xscale;
      for (int k = 0; k < I.nst; ++k, ++g) {
        const int s = (int)(g % kStages);
        const uint32_t use = (uint32_t)(g / kStages);
        if (!tc::mbar_wait_warp(&bars.full[s], use & 1, &abort_flag, err, wb)) {
          ok = false;
          break;
        }
        const float* xs = reinterpret_cast<const float*>(st_x(s));
        uint32_t b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int cl = 8 * g8 + i;
          const float2 sc = xsc[k * kK + cl];  // zero beyond m and for zero or non-finite columns
          b[i] = (uint32_t)__float2int_rn((xs[cl * kRowsT + r] * sc.x) * sc.y) + 0x80808080u;
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bars.xfree[s]);  // this warp's staging reads are done
        if (g >= kStages && !tc::mbar_wait_warp(&bars.ofree[s], (use - 1) & 1, &abort_flag, err, wb)) {
          ok = false;
          break;
        }
#pragma unroll
        for (int t = 0; t < kDigits; ++t) {
          const uint32_t bs = 3u - (uint32_t)t;  // digit t = byte 3 - t
          const uint32_t sel = bs | (bs << 4) | ((bs + 4u) << 8) | ((bs + 4u) << 12);
          *reinterpret_cast<uint4*>(op_x(s) + t * kPlaneX + off) =
              make_uint4(digit_pair(b[0], b[1], sel), digit_pair(b[2], b[3], sel), digit_pair(b[4], b[5], sel),
                         digit_pair(b[6], b[7], sel));
        }
        tc::fence_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bars.ofull[s]);
      }
    }
  } else {
    // ------------------------------------------------------------ output
    const int ow = warp - kFirstOutWarp;  // 0..7
    const int q = warp & 3;               // TMEM lane quarter = rows 32 q .. 32 q + 31
    const int h = ow >> 2;                // modes 32 h .. 32 h + 31 of the tile
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    int64_t ch = 0;
    bool ok = true;
    for (int64_t it = it_begin; it < it_end && ok; ++it) {
      const Item I = item_of(jobs, njobs, it);
      const FxModesJob& J = jobs[I.jb];
      const int nchunk = (I.nst + kChunkStages - 1) / kChunkStages;
      long long acc[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[c] = 0;
      for (int c = 0; c < nchunk; ++c, ++ch) {
        const int set = (int)(ch & 1);
        if (!tc::mbar_wait_warp(&bars.acc_full[set], (uint32_t)(ch >> 1) & 1, &abort_flag, err, wb)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8) {
          const uint32_t col = (uint32_t)set * kSetCols + (uint32_t)(32 * h + 8 * g8);
          uint32_t l2[8], l3[8], l4[8], l5[8];
          tc::tmem_ld8_raw(tbase + lanes + col, l2);
          tc::tmem_ld8_raw(tbase + lanes + col + kModesT, l3);
          tc::tmem_ld8_raw(tbase + lanes + col + 2 * kModesT, l4);
          tc::tmem_ld8_raw(tbase + lanes + col + 3 * kModesT, l5);
          tc::tmem_wait_ld();
          tc::reg_barrier8(l2);
          tc::reg_barrier8(l3);
          tc::reg_barrier8(l4);
          tc::reg_barrier8(l5);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            acc[8 * g8 + i] += (long long)__float2int_rn(__uint_as_float(l2[i])) * 16777216LL +
                               (long long)__float2int_rn(__uint_as_float(l3[i])) * 65536LL +
                               (long long)__float2int_rn(__uint_as_float(l4[i])) * 256LL +
                               (long long)__float2int_rn(__uint_as_float(l5[i]));
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bars.acc_empty[set]);
      }
      if (!ok || abort_flag) break;
      // y = acc 2^(F_c - 37) scale_c in FP32 arithmetic (GB300 runs FP64 at 1/64 of the
      // FP32 rate): at most two roundings of the int64 sum times the mode's factor
      // 2^(F_c - 37) scale_c (exact when it is a normal float; ldexpf otherwise)
      const int64_t row = I.row0 + 32 * q + lane;
      float* __restrict__ ycol = J.Y + (size_t)(I.mt * kModesT + 32 * h) * J.ldy + row;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int col = I.mt * kModesT + 32 * h + c;
        if (col >= J.k || row >= J.n) continue;
        const float f = J.ymul[col];  // > 0 factor, 0 zero mode, NaN bad mode, -1 out of range
        float y;
        if (f > 0.f)
          y = i64_to_f32(acc[c]) * f;
        else if (f == 0.f || f != f)
          y = f;
        else
          y = ldexpf(i64_to_f32(acc[c]), J.fexp[col] - 37) * J.yscale[col];
        ycol[(size_t)c * J.ldy] = y;
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, kTmemCols);
}

// V_k digits: per mode c, F_c with max_j 2^E_j |V_jc| < 2^F_c, then the four digits of
// rint(V_jc 2^(E_j + 31 - F_c)) in the K-major operand layout of the X V kernel:
// [mode tile][16-column chunk][digit][8-mode group][column octet][8 modes x 8 columns].
// One block per mode.
__global__ void __launch_bounds__(256) modes_fx_vsplit(const FxVSplitJob* __restrict__ jobs, int njobs) {
  const FxVSplitJob& J = jobs[blockIdx.y];
  const int c = blockIdx.x;
  if (c >= J.kpad) return;
  __shared__ int s_max[8];
  __shared__ int s_bad[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // F_c from the exponents of |V_jc| 2^E_j (valid columns); a bad column with V_jc != 0 -> bad
  int fmax = kExpZero, bad = 0;
  if (c < J.k) {
    for (int j = tid; j < J.m; j += blockDim.x) {
      const double v = J.V[(size_t)c * J.ldv + j];
      const int E = J.exps[j];
      if (!isfinite(v) || (E >= kExpBad && v != 0.0)) bad = 1;
      if (E <= kExpZero || E >= kExpBad || v == 0.0 || !isfinite(v)) continue;
      int e;
      frexp(v, &e);  // |v| < 2^e
      fmax = max(fmax, e + E);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fmax = max(fmax, __shfl_xor_sync(0xffffffffu, fmax, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (lane == 0) {
    s_max[warp] = fmax;
    s_bad[warp] = bad;
  }
  __syncthreads();
  if (tid == 0) {
    int f = kExpZero, b = 0;
    for (int w = 0; w < 8; ++w) {
      f = max(f, s_max[w]);
      b |= s_bad[w];
    }
    s_max[0] = b ? kExpBad : f;
  }
  __syncthreads();
  const int F = s_max[0];
  if (tid == 0) {
    J.fexp[c] = F;
    const float ys = c < J.k && J.scale ? (float)J.scale[c] : 1.0f;
    J.yscale[c] = ys;
    // one FP32 factor 2^(F - 37) ys for the output, when it is a normal float
    float f;
    if (F >= kExpBad) {
      f = __int_as_float(0x7FC00000);
    } else if (F <= kExpZero || ys == 0.f) {
      f = 0.f;
    } else {
      const double fd = ldexp((double)ys, F - 37);
      f = (fabs(fd) >= 0x1.0p-126 && fabs(fd) < 0x1.0p+127 && ys > 0.f) ? (float)fd : -1.f;
    }
    J.ymul[c] = f;
  }
  // the block of mode 0 also writes the X scale pairs s1 s2 = 2^(30 - E_j) of the
  // converters (zero for zero or non-finite columns and for the padding up to whole
  // 16-column stages)
  if (c == 0) {
    const int npad = (J.m + kK - 1) / kK * kK;
    for (int j = tid; j < npad; j += blockDim.x) {
      float s1 = 0.f, s2 = 0.f;
      const int E = j < J.m ? J.exps[j] : kExpZero;
      if (E > kExpZero && E < kExpBad) {
        const int e = 30 - E, e1 = max(-126, min(127, e));
        s1 = ldexpf(1.0f, e1);
        s2 = ldexpf(1.0f, e - e1);
      }
      J.xscale[j] = make_float2(s1, s2);
    }
  }
  // digits, column by column of V (the contraction index j), zero beyond m and k
  const int mt = c / kModesT, cc = c % kModesT;
  const int nst = (J.m + kK - 1) / kK;
  for (int j = tid; j < nst * kK; j += blockDim.x) {
    double a = 0.0;
    if (c < J.k && j < J.m && F > kExpZero && F < kExpBad) {
      const int E = J.exps[j];
      if (E > kExpZero && E < kExpBad) a = rint(ldexp(J.V[(size_t)c * J.ldv + j], E + 31 - F));
    }
    // balanced base-256 digits of the integer a (|a| <= 2^31)
    double rem = a;
    float d[kDigits];
#pragma unroll
    for (int t = 0; t < kDigits; ++t) {
      const double w = ldexp(1.0, 8 * (kDigits - 1 - t));
      const double q = rint(rem / w);
      d[t] = (float)q;
      rem -= q * w;
    }
    const int k = j / kK, jj = j % kK;
    uint8_t* base = reinterpret_cast<uint8_t*>(J.vdig) + ((size_t)mt * nst + k) * kOpV;
    const uint32_t off = (uint32_t)(cc >> 3) * kSbo + (uint32_t)(jj >> 3) * kLbo + (uint32_t)(cc & 7) * 16 +
                         (uint32_t)(jj & 7) * 2;
#pragma unroll
    for (int t = 0; t < kDigits; ++t) *reinterpret_cast<__half*>(base + t * kPlaneV + off) = __float2half_rn(d[t]);
  }
}

// Column exponents of FP32 X (max |x_rj| < 2^E_j; kExpZero for a zero column, kExpBad
// for a column holding Inf or NaN): one block per (column, chunk of 2^16 rows), four
// independent float4 loads in flight per thread, one atomicMax per block (the array
// starts below kExpZero).
constexpr int64_t kColexpRows = 1 << 16;

__global__ void __launch_bounds__(256) fx_colexp(const float* __restrict__ X, int64_t ldx, int64_t n, int* exps) {
  const int j = blockIdx.y;
  const float* x = X + (size_t)j * ldx;
  const int64_t r0 = (int64_t)blockIdx.x * kColexpRows, r1 = min(n, r0 + kColexpRows);
  float mx = 0.f;
  int bad = 0;
  if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
    const int64_t q0 = r0 / 4, q1 = r1 / 4;  // whole float4s, r0 is a multiple of 4
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (int64_t q = q0 + threadIdx.x; q < q1; q += 4 * blockDim.x) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = q + u * blockDim.x < q1 ? x4[q + u * blockDim.x] : make_float4(0, 0, 0, 0);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float m4 = fmaxf(fmaxf(fabsf(v[u].x), fabsf(v[u].y)), fmaxf(fabsf(v[u].z), fabsf(v[u].w)));
        bad |= !(m4 <= 3.402823466e38f) | (v[u].x != v[u].x) | (v[u].y != v[u].y) | (v[u].z != v[u].z) |
               (v[u].w != v[u].w);
        mx = fmaxf(mx, m4);
      }
    }
    for (int64_t r = 4 * q1 + threadIdx.x; r < r1; r += blockDim.x) {  // ragged tail
      const float v = fabsf(x[r]);
      bad |= !(v <= 3.402823466e38f);
      mx = fmaxf(mx, v);
    }
  } else {
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      const float v = fabsf(x[r]);
      bad |= !(v <= 3.402823466e38f);
      mx = fmaxf(mx, v);
    }
  }
  __shared__ float s_m[8];
  __shared__ int s_b[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_m[threadIdx.x >> 5] = mx;
    s_b[threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    int b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      m = fmaxf(m, s_m[w]);
      b |= s_b[w];
    }
    int e = kExpZero;
    if (b)
      e = kExpBad;
    else if (m > 0.f)
      frexpf(m, &e);
    atomicMax(&exps[j], e);
  }
}

}  // namespace

int fx_modes_tile() { return kModesT; }
size_t fx_xscale_bytes(int64_t m) { return (size_t)((m + kK - 1) / kK * kK) * sizeof(float2); }
size_t fx_vdig_bytes(int64_t m, int64_t k) {
  const int64_t nst = (m + kK - 1) / kK, mtiles = (k + kModesT - 1) / kModesT;
  return (size_t)(mtiles * nst) * kOpV;
}

cudaError_t launch_fx_colexp(const float* X, int64_t ldx, int64_t n, int64_t m, int* exps, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(exps, 0x80, sizeof(int) * (size_t)m, s);  // below kExpZero
  if (e != cudaSuccess) return e;
  const unsigned chunks = (unsigned)std::max<int64_t>(1, (n + kColexpRows - 1) / kColexpRows);
  fx_colexp<<<dim3(chunks, (unsigned)m), 256, 0, s>>>(X, ldx, n, exps);
  return cudaGetLastError();
}

cudaError_t launch_modes_fx(const FxVSplitJob* vjobs_dev, int njobs, int max_kpad, const FxModesJob* jobs_dev,
                            const CUtensorMap* maps_dev, int64_t total_items, int* err_flag, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(modes_fx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (njobs <= 0 || total_items <= 0) return cudaSuccess;
  modes_fx_vsplit<<<dim3((unsigned)max_kpad, (unsigned)njobs), 256, 0, s>>>(vjobs_dev, njobs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  }
  const int64_t grid = total_items < sms ? total_items : sms;
  modes_fx_kernel<<<(unsigned)grid, kThreads, kSmemBytes, s>>>(jobs_dev, maps_dev, njobs, total_items, err_flag);
  return cudaGetLastError();
}

}  // namespace hapod
