// K4, fixed-point mixed form: Y = X V_k diag(scale) (Sec. 2, Remark
// def:method_of_snapshots: sigma_k phi_k = X psi_k, or phi_k with scale = 1/sigma)
// of FP32 snapshots on the 5th-generation tensor cores (tcgen05, kind::f16, fp16
// digit operands) with exact accumulation.
//
// With E_j the exponent of column j's largest |x| (2^(E_j-1) <= max < 2^E_j, recorded
// by the Gram kernel) and F_c that of max_j 2^E_j |V_jc|, every x_rj is the 32-bit
// integer A_rj = rint(x_rj 2^(31-E_j)) and every V_jc the 32-bit integer
// B_jc = rint(V_jc 2^(E_j+31-F_c)), each written as four balanced base-256 digits, so
//   Y_rc = sum_j x_rj V_jc = 2^(F_c-62) sum_j A_rj B_jc   (the column scales cancel),
// sum_j A_rj B_jc = sum_{t,u} 2^(8(8-t-u)) L_{t+u} with L_s the level sums of digit
// products.  Levels 2..5 (ten digit pairs) are kept; over a chunk of 64 columns every
// L_s <= 64 * 4 * 2^14 = 2^22 is an exact integer in the FP32 accumulator; the chunks
// are added exactly into int64 sums (unit 2^(F_c-38)) and rounded once to FP32 at the
// end.  The error of an entry is at most 2^(-30) sum_j 2^(E_j+F_c-E_j) per column
// pair: about m 2^-30 max|x| max|V|, against the 2^-24 m max|x| max|V| of an FP32
// dot product.  Columns holding Inf or NaN give NaN columns of Y.
//
// Work item = (node, 128-row tile, 64-mode tile).  One CTA per item, 14 warps:
//   warp 0        loader: TMA box of X (128 rows x 16 columns FP32) and a bulk copy
//                 of the 16-column chunk of V digits (8 KB), 4 stages deep
//   warp 1        TMEM owner and single-thread MMA issuer: per 16 columns four MMAs,
//                 X digit t against the V digits 1 .. 5 - t (N = 64 (5 - t)) into
//                 the level accumulators L_{t+1} .. L_5; two accumulator sets
//                 (2 x 256 TMEM columns) alternate between 64-column chunks
//   warps 2..5    converters: X -> four digit planes (K-major core matrices)
//   warps 6..13   output: int64 sums of 32 entries per thread, then Y
// Every mbarrier wait is bounded: a timeout raises the error flag, the CTA drains
// its copies and MMAs and frees TMEM.
#include <cuda_fp16.h>

#include <vector>

#include "hapod_internal.cuh"
#include "tc_common.cuh"

namespace hapod {
namespace {

constexpr int kDigits = 4;
constexpr int kRowsT = 128;                          // rows of X per item (M)
constexpr int kModesT = 64;                          // modes per item
constexpr int kK = 16;                               // columns of X per stage (one MMA K)
constexpr int kChunkStages = 4;                      // 64 columns between exact flushes
constexpr int kStX = kRowsT * kK * 4;                // FP32 staging of X, 8 KB
constexpr int kPlaneX = kRowsT * kK * 2;             // one digit plane of X, 4 KB
constexpr int kPlaneV = kModesT * kK * 2;            // one digit plane of V, 2 KB
constexpr int kOpX = kDigits * kPlaneX;              // 16 KB
constexpr int kOpV = kDigits * kPlaneV;              // 8 KB
constexpr int kStages = 4;
constexpr int kSmemBytes = kStages * (kStX + kOpX + kOpV) + 1024;
constexpr int kConvWarps = 4;
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

struct Bars {
  uint64_t full[kStages];    // loader: X (TMA) and V digits (bulk), transaction bytes
  uint64_t xfree[kStages];   // converters: X staging read
  uint64_t ofull[kStages];   // converters: X digits written
  uint64_t ofree[kStages];   // MMA completion: operands free
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t mma_done;
};

__device__ __forceinline__ void digits4(float a, float (&d)[4]) {
  const float C = 12582912.0f;  // 1.5 2^23: (y + C) - C = rint(y) for |y| < 2^22
  d[0] = __fadd_rn(__fmaf_rn(a, 1.0f / 16777216.0f, C), -C);
  const float r1 = __fmaf_rn(d[0], -16777216.0f, a);
  d[1] = __fadd_rn(__fmaf_rn(r1, 1.0f / 65536.0f, C), -C);
  const float r2 = __fmaf_rn(d[1], -65536.0f, r1);
  d[2] = __fadd_rn(__fmaf_rn(r2, 1.0f / 256.0f, C), -C);
  const float r3 = __fmaf_rn(d[2], -256.0f, r2);
  d[3] = __fadd_rn(__fadd_rn(r3, C), -C);
}

__device__ __forceinline__ uint32_t h2bits(float lo, float hi) {
  const __half2 v = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ int find_job(const FxModesJob* jobs, int njobs, int64_t item) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].item_base <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kThreads, 1)
    modes_fx_kernel(const FxModesJob* __restrict__ jobs, const CUtensorMap* __restrict__ maps, int njobs,
                    int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ Bars bars;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const tc::WaitBudget wb = tc::wait_budget(err);

  const int jb = find_job(jobs, njobs, blockIdx.x);
  const FxModesJob& J = jobs[jb];
  const int64_t local = blockIdx.x - J.item_base;
  const int row0 = (int)((local % J.row_tiles) * kRowsT);
  const int mt = (int)(local / J.row_tiles);
  const int nst = (J.m + kK - 1) / kK;
  const int nchunk = (nst + kChunkStages - 1) / kChunkStages;
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
    if (lane == 0 && nst > 0) {
      const CUtensorMap* map = maps + jb;
      tc::tensormap_acquire(map);
      const uint8_t* vsrc = reinterpret_cast<const uint8_t*>(J.vdig) + (size_t)mt * nst * kOpV;
      int issued = 0;
      for (int k = 0; k < nst; ++k) {
        const int s = k % kStages;
        // the slot's X staging and its operand area must both be free
        if (k >= kStages && (!tc::mbar_wait(&bars.xfree[s], ((k / kStages) - 1) & 1, &abort_flag, err, wb) ||
                             !tc::mbar_wait(&bars.ofree[s], ((k / kStages) - 1) & 1, &abort_flag, err, wb)))
          break;
        tc::mbar_expect_tx(&bars.full[s], (uint32_t)(kStX + kOpV));
        tc::tma_load_2d(st_x(s), map, row0, k * kK, &bars.full[s]);
        tc::bulk_load(op_v(s), vsrc + (size_t)k * kOpV, (uint32_t)kOpV, &bars.full[s]);
        issued = k + 1;
      }
      if (abort_flag) {
        for (int k = max(0, issued - kStages); k < issued; ++k) {
          const long long t0 = clock64();
          while (!tc::mbar_try(&bars.full[k % kStages], (k / kStages) & 1) && clock64() - t0 < tc::kWaitBudget) {
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
      for (int k = 0; k < nst; ++k) {
        const int s = k % kStages;
        const int ch = k / kChunkStages;
        const bool first = (k % kChunkStages) == 0;
        const bool last = (k % kChunkStages) == kChunkStages - 1 || k == nst - 1;
        const int set = ch & 1;
        if (first && ch >= 2 && !tc::mbar_wait(&bars.acc_empty[set], ((ch >> 1) - 1) & 1, &abort_flag, err, wb))
          break;
        if (!tc::mbar_wait(&bars.ofull[s], (k / kStages) & 1, &abort_flag, err, wb) ||
            !tc::mbar_wait(&bars.full[s], (k / kStages) & 1, &abort_flag, err, wb))  // the V digits landed
          break;
        tc::tc_fence_after();
        const uint32_t px = tc::smem_u32(op_x(s)), pv = tc::smem_u32(op_v(s));
        const uint32_t d = tbase + (uint32_t)set * kSetCols;
#pragma unroll
        for (int t = 0; t < kDigits; ++t)
          tc::umma_f16(d + (uint32_t)(kModesT * t), tc::ns_desc(px + (uint32_t)t * kPlaneX, kLbo, kSbo),
                       tc::ns_desc(pv, kLbo, kSbo), idn[t], (first && t == 0) ? 0u : 1u);
        tc::umma_commit(&bars.ofree[s]);
        if (last) tc::umma_commit(&bars.acc_full[set]);
      }
      tc::umma_commit(&bars.mma_done);
      const long long t0 = clock64();
      while (!tc::mbar_try(&bars.mma_done, 0) && clock64() - t0 < tc::kWaitBudget) {
      }
    }
  } else if (warp < kFirstOutWarp) {
    // ------------------------------------------------------------ converters
    // thread ct takes row r = ct for both column octets g of a stage (a warp: 32
    // consecutive rows, so every staging load reads 128 contiguous bytes); the 16-byte
    // digit stores of 8 consecutive rows fill one core matrix (128 contiguous bytes)
    const int r = tid - kFirstConvWarp * 32;  // 0..127
    for (int k = 0; k < nst; ++k) {
      const int s = k % kStages;
      if (!tc::mbar_wait_warp(&bars.full[s], (k / kStages) & 1, &abort_flag, err, wb)) break;
      const float* xs = reinterpret_cast<const float*>(st_x(s));
      uint32_t w[2][kDigits][4];
#pragma unroll
      for (int g = 0; g < 2; ++g) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int cl = 8 * g + 2 * i;  // column within the stage
          const int c0 = k * kK + cl;     // column of X
          const int e0 = c0 < J.m ? J.exps[c0] : kExpZero;
          const int e1 = c0 + 1 < J.m ? J.exps[c0 + 1] : kExpZero;
          const float x0 = xs[cl * kRowsT + r], x1 = xs[(cl + 1) * kRowsT + r];
          const bool v0 = e0 > kExpZero && e0 < kExpBad, v1 = e1 > kExpZero && e1 < kExpBad;
          float da[kDigits], db[kDigits];
          digits4(v0 ? ldexpf(x0, 31 - e0) : 0.f, da);
          digits4(v1 ? ldexpf(x1, 31 - e1) : 0.f, db);
#pragma unroll
          for (int t = 0; t < kDigits; ++t) w[g][t][i] = h2bits(da[t], db[t]);
        }
      }
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars.xfree[s]);  // this warp's staging reads are done
      if (k >= kStages && !tc::mbar_wait_warp(&bars.ofree[s], ((k / kStages) - 1) & 1, &abort_flag, err, wb)) break;
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const uint32_t off = (uint32_t)(r >> 3) * kSbo + (uint32_t)g * kLbo + (uint32_t)(r & 7) * 16;
#pragma unroll
        for (int t = 0; t < kDigits; ++t)
          *reinterpret_cast<uint4*>(op_x(s) + t * kPlaneX + off) =
              make_uint4(w[g][t][0], w[g][t][1], w[g][t][2], w[g][t][3]);
      }
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars.ofull[s]);
    }
  } else {
    // ------------------------------------------------------------ output
    const int ow = warp - kFirstOutWarp;  // 0..7
    const int q = warp & 3;               // TMEM lane quarter = rows 32 q .. 32 q + 31
    const int h = ow >> 2;                // modes 32 h .. 32 h + 31 of the tile
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    long long acc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = 0;
    bool ok = true;
    for (int ch = 0; ch < nchunk && ok; ++ch) {
      const int set = ch & 1;
      ok = tc::mbar_wait_warp(&bars.acc_full[set], (ch >> 1) & 1, &abort_flag, err, wb);
      if (!ok) break;
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
    if (__all_sync(0xffffffffu, ok && !abort_flag)) {
      const int64_t row = row0 + 32 * q + lane;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int col = mt * kModesT + 32 * h + c;
        if (col >= J.k || row >= J.n) continue;
        const int F = J.fexp[col];
        float y;
        if (F >= kExpBad)
          y = __int_as_float(0x7FC00000);
        else if (F <= kExpZero)
          y = 0.f;
        else
          y = (float)(ldexp((double)acc[c], F - 38) * (J.scale ? J.scale[col] : 1.0));
        J.Y[(size_t)col * J.ldy + row] = y;
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
  if (tid == 0) J.fexp[c] = F;
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
// for a column holding Inf or NaN): one block per column.
__global__ void __launch_bounds__(256) fx_colexp(const float* __restrict__ X, int64_t ldx, int64_t n, int* exps) {
  const int j = blockIdx.x;
  const float* x = X + (size_t)j * ldx;
  float mx = 0.f;
  int bad = 0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const float v = fabsf(x[r]);
    bad |= !(v <= 3.402823466e38f);
    mx = fmaxf(mx, v);
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
    exps[j] = e;
  }
}

}  // namespace

int fx_modes_tile() { return kModesT; }
size_t fx_vdig_bytes(int64_t m, int64_t k) {
  const int64_t nst = (m + kK - 1) / kK, mtiles = (k + kModesT - 1) / kModesT;
  return (size_t)(mtiles * nst) * kOpV;
}

cudaError_t launch_fx_colexp(const float* X, int64_t ldx, int64_t n, int64_t m, int* exps, cudaStream_t s) {
  if (m > 0) fx_colexp<<<(unsigned)m, 256, 0, s>>>(X, ldx, n, exps);
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
  modes_fx_kernel<<<(unsigned)total_items, kThreads, kSmemBytes, s>>>(jobs_dev, maps_dev, njobs, err_flag);
  return cudaGetLastError();
}

}  // namespace hapod
