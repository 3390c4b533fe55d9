// K4, fixed-point mixed form: Y = X V_k diag(scale) (Sec. 2, Remark
// def:method_of_snapshots: sigma_k phi_k = X psi_k, or phi_k with scale = 1/sigma)
// of FP32 snapshots on the 5th-generation tensor cores (tcgen05, kind::f16, fp16
// digit operands).
//
// With E_j the exponent of column j's largest |x| (2^(E_j-1) <= max < 2^E_j) and F_c
// that of max_j 2^E_j |V_jc|, every x_rj is the integer A_rj = rint(x_rj 2^(30-E_j))
// (|A| <= 2^30) and every V_jc the integer B_jc = rint(V_jc 2^(E_j+31-F_c)) (|B| < 2^31),
// each written as four base-256 digits a_0..a_3, b_0..b_3 (most significant first):
//   Y_rc = sum_j x_rj V_jc = 2^(F_c-61) sum_j A_rj B_jc   (the column scales cancel),
//   sum_j A B = 2^48 D2 + 2^40 D3 + (digit pairs t + u >= 4, at most 3.008 2^30 each),
//   D2 = sum_j a_0 b_0,
//   D3 = sum_j [a_0 b_1 + a_1 b_0 + 2^-8 (a_0 b_2 + a_1 b_1 + a_2 b_0)
//               + 2^-16 (a_0 b_3 + a_1 b_2 + a_2 b_1 + a_3 b_0)].
// The digits of A are the bytes of A + 0x80808080 less 128 (|a_0| <= 64, the others in
// [-128, 127]), those of B balanced (|b| <= 128).  D2 is exact: each a_0 b_0 is an
// integer of at most 2^13, and a group of up to 2048 columns keeps |D2| <= 2^24 in the
// FP32 accumulator.  D3 is accumulated in FP32 by the tensor cores from exact products:
// its 2^-8 and 2^-16 weights ride on scaled digit planes (a_2 2^-8 and a_3 2^-16 on the
// X side; b_1 2^-8, b_2 2^-8, b_2 2^-16, b_3 2^-16 on the V side; all exact in fp16), so
// it carries the rounding of an FP32 dot product at 2^-7 of D2's scale.  Output:
// y = (256 D2 + D3) 2^(F_c-21) scale_c, one fused FP32 rounding and one product with
// the mode's factor; columns holding Inf or NaN give NaN modes.  Contractions longer
// than one group keep the D2 of the earlier groups exactly as int32 sums in a scratch
// array and their D3 in Y; the last group combines them.
//
// Persistent: one CTA per SM walks a contiguous range of the items (node, 128-row tile,
// mode tile of at most 128 modes), so a node with k <= 128 converts its X once.  The
// X staging ring (8 deep) and the operand ring (4 deep) run on across items and the
// two TMEM accumulator sets alternate between groups.  19 warps:
//   warp 0        X loader: TMA box of X (128 rows x 16 columns FP32)
//   warp 1        TMEM owner and single-thread MMA issuer: per 16 columns nine MMAs,
//                 a_0 x [b_0 | b_1] into [D2 | D3] and eight more into D3
//   warp 2        V loader: bulk copy of the six V digit planes of 16 columns
//   warps 3..10   converters: X -> four digit planes (K-major core matrices)
//   warps 11..18  output: Y from D2 and D3
// Every mbarrier wait is bounded: a timeout raises the error flag, the CTA drains
// its copies and MMAs and frees TMEM.
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "hapod_internal.cuh"
#include "tc_common.cuh"

namespace hapod {
namespace {

constexpr int kXDigits = 4;
constexpr int kVPlanes = 6;                          // b0, b1, b1/2^8, b2/2^8, b2/2^16, b3/2^16
constexpr int kRowsT = 128;                          // rows of X per item (M)
constexpr int kMaxModes = 128;                       // modes per item
constexpr int kK = 16;                               // columns of X per stage (one MMA K)
constexpr int kGroupStages = 128;                    // 2048 columns per exact D2 group
constexpr int kStX = kRowsT * kK * 4;                // FP32 staging of X, 8 KB
constexpr int kPlaneX = kRowsT * kK * 2;             // one digit plane of X, 4 KB
constexpr int kOpX = kXDigits * kPlaneX;             // 16 KB
constexpr int kOpV = kVPlanes * kMaxModes * kK * 2;  // 24 KB at 128 modes
constexpr int kXStages = 8;
constexpr int kOpStages = 4;
constexpr int kSmemBytes = kXStages * kStX + kOpStages * (kOpX + kOpV) + 1024;
constexpr int kXLoadWarp = 0;
constexpr int kMmaWarp = 1;
constexpr int kVLoadWarp = 2;
constexpr int kFirstConvWarp = 3;
constexpr int kConvWarps = 8;
constexpr int kFirstOutWarp = kFirstConvWarp + kConvWarps;
constexpr int kOutWarps = 8;
constexpr int kThreads = (kFirstOutWarp + kOutWarps) * 32;
constexpr uint32_t kLbo = 128;                       // next core matrix along K
constexpr uint32_t kSbo = (kK / 8) * 128;            // next core matrix along M / N
constexpr uint32_t kSetCols = 256;                   // D2 | D3 of up to 128 modes
constexpr uint32_t kTmemCols = 512;
constexpr int kExpZero = kFxExpZero;
constexpr int kExpBad = kFxExpBad;
static_assert(kSmemBytes <= 227 * 1024 - 512, "shared memory");

struct Bars {
  uint64_t xfull[kXStages];   // X loader: TMA box landed (transaction bytes)
  uint64_t xfree[kXStages];   // converters: staging read
  uint64_t vfull[kOpStages];  // V loader: digit planes landed (transaction bytes)
  uint64_t ofull[kOpStages];  // converters: X digits written
  uint64_t ofree[kOpStages];  // MMA completion: operands free
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

// fp16 pair (lo, hi) = ((byte b of u0) - 128, (byte b of u1) - 128) 2^-s: the bytes are
// placed in the low mantissa bits of `base` (1024, 4 or 2^-6, whose unit in the last
// place is 1, 2^-8 or 2^-16) and base + 128 ulp is subtracted, exactly.
__device__ __forceinline__ uint32_t digit_pair(uint32_t u0, uint32_t u1, uint32_t sel, uint32_t base, __half2 sub) {
  const uint32_t w = (__byte_perm(u0, u1, sel) & 0x00FF00FFu) | base;
  const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&w), sub);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Output of one mode: t = 256 D2 + D3 (units 2^(F-21)) times the mode's factor.
__device__ __forceinline__ float apply_factor(float t, float f, const FxModesJob& J, int col) {
  if (f > 0.f) return t * f;
  if (f == 0.f || f != f) return f;  // zero mode / NaN mode
  return ldexpf(t, J.fexp[col] - 21) * J.yscale[col];
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
  // other, so a second read of the tile's X comes from L2
  const int64_t per_cta = (total_items + gridDim.x - 1) / gridDim.x;
  const int64_t it_begin = (int64_t)blockIdx.x * per_cta;
  const int64_t it_end = it_begin + per_cta < total_items ? it_begin + per_cta : total_items;
  auto st_x = [&](int s) -> uint8_t* { return smem + (size_t)s * kStX; };
  auto op_x = [&](int s) -> uint8_t* { return smem + (size_t)kXStages * kStX + (size_t)s * (kOpX + kOpV); };
  auto op_v = [&](int s) -> uint8_t* { return op_x(s) + kOpX; };

  if (tid == 0) {
    for (int s = 0; s < kXStages; ++s) {
      tc::mbar_init(&bars.xfull[s], 1);
      tc::mbar_init(&bars.xfree[s], kConvWarps);
    }
    for (int s = 0; s < kOpStages; ++s) {
      tc::mbar_init(&bars.vfull[s], 1);
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
  if (warp == kMmaWarp) tc::tmem_alloc(&tmem_base, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == kXLoadWarp) {
    // ------------------------------------------------------------ X loader
    if (lane == 0) {
      int64_t g = 0;  // stages issued by this CTA
      int cur_jb = -1;
      bool ok = true;
      for (int64_t it = it_begin; it < it_end && ok; ++it) {
        const Item I = item_of(jobs, njobs, it);
        const CUtensorMap* map = maps + I.jb;
        if (I.jb != cur_jb) {
          tc::tensormap_acquire(map);
          cur_jb = I.jb;
        }
        for (int k = 0; k < I.nst; ++k, ++g) {
          const int s = (int)(g % kXStages);
          const uint32_t use = (uint32_t)(g / kXStages);
          if (g >= kXStages && !tc::mbar_wait(&bars.xfree[s], (use - 1) & 1, &abort_flag, err, wb)) {
            ok = false;
            break;
          }
          tc::mbar_expect_tx(&bars.xfull[s], (uint32_t)kStX);
          tc::tma_load_2d(st_x(s), map, I.row0, k * kK, &bars.xfull[s]);
        }
      }
      if (abort_flag) {  // wait (bounded) for the copies still in flight
        for (int64_t k = (g > kXStages ? g - kXStages : 0); k < g; ++k) {
          const long long t0 = clock64();
          while (!tc::mbar_try(&bars.xfull[k % kXStages], (uint32_t)(k / kXStages) & 1) &&
                 clock64() - t0 < tc::kWaitBudget) {
          }
        }
      }
    }
  } else if (warp == kVLoadWarp) {
    // ------------------------------------------------------------ V loader
    if (lane == 0) {
      int64_t g = 0;
      bool ok = true;
      for (int64_t it = it_begin; it < it_end && ok; ++it) {
        const Item I = item_of(jobs, njobs, it);
        const FxModesJob& J = jobs[I.jb];
        const uint32_t vbytes = (uint32_t)(kVPlanes * kK * 2 * J.nt);
        const uint8_t* vsrc = reinterpret_cast<const uint8_t*>(J.vdig) + (size_t)I.mt * I.nst * vbytes;
        for (int k = 0; k < I.nst; ++k, ++g) {
          const int s = (int)(g % kOpStages);
          const uint32_t use = (uint32_t)(g / kOpStages);
          if (g >= kOpStages && !tc::mbar_wait(&bars.ofree[s], (use - 1) & 1, &abort_flag, err, wb)) {
            ok = false;
            break;
          }
          tc::mbar_expect_tx(&bars.vfull[s], vbytes);
          tc::bulk_load(op_v(s), vsrc + (size_t)k * vbytes, vbytes, &bars.vfull[s]);
        }
      }
      if (abort_flag) {
        for (int64_t k = (g > kOpStages ? g - kOpStages : 0); k < g; ++k) {
          const long long t0 = clock64();
          while (!tc::mbar_try(&bars.vfull[k % kOpStages], (uint32_t)(k / kOpStages) & 1) &&
                 clock64() - t0 < tc::kWaitBudget) {
          }
        }
      }
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int64_t g = 0, ch = 0;
      int cur_jb = -1;
      uint32_t id1 = 0, id2 = 0, nt = 0;
      bool ok = true;
      for (int64_t it = it_begin; it < it_end && ok; ++it) {
        const Item I = item_of(jobs, njobs, it);
        if (I.jb != cur_jb) {
          cur_jb = I.jb;
          nt = (uint32_t)jobs[I.jb].nt;
          id1 = tc::idesc_f16_f32_major(128, nt, 0, 0);
          id2 = tc::idesc_f16_f32_major(128, 2 * nt, 0, 0);
        }
        const uint32_t pl = (uint32_t)(kK * 2) * nt;  // bytes of one V digit plane
        for (int k = 0; k < I.nst; ++k, ++g) {
          const int s = (int)(g % kOpStages);
          const uint32_t use = (uint32_t)(g / kOpStages);
          const bool first = (k % kGroupStages) == 0;
          const bool last = (k % kGroupStages) == kGroupStages - 1 || k == I.nst - 1;
          const int set = (int)(ch & 1);
          if (first && ch >= 2 &&
              !tc::mbar_wait(&bars.acc_empty[set], (uint32_t)((ch >> 1) - 1) & 1, &abort_flag, err, wb)) {
            ok = false;
            break;
          }
          if (!tc::mbar_wait(&bars.ofull[s], use & 1, &abort_flag, err, wb) ||
              !tc::mbar_wait(&bars.vfull[s], use & 1, &abort_flag, err, wb)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t px = tc::smem_u32(op_x(s)), pv = tc::smem_u32(op_v(s));
          const uint32_t d2 = tbase + (uint32_t)set * kSetCols, d3 = d2 + nt;
          auto A = [&](int t) { return tc::ns_desc(px + (uint32_t)t * kPlaneX, kLbo, kSbo); };
          auto B = [&](int p) { return tc::ns_desc(pv + (uint32_t)p * pl, kLbo, kSbo); };
          tc::umma_f16(d2, A(0), B(0), id2, first ? 0u : 1u);  // a0 [b0 | b1] -> [D2 | D3]
          tc::umma_f16(d3, A(0), B(3), id1, 1u);               // a0 b2 2^-8
          tc::umma_f16(d3, A(0), B(5), id1, 1u);               // a0 b3 2^-16
          tc::umma_f16(d3, A(1), B(0), id1, 1u);               // a1 b0
          tc::umma_f16(d3, A(1), B(2), id1, 1u);               // a1 b1 2^-8
          tc::umma_f16(d3, A(1), B(4), id1, 1u);               // a1 b2 2^-16
          tc::umma_f16(d3, A(2), B(0), id1, 1u);               // (a2 2^-8) b0
          tc::umma_f16(d3, A(2), B(2), id1, 1u);               // (a2 2^-8) (b1 2^-8)
          tc::umma_f16(d3, A(3), B(0), id1, 1u);               // (a3 2^-16) b0
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
    const __half2 sub01 = __floats2half2_rn(1152.f, 1152.f);            // 1024 + 128
    const __half2 sub2 = __floats2half2_rn(4.5f, 4.5f);                 // 4 + 128 2^-8
    const __half2 sub3 = __floats2half2_rn(0.017578125f, 0.017578125f);  // 2^-6 + 128 2^-16
    int64_t g = 0;
    bool ok = true;
    for (int64_t it = it_begin; it < it_end && ok; ++it) {
      const Item I = item_of(jobs, njobs, it);
      const float2* __restrict__ xsc = jobs[I.jb].xscale;
      for (int k = 0; k < I.nst; ++k, ++g) {
        const int sx = (int)(g % kXStages), so = (int)(g % kOpStages);
        if (!tc::mbar_wait_warp(&bars.xfull[sx], (uint32_t)(g / kXStages) & 1, &abort_flag, err, wb)) {
          ok = false;
          break;
        }
        const float* xs = reinterpret_cast<const float*>(st_x(sx));
        uint32_t b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int cl = 8 * g8 + i;
          const float2 sc = xsc[k * kK + cl];  // zero beyond m and for zero or non-finite columns
          b[i] = (uint32_t)__float2int_rn((xs[cl * kRowsT + r] * sc.x) * sc.y) + 0x80808080u;
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bars.xfree[sx]);  // this warp's staging reads are done
        const uint32_t use = (uint32_t)(g / kOpStages);
        if (g >= kOpStages && !tc::mbar_wait_warp(&bars.ofree[so], (use - 1) & 1, &abort_flag, err, wb)) {
          ok = false;
          break;
        }
#pragma unroll
        for (int t = 0; t < kXDigits; ++t) {
          const uint32_t bs = 3u - (uint32_t)t;  // digit t = byte 3 - t
          const uint32_t sel = bs | (bs << 4) | ((bs + 4u) << 8) | ((bs + 4u) << 12);
          const uint32_t base = t < 2 ? 0x64006400u : (t == 2 ? 0x44004400u : 0x24002400u);
          const __half2 sub = t < 2 ? sub01 : (t == 2 ? sub2 : sub3);
          *reinterpret_cast<uint4*>(op_x(so) + t * kPlaneX + off) =
              make_uint4(digit_pair(b[0], b[1], sel, base, sub), digit_pair(b[2], b[3], sel, base, sub),
                         digit_pair(b[4], b[5], sel, base, sub), digit_pair(b[6], b[7], sel, base, sub));
        }
        tc::fence_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bars.ofull[so]);
      }
    }
  } else {
    // ------------------------------------------------------------ output
    const int ow = warp - kFirstOutWarp;  // 0..7
    const int q = warp & 3;               // TMEM lane quarter = rows 32 q .. 32 q + 31
    const int h = ow >> 2;                // half h of the tile's modes
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    int64_t ch = 0;
    bool ok = true;
    for (int64_t it = it_begin; it < it_end && ok; ++it) {
      const Item I = item_of(jobs, njobs, it);
      const FxModesJob& J = jobs[I.jb];
      const int nt = J.nt, half = nt >> 1;
      const int ngroups = (I.nst + kGroupStages - 1) / kGroupStages;
      const int64_t row = I.row0 + 32 * q + lane;
      const bool live = row < J.n;
      const int cfirst = I.mt * nt + h * half;  // this warp's first mode
      for (int grp = 0; grp < ngroups; ++grp, ++ch) {
        const int set = (int)(ch & 1);
        if (!tc::mbar_wait_warp(&bars.acc_full[set], (uint32_t)(ch >> 1) & 1, &abort_flag, err, wb)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        for (int c8 = 0; c8 < half; c8 += 8) {
          __syncwarp();  // the TMEM loads are warp-collective
          const uint32_t tc2 = tbase + lanes + (uint32_t)set * kSetCols + (uint32_t)(h * half + c8);
          uint32_t r2[8], r3[8];
          tc::tmem_ld8_raw(tc2, r2);
          tc::tmem_ld8_raw(tc2 + (uint32_t)nt, r3);
          tc::tmem_wait_ld();
          tc::reg_barrier8(r2);
          tc::reg_barrier8(r3);
          const int col0 = cfirst + c8;
          if (!live || col0 >= J.k) continue;  // after the loads
          const float4 fa = __ldg(reinterpret_cast<const float4*>(J.ymul + col0));
          const float4 fb = __ldg(reinterpret_cast<const float4*>(J.ymul + col0 + 4));
          const float f[8] = {fa.x, fa.y, fa.z, fa.w, fb.x, fb.y, fb.z, fb.w};
          float* yp = J.Y + (size_t)col0 * J.ldy + row;
#pragma unroll
          for (int i = 0; i < 8; ++i, yp += J.ldy) {
            if (col0 + i >= J.k) break;
            const float D2 = __uint_as_float(r2[i]), D3 = __uint_as_float(r3[i]);
            if (ngroups == 1) {
              *yp = apply_factor(fmaf(D2, 256.f, D3), f[i], J, col0 + i);
            } else {
              int32_t* zp = J.Z + (size_t)(col0 + i) * J.ldz + row;
              const int32_t z = __float2int_rn(D2);  // an integer of at most 2^24
              if (grp == 0) {
                *zp = z;
                *yp = D3;
              } else if (grp < ngroups - 1) {
                *zp += z;
                *yp += D3;
              } else {
                const double tz = fma((double)(*zp + z), 256.0, (double)(*yp + D3));
                *yp = apply_factor((float)tz, f[i], J, col0 + i);
              }
            }
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bars.acc_empty[set]);
      }
      if (!ok || abort_flag) break;
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == kMmaWarp) tc::tmem_dealloc(tbase, kTmemCols);
}

// V_k digits: per mode c, F_c with max_j 2^E_j |V_jc| < 2^F_c, then the four balanced
// digits b_0..b_3 of rint(V_jc 2^(E_j + 31 - F_c)) as the six planes b_0, b_1, b_1 2^-8,
// b_2 2^-8, b_2 2^-16, b_3 2^-16 in the K-major operand layout of the X V kernel:
// [mode tile][16-column chunk][plane][8-mode group][column octet][8 modes x 8 columns].
// One block per mode; the block of mode 0 also writes the converters' column scales.
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
    // one FP32 factor 2^(F - 21) ys for the output, when it is a normal float
    float f;
    if (F >= kExpBad) {
      f = __int_as_float(0x7FC00000);
    } else if (F <= kExpZero || ys == 0.f) {
      f = 0.f;
    } else {
      const double fd = ldexp((double)ys, F - 21);
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
  const int nt = J.nt, mt = c / nt, cc = c % nt;
  const int nst = (J.m + kK - 1) / kK;
  const size_t pl = (size_t)kK * 2 * nt, blk = kVPlanes * pl;  // bytes of a plane, of a 16-column chunk
  for (int j = tid; j < nst * kK; j += blockDim.x) {
    double a = 0.0;
    if (c < J.k && j < J.m && F > kExpZero && F < kExpBad) {
      const int E = J.exps[j];
      if (E > kExpZero && E < kExpBad) a = rint(ldexp(J.V[(size_t)c * J.ldv + j], E + 31 - F));
    }
    // balanced base-256 digits of the integer a (|a| < 2^31)
    double rem = a;
    float d[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const double w = ldexp(1.0, 8 * (3 - t));
      const double q = rint(rem / w);
      d[t] = (float)q;
      rem -= q * w;
    }
    const float p[kVPlanes] = {d[0], d[1], d[1] * 0x1.0p-8f, d[2] * 0x1.0p-8f, d[2] * 0x1.0p-16f, d[3] * 0x1.0p-16f};
    const int k = j / kK, jj = j % kK;
    uint8_t* base = reinterpret_cast<uint8_t*>(J.vdig) + ((size_t)mt * nst + k) * blk;
    const uint32_t off = (uint32_t)(cc >> 3) * kSbo + (uint32_t)(jj >> 3) * kLbo + (uint32_t)(cc & 7) * 16 +
                         (uint32_t)(jj & 7) * 2;
#pragma unroll
    for (int t = 0; t < kVPlanes; ++t) *reinterpret_cast<__half*>(base + t * pl + off) = __float2half_rn(p[t]);
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

int fx_mode_tiles(int64_t k) { return (int)std::max<int64_t>(1, (k + kMaxModes - 1) / kMaxModes); }
int fx_mode_width(int64_t k) {
  const int64_t tiles = fx_mode_tiles(k), w = (std::max<int64_t>(k, 1) + tiles - 1) / tiles;
  return (int)((w + 15) / 16 * 16);
}
int64_t fx_modes_max_m() { return (int64_t)kGroupStages * kK * 120; }
bool fx_modes_needs_scratch(int64_t m) { return (m + kK - 1) / kK > kGroupStages; }
size_t fx_xscale_bytes(int64_t m) { return (size_t)((m + kK - 1) / kK * kK) * sizeof(float2); }
size_t fx_vdig_bytes(int64_t m, int64_t k) {
  const int64_t nst = (m + kK - 1) / kK;
  return (size_t)(fx_mode_tiles(k) * nst) * kVPlanes * kK * 2 * (size_t)fx_mode_width(k);
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
