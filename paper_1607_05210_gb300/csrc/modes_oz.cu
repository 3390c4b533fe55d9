// K4, digit-slice FP64 form: Y = X V_k diag(scale) (Sec. 2, Remark
// def:method_of_snapshots: sigma_k phi_k = X psi_k, or phi_k with scale = 1/sigma)
// from exact digits on the tensor cores (tcgen05 kind::f16, fp16 x fp16 -> FP32).
//
// X is split per column as for the Gram, x_rj = 2^E_j xt_rj (oz_common.cuh).
// Moving the column scale into V, Y_rc = sum_j xt_rj (2^E_j V_jc) = 2^F_c sum_j
// xt_rj vt_jc with 2^F_c > max_j 2^E_j |V_jc| and vt_jc = 2^(E_j - F_c) V_jc, split
// into 7 base-256 digits the same way (oz_vsplit_kernel: the digits of V_jc against
// the bound 2^(F_c - E_j), so nothing overflows).  The 28 digit pairs of level
// t + u <= 8 are summed exactly over blocks of 128 columns, flushed exactly into
// int64 sums, rounded to FP64 per block (Y_rc = 2^(F_c - 62) (hi 2^32 + lo)) and
// summed over the blocks in FP64 (one rounding for m <= 128), times scale_c.
//
// Persistent kernel, one CTA per SM, looping over items (node, 128-row tile,
// 32-mode tile).  Per 16-column stage the loader brings the FP64 X tile (128 rows x
// 16 columns, one TMA box, zero-filled outside X) into a 5-deep staging ring and the
// V digits (K-major B operand) into the 4-deep operand ring; the converter warps
// write the tile's 7 digit planes into the operand ring as the MN-major A operand
// (M = rows; row groups padded by 16 bytes so the digit stores are conflict-free).
// Warps:
//   warp 0       loader (TMA X tiles, bulk copies of V digits)
//   warp 1       TMEM owner and single-thread UMMA issuer: per stage 10 MMAs
//                128 x (32..128) x 16 (one X digit against up to 4 V digits) into
//                7 level accumulators; two accumulator sets alternating per
//                128-column block, so a block's output overlaps the next
//                block's products
//   warps 2..9   converters (FP64 -> digits)
//   warps 10..13 output (32 modes x 32 rows each; 14 warps leave 128 registers a thread)
#include <climits>

#include "hapod_internal.cuh"
#include "oz_common.cuh"
#include "tc_common.cuh"

namespace hapod {
namespace {

constexpr int NT = 32;                              // modes per item
constexpr int kStages = 4;
constexpr int kRowGroupBytes = 2 * kOzGroupBytes + 16;  // padded: conflict-free digit stores
constexpr int kStageA = 16 * kRowGroupBytes;        // 128 rows x 16 columns, all digits
constexpr int kStageB = 2 * (NT / 8) * kOzGroupBytes;
constexpr int kStageBytes = kStageA + kStageB;
constexpr int kXSlots = 5;                         // FP64 staging ring (TMA boxes of 128 rows x 16 columns)
constexpr int kXSlotBytes = 128 * 16 * 8;
constexpr int kSmemBytes = kStages * kStageBytes + kXSlots * kXSlotBytes + 128;
constexpr int kKBlockStages = kOzKBlock / 16;       // 128 columns between exact flushes
constexpr int kLevels = kOzLevels;
constexpr int kConvWarps = 8;
constexpr int kFirstConvWarp = 2;
constexpr int kFirstOutWarp = kFirstConvWarp + kConvWarps;
constexpr int kOutWarps = 4;
constexpr int kThreads = (kFirstOutWarp + kOutWarps) * 32;
constexpr uint32_t kAccCols = kLevels * NT;         // one accumulator set
constexpr uint32_t kTmemCols = 512;

struct Bars {
  uint64_t xfull[kXSlots];   // TMA (transaction bytes)
  uint64_t xempty[kXSlots];  // converters (8 arrivals)
  uint64_t vfull[kStages];   // loader (transaction bytes of the V digits)
  uint64_t full[kStages];    // converters (8 arrivals)
  uint64_t empty[kStages];   // MMA completion
  uint64_t acc_full[2];
  uint64_t acc_empty[2];    // output warps (8 arrivals)
  uint64_t mma_done;
};

__device__ __forceinline__ int find_job(const OzModesJob* jobs, int njobs, int64_t item) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].item_base <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kThreads, 1)
    modes_oz_kernel(const OzModesJob* __restrict__ jobs, const CUtensorMap* __restrict__ maps, int njobs,
                    int64_t total_items, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  __shared__ Bars bars;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const tc::WaitBudget wb = tc::wait_budget(err);
  auto stage_a = [&](int s) -> uint8_t* { return smem + (size_t)s * kStageBytes; };
  auto stage_b = [&](int s) -> uint8_t* { return smem + (size_t)s * kStageBytes + kStageA; };

  if (tid == 0) {
    for (int s = 0; s < kXSlots; ++s) {
      tc::mbar_init(&bars.xfull[s], 1);
      tc::mbar_init(&bars.xempty[s], kConvWarps);
    }
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&bars.vfull[s], 1);
      tc::mbar_init(&bars.full[s], kConvWarps);
      tc::mbar_init(&bars.empty[s], 1);
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

  // Every role walks the same item sequence; `gk` counts 16-column stages over it.
  double* xs = reinterpret_cast<double*>(smem + (size_t)kStages * kStageBytes);
  if (warp == 0) {
    // ------------------------------------------------------------ loader: X tiles (TMA), V digits
    if (lane == 0) {
      int64_t gx = 0, gv = 0;  // X tiles and V stages issued
      int last_job = -1;
      for (int64_t it = blockIdx.x; it < total_items && !abort_flag; it += gridDim.x) {
        const int jb = find_job(jobs, njobs, it);
        const OzModesJob& J = jobs[jb];
        if (jb != last_job) {
          tc::tensormap_acquire(maps + jb);
          last_job = jb;
        }
        const int64_t local = it - J.item_base;
        const int row0 = (int)((local % J.row_tiles) * 128);
        const int nt = (int)(local / J.row_tiles);
        const uint8_t* vd = reinterpret_cast<const uint8_t*>(J.vdig);
        const int nst = (J.m + 15) / 16;
        bool ok = true;
        for (int k = 0; k < nst; ++k) {
          const int x = (int)(gx % kXSlots);
          if (gx >= kXSlots && !tc::mbar_wait(&bars.xempty[x], ((gx / kXSlots) - 1) & 1, &abort_flag, err, wb)) {
            ok = false;
            break;
          }
          tc::mbar_expect_tx(&bars.xfull[x], kXSlotBytes);
          tc::tma_load_2d(xs + (size_t)x * (kXSlotBytes / 8), maps + jb, row0, 16 * k, &bars.xfull[x]);
          ++gx;
          const int s = (int)(gv % kStages);
          if (gv >= kStages && !tc::mbar_wait(&bars.empty[s], ((gv / kStages) - 1) & 1, &abort_flag, err, wb)) {
            ok = false;
            break;
          }
          tc::mbar_expect_tx(&bars.vfull[s], kStageB);
#pragma unroll
          for (int q = 0; q < 2; ++q)
            tc::bulk_load(stage_b(s) + q * (kStageB / 2),
                          vd + ((int64_t)(2 * k + q) * J.n_tiles + nt) * (kStageB / 2), kStageB / 2,
                          &bars.vfull[s]);
          ++gv;
        }
        if (!ok) break;
      }
      // copies in flight must land before shared memory is released
      for (int64_t k = max((int64_t)0, gv - kStages); k < gv; ++k) {
        const long long t0 = clock64();
        while (!tc::mbar_try(&bars.vfull[k % kStages], (k / kStages) & 1) && clock64() - t0 < tc::kWaitBudget) {
        }
      }
      const int64_t gk = gx;
      for (int64_t k = max((int64_t)0, gk - kXSlots); k < gk; ++k) {
        const long long t0 = clock64();
        while (!tc::mbar_try(&bars.xfull[k % kXSlots], (k / kXSlots) & 1) && clock64() - t0 < tc::kWaitBudget) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ UMMA issuer
    if (lane == 0) {
      int64_t gk = 0;
      int uses[2] = {0, 0};  // K-blocks accumulated per accumulator set
      int kbg = 0;           // K-blocks so far: the sets alternate per 128-column block
      bool ok = true;
      for (int64_t it = blockIdx.x; it < total_items && ok; it += gridDim.x) {
        const OzModesJob& J = jobs[find_job(jobs, njobs, it)];
        const int nst = (J.m + 15) / 16;
        int b = 0;
        uint32_t acc = tbase;
        for (int k = 0; k < nst && ok; ++k, ++gk) {
          const int s = (int)(gk % kStages);
          const int pos = k % kKBlockStages;
          if (pos == 0) {
            b = kbg & 1;
            acc = tbase + (uint32_t)b * kAccCols;
          }
          if (pos == 0 && uses[b] > 0 &&
              !tc::mbar_wait(&bars.acc_empty[b], (uses[b] - 1) & 1, &abort_flag, err, wb)) {
            ok = false;
            break;
          }
          if (!tc::mbar_wait(&bars.vfull[s], (gk / kStages) & 1, &abort_flag, err, wb) ||
              !tc::mbar_wait(&bars.full[s], (gk / kStages) & 1, &abort_flag, err, wb)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t a0 = tc::smem_u32(stage_a(s)), b0 = tc::smem_u32(stage_b(s));
          // digit t of X against digits u0 .. u0 + len - 1 of V in one MMA: the B planes
          // are consecutive (N = 32 len) and so are the level accumulators t + u.
          // A (MN-major): LBO = column-group stride (K), SBO = padded row-group stride (M);
          // B (K-major): LBO = column-group stride (K), SBO = 128 (mode groups, then planes)
#pragma unroll
          for (int t = 1; t <= kOzDigits; ++t) {
#pragma unroll
            for (int u0 = 1; u0 <= kLevels + 1 - t; u0 += 4) {
              const int len = min(4, kLevels + 2 - t - u0);
              const uint32_t idesc = tc::idesc_f16_f32_major(128, NT * len, 1, 0);
              tc::umma_f16(acc + (uint32_t)((t + u0 - 2) * NT),
                            tc::ns_desc(a0 + (uint32_t)(t - 1) * 128u, kOzGroupBytes, kRowGroupBytes),
                            tc::ns_desc(b0 + (uint32_t)(u0 - 1) * (NT / 8) * 128u, kStageB / 2, 128u), idesc,
                            (pos == 0 && t == 1) ? 0u : 1u);
            }
          }
          tc::umma_commit(&bars.empty[s]);
          if (pos == kKBlockStages - 1 || k == nst - 1) {
            tc::umma_commit(&bars.acc_full[b]);
            ++uses[b];
            ++kbg;
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
    // warp cw: columns 2 cw, 2 cw + 1 of each stage; lane: rows 4 lane .. 4 lane + 3
    // (one 8-byte half of a 16-byte core-matrix row per digit plane and column).  The
    // job is copied to registers per item and the next stage's column exponents are
    // loaded before the current stage's wait, off the conversion's critical path.
    const int cw = warp - kFirstConvWarp;
    int64_t gk = 0;
    for (int64_t it = blockIdx.x; it < total_items && !abort_flag; it += gridDim.x) {
      const OzModesJob J = jobs[find_job(jobs, njobs, it)];
      const int nst = (J.m + 15) / 16;
      auto exps_of = [&](int k, int jj) -> int {
        const int j = 16 * k + 2 * cw + jj;
        return j < J.m ? __ldg(J.exps + j) : kOzNonFinite;
      };
      int En[2] = {exps_of(0, 0), exps_of(0, 1)};
      bool ok = true;
      for (int k = 0; k < nst; ++k, ++gk) {
        const int x = (int)(gk % kXSlots);
        const int s = (int)(gk % kStages);
        const int E[2] = {En[0], En[1]};
        if (k + 1 < nst) {
          En[0] = exps_of(k + 1, 0);
          En[1] = exps_of(k + 1, 1);
        }
        if (!tc::mbar_wait_warp(&bars.xfull[x], (gk / kXSlots) & 1, &abort_flag, err, wb)) {
          ok = false;
          break;
        }
        const double* xsl = xs + (size_t)x * (kXSlotBytes / 8);
        double v[2][4];
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int jl = 2 * cw + jj;
          const double2* src = reinterpret_cast<const double2*>(xsl + jl * 128 + 4 * lane);
          const double2 a = src[0], b2 = src[1];
          v[jj][0] = a.x;
          v[jj][1] = a.y;
          v[jj][2] = b2.x;
          v[jj][3] = b2.y;
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bars.xempty[x]);
        // digits of 4 consecutive rows, packed two fp16 per word
        uint32_t w[2][2][kOzDigits];
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (E[jj] != kOzNonFinite) {
              oz_digits2(v[jj][2 * h], v[jj][2 * h + 1], E[jj], w[jj][h]);
            } else {
#pragma unroll
              for (int q = 0; q < kOzDigits; ++q) w[jj][h][q] = 0u;
            }
          }
        }
        if (gk >= kStages && !tc::mbar_wait_warp(&bars.empty[s], ((gk / kStages) - 1) & 1, &abort_flag, err, wb)) {
          ok = false;
          break;
        }
        uint8_t* A = stage_a(s) + (lane >> 1) * kRowGroupBytes + (lane & 1) * 8;
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int jl = 2 * cw + jj;
          uint8_t* p = A + (jl >> 3) * kOzGroupBytes + (jl & 7) * 16;
#pragma unroll
          for (int q = 0; q < kOzDigits; ++q)
            *reinterpret_cast<uint2*>(p + q * 128) = make_uint2(w[jj][0][q], w[jj][1][q]);
        }
        tc::fence_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bars.full[s]);
      }
      if (!ok) break;
    }
  } else {
    // ------------------------------------------------------------ output
    // Per 128-column block: 8 modes at a time, the exact level sums -> FP64 (one
    // rounding); blocks after the first are added to the partial result in Y.
    const int q = warp & 3;
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    int uses[2] = {0, 0};
    int kbg = 0;
    for (int64_t it = blockIdx.x; it < total_items; it += gridDim.x) {
      // by value: the stores to Y must not force reloads of the job's fields
      const OzModesJob J = jobs[find_job(jobs, njobs, it)];
      const int64_t local = it - J.item_base;
      const int64_t rt = local % J.row_tiles;
      const int nt = (int)(local / J.row_tiles);
      const int nkb = ((J.m + 15) / 16 + kKBlockStages - 1) / kKBlockStages;
      const int64_t r = rt * 128 + 32 * q + lane;
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb, ++kbg) {
        const int b = kbg & 1;
        const uint32_t acc = tbase + lanes + (uint32_t)b * kAccCols;
        if (!tc::mbar_wait_warp(&bars.acc_full[b], uses[b] & 1, &abort_flag, err, wb)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const bool last = kb == nkb - 1;
        // mode chunks of 8 that hold a mode < k (the rest of the tile is padding)
        const int nc8 = min(NT / 8, (J.k - nt * NT + 7) / 8);
#pragma unroll 1
        for (int c8 = 0; c8 < nc8; ++c8) {
          const int col0 = nt * NT + 8 * c8;
          // the partial sums of the earlier blocks, the column exponents and scales are
          // loaded first, under the TMEM loads
          double yp[8], sc[8];
          int F[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const bool in = col0 + c < J.k;
            yp[c] = (kb > 0 && r < J.n && in) ? J.Y[(size_t)(col0 + c) * J.ldy + r] : 0.0;
            F[c] = in ? __ldg(J.fexp + col0 + c) : 0;
            sc[c] = (last && in && J.scale) ? __ldg(J.scale + col0 + c) : 1.0;
          }
          uint32_t lv8[kLevels][8];
#pragma unroll
          for (int lv = 0; lv < kLevels; ++lv) tc::tmem_ld8_raw(acc + (uint32_t)(lv * NT + 8 * c8), lv8[lv]);
          tc::tmem_wait_ld();
          long long hi[8], lo[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) hi[c] = lo[c] = 0;
#pragma unroll
          for (int lv = 0; lv < kLevels; ++lv) {
            tc::reg_barrier8(lv8[lv]);  // every use of the loaded registers after the wait
            const long long w = oz_level_weight(lv);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const long long xv = (long long)__float2int_rn(__uint_as_float(lv8[lv][c])) * w;
              if (lv < 3) hi[c] += xv; else lo[c] += xv;
            }
          }
          if (r < J.n) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const int col = col0 + c;
              if (col >= J.k) break;
              double v = F[c] == kOzNonFinite ? 0.0 : oz_combine(hi[c], lo[c], F[c] - 62);
              v += yp[c];
              if (last) v = F[c] == kOzNonFinite ? __longlong_as_double(0x7FF8000000000000ll) : v * sc[c];
              J.Y[(size_t)col * J.ldy + r] = v;
            }
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bars.acc_empty[b]);
        ++uses[b];
      }
      if (!__all_sync(0xffffffffu, ok && !abort_flag)) break;
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, kTmemCols);
}

// One block per mode column c (of kpad = 8 NG): F_c = max_j (E_j + e(V_jc)) with
// |V_jc| < 2^e(V_jc), then the digits of V_jc against 2^(F_c - E_j) into
// [column group j/8][32-mode tile c/32][digit][mode group (c%32)/8][c % 8][j % 8], so
// that consecutive digit planes of one tile form one K-major operand of up to 128
// modes.  Columns c >= k and rows j >= m are zero.  A non-finite X column (E_j
// marker) or V entry marks F_c.
__global__ void __launch_bounds__(256) oz_vsplit_kernel(const OzVSplitJob* __restrict__ jobs, int njobs) {
  const int64_t b = blockIdx.x;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].col_base <= b) lo = mid; else hi = mid - 1;
  }
  const OzVSplitJob J = jobs[lo];
  const int c = (int)(b - J.col_base);
  if (c >= J.NG * 8) return;
  __shared__ int fmax_sh;
  __shared__ int bad_sh;
  if (threadIdx.x == 0) {
    fmax_sh = INT_MIN;
    bad_sh = 0;
  }
  __syncthreads();
  const double* v = J.V + (size_t)c * J.ldv;
  if (c < J.k) {
    int f = INT_MIN, bad = 0;
    for (int j = threadIdx.x; j < J.m; j += blockDim.x) {
      const int E = J.exps[j];
      const double x = v[j];
      if (E == kOzNonFinite || !isfinite(x)) {
        bad = 1;
      } else if (x != 0.0) {
        int e;
        frexp(x, &e);
        f = max(f, E + e);
      }
    }
    if (bad) atomicExch(&bad_sh, 1);
    if (f != INT_MIN) atomicMax(&fmax_sh, f);
  }
  __syncthreads();
  const int F = bad_sh ? kOzNonFinite : (fmax_sh == INT_MIN ? 0 : fmax_sh);
  if (threadIdx.x == 0) J.fexp[c] = F;
  // digits: thread = 8 consecutive rows j of this column
  for (int g = threadIdx.x; g < J.CGp; g += blockDim.x) {
    uint32_t w[kOzDigits][4];
#pragma unroll
    for (int q = 0; q < kOzDigits; ++q) w[q][0] = w[q][1] = w[q][2] = w[q][3] = 0u;
    if (c < J.k && F != kOzNonFinite) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int j = 8 * g + r;
        const double x = j < J.m ? v[j] : 0.0;
        uint32_t d[kOzDigits];
        oz_digits(x, j < J.m ? F - J.exps[j] : 0, d);
#pragma unroll
        for (int q = 0; q < kOzDigits; ++q) w[q][r >> 1] |= d[q] << (16 * (r & 1));
      }
    }
    const int tiles = J.NG / (NT / 8);
    uint4* out = reinterpret_cast<uint4*>(J.vdig) + (((size_t)g * tiles + (c / NT)) * kOzDigits) * (NT / 8) * 8 +
                 ((c % NT) >> 3) * 8 + (c & 7);
#pragma unroll
    for (int q = 0; q < kOzDigits; ++q) out[q * (NT / 8) * 8] = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
  }
}

}  // namespace

int oz_modes_tile(int) { return NT; }

cudaError_t launch_modes_oz(const OzModesJob* jobs_dev, const CUtensorMap* maps_dev, int njobs, int64_t total_items,
                            int* err_flag, cudaStream_t s) {
  if (njobs <= 0 || total_items <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(modes_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int grid = (int)(total_items < kNumSMs ? total_items : kNumSMs);
  modes_oz_kernel<<<grid, kThreads, kSmemBytes, s>>>(jobs_dev, maps_dev, njobs, total_items, err_flag);
  return cudaGetLastError();
}

cudaError_t launch_oz_vsplit(const OzVSplitJob* jobs_dev, int njobs, int64_t total_cols, cudaStream_t s) {
  if (njobs <= 0 || total_cols <= 0) return cudaSuccess;
  if (total_cols > 0x7FFFFFFF) return cudaErrorInvalidValue;
  oz_vsplit_kernel<<<(unsigned)total_cols, 256, 0, s>>>(jobs_dev, njobs);
  return cudaGetLastError();
}

}  // namespace hapod
