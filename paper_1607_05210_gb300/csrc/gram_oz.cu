// K1, digit-slice FP64 form: G = X^T X (Sec. 2, Remark def:method_of_snapshots)
// from the exact digit planes of X (oz_split.cu) on the 5th-generation tensor cores
// (tcgen05 kind::f16, fp16 x fp16 -> FP32).
//
// With x_ri = 2^(E_i+1) sum_t d_t(r,i) 2^(-8t) (7 balanced base-256 digits),
//   G_ij = 2^(E_i + E_j + 2) sum_{s=2}^{8} 2^(-8 s) L_s(i, j),
//   L_s(i, j) = sum_r sum_{t+u=s} d_t(r,i) d_u(r,j),
// keeping the 28 digit pairs with t + u <= 8 (the dropped pairs weigh < 2^-57 of
// 2^(E_i + E_j) per row, below the truncation of the digits).  Over a block of 128
// rows every level sum is an integer below 7 * 2^21 < 2^24, so the FP32 tensor-core
// accumulation of digit products is exact; after each block the seven level
// accumulators are converted to integers and added exactly into two int64
// fixed-point sums per entry: hi = sum (L_2 2^16 + L_3 2^8 + L_4),
// lo = sum (L_5 2^24 + L_6 2^16 + L_7 2^8 + L_8), G_ij = 2^(E_i+E_j-62) (hi 2^32 + lo),
// rounded once to FP64.  The only rounding of the whole Gram is that final one and the FP64
// sum over row splits.
//
// Work item = one 128 x 64 tile (columns 128 I.. x 64 J..) over one row split.  A
// digit plane of a row group holds ceil(m / 8) column groups; a block that runs past
// them reads the next plane or the buffer's slack, which only reach tile rows /
// columns >= m, never written back.  One CTA per item, 18 warps:
//   warp 0       bulk-copy producer: 4-deep ring of 16-row stages (all 7 digit
//                planes of the 128 A columns and the 64 B columns, 42 KB; one copy
//                per row group and digit plane of each block)
//   warp 1       TMEM owner and single-thread UMMA issuer: per stage 10 MMAs
//                128 x (64..256) x 16, digit t of the A columns against up to 4
//                consecutive digits u of the B columns (consecutive planes form one
//                K-major operand; the level accumulators t + u are adjacent 64-column
//                blocks of TMEM): an MMA costs ~72 cycles at N = 64 and ~150 at
//                N = 256 (measured), so grouping the planes halves the issue time
//   warps 2..17  flushers: after every 128-row block, 16 columns x 32 lanes each
// Every mbarrier wait is bounded: a timeout raises the error flag, the CTA drains
// its copies and MMAs and frees TMEM.
#include "hapod_internal.cuh"
#include "oz_common.cuh"
#include "tc_common.cuh"

namespace hapod {
namespace {

constexpr int kAGroups = 16;                                  // column groups of the A block (128 columns)
constexpr int kBGroups = 8;                                   // column groups of the B block (64 columns)
constexpr int kPlaneA = kAGroups * 128;                       // one digit plane of one row group: 2 KB
constexpr int kPlaneB = kBGroups * 128;                       // 1 KB
constexpr int kStageA = 2 * kOzDigits * kPlaneA;              // [row group][digit][16 groups]: 28672 B
constexpr int kStageB = 2 * kOzDigits * kPlaneB;              // [row group][digit][8 groups]: 14336 B
constexpr int kStageBytes = kStageA + kStageB;
constexpr int kStages = 4;
constexpr int kSmemBytes = kStages * kStageBytes + 128;
constexpr int kBlockStages = kOzKBlock / 16;                  // stages per exact block
constexpr int kThreads = 576;
constexpr int kFirstFlushWarp = 2;
constexpr int kFlushWarps = 16;
constexpr int kLevels = kOzLevels;
constexpr uint32_t kLevelCols = 64;
constexpr uint32_t kTmemCols = 512;

struct Bars {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t acc_full;
  uint64_t acc_empty;
  uint64_t mma_done;
};

// tile index -> (I, J), J from 2 I up to ceil(m / 64) - 1
__device__ __forceinline__ void tile_of(int tile, int m, int* I, int* J) {
  const int jmax = (m + 63) / 64;
  int i = 0;
  for (;; ++i) {
    const int cnt = jmax - 2 * i;
    if (cnt <= 0 || tile < cnt) break;
    tile -= cnt;
  }
  *I = i;
  *J = 2 * i + tile;
}

__global__ void __launch_bounds__(kThreads, 1) gram_oz_kernel(const OzGramJob* __restrict__ jobs, int njobs, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  __shared__ Bars bars;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  const int64_t b = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
  int jlo = 0, jhi = njobs - 1;
  while (jlo < jhi) {
    const int mid = (jlo + jhi + 1) >> 1;
    if (jobs[mid].item_base <= b) jlo = mid; else jhi = mid - 1;
  }
  const OzGramJob J = jobs[jlo];
  const int64_t local = b - J.item_base;
  if (local >= (int64_t)J.splits * J.tiles) return;  // whole CTA leaves before any barrier
  const int sp = (int)(local / J.tiles);
  int TI, TJ;
  tile_of((int)(local % J.tiles), J.m, &TI, &TJ);
  const int total_stages = J.RG / 2;
  const int st0 = sp * J.stages_per_split;
  const int nst = max(0, min(total_stages - st0, J.stages_per_split));
  const int nkb = (nst + kBlockStages - 1) / kBlockStages;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto stage_a = [&](int s) -> uint8_t* { return smem + (size_t)s * kStageBytes; };
  auto stage_b = [&](int s) -> uint8_t* { return smem + (size_t)s * kStageBytes + kStageA; };

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&bars.full[s], 1);
      tc::mbar_init(&bars.empty[s], 1);
    }
    tc::mbar_init(&bars.acc_full, 1);
    tc::mbar_init(&bars.acc_empty, kFlushWarps);
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
    // ------------------------------------------------------------ producer
    if (lane == 0 && nst > 0) {
      const uint8_t* base = reinterpret_cast<const uint8_t*>(J.digits);
      int issued = 0;
      for (int k = 0; k < nst; ++k) {
        const int s = k % kStages;
        if (k >= kStages && !tc::mbar_wait(&bars.empty[s], ((k / kStages) - 1) & 1, &abort_flag, err)) break;
        tc::mbar_expect_tx(&bars.full[s], kStageBytes);
        const int64_t rg0 = 2 * (int64_t)(st0 + k);
        const int64_t plane_bytes = (int64_t)J.CGs * 128;  // one digit plane of one row group
#pragma unroll
        for (int q = 0; q < 2; ++q) {
#pragma unroll
          for (int p = 0; p < kOzDigits; ++p) {
            // the A / B blocks may run past the stored groups (into the next plane / slack)
            const uint8_t* row = base + ((rg0 + q) * kOzDigits + p) * plane_bytes;
            tc::bulk_load(stage_a(s) + (q * kOzDigits + p) * kPlaneA, row + (int64_t)kPlaneA * TI, kPlaneA,
                          &bars.full[s]);
            tc::bulk_load(stage_b(s) + (q * kOzDigits + p) * kPlaneB, row + (int64_t)kPlaneB * TJ, kPlaneB,
                          &bars.full[s]);
          }
        }
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
    // ------------------------------------------------------------ UMMA issuer
    if (lane == 0) {
      for (int k = 0; k < nst; ++k) {
        const int s = k % kStages;
        const int pos = k % kBlockStages;
        if (pos == 0 && k > 0 && !tc::mbar_wait(&bars.acc_empty, ((k / kBlockStages) - 1) & 1, &abort_flag, err))
          break;
        if (!tc::mbar_wait(&bars.full[s], (k / kStages) & 1, &abort_flag, err)) break;
        tc::tc_fence_after();
        const uint32_t a0 = tc::smem_u32(stage_a(s)), b0 = tc::smem_u32(stage_b(s));
        // A (digit t): LBO = row-group stride (K), SBO = 128 (column groups, M).
        // B (digits u0 .. u0 + len - 1): LBO = row-group stride, SBO = 128 (column
        // groups of one digit, then of the next: N = 64 len).
#pragma unroll
        for (int t = 1; t <= kOzDigits; ++t) {
#pragma unroll
          for (int u0 = 1; u0 <= kLevels + 1 - t; u0 += 4) {
            const int len = min(4, kLevels + 2 - t - u0);
            const uint32_t idesc = tc::idesc_f16_f32_major(128, kLevelCols * len, 0, 0);
            tc::umma_f16(tbase + (uint32_t)(t + u0 - 2) * kLevelCols,
                         tc::ns_desc(a0 + (uint32_t)(t - 1) * kPlaneA, kOzDigits * kPlaneA, 128u),
                         tc::ns_desc(b0 + (uint32_t)(u0 - 1) * kPlaneB, kOzDigits * kPlaneB, 128u), idesc,
                         (pos == 0 && t == 1) ? 0u : 1u);
          }
        }
        tc::umma_commit(&bars.empty[s]);
        if (pos == kBlockStages - 1 || k == nst - 1) tc::umma_commit(&bars.acc_full);
      }
      tc::umma_commit(&bars.mma_done);
      const long long t0 = clock64();
      while (!tc::mbar_try(&bars.mma_done, 0) && clock64() - t0 < tc::kWaitBudget) {
      }
    }
  } else {
    // ------------------------------------------------------------ flushers + result
    const int q = warp & 3;                          // TMEM lane quarter
    const int cw = (warp - kFirstFlushWarp) >> 2;    // 16-column slice of the 64-column tile
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    long long hi[16], lo[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0;
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      if (!tc::mbar_wait_warp(&bars.acc_full, kb & 1, &abort_flag, err)) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
#pragma unroll
      for (int lv = 0; lv < kLevels; ++lv) {
        float v[16];
        tc::tmem_ld16(tbase + lanes + (uint32_t)lv * kLevelCols + (uint32_t)(16 * cw), v);
        tc::tmem_wait_ld();
        const long long w = oz_level_weight(lv);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const long long x = (long long)__float2int_rn(v[c]) * w;
          if (lv < 3) hi[c] += x; else lo[c] += x;
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars.acc_empty);
    }
    if (__all_sync(0xffffffffu, ok && !abort_flag)) {
      const int mp = J.mp;
      const int i = 128 * TI + 32 * q + lane;
      const int Ei = i < J.m ? J.exps[i] : 0;
      double* out = J.partial + (size_t)sp * mp * mp;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int j = 64 * TJ + 16 * cw + c;
        if (i < J.m && j < J.m) {  // rows / columns past m come from slack digits
          const int Ej = J.exps[j];
          double v;
          if (Ei == kOzNonFinite || Ej == kOzNonFinite)
            v = __longlong_as_double(0x7FF8000000000000ll);
          else
            v = oz_combine(hi[c], lo[c], Ei + Ej - 62);
          out[(size_t)j * mp + i] = v;
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, kTmemCols);
}

// One block per column j of one node: G[:, j] and G[j, :] from the upper triangle
// (rows i <= j) of the partial slots, summed in slot order.
__global__ void __launch_bounds__(256) oz_reduce_kernel(const OzReduceJob* __restrict__ jobs, int njobs) {
  const int64_t b = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].col_base <= b) lo = mid; else hi = mid - 1;
  }
  const OzReduceJob J = jobs[lo];
  const int64_t j = b - J.col_base;
  if (j >= J.m) return;
  const size_t slot = (size_t)J.mp * J.mp;
  for (int64_t i = threadIdx.x; i <= j; i += blockDim.x) {
    const double* p = J.partial + (size_t)j * J.mp + i;
    double s = 0.0;
    for (int k = 0; k < J.slots; ++k) s += p[k * slot];
    J.G[(size_t)j * J.m + i] = s;
    J.G[(size_t)i * J.m + j] = s;
  }
}

dim3 grid_for(int64_t blocks) {
  const int64_t gx = blocks < 65535 ? blocks : 65535;
  return dim3((unsigned)gx, (unsigned)((blocks + gx - 1) / gx));
}

}  // namespace

int oz_gram_tiles(int32_t m) {
  const int jmax = (m + 63) / 64;
  int n = 0;
  for (int i = 0; 2 * i < jmax; ++i) n += jmax - 2 * i;
  return n;
}

cudaError_t launch_gram_oz(const OzGramJob* jobs_dev, int njobs, int64_t total_items, int* err_flag, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gram_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (njobs <= 0 || total_items <= 0) return cudaSuccess;
  gram_oz_kernel<<<grid_for(total_items), kThreads, kSmemBytes, s>>>(jobs_dev, njobs, err_flag);
  return cudaGetLastError();
}

cudaError_t launch_oz_reduce(const OzReduceJob* jobs_dev, int njobs, int64_t total_cols, cudaStream_t s) {
  if (njobs <= 0 || total_cols <= 0) return cudaSuccess;
  oz_reduce_kernel<<<grid_for(total_cols), 256, 0, s>>>(jobs_dev, njobs);
  return cudaGetLastError();
}

}  // namespace hapod
