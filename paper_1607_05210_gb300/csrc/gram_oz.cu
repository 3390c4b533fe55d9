// K1, digit-slice FP64 form: G = X^T X (Sec. 2, Remark def:method_of_snapshots)
// from the exact digit planes of X (oz_split.cu) on the 5th-generation tensor cores
// (tcgen05 kind::f16, fp16 x fp16 -> FP32).
//
// With x_ri = 2^(E_i+1) sum_t d_t(r,i) 2^(-8t) (7 balanced base-256 digits),
//   G_ij = 2^(E_i + E_j + 2) sum_{s=2}^{8} 2^(-8 s) L_s(i, j),
//   L_s(i, j) = sum_r sum_{t+u=s} d_t(r,i) d_u(r,j),
// keeping the 28 digit pairs with t + u <= 8.  The dropped pairs weigh at most
// 6.02 * 2^(E_i + E_j - 56) per row (the six level-9 pairs of digits in [-128, 127]);
// with the digit truncation, 2^(E_i + E_j - 54), a row's product is off by less than
// 1.26 * 2^(E_i + E_j - 53).  Over a block of 128 rows every level sum is an integer
// below 7 * 2^21 < 2^24, so the FP32 tensor-core accumulation of digit products is
// exact; after each block the seven level accumulators are converted to integers and
// added exactly into two int64 fixed-point sums per entry:
//   hi = sum (L_2 2^16 + L_3 2^8 + L_4),   lo = sum (L_5 2^24 + L_6 2^16 + L_7 2^8 + L_8),
//   G_ij = 2^(E_i + E_j - 62) (hi 2^32 + lo), rounded once to FP64 per row split;
// the splits are summed in FP64 (oz_reduce_kernel).
//
// Work item = one 128 x 32 tile (columns 128 I.. x 32 J..) over one row split.  A
// digit plane of a row group holds ceil(m / 8) column groups; tile rows / columns
// >= m are never written back.  One CTA per item, 18 warps:
//   warp 0       TMA producer: 6-deep ring of 16-row stages (all 7 digit planes of
//                the 128 A columns and the 32 B columns, 35 KB) in two 3-D tensor
//                copies per stage (one per block: 2 row groups x 7 digits x one run
//                of whole column groups); column groups past the stored ones read
//                as zero
//   warp 1       TMEM owner and single-thread UMMA issuer: per stage 7 MMAs
//                128 x 32 (8 - t) x 16, digit t of the A columns against the digits
//                u = 1 .. 8 - t of the B columns (consecutive planes form one K-major
//                operand; the level accumulators t + u are adjacent 32-column blocks of
//                TMEM).  Two sets of the seven level accumulators (2 x 224 columns)
//                alternate between 128-row blocks, so the flush of one block runs
//                under the MMAs of the next.
//   warps 2..17  flushers: after every 128-row block, 8 columns x 32 lanes each
// (18 warps put 5 on two of the four SM sub-partitions, whose 16K registers cap a
// thread at 96).
#include "hapod_internal.cuh"
#include "oz_common.cuh"
#include "tc_common.cuh"

namespace hapod {
namespace {

constexpr int kAGroups = kOzGramAGroups;                      // column groups of the A block (128 columns)
constexpr int kBGroups = kOzGramBGroups;                      // column groups of the B block (32 columns)
constexpr int kPlaneA = kAGroups * 128;                       // one digit plane of one row group: 2 KB
constexpr int kPlaneB = kBGroups * 128;                       // 512 B
constexpr int kStageA = 2 * kOzDigits * kPlaneA;              // [row group][digit][16 groups]: 28672 B
constexpr int kStageB = 2 * kOzDigits * kPlaneB;              // [row group][digit][4 groups]: 7168 B
constexpr int kStageBytes = kStageA + kStageB;
constexpr int kStages = 6;
constexpr int kSmemBytes = kStages * kStageBytes + 128;
constexpr int kBlockStages = kOzKBlock / 16;                  // stages per exact block
constexpr int kThreads = 576;
constexpr int kFirstFlushWarp = 2;
constexpr int kFlushWarps = 16;
constexpr int kLevels = kOzLevels;
constexpr int kTileCols = kBGroups * 8;                       // 32
constexpr uint32_t kLevelCols = kTileCols;
constexpr uint32_t kSetCols = kLevels * kLevelCols;           // 224: one set of level accumulators
constexpr uint32_t kTmemCols = 512;
constexpr int kFlushCols = kTileCols / 4;                     // columns per flusher warp
static_assert(2 * kSetCols <= kTmemCols, "two accumulator sets must fit in TMEM");
static_assert(kSmemBytes <= 227 * 1024, "shared memory");

struct Bars {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t mma_done;
};

constexpr int kJPerI = 128 / kTileCols;  // B blocks per A block

// tile index -> (I, J), J from 4 I up to ceil(m / 32) - 1
__device__ __forceinline__ void tile_of(int tile, int m, int* I, int* J) {
  const int jmax = (m + kTileCols - 1) / kTileCols;
  int i = 0;
  for (;; ++i) {
    const int cnt = jmax - kJPerI * i;
    if (cnt <= 0 || tile < cnt) break;
    tile -= cnt;
  }
  *I = i;
  *J = kJPerI * i + tile;
}

__global__ void __launch_bounds__(kThreads, 1) gram_oz_kernel(const OzGramJob* __restrict__ jobs, const CUtensorMap* __restrict__ maps, int njobs, int* err) {
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
  const tc::WaitBudget wb = tc::wait_budget(err);
  auto stage_a = [&](int s) -> uint8_t* { return smem + (size_t)s * kStageBytes; };
  auto stage_b = [&](int s) -> uint8_t* { return smem + (size_t)s * kStageBytes + kStageA; };

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&bars.full[s], 1);
      tc::mbar_init(&bars.empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&bars.acc_full[a], 1);
      tc::mbar_init(&bars.acc_empty[a], kFlushWarps);
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
    // ------------------------------------------------------------ producer
    if (lane == 0 && nst > 0) {
      const CUtensorMap* mapA = maps + 2 * jlo;
      const CUtensorMap* mapB = mapA + 1;
      tc::tensormap_acquire(mapA);
      tc::tensormap_acquire(mapB);
      int issued = 0;
      for (int k = 0; k < nst; ++k) {
        const int s = k % kStages;
        if (k >= kStages && !tc::mbar_wait(&bars.empty[s], ((k / kStages) - 1) & 1, &abort_flag, err, wb)) break;
        tc::mbar_expect_tx(&bars.full[s], kStageBytes);
        const int rg0 = 2 * (st0 + k);
        tc::tma_load_3d(stage_a(s), mapA, 16 * kAGroups * TI, 0, rg0, &bars.full[s]);
        tc::tma_load_3d(stage_b(s), mapB, 16 * kBGroups * TJ, 0, rg0, &bars.full[s]);
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
        const int kb = k / kBlockStages;
        const int set = kb & 1;
        if (pos == 0 && kb >= 2 && !tc::mbar_wait(&bars.acc_empty[set], ((kb >> 1) - 1) & 1, &abort_flag, err, wb))
          break;
        if (!tc::mbar_wait(&bars.full[s], (k / kStages) & 1, &abort_flag, err, wb)) break;
        tc::tc_fence_after();
        const uint32_t a0 = tc::smem_u32(stage_a(s)), b0 = tc::smem_u32(stage_b(s));
        const uint32_t acc = tbase + (uint32_t)set * kSetCols;
        // A (digit t): LBO = row-group stride (K), SBO = 128 (column groups, M).
        // B (digits 1 .. 8 - t): LBO = row-group stride, SBO = 128 (column groups of
        // one digit, then of the next: N = 32 (8 - t)); D = levels t + 1 .. 8.
#pragma unroll
        for (int t = 1; t <= kOzDigits; ++t) {
          const uint32_t idesc = tc::idesc_f16_f32_major(128, kLevelCols * (kLevels + 1 - t), 0, 0);
          tc::umma_f16(acc + (uint32_t)(t - 1) * kLevelCols,
                       tc::ns_desc(a0 + (uint32_t)(t - 1) * kPlaneA, kOzDigits * kPlaneA, 128u),
                       tc::ns_desc(b0, kOzDigits * kPlaneB, 128u), idesc, (pos == 0 && t == 1) ? 0u : 1u);
        }
        tc::umma_commit(&bars.empty[s]);
        if (pos == kBlockStages - 1 || k == nst - 1) tc::umma_commit(&bars.acc_full[set]);
      }
      tc::umma_commit(&bars.mma_done);
      const long long t0 = clock64();
      while (!tc::mbar_try(&bars.mma_done, 0) && clock64() - t0 < tc::kWaitBudget) {
      }
    }
  } else {
    // ------------------------------------------------------------ flushers + result
    const int q = warp & 3;                          // TMEM lane quarter
    const int cw = (warp - kFirstFlushWarp) >> 2;    // 8-column slice of the 32-column tile
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    long long hi[kFlushCols], lo[kFlushCols];
#pragma unroll
    for (int c = 0; c < kFlushCols; ++c) hi[c] = lo[c] = 0;
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      const int set = kb & 1;
      if (!tc::mbar_wait_warp(&bars.acc_full[set], (kb >> 1) & 1, &abort_flag, err, wb)) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
      // all seven levels in flight at once, then one wait
      uint32_t r[kLevels][kFlushCols];
      const uint32_t col = tbase + lanes + (uint32_t)set * kSetCols + (uint32_t)(kFlushCols * cw);
#pragma unroll
      for (int lv = 0; lv < kLevels; ++lv) tc::tmem_ld8_raw(col + (uint32_t)lv * kLevelCols, r[lv]);
      tc::tmem_wait_ld();
#pragma unroll
      for (int lv = 0; lv < kLevels; ++lv) {
        tc::reg_barrier8(r[lv]);  // keep every use of the loaded registers after the wait
        const long long w = oz_level_weight(lv);
#pragma unroll
        for (int c = 0; c < kFlushCols; ++c) {
          const long long x = (long long)__float2int_rn(__uint_as_float(r[lv][c])) * w;
          if (lv < 3) hi[c] += x; else lo[c] += x;
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars.acc_empty[set]);
    }
    if (__all_sync(0xffffffffu, ok && !abort_flag)) {
      const int mp = J.mp;
      const int i = 128 * TI + 32 * q + lane;
      const int Ei = i < J.m ? J.exps[i] : 0;
      double* out = J.partial + (size_t)sp * mp * mp;
#pragma unroll
      for (int c = 0; c < kFlushCols; ++c) {
        const int j = kTileCols * TJ + kFlushCols * cw + c;
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
  const int jmax = (m + kTileCols - 1) / kTileCols;
  int n = 0;
  for (int i = 0; kJPerI * i < jmax; ++i) n += jmax - kJPerI * i;
  return n;
}

cudaError_t launch_gram_oz(const OzGramJob* jobs_dev, const CUtensorMap* maps_dev, int njobs, int64_t total_items,
                           int* err_flag, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gram_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (njobs <= 0 || total_items <= 0) return cudaSuccess;
  gram_oz_kernel<<<grid_for(total_items), kThreads, kSmemBytes, s>>>(jobs_dev, maps_dev, njobs, err_flag);
  return cudaGetLastError();
}

cudaError_t launch_oz_reduce(const OzReduceJob* jobs_dev, int njobs, int64_t total_cols, cudaStream_t s) {
  if (njobs <= 0 || total_cols <= 0) return cudaSuccess;
  oz_reduce_kernel<<<grid_for(total_cols), 256, 0, s>>>(jobs_dev, njobs);
  return cudaGetLastError();
}

}  // namespace hapod
