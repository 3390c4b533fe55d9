// K1, mixed form: Gramian G = X^T X (Sec. 2, Remark def:method_of_snapshots)
// on the 5th-generation tensor cores (tcgen05, kind::tf32), for every node of a
// batch in one launch.
//
// Split: x = hi + lo with hi = x truncated to TF32 (what kind::tf32 reads from an
// FP32 word) and lo = x - hi (exact in FP32); the products hi*hi^T + hi*lo^T +
// lo*hi^T represent x_i x_j to ~2^-20 relative.  TMA writes each FP32 panel block
// (32 rows x 128 columns) in the 128-byte-swizzled K-major layout the UMMA reads,
// so hi needs no conversion; converter warps write lo at the same offsets.
//
// Work item = one 128 x 128 tile (ti <= tj) of one node's G over one row range.
// Items are ordered by row range first, so the tiles of one range run together and
// share their column panels through L2.  One CTA per item, 18 warps:
//   warp 0        TMA producer: 4-deep ring of hi blocks (32 rows of the ti and tj
//                 panels, as loaded)
//   warp 1        TMEM owner and single-thread UMMA issuer
//   warps 2..9    converters: lo = x - trunc(x) into a 2-deep lo ring
//   warps 10..17  flushers
// The tensor core's FP32 accumulation truncates (measured: ~0.85 ulp lost per
// accumulate step), so the accumulator restarts every kSegStages blocks (128 rows,
// 48 accumulate steps; the resulting bias is a near-uniform relative shrink of the
// segment sums) and the flushers add each finished segment into a Kahan-compensated
// FP32 pair (running sum s and compensation c) kept in the other half of TMEM; the
// item's compensated sum s - c is written in FP64 and splits are summed in FP64 by
// gram_reduce in a fixed order.  Every mbarrier wait is
// bounded: a timeout raises the error flag, the CTA drains its copies and MMAs and
// frees TMEM.
#include <vector>

#include "hapod_internal.cuh"
#include "tc_common.cuh"

namespace hapod {
namespace {

constexpr int kRowsPerStage = 32;                               // K per block (one 128-byte row)
constexpr int kPanelCols = 128;
constexpr int kBlockBytes = kRowsPerStage * kPanelCols * 4;     // 16 KB FP32 (hi as loaded)
constexpr int kPairBytes = 2 * kBlockBytes;                     // ti and tj panels
constexpr int kStages = 4;                                      // hi ring (TMA targets)
constexpr int kLoStages = 2;                                    // lo ring
constexpr int kSegStages = 4;                                   // blocks per TMEM accumulation
constexpr int kSmemBytes = (kStages + kLoStages) * kPairBytes + 1024;
constexpr int kThreads = 576;
constexpr int kConvThreads = 256;
constexpr int kFirstFlushWarp = 10;
// TMEM columns: [0,128) and [128,256) segment accumulators, [256,384) running sum s,
// [384,512) its TwoSum compensation c (all FP32, lane = tile row).
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kSumCol = 256;
constexpr uint32_t kCompCol = 384;

struct Bars {
  uint64_t full[kStages];     // TMA -> converters (transaction bytes)
  uint64_t cvt[kStages];      // converters -> issuer
  uint64_t empty[kStages];    // issuer (MMA completion) -> TMA: hi block free
  uint64_t lo_free[kLoStages];  // issuer (MMA completion) -> converters: lo block free
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t mma_done;
};

// lo = x - trunc_tf32(x) for one 16 KB block (1024 chunks of 16 bytes, same offsets)
__device__ __forceinline__ void make_lo(const float* __restrict__ hi, float* __restrict__ lo, int ct) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int c = ct + i * kConvThreads;
    const float4 x = reinterpret_cast<const float4*>(hi)[c];
    float4 l;
    l.x = x.x - __uint_as_float(__float_as_uint(x.x) & 0xFFFFE000u);
    l.y = x.y - __uint_as_float(__float_as_uint(x.y) & 0xFFFFE000u);
    l.z = x.z - __uint_as_float(__float_as_uint(x.z) & 0xFFFFE000u);
    l.w = x.w - __uint_as_float(__float_as_uint(x.w) & 0xFFFFE000u);
    reinterpret_cast<float4*>(lo)[c] = l;
  }
}

// Add the finished segment j (TMEM accumulator j % 2) into the running compensated
// pair (s, c) in TMEM for this warp's 32 lanes and columns 64 h .. 64 h + 63, then
// hand the accumulator back to the issuer.  Segment 0 initialises s and c.
__device__ __forceinline__ bool flush_segment(int j, uint32_t tbase, int q, int h, int lane, Bars& bars,
                                              volatile int* abort_flag, int* err, tc::WaitBudget wb) {
  const int b = j & 1;
  if (!tc::mbar_wait_warp(&bars.acc_full[b], (j >> 1) & 1, abort_flag, err, wb)) return false;
  tc::tc_fence_after();
  const uint32_t lanes = (uint32_t)(32 * q) << 16;
#pragma unroll 1
  for (int g = 0; g < 4; ++g) {
    const uint32_t col = (uint32_t)(64 * h + 16 * g);
    float v[16], sv[16], cv[16];
    tc::tmem_ld16(tbase + lanes + (uint32_t)b * 128u + col, v);
    if (j > 0) {
      tc::tmem_ld16(tbase + lanes + kSumCol + col, sv);
      tc::tmem_ld16(tbase + lanes + kCompCol + col, cv);
    }
    tc::tmem_wait_ld();
    if (j == 0) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        sv[i] = v[i];
        cv[i] = 0.f;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) tc::kahan_acc(sv[i], cv[i], v[i]);
    }
    tc::tmem_st16(tbase + lanes + kSumCol + col, sv);
    tc::tmem_st16(tbase + lanes + kCompCol + col, cv);
  }
  tc::tmem_wait_st();
  tc::tc_fence_before();
  __syncwarp();
  if (lane == 0) tc::mbar_arrive(&bars.acc_empty[b]);
  return true;
}

__global__ void __launch_bounds__(kThreads, 1)
    gram_tc_kernel(const GramJob* __restrict__ jobs, const CUtensorMap* __restrict__ maps, const int4* __restrict__ items,
                   double* __restrict__ partials, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ Bars bars;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  const int4 it = items[blockIdx.x];
  const GramJob J = jobs[it.x];
  const CUtensorMap* map = maps + it.x;
  const int ti = it.y, tj = it.z, sp = it.w;
  const bool diag = ti == tj;
  const int64_t r0 = (int64_t)sp * J.rows_per_split;
  const int64_t r1 = min(J.n, r0 + J.rows_per_split);
  const int nst = r1 > r0 ? (int)((r1 - r0 + kRowsPerStage - 1) / kRowsPerStage) : 0;
  const int nseg = (nst + kSegStages - 1) / kSegStages;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const tc::WaitBudget wb = tc::wait_budget(err);
  // hi ring slot s: [A hi | B hi]; lo ring slot t (after the hi ring): [A lo | B lo]; 16 KB each
  auto hi_blk = [&](int s, int panel) -> uint8_t* { return smem + (size_t)s * kPairBytes + (size_t)panel * kBlockBytes; };
  auto lo_blk = [&](int t, int panel) -> uint8_t* {
    return smem + (size_t)(kStages + t) * kPairBytes + (size_t)panel * kBlockBytes;
  };

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&bars.full[s], 1);
      tc::mbar_init(&bars.cvt[s], 8);
      tc::mbar_init(&bars.empty[s], 1);
    }
    for (int t = 0; t < kLoStages; ++t) tc::mbar_init(&bars.lo_free[t], 1);
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bars.acc_full[b], 1);
      tc::mbar_init(&bars.acc_empty[b], 8);
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
    // ------------------------------------------------------------ TMA producer
    if (lane == 0 && nst > 0) {
      tc::tensormap_acquire(map);
      const uint32_t bytes = diag ? kBlockBytes : kPairBytes;
      int issued = 0;
      for (int k = 0; k < nst; ++k) {
        const int s = k % kStages;
        if (k >= kStages && !tc::mbar_wait(&bars.empty[s], ((k / kStages) - 1) & 1, &abort_flag, err, wb)) break;
        tc::mbar_expect_tx(&bars.full[s], bytes);
        const int row = (int)(r0 + (int64_t)k * kRowsPerStage);
        tc::tma_load_2d(hi_blk(s, 0), map, row, ti * kPanelCols, &bars.full[s]);
        if (!diag) tc::tma_load_2d(hi_blk(s, 1), map, row, tj * kPanelCols, &bars.full[s]);
        issued = k + 1;
      }
      if (abort_flag) {
        // drain: copies in flight must land before the CTA's shared memory is released
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
      constexpr uint32_t idesc = tc::idesc_tf32_f32(128, 128);
      for (int k = 0; k < nst; ++k) {
        const int s = k % kStages;
        const int seg = k / kSegStages;
        const bool seg_first = (k % kSegStages) == 0;
        const bool seg_last = (k % kSegStages) == kSegStages - 1 || k == nst - 1;
        const int b = seg & 1;
        if (seg_first && seg >= 2 &&
            !tc::mbar_wait(&bars.acc_empty[b], ((seg >> 1) - 1) & 1, &abort_flag, err, wb))
          break;
        if (!tc::mbar_wait(&bars.cvt[s], (k / kStages) & 1, &abort_flag, err, wb)) break;
        tc::tc_fence_after();
        const int t = k % kLoStages;
        const uint32_t ah = tc::smem_u32(hi_blk(s, 0)), al = tc::smem_u32(lo_blk(t, 0));
        const uint32_t bh = diag ? ah : tc::smem_u32(hi_blk(s, 1)), bl = diag ? al : tc::smem_u32(lo_blk(t, 1));
        const uint32_t d = tbase + (uint32_t)b * 128u;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {  // K = 8 per tf32 MMA: 32 bytes of the 128-byte row
          const uint32_t off = kk * 32;
          tc::umma_tf32(d, tc::sw128_desc(ah + off), tc::sw128_desc(bh + off), idesc,
                        (seg_first && kk == 0) ? 0u : 1u);
          tc::umma_tf32(d, tc::sw128_desc(ah + off), tc::sw128_desc(bl + off), idesc, 1u);
          tc::umma_tf32(d, tc::sw128_desc(al + off), tc::sw128_desc(bh + off), idesc, 1u);
        }
        tc::umma_commit(&bars.empty[s]);
        tc::umma_commit(&bars.lo_free[t]);
        if (seg_last) tc::umma_commit(&bars.acc_full[b]);
      }
      // no MMA may be in flight when TMEM or shared memory is released
      tc::umma_commit(&bars.mma_done);
      const long long t0 = clock64();
      while (!tc::mbar_try(&bars.mma_done, 0) && clock64() - t0 < tc::kWaitBudget) {
      }
    }
  } else if (warp < kFirstFlushWarp) {
    // ------------------------------------------------------------ converters
    const int ct = tid - 64;
    for (int k = 0; k < nst; ++k) {
      const int s = k % kStages, t = k % kLoStages;
      if (!tc::mbar_wait_warp(&bars.full[s], (k / kStages) & 1, &abort_flag, err, wb)) break;
      if (k >= kLoStages && !tc::mbar_wait_warp(&bars.lo_free[t], ((k / kLoStages) - 1) & 1, &abort_flag, err, wb)) break;
      make_lo(reinterpret_cast<const float*>(hi_blk(s, 0)), reinterpret_cast<float*>(lo_blk(t, 0)), ct);
      if (!diag) make_lo(reinterpret_cast<const float*>(hi_blk(s, 1)), reinterpret_cast<float*>(lo_blk(t, 1)), ct);
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars.cvt[s]);
    }
  } else {
    // ------------------------------------------------------------ flushers + result
    const int q = warp & 3;                       // TMEM lane quarter this warp may access
    const int h = (warp - kFirstFlushWarp) >> 2;  // column half of the tile
    bool ok = true;
    for (int j = 0; j < nseg && ok; ++j) ok = flush_segment(j, tbase, q, h, lane, bars, &abort_flag, err, wb);
    if (__all_sync(0xffffffffu, ok && !abort_flag)) {
      const int a = 32 * q + lane;  // tile row
      const int gi = ti * kPanelCols + a;
      const uint32_t lanes = (uint32_t)(32 * q) << 16;
      // tile-major partial slot: J.item_base + (row-major upper-triangle index) * splits + split
      const int tile_idx = ti * J.tiles - ti * (ti - 1) / 2 + (tj - ti);
      double* out = J.splits == 1 ? nullptr
                                  : partials + ((size_t)J.item_base + (size_t)tile_idx * J.splits + sp) *
                                                   (kPanelCols * kPanelCols) +
                                        (size_t)a * kPanelCols;
#pragma unroll 1
      for (int g = 0; g < 4; ++g) {
        const int c0 = 64 * h + 16 * g;
        float sv[16], cv[16];
        if (nseg > 0) {
          tc::tmem_ld16(tbase + lanes + kSumCol + (uint32_t)c0, sv);
          tc::tmem_ld16(tbase + lanes + kCompCol + (uint32_t)c0, cv);
          tc::tmem_wait_ld();
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) sv[i] = cv[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const double v = (double)sv[i] - (double)cv[i];  // the compensated sum: c holds the excess of s
          if (out) {
            out[c0 + i] = v;
          } else {
            const int gj = tj * kPanelCols + c0 + i;
            if (gi < J.m && gj < J.m && gj >= gi) {  // one writer per symmetric pair (diagonal tiles)
              J.G[(size_t)gj * J.m + gi] = v;
              J.G[(size_t)gi * J.m + gj] = v;
            }
          }
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, kTmemCols);
}

}  // namespace

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  }
  return fn;
}

bool tma_compatible_f32(const void* base, int64_t ld) {
  return base && (reinterpret_cast<uintptr_t>(base) % 16 == 0) && (ld % 4 == 0);
}

bool encode_colmajor_f32(CUtensorMap* out, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                         int box_cols, bool swizzle128) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !tma_compatible_f32(base, ld) || rows < 1 || cols < 1) return false;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
  cuuint32_t es[2] = {1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tma_compatible_f64(const void* base, int64_t ld) {
  return base && (reinterpret_cast<uintptr_t>(base) % 16 == 0) && (ld % 2 == 0);
}

bool encode_colmajor_f64(CUtensorMap* out, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                         int box_cols) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !tma_compatible_f64(base, ld) || rows < 1 || cols < 1) return false;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
  cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
  cuuint32_t es[2] = {1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_oz_digits(CUtensorMap* out, const void* base, int32_t CGs, int64_t RG, int box_groups) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !base || reinterpret_cast<uintptr_t>(base) % 16 != 0 || CGs < 1 || RG < 2 || box_groups > 16) return false;
  // [row group][digit][column groups x 128 B], addressed in 8-byte units so that a box
  // row is box_groups whole column groups (up to 2 KB) of one digit plane
  cuuint64_t dims[3] = {(cuuint64_t)CGs * 16, (cuuint64_t)kOzDigits, (cuuint64_t)RG};
  cuuint64_t strides[2] = {(cuuint64_t)CGs * 128, (cuuint64_t)CGs * 128 * kOzDigits};
  cuuint32_t box[3] = {(cuuint32_t)box_groups * 16, (cuuint32_t)kOzDigits, 2};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int gram_tc_rows_per_stage() { return kRowsPerStage; }

cudaError_t launch_gram_tc(const GramJob* jobs_dev, const CUtensorMap* maps_dev, const int4* items_dev, int num_items,
                           const int4* reduce_dev, int num_reduce, double* partials, int* err_flag, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (num_items > 0)
    gram_tc_kernel<<<num_items, kThreads, kSmemBytes, s>>>(jobs_dev, maps_dev, items_dev, partials, err_flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gram_reduce(128, jobs_dev, reduce_dev, num_reduce, partials, s);
}

}  // namespace hapod
