// K1, split-BF16 mixed form: Gramian G = X^T X (Sec. 2, Remark
// def:method_of_snapshots) of FP32 snapshots on the 5th-generation tensor cores
// (tcgen05, kind::f16 with bf16 operands), for every node of a batch in one launch.
//
// Split: every FP32 value is written exactly as x = b1 + b2 + b3 + r, b_p bf16
// (round to nearest at each step, b1 = bf16(x), b2 = bf16(x - b1), b3 = bf16(x - b1
// - b2)), |r| <= 2^-27 |x|.  The six products whose levels add to at most 2 --
// b1 b1, b1 b2, b2 b1, b2 b2, b1 b3, b3 b1 -- are formed on the tensor cores (each
// product of two bf16 values is exact in FP32); the dropped ones are below
// 2^-26 |x_i x_j| and of random sign.  The squared condition number of the Gram
// matrix (footnote of the method-of-snapshots remark) is what makes the split
// necessary: a single bf16 or TF32 product leaves errors of 2^-8 or 2^-11 of
// x_i x_j, far above the tail sums the truncation compares with eps^2.
//
// Accumulation: the FP32 tensor-core accumulator truncates at every step, so it
// restarts every kSegStages stages (64 rows, 24 MMAs) and each finished segment is
// added into a compensated FP32 pair (running sum s, compensation c, TwoSum) kept in
// TMEM; the item's compensated sum s - c is written in FP64 and row splits are summed in FP64 by
// gram_reduce in a fixed order.  GB300 runs FP64 at 1/64 of the FP32 rate, so the
// per-segment additions stay in FP32 pairs, whose 2^-44 relative resolution is far
// below the accumulation error of the segments themselves.
//
// Work item = one 128 x 128 tile (ti <= tj) of one node's G over one row range; items
// are ordered by row range first so that the tiles of one range share their panels
// through L2.  One CTA per item, 18 warps:
//   warp 0        TMA producer: FP32 panel blocks of 32 rows x 128 columns (128-byte
//                 swizzled), 6 deep (diagonal tile) or 3 deep (two panels)
//   warp 1        TMEM owner and single-thread MMA issuer
//   warps 2..9    converters: FP32 block -> the three bf16 pieces, written as K-major
//                 8 x 8 core matrices (no swizzle), 4 deep (diagonal) or 2 deep
//   warps 10..17  flushers
// Every mbarrier wait is bounded: a timeout raises the error flag, the CTA drains
// its copies and MMAs and frees TMEM.
#include <cuda_bf16.h>

#include <vector>

#include "hapod_internal.cuh"
#include "tc_common.cuh"

namespace hapod {
namespace {

constexpr int kRows = 32;                              // rows (K) per stage
constexpr int kPanel = 128;                            // columns per panel
constexpr int kStageBytes = kRows * kPanel * 4;        // FP32 block of one panel, 16 KB
constexpr int kPieceBytes = kRows * kPanel * 2;        // one bf16 piece of one panel, 8 KB
constexpr int kOpBytes = 3 * kPieceBytes;              // the three pieces of one panel, 24 KB
constexpr int kRingBytes = 96 * 1024;                  // staging ring and operand ring, each
constexpr int kMaxSt = kRingBytes / kStageBytes;       // 6 staging slots (diagonal tiles)
constexpr int kMaxOp = kRingBytes / kOpBytes;          // 4 operand slots (diagonal tiles)
constexpr int kSegStages = 2;                          // stages per TMEM accumulation (64 rows)
constexpr int kSmemBytes = 2 * kRingBytes + 1024;
constexpr int kThreads = 576;
constexpr int kConvThreads = 256;
constexpr int kFirstFlushWarp = 10;
// Core-matrix layout of a piece: column group (8 columns) g_c, row octet g_r:
// offset g_c * kSbo + g_r * kLbo, 16 bytes per column inside the core matrix.
constexpr uint32_t kLbo = 128;                         // next core matrix along K (8 rows)
constexpr uint32_t kSbo = (kRows / 8) * 128;           // next core matrix along M/N (8 columns)
// TMEM: [0,128) and [128,256) segment accumulators, [256,384) running sum s,
// [384,512) its compensation c (FP32, lane = tile row).
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kSumCol = 256;
constexpr uint32_t kCompCol = 384;

struct Bars {
  uint64_t full[kMaxSt];     // TMA -> converters (transaction bytes)
  uint64_t st_free[kMaxSt];  // converters -> TMA: staging slot read
  uint64_t op_full[kMaxOp];  // converters -> issuer
  uint64_t op_free[kMaxOp];  // issuer (MMA completion) -> converters
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t mma_done;
};

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// Split 8 consecutive rows of one column into the three bf16 pieces (8 values each,
// row order = ascending address).
__device__ __forceinline__ void split8(const float (&x)[8], uint4& p1, uint4& p2, uint4& p3) {
  uint32_t w1[4], w2[4], w3[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float a = x[2 * i], b = x[2 * i + 1];
    w1[i] = bf16x2(a, b);
    const float ra = a - bf_lo(w1[i]), rb = b - bf_hi(w1[i]);  // exact
    w2[i] = bf16x2(ra, rb);
    const float sa = ra - bf_lo(w2[i]), sb = rb - bf_hi(w2[i]);  // exact
    w3[i] = bf16x2(sa, sb);
  }
  p1 = make_uint4(w1[0], w1[1], w1[2], w1[3]);
  p2 = make_uint4(w2[0], w2[1], w2[2], w2[3]);
  p3 = make_uint4(w3[0], w3[1], w3[2], w3[3]);
}

// One panel's FP32 block (128-byte swizzled: the 16-byte chunk j of column c sits at
// c * 128 + ((j ^ (c % 8)) * 16)) -> its three pieces.  Thread ct handles the units
// (column c, row octet g) with c = u % 128, g = u / 128, u = ct and ct + 256: eight
// consecutive threads take eight consecutive columns of one octet, so both the reads
// (chunks 2g, 2g + 1 xor c % 8) and the writes (16 bytes at c % 8 of a core matrix)
// hit eight different bank groups.
__device__ __forceinline__ void convert_panel(const uint8_t* __restrict__ st, uint8_t* __restrict__ op, int ct) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int u = ct + h * kConvThreads;
    const int c = u & (kPanel - 1), g = u >> 7;
    const float4 v0 = *reinterpret_cast<const float4*>(st + c * 128 + (((2 * g) ^ (c & 7)) << 4));
    const float4 v1 = *reinterpret_cast<const float4*>(st + c * 128 + (((2 * g + 1) ^ (c & 7)) << 4));
    const float x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    uint4 p1, p2, p3;
    split8(x, p1, p2, p3);
    const uint32_t off = (uint32_t)(c >> 3) * kSbo + (uint32_t)g * kLbo + (uint32_t)(c & 7) * 16;
    *reinterpret_cast<uint4*>(op + off) = p1;
    *reinterpret_cast<uint4*>(op + kPieceBytes + off) = p2;
    *reinterpret_cast<uint4*>(op + 2 * kPieceBytes + off) = p3;
  }
}

// Add the finished segment j (TMEM accumulator j % 2) into the compensated pair
// (s, c) in TMEM for this warp's 32 lanes and columns 64 h .. 64 h + 63, then hand
// the accumulator back to the issuer.  Segment 0 initialises s and c.
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
    gram_bf3_kernel(const GramJob* __restrict__ jobs, const CUtensorMap* __restrict__ maps,
                    const int4* __restrict__ items, double* __restrict__ partials, int* err) {
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
  const int panels = diag ? 1 : 2;
  const int n_st = diag ? kMaxSt : kMaxSt / 2;  // staging slots (one slot = all panels of a stage)
  const int n_op = diag ? kMaxOp : kMaxOp / 2;  // operand slots
  const int64_t r0 = (int64_t)sp * J.rows_per_split;
  const int64_t r1 = min(J.n, r0 + J.rows_per_split);
  const int nst = r1 > r0 ? (int)((r1 - r0 + kRows - 1) / kRows) : 0;
  const int nseg = (nst + kSegStages - 1) / kSegStages;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const tc::WaitBudget wb = tc::wait_budget(err);
  uint8_t* st_ring = smem;
  uint8_t* op_ring = smem + kRingBytes;
  auto st_blk = [&](int s, int panel) -> uint8_t* { return st_ring + (size_t)(s * panels + panel) * kStageBytes; };
  auto op_blk = [&](int t, int panel) -> uint8_t* { return op_ring + (size_t)(t * panels + panel) * kOpBytes; };

  if (tid == 0) {
    for (int s = 0; s < kMaxSt; ++s) {
      tc::mbar_init(&bars.full[s], 1);
      tc::mbar_init(&bars.st_free[s], 8);
    }
    for (int t = 0; t < kMaxOp; ++t) {
      tc::mbar_init(&bars.op_full[t], 8);
      tc::mbar_init(&bars.op_free[t], 1);
    }
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
      const uint32_t bytes = (uint32_t)(panels * kStageBytes);
      int issued = 0;
      for (int k = 0; k < nst; ++k) {
        const int s = k % n_st;
        if (k >= n_st && !tc::mbar_wait(&bars.st_free[s], ((k / n_st) - 1) & 1, &abort_flag, err, wb)) break;
        tc::mbar_expect_tx(&bars.full[s], bytes);
        const int row = (int)(r0 + (int64_t)k * kRows);
        tc::tma_load_2d(st_blk(s, 0), map, row, ti * kPanel, &bars.full[s]);
        if (!diag) tc::tma_load_2d(st_blk(s, 1), map, row, tj * kPanel, &bars.full[s]);
        issued = k + 1;
      }
      if (abort_flag) {
        // drain: copies in flight must land before the CTA's shared memory is released
        for (int k = max(0, issued - n_st); k < issued; ++k) {
          const long long t0 = clock64();
          while (!tc::mbar_try(&bars.full[k % n_st], (k / n_st) & 1) && clock64() - t0 < tc::kWaitBudget) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32_major(128, 128, 0, 0);
      for (int k = 0; k < nst; ++k) {
        const int t = k % n_op;
        const int seg = k / kSegStages;
        const bool seg_first = (k % kSegStages) == 0;
        const bool seg_last = (k % kSegStages) == kSegStages - 1 || k == nst - 1;
        const int b = seg & 1;
        if (seg_first && seg >= 2 && !tc::mbar_wait(&bars.acc_empty[b], ((seg >> 1) - 1) & 1, &abort_flag, err, wb))
          break;
        if (!tc::mbar_wait(&bars.op_full[t], (k / n_op) & 1, &abort_flag, err, wb)) break;
        tc::tc_fence_after();
        const uint32_t a0 = tc::smem_u32(op_blk(t, 0));
        const uint32_t b0 = diag ? a0 : tc::smem_u32(op_blk(t, 1));
        const uint32_t d = tbase + (uint32_t)b * 128u;
        // products (A piece, B piece) whose levels add to at most 2
        constexpr int pa[6] = {0, 0, 1, 1, 0, 2};
        constexpr int pb[6] = {0, 1, 0, 1, 2, 0};
#pragma unroll
        for (int kk = 0; kk < kRows / 16; ++kk) {  // K = 16 per MMA: two core matrices along K
#pragma unroll
          for (int p = 0; p < 6; ++p) {
            const uint32_t aa = a0 + (uint32_t)pa[p] * kPieceBytes + (uint32_t)kk * 2 * kLbo;
            const uint32_t bb = b0 + (uint32_t)pb[p] * kPieceBytes + (uint32_t)kk * 2 * kLbo;
            tc::umma_f16(d, tc::ns_desc(aa, kLbo, kSbo), tc::ns_desc(bb, kLbo, kSbo), idesc,
                         (seg_first && kk == 0 && p == 0) ? 0u : 1u);
          }
        }
        tc::umma_commit(&bars.op_free[t]);
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
      const int s = k % n_st, t = k % n_op;
      if (!tc::mbar_wait_warp(&bars.full[s], (k / n_st) & 1, &abort_flag, err, wb)) break;
      if (k >= n_op && !tc::mbar_wait_warp(&bars.op_free[t], ((k / n_op) - 1) & 1, &abort_flag, err, wb)) break;
      for (int p = 0; p < panels; ++p) convert_panel(st_blk(s, p), op_blk(t, p), ct);
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&bars.st_free[s]);
        tc::mbar_arrive(&bars.op_full[t]);
      }
    }
  } else {
    // ------------------------------------------------------------ flushers + result
    const int q = warp & 3;                       // TMEM lane quarter this warp may access
    const int h = (warp - kFirstFlushWarp) >> 2;  // column half of the tile
    bool ok = true;
    for (int j = 0; j < nseg && ok; ++j) ok = flush_segment(j, tbase, q, h, lane, bars, &abort_flag, err, wb);
    if (__all_sync(0xffffffffu, ok && !abort_flag)) {
      const int a = 32 * q + lane;  // tile row
      const int gi = ti * kPanel + a;
      const uint32_t lanes = (uint32_t)(32 * q) << 16;
      // tile-major partial slot: J.item_base + (row-major upper-triangle index) * splits + split
      const int tile_idx = ti * J.tiles - ti * (ti - 1) / 2 + (tj - ti);
      double* out = J.splits == 1 ? nullptr
                                  : partials + ((size_t)J.item_base + (size_t)tile_idx * J.splits + sp) *
                                                   (kPanel * kPanel) +
                                        (size_t)a * kPanel;
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
            const int gj = tj * kPanel + c0 + i;
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

int gram_bf3_rows_per_stage() { return kRows; }

cudaError_t launch_gram_bf3(const GramJob* jobs_dev, const CUtensorMap* maps_dev, const int4* items_dev,
                            int num_items, const int4* reduce_dev, int num_reduce, double* partials, int* err_flag,
                            cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gram_bf3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (num_items > 0)
    gram_bf3_kernel<<<num_items, kThreads, kSmemBytes, s>>>(jobs_dev, maps_dev, items_dev, partials, err_flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gram_reduce(128, jobs_dev, reduce_dev, num_reduce, partials, s);
}

}  // namespace hapod
