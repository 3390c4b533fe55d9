// K4, digit-slice FP64 form: Y = X V_k diag(scale) (Sec. 2, Remark
// def:method_of_snapshots: sigma_k phi_k = X psi_k, or phi_k with scale = 1/sigma)
// from exact digits on the tensor cores (tcgen05 kind::f16, bf16 x bf16 -> FP32).
//
// X is split per column as for the Gram, x_rj = 2^E_j xt_rj (oz_split.cu).  Moving
// the column scale into V, Y_rc = sum_j xt_rj (2^E_j V_jc) = 2^F_c sum_j xt_rj vt_jc
// with 2^F_c > max_j 2^E_j |V_jc| and vt_jc = 2^(E_j - F_c) V_jc < 1, split into 7
// base-128 digits the same way (oz_vsplit_kernel below: the digits of V_jc against
// the bound 2^(F_c - E_j), so nothing overflows).  Level sums over the columns are
// exact integers below 2^24 for up to kKBlock = 448 columns; longer rows are cut
// into 448-column blocks whose level sums are flushed exactly into int64 sums as
// in the Gram kernel, and Y_rc = 2^(F_c - 56) (hi 2^28 + lo) scale_c is rounded
// once to FP64.
//
// Work item = 128 rows x NT modes.  The X digit block is read as the MN-major A
// operand (M = rows: 16 row groups x 2 column groups per 16-column stage), the V
// digits as the K-major B operand.  One CTA per item:
//   warp 0       bulk-copy producer (3-deep ring: 16 x 1792 B of X digits and
//                2 x NT/8 x 896 B of V digits per 16-column stage)
//   warp 1       TMEM owner and single-thread UMMA issuer (28 MMAs 128 x NT x 16
//                per stage into 7 level accumulators of NT TMEM columns)
//   warps 2..    NT/4 flusher warps (16 modes x 32 rows each)
#include <climits>

#include "hapod_internal.cuh"
#include "oz_common.cuh"
#include "tc_common.cuh"

namespace hapod {
namespace {

constexpr int kStages = 3;
constexpr int kStageA = 16 * 2 * kOzGroupBytes;  // 28672 B: 128 rows x 16 columns, all digits
constexpr int kKBlockStages = 28;                // 448 columns between exact flushes
constexpr int kLevels = 7;

template <int NT>
struct Cfg {
  static constexpr int kStageB = 2 * (NT / 8) * kOzGroupBytes;
  static constexpr int kStageBytes = kStageA + kStageB;
  static constexpr int kSmemBytes = kStages * kStageBytes + 128;
  static constexpr int kFlushWarps = NT / 4;
  static constexpr int kThreads = (2 + kFlushWarps) * 32;
  static constexpr uint32_t kTmemCols = NT == 64 ? 512 : 256;
};

struct Bars {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t acc_full;
  uint64_t acc_empty;
  uint64_t mma_done;
};

template <int NT>
__global__ void __launch_bounds__(Cfg<NT>::kThreads, 1)
    modes_oz_kernel(const OzModesJob* __restrict__ jobs, int njobs, int* err) {
  using C = Cfg<NT>;
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
  const OzModesJob J = jobs[jlo];
  const int64_t local = b - J.item_base;
  if (local >= (int64_t)J.row_tiles * J.n_tiles) return;
  const int64_t rt = local % J.row_tiles;
  const int nt = (int)(local / J.row_tiles);
  const int rg0 = (int)(rt * 16);
  const int nrg = min(16, J.RG - rg0);  // row groups present in this tile
  const int nst = J.CGp / 2;            // 16-column stages
  const int nkb = (nst + kKBlockStages - 1) / kKBlockStages;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto stage_a = [&](int s) -> uint8_t* { return smem + (size_t)s * C::kStageBytes; };
  auto stage_b = [&](int s) -> uint8_t* { return smem + (size_t)s * C::kStageBytes + kStageA; };

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&bars.full[s], 1);
      tc::mbar_init(&bars.empty[s], 1);
    }
    tc::mbar_init(&bars.acc_full, 1);
    tc::mbar_init(&bars.acc_empty, C::kFlushWarps);
    tc::mbar_init(&bars.mma_done, 1);
    abort_flag = 0;
    tc::mbar_fence_init();
  }
  if (warp == 1) tc::tmem_alloc(&tmem_base, C::kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      const uint8_t* xd = reinterpret_cast<const uint8_t*>(J.xdig);
      const uint8_t* vd = reinterpret_cast<const uint8_t*>(J.vdig);
      const uint32_t bytes = (uint32_t)nrg * (2 * kOzGroupBytes) + C::kStageB;
      int issued = 0;
      for (int k = 0; k < nst; ++k) {
        const int s = k % kStages;
        if (k >= kStages && !tc::mbar_wait(&bars.empty[s], ((k / kStages) - 1) & 1, &abort_flag, err)) break;
        tc::mbar_expect_tx(&bars.full[s], bytes);
        for (int q = 0; q < nrg; ++q)
          tc::bulk_load(stage_a(s) + q * (2 * kOzGroupBytes),
                        xd + ((int64_t)(rg0 + q) * J.CGp + 2 * k) * kOzGroupBytes, 2 * kOzGroupBytes, &bars.full[s]);
#pragma unroll
        for (int q = 0; q < 2; ++q)
          tc::bulk_load(stage_b(s) + q * (C::kStageB / 2),
                        vd + ((int64_t)(2 * k + q) * J.NG + nt * (NT / 8)) * kOzGroupBytes, C::kStageB / 2,
                        &bars.full[s]);
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
      constexpr uint32_t idesc = tc::idesc_bf16_f32_major(128, NT, 1, 0);
      for (int k = 0; k < nst; ++k) {
        const int s = k % kStages;
        const int pos = k % kKBlockStages;
        if (pos == 0 && k > 0 && !tc::mbar_wait(&bars.acc_empty, ((k / kKBlockStages) - 1) & 1, &abort_flag, err))
          break;
        if (!tc::mbar_wait(&bars.full[s], (k / kStages) & 1, &abort_flag, err)) break;
        tc::tc_fence_after();
        const uint32_t a0 = tc::smem_u32(stage_a(s)), b0 = tc::smem_u32(stage_b(s));
#pragma unroll
        for (int lv = 2; lv <= 8; ++lv) {
          const int t_lo = lv - 7 > 1 ? lv - 7 : 1;
          const int t_hi = lv - 1 < 7 ? lv - 1 : 7;
#pragma unroll
          for (int t = t_lo; t <= t_hi; ++t) {
            const int u = lv - t;
            // A (MN-major): LBO = column-group stride (K), SBO = row-group stride (M);
            // B (K-major): LBO = column-group stride (K), SBO = mode-group stride (N)
            tc::umma_bf16(tbase + (uint32_t)((lv - 2) * NT),
                          tc::ns_desc(a0 + (uint32_t)(t - 1) * 128u, kOzGroupBytes, 2 * kOzGroupBytes),
                          tc::ns_desc(b0 + (uint32_t)(u - 1) * 128u, C::kStageB / 2, kOzGroupBytes), idesc,
                          (pos == 0 && t == t_lo) ? 0u : 1u);
          }
        }
        tc::umma_commit(&bars.empty[s]);
        if (pos == kKBlockStages - 1 || k == nst - 1) tc::umma_commit(&bars.acc_full);
      }
      tc::umma_commit(&bars.mma_done);
      const long long t0 = clock64();
      while (!tc::mbar_try(&bars.mma_done, 0) && clock64() - t0 < tc::kWaitBudget) {
      }
    }
  } else {
    // ------------------------------------------------------------ flushers + output
    const int q = warp & 3;
    const int cw = (warp - 2) >> 2;  // 16-mode slice of the NT-mode tile
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
        tc::tmem_ld16(tbase + lanes + (uint32_t)(lv * NT + 16 * cw), v);
        tc::tmem_wait_ld();
        const long long w = lv < 3 ? (1ll << (7 * (2 - lv))) : (1ll << (7 * (6 - lv)));
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
      const int64_t r = (int64_t)rg0 * 8 + 32 * q + lane;
      if (r < J.rows) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int col = nt * NT + 16 * cw + c;
          if (col >= J.k) break;
          const int F = J.fexp[col];
          double v;
          if (F == kOzNonFinite) {
            v = __longlong_as_double(0x7FF8000000000000ll);
          } else {
            v = scalbn((double)hi[c] * 268435456.0 + (double)lo[c], F - 56);
            if (J.scale) v *= J.scale[col];
          }
          J.Y[(size_t)col * J.ldy + r] = v;
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, C::kTmemCols);
}

// One block per mode column c (of kpad = 8 NG): F_c = max_j (E_j + e(V_jc)) with
// |V_jc| < 2^e(V_jc), then the digits of V_jc against 2^(F_c - E_j) into
// [column group j/8][mode group c/8][digit][c % 8][j % 8].  Columns c >= k and rows
// j >= m are zero.  A non-finite X column (E_j marker) or V entry marks F_c.
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
    uint4* out = reinterpret_cast<uint4*>(J.vdig) + (((size_t)g * J.NG + (c >> 3)) * kOzDigits) * 8 + (c & 7);
#pragma unroll
    for (int q = 0; q < kOzDigits; ++q) out[q * 8] = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
  }
}

dim3 grid_for(int64_t blocks) {
  const int64_t gx = blocks < 65535 ? blocks : 65535;
  return dim3((unsigned)gx, (unsigned)((blocks + gx - 1) / gx));
}

template <int NT>
cudaError_t launch_nt(const OzModesJob* jobs_dev, int njobs, int64_t total_items, int* err_flag, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(modes_oz_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<NT>::kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  modes_oz_kernel<NT><<<grid_for(total_items), Cfg<NT>::kThreads, Cfg<NT>::kSmemBytes, s>>>(jobs_dev, njobs, err_flag);
  return cudaGetLastError();
}

}  // namespace

int oz_modes_tile(int k) { return k <= 32 ? 32 : 64; }

cudaError_t launch_modes_oz(const OzModesJob* jobs_dev, int njobs, int64_t total_items, int nt, int* err_flag,
                            cudaStream_t s) {
  if (njobs <= 0 || total_items <= 0) return cudaSuccess;
  if (nt == 32) return launch_nt<32>(jobs_dev, njobs, total_items, err_flag, s);
  if (nt == 64) return launch_nt<64>(jobs_dev, njobs, total_items, err_flag, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_oz_vsplit(const OzVSplitJob* jobs_dev, int njobs, int64_t total_cols, cudaStream_t s) {
  if (njobs <= 0 || total_cols <= 0) return cudaSuccess;
  if (total_cols > 0x7FFFFFFF) return cudaErrorInvalidValue;
  oz_vsplit_kernel<<<(unsigned)total_cols, 256, 0, s>>>(jobs_dev, njobs);
  return cudaGetLastError();
}

}  // namespace hapod
