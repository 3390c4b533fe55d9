// K4, mixed form: scaled POD modes Y = X V_k diag(scale) (Sec. 2, Remark
// def:method_of_snapshots; Def. HAPOD passes sigma_k phi_k = X psi_k to the parent)
// for FP32 snapshots, on the FP32 CUDA cores (fused multiply-add, round-to-nearest).
//
// V_k (FP64 m x k) is rounded to FP32 once per CTA into shared memory, KT modes
// at a time.  Each thread owns RPT = 64 / KT consecutive rows, read as one vector
// per column (a warp touches 32 RPT consecutive floats of one column), and KT
// accumulators per row; every X element is read from HBM once per mode tile and
// multiplied with KT shared-memory broadcasts.  For the kept ranks of this method
// (k of a few tens) one mode tile covers k, so X is read once: the kernel streams
// b n m bytes in and b n k out.
#include "hapod_internal.cuh"

namespace hapod {
namespace {

constexpr int kThreadsM = 256;

__device__ __forceinline__ int find_job_m(const ModesJob* jobs, int njobs, int64_t b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].block_base <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// RPT = 64 / KT consecutive rows per thread (one vector load per column when VEC),
// KT modes per launch tile, 64 FP32 accumulators per thread.
template <int KT, int RPT, bool VEC>
__global__ void __launch_bounds__(kThreadsM, 2) modes_mixed_kernel(const ModesJob* __restrict__ jobs, int njobs) {
  constexpr int kMaxMChunk = 8192 / KT;  // columns of X per staged slice of V (32 KB)
  __shared__ __align__(16) float Vs[kMaxMChunk * KT];
  const int64_t b = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
  const ModesJob J = jobs[find_job_m(jobs, njobs, b)];
  const int64_t local = b - J.block_base;
  if (local >= (int64_t)J.row_tiles * J.col_tiles) return;
  const int64_t rt = local % J.row_tiles;
  const int ct = (int)(local / J.row_tiles);
  const int j0 = ct * KT;
  const int64_t row0 = rt * (int64_t)(kThreadsM * RPT) + (int64_t)threadIdx.x * RPT;
  const float* __restrict__ X = static_cast<const float*>(J.X);
  float* __restrict__ Y = static_cast<float*>(J.Y);
  const bool full = row0 + RPT <= J.n;

  float acc[RPT][KT];
#pragma unroll
  for (int i = 0; i < RPT; ++i)
#pragma unroll
    for (int j = 0; j < KT; ++j) acc[i][j] = 0.f;

  for (int c0 = 0; c0 < J.m; c0 += kMaxMChunk) {
    const int cn = min(kMaxMChunk, J.m - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < cn * KT; e += kThreadsM) {
      const int c = e / KT, j = e % KT;
      Vs[e] = (j0 + j < J.k) ? (float)J.Vk[(size_t)(j0 + j) * J.ldv + c0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < cn; ++c) {
      const float* col = X + (size_t)(c0 + c) * J.ldx + row0;
      float x[RPT];
      if (VEC && full) {
        if constexpr (RPT == 4) {
          const float4 t = *reinterpret_cast<const float4*>(col);
          x[0] = t.x;
          x[1] = t.y;
          x[2] = t.z;
          x[3] = t.w;
        } else if constexpr (RPT == 2) {
          const float2 t = *reinterpret_cast<const float2*>(col);
          x[0] = t.x;
          x[1] = t.y;
        } else {
          x[0] = col[0];
        }
      } else {
#pragma unroll
        for (int i = 0; i < RPT; ++i) x[i] = row0 + i < J.n ? col[i] : 0.f;
      }
      const float4* v4 = reinterpret_cast<const float4*>(Vs + c * KT);
#pragma unroll
      for (int j4 = 0; j4 < KT / 4; ++j4) {
        const float4 v = v4[j4];
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          acc[i][4 * j4 + 0] = fmaf(x[i], v.x, acc[i][4 * j4 + 0]);
          acc[i][4 * j4 + 1] = fmaf(x[i], v.y, acc[i][4 * j4 + 1]);
          acc[i][4 * j4 + 2] = fmaf(x[i], v.z, acc[i][4 * j4 + 2]);
          acc[i][4 * j4 + 3] = fmaf(x[i], v.w, acc[i][4 * j4 + 3]);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < KT; ++j) {
    if (j0 + j >= J.k) break;
    const float sc = J.scale ? (float)J.scale[j0 + j] : 1.f;
    float* out = Y + (size_t)(j0 + j) * J.ldy + row0;
    if (VEC && full && RPT == 4) {
      *reinterpret_cast<float4*>(out) = make_float4(acc[0][j] * sc, acc[RPT > 1 ? 1 : 0][j] * sc,
                                                    acc[RPT > 2 ? 2 : 0][j] * sc, acc[RPT > 3 ? 3 : 0][j] * sc);
    } else {
#pragma unroll
      for (int i = 0; i < RPT; ++i)
        if (row0 + i < J.n) out[i] = acc[i][j] * sc;
    }
  }
}

}  // namespace

// Mode tile: 16 modes for k <= 16 (4 rows per thread), 32 for k <= 32 (2 rows),
// else 64 (1 row).
int modes_mixed_tile_cols(int k) { return k <= 16 ? 16 : (k <= 32 ? 32 : 64); }
int modes_mixed_rows_per_block(int k) { return kThreadsM * (64 / modes_mixed_tile_cols(k)); }

template <int KT>
static void launch_kt(dim3 grid, const ModesJob* jobs_dev, int njobs, bool vec, cudaStream_t s) {
  if (vec)
    modes_mixed_kernel<KT, 64 / KT, true><<<grid, kThreadsM, 0, s>>>(jobs_dev, njobs);
  else
    modes_mixed_kernel<KT, 64 / KT, false><<<grid, kThreadsM, 0, s>>>(jobs_dev, njobs);
}

cudaError_t launch_modes_mixed(const ModesJob* jobs_dev, int njobs, int64_t total_blocks, int kt, bool vec,
                               cudaStream_t s) {
  if (njobs <= 0 || total_blocks <= 0) return cudaSuccess;
  const int64_t gx = total_blocks < 65535 ? total_blocks : 65535;
  const int64_t gy = (total_blocks + gx - 1) / gx;
  dim3 grid((unsigned)gx, (unsigned)gy);
  if (kt == 16)
    launch_kt<16>(grid, jobs_dev, njobs, vec, s);
  else if (kt == 32)
    launch_kt<32>(grid, jobs_dev, njobs, vec, s);
  else
    launch_kt<64>(grid, jobs_dev, njobs, vec, s);
  return cudaGetLastError();
}

}  // namespace hapod
