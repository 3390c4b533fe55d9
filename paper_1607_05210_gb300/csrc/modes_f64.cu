// K4, FP64 form: scaled POD modes Y = X V_k (Sec. 2, Remark
// def:method_of_snapshots: sigma_k phi_k = sum_i psi_{k,i} s_i), the quantity
// Def. HAPOD passes to the parent; at the root the epilogue multiplies column j
// by 1/sigma_j to return phi_j.  Also the gather V_k[:, j] = V[:, perm[j]] that
// orders the eigenvectors by descending eigenvalue.
//
// Tile: ROWS x COLS (rows x modes) per CTA with COLS = 16, 32 or 64 chosen from the
// largest kept rank of the launch (ROWS = 4096 / COLS), so a rank of ~20 does not
// pay for 64-wide tiles; K (= m) in chunks of 16.  Columns of X are contiguous, so a
// warp reads 32 consecutive rows of one column; every store instruction writes
// consecutive rows of one output column.  Bound by the FP64 pipe on GB300.
#include "hapod_internal.cuh"

namespace hapod {
namespace {

constexpr int kBK = 16;

template <typename T>
__global__ void gather_kernel(const GatherJob* __restrict__ jobs) {
  const GatherJob J = jobs[blockIdx.y];
  const T* V = static_cast<const T*>(J.V);
  const size_t total = (size_t)J.m * J.k;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / J.m), i = (int)(e % J.m);
    J.Vk[e] = (double)V[(size_t)J.perm[j] * J.m + i];
  }
}

__device__ __forceinline__ int find_job(const ModesJob* jobs, int njobs, int64_t b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].block_base <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ROWS x COLS output tile, 256 threads as (ROWS/4) x (COLS/4), 4 x 4 outputs each:
// thread t owns rows t % (ROWS/4) + (ROWS/4) p and modes t / (ROWS/4) + (COLS/4) q.
template <int ROWS, int COLS>
__global__ void __launch_bounds__(256) modes_f64_kernel(const ModesJob* __restrict__ jobs, int njobs) {
  constexpr int TR = ROWS / 4, TC = COLS / 4;
  static_assert(TR * TC == 256, "256 threads");
  const int64_t b = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
  const int jb = find_job(jobs, njobs, b);
  const ModesJob J = jobs[jb];
  const int64_t local = b - J.block_base;
  if (local >= (int64_t)J.row_tiles * J.col_tiles) return;
  const int64_t rt = local % J.row_tiles;
  const int ct = (int)(local / J.row_tiles);
  const int64_t r0 = rt * ROWS;
  const int c0 = ct * COLS;
  const double* __restrict__ X = static_cast<const double*>(J.X);
  double* __restrict__ Y = static_cast<double*>(J.Y);

  __shared__ double Xs[kBK][ROWS + 1];
  __shared__ double Vs[kBK][COLS + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tr = tid % TR, tc = tid / TR;
  double acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;

  for (int k0 = 0; k0 < J.m; k0 += kBK) {
    // X tile: kBK columns x ROWS rows; warp w loads columns w, w + 8 (lanes along rows)
    for (int c = warp; c < kBK; c += 8) {
      const int col = k0 + c;
#pragma unroll
      for (int h = 0; h < ROWS / 32; ++h) {
        const int64_t r = r0 + lane + 32 * h;
        Xs[c][lane + 32 * h] = (col < J.m && r < J.n) ? X[(size_t)col * J.ldx + r] : 0.0;
      }
    }
    // V tile: kBK rows (k) x COLS modes
    for (int e = tid; e < kBK * COLS; e += 256) {
      const int kk = e % kBK, j = e / kBK;
      const int row = k0 + kk, col = c0 + j;
      Vs[kk][j] = (row < J.m && col < J.k) ? J.Vk[(size_t)col * J.ldv + row] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kBK; ++kk) {
      double a[4], v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = Xs[kk][tr + TR * q];
        v[q] = Vs[kk][tc + TC * q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], v[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int col = c0 + tc + TC * q;
    if (col >= J.k) continue;
    const double sc = J.scale ? J.scale[col] : 1.0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t r = r0 + tr + TR * p;
      if (r < J.n) Y[(size_t)col * J.ldy + r] = acc[p][q] * sc;
    }
  }
}

}  // namespace

int modes_f64_tile_cols(int k) { return k <= 16 ? 16 : (k <= 32 ? 32 : 64); }
int modes_f64_tile_rows(int k) { return 4096 / modes_f64_tile_cols(k); }

cudaError_t launch_gather(bool fp64_src, const GatherJob* jobs_dev, int njobs, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  dim3 grid(64, njobs);
  if (fp64_src)
    gather_kernel<double><<<grid, 256, 0, s>>>(jobs_dev);
  else
    gather_kernel<float><<<grid, 256, 0, s>>>(jobs_dev);
  return cudaGetLastError();
}

cudaError_t launch_modes_f64(const ModesJob* jobs_dev, int njobs, int64_t total_blocks, int tile_cols, cudaStream_t s) {
  if (njobs <= 0 || total_blocks <= 0) return cudaSuccess;
  const int64_t gx = total_blocks < 65535 ? total_blocks : 65535;
  const int64_t gy = (total_blocks + gx - 1) / gx;
  const dim3 grid((unsigned)gx, (unsigned)gy);
  if (tile_cols == 16)
    modes_f64_kernel<256, 16><<<grid, 256, 0, s>>>(jobs_dev, njobs);
  else if (tile_cols == 32)
    modes_f64_kernel<128, 32><<<grid, 256, 0, s>>>(jobs_dev, njobs);
  else
    modes_f64_kernel<64, 64><<<grid, 256, 0, s>>>(jobs_dev, njobs);
  return cudaGetLastError();
}

}  // namespace hapod
