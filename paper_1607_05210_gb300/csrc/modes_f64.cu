// K4, FP64 form: scaled POD modes Y = X V_k (Sec. 2, Remark
// def:method_of_snapshots: sigma_k phi_k = sum_i psi_{k,i} s_i), the quantity
// Def. HAPOD passes to the parent; at the root the epilogue multiplies column j
// by 1/sigma_j to return phi_j.  Also the gather V_k[:, j] = V[:, perm[j]] that
// orders the eigenvectors by descending eigenvalue.
//
// Tile: 64 rows x 64 modes per CTA, K (= m) in chunks of 32.  Columns of X are
// contiguous, so a warp reads 32 consecutive rows of one column; thread t owns
// rows t%16 + 16i and modes t/16 + 16j, so each store instruction writes 16
// consecutive rows of one output column.  Bound by the FP64 pipe on GB300.
#include "hapod_internal.cuh"

namespace hapod {
namespace {

constexpr int kRows = 64, kCols = 64, kBK = 32;

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

__global__ void __launch_bounds__(256) modes_f64_kernel(const ModesJob* __restrict__ jobs, int njobs) {
  const int64_t b = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
  const int jb = find_job(jobs, njobs, b);
  const ModesJob J = jobs[jb];
  const int64_t local = b - J.block_base;
  if (local >= (int64_t)J.row_tiles * J.col_tiles) return;
  const int64_t rt = local % J.row_tiles;
  const int ct = (int)(local / J.row_tiles);
  const int64_t r0 = rt * kRows;
  const int c0 = ct * kCols;
  const double* __restrict__ X = static_cast<const double*>(J.X);
  double* __restrict__ Y = static_cast<double*>(J.Y);

  __shared__ double Xs[kBK][kRows + 1];
  __shared__ double Vs[kBK][kCols + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tr = tid & 15, tc = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;

  for (int k0 = 0; k0 < J.m; k0 += kBK) {
    // X tile: kBK columns x 64 rows; warp w loads columns w, w+8, ...; two rows per lane
    for (int c = warp; c < kBK; c += 8) {
      const int col = k0 + c;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t r = r0 + lane + 32 * h;
        Xs[c][lane + 32 * h] = (col < J.m && r < J.n) ? X[(size_t)col * J.ldx + r] : 0.0;
      }
    }
    // V tile: kBK rows (k) x 64 modes
    for (int e = tid; e < kBK * kCols; e += 256) {
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
        a[q] = Xs[kk][tr + 16 * q];
        v[q] = Vs[kk][tc + 16 * q];
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
    const int col = c0 + tc + 16 * q;
    if (col >= J.k) continue;
    const double sc = J.scale ? J.scale[col] : 1.0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t r = r0 + tr + 16 * p;
      if (r < J.n) Y[(size_t)col * J.ldy + r] = acc[p][q] * sc;
    }
  }
}

}  // namespace

int modes_tile_rows(bool fp64) { return fp64 ? kRows : 128; }
int modes_tile_cols(bool fp64) { return fp64 ? kCols : 256; }

cudaError_t launch_gather(bool fp64_src, const GatherJob* jobs_dev, int njobs, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  dim3 grid(64, njobs);
  if (fp64_src)
    gather_kernel<double><<<grid, 256, 0, s>>>(jobs_dev);
  else
    gather_kernel<float><<<grid, 256, 0, s>>>(jobs_dev);
  return cudaGetLastError();
}

cudaError_t launch_modes_f64(const ModesJob* jobs_dev, int njobs, int64_t total_blocks, cudaStream_t s) {
  if (njobs <= 0 || total_blocks <= 0) return cudaSuccess;
  const int64_t gx = total_blocks < 65535 ? total_blocks : 65535;
  const int64_t gy = (total_blocks + gx - 1) / gx;
  modes_f64_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(jobs_dev, njobs);
  return cudaGetLastError();
}

}  // namespace hapod
