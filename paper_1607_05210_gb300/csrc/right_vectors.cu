// Right singular vectors of the HAPOD (Sec. 3.3, Remark "Low-rank approximation of
// the snapshot mapping", with Def. "Additional notation"): the cumulative map
// Lambda~_a = diag(Lambda~_c over the children c) o Lambda_a, Lambda_a the node's
// right singular vectors (its Gram eigenvectors V_N), composed from the root down.
// The only arithmetic is small dense products C = A B in FP64 (rows of the parent's
// composed map times a child's V_N), one launch per node.
#include "hapod_internal.cuh"

namespace hapod {
namespace {

constexpr int kT = 32;  // output tile kT x kT, K in slices of kT

// C (M x N, ldc) = A (M x K, lda) B (K x N, ldb), column-major, FP64.
__global__ void __launch_bounds__(256) gemm_nn_f64(int64_t M, int64_t N, int64_t K, const double* __restrict__ A,
                                                   int64_t lda, const double* __restrict__ B, int64_t ldb,
                                                   double* __restrict__ C, int64_t ldc) {
  __shared__ double sa[kT][kT + 1];  // sa[k][i] = A(i0 + i, k0 + k)
  __shared__ double sb[kT][kT + 1];  // sb[j][k] = B(k0 + k, j0 + j)
  const int64_t i0 = (int64_t)blockIdx.x * kT, j0 = (int64_t)blockIdx.y * kT;
  const int tx = threadIdx.x % kT, ty = threadIdx.x / kT;  // 32 x 8 threads
  double acc[kT / 8];
#pragma unroll
  for (int r = 0; r < kT / 8; ++r) acc[r] = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += kT) {
    for (int r = ty; r < kT; r += 8) {
      const int64_t i = i0 + tx, k = k0 + r;
      sa[r][tx] = (i < M && k < K) ? A[k * lda + i] : 0.0;
      const int64_t kk = k0 + tx, j = j0 + r;
      sb[r][tx] = (kk < K && j < N) ? B[j * ldb + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kT; ++k) {
      const double a = sa[k][tx];
#pragma unroll
      for (int r = 0; r < kT / 8; ++r) acc[r] = fma(a, sb[ty + 8 * r][k], acc[r]);
    }
    __syncthreads();
  }
  const int64_t i = i0 + tx;
#pragma unroll
  for (int r = 0; r < kT / 8; ++r) {
    const int64_t j = j0 + ty + 8 * r;
    if (i < M && j < N) C[j * ldc + i] = acc[r];
  }
}

}  // namespace

cudaError_t launch_gemm_nn_f64(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
                               int64_t ldb, double* C, int64_t ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((M + kT - 1) / kT), (unsigned)((N + kT - 1) / kT));
  gemm_nn_f64<<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
  return cudaGetLastError();
}

}  // namespace hapod
