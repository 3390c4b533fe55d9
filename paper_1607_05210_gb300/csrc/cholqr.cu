// A6, mixed form, root only: CholQR2 re-orthogonalisation of the root's modes and
// refresh of its singular values.  Not a step of the paper: the method of
// snapshots forms phi_k = lambda_k^{-1/2} X psi_k (Sec. 2, Remark
// def:method_of_snapshots), whose orthogonality degrades with cond(G) = cond(X)^2
// (the remark's footnote); with FP32 data and tensor-core products that loss is
// visible, so the root's output is re-orthogonalised.
//
// With Y = X V_k (n x k, sigma-scaled modes):
//   W  = Y^T Y,   R1 = chol(W),   Q1 = Y R1^{-1}          (pass 1)
//   W2 = Q1^T Q1, R2 = chol(W2),  R = R2 R1 (so Y = Q R, Q = Q1 R2^{-1})
//   R = P S Z^T (one-sided Jacobi on R^T, FP64), U = Q P = Q1 (R2^{-1} P), sigma = S.
// The two k x k kernels below run on one CTA in FP64 (k is the kept rank, a few
// tens); the n x k passes reuse the Gram and modes kernels.
#include "hapod_internal.cuh"

namespace hapod {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Upper Cholesky factor R (R^T R = W) in place of an upper-triangular work array,
// then its inverse Rinv (upper).  W, R, Rinv: k x k column-major.  Right-looking,
// one column per step; a non-positive pivot (numerically rank-deficient W) is
// replaced by a tiny positive value and flagged.
__device__ void chol_upper_inv(const double* W, double* R, double* Rinv, int k, int* flag) {
  const int tid = threadIdx.x;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;
    R[e] = i <= j ? W[e] : 0.0;
    Rinv[e] = 0.0;
  }
  __syncthreads();
  __shared__ double piv;
  for (int c = 0; c < k; ++c) {
    if (tid == 0) {
      double d = R[(size_t)c * k + c];
      if (!(d > 0.0)) {
        d = 1e-300;
        *flag = 1;
      }
      piv = sqrt(d);
      R[(size_t)c * k + c] = piv;
    }
    __syncthreads();
    // row c to the right of the pivot
    for (int j = c + 1 + tid; j < k; j += blockDim.x) R[(size_t)j * k + c] /= piv;
    __syncthreads();
    // trailing update R[i][j] -= R[c][i] R[c][j], c < i <= j
    for (int e = tid; e < (k - c - 1) * (k - c - 1); e += blockDim.x) {
      const int i = c + 1 + e % (k - c - 1), j = c + 1 + e / (k - c - 1);
      if (i <= j) R[(size_t)j * k + i] -= R[(size_t)i * k + c] * R[(size_t)j * k + c];
    }
    __syncthreads();
  }
  // Rinv: back substitution column by column (column j of Rinv solves R x = e_j)
  for (int j = tid; j < k; j += blockDim.x) {
    for (int i = j; i >= 0; --i) {
      double s = (i == j) ? 1.0 : 0.0;
      for (int l = i + 1; l <= j; ++l) s -= R[(size_t)l * k + i] * Rinv[(size_t)j * k + l];
      Rinv[(size_t)j * k + i] = s / R[(size_t)i * k + i];
    }
  }
  __syncthreads();
}

// pass-1 factors: R1 = chol(W), M1 = R1^{-1}
__global__ void __launch_bounds__(kThreads) cholqr_first(const double* W, double* R1, double* M1, int k, int* flag) {
  chol_upper_inv(W, R1, M1, k, flag);
}

// pass-2 factors: R2 = chol(W2), R = R2 R1, SVD of R by one-sided Jacobi on R^T with
// the rotations accumulated in P; outputs M = R2^{-1} P (columns sorted by singular
// value, descending) and sigma.
__global__ void __launch_bounds__(kThreads) cholqr_second(const double* W2, const double* R1, double* R2, double* R2inv,
                                                         double* B, double* P, double* M, double* sigma, int k,
                                                         int* flag, int max_sweeps) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  chol_upper_inv(W2, R2, R2inv, k, flag);
  // B = (R2 R1)^T, P = I
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;  // B[i][j] = R[j][i] = sum_l R2[j][l] R1[l][i]
    double s = 0.0;
    for (int l = j; l <= i; ++l) s += R2[(size_t)l * k + j] * R1[(size_t)i * k + l];
    B[e] = s;
    P[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  __shared__ int rotated_sh;
  const double tol = (double)k * 1.1102230246251565e-16;
  const int kp = k + (k & 1);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rotated_sh = 0;
    __syncthreads();
    for (int t = 0; t < kp - 1; ++t) {
      for (int pr = warp; pr < kp / 2; pr += nw) {
        int p, q;
        const int r = kp - 1;
        if (pr == 0) {
          p = t;
          q = r;
        } else {
          p = (t + pr) % r;
          q = (t - pr + r) % r;
        }
        if (p >= k || q >= k) continue;
        double al = 0, be = 0, ga = 0;
        for (int i = lane; i < k; i += 32) {
          const double x = B[(size_t)p * k + i], y = B[(size_t)q * k + i];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga == 0.0 || !(fabs(ga) > tol * sqrt(al * be))) continue;
        if (lane == 0) rotated_sh = 1;
        const double zeta = (be - al) / (2.0 * ga);
        const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
        for (int i = lane; i < k; i += 32) {
          const double x = B[(size_t)p * k + i], y = B[(size_t)q * k + i];
          B[(size_t)p * k + i] = c * x - s * y;
          B[(size_t)q * k + i] = s * x + c * y;
          const double u = P[(size_t)p * k + i], v = P[(size_t)q * k + i];
          P[(size_t)p * k + i] = c * u - s * v;
          P[(size_t)q * k + i] = s * u + c * v;
        }
      }
      __syncthreads();
    }
    const int any = rotated_sh;
    __syncthreads();
    if (!any) break;
  }
  // sigma_j = ||B P e_j||; sort descending; M = R2^{-1} P (sorted columns)
  __shared__ double sv[256];
  __shared__ int order[256];
  for (int j = warp; j < k; j += nw) {
    double s = 0.0;
    for (int i = lane; i < k; i += 32) s += B[(size_t)j * k + i] * B[(size_t)j * k + i];
    s = warp_sum(s);
    if (lane == 0) sv[j] = sqrt(s);
  }
  __syncthreads();
  for (int j = tid; j < k; j += blockDim.x) {
    int rank = 0;
    for (int i = 0; i < k; ++i) rank += (sv[i] > sv[j]) || (sv[i] == sv[j] && i < j);
    order[rank] = j;
  }
  __syncthreads();
  for (int j = tid; j < k; j += blockDim.x) sigma[j] = sv[order[j]];
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;  // M[i][j] = sum_l R2inv[i][l] P[l][order[j]]
    double s = 0.0;
    for (int l = i; l < k; ++l) s += R2inv[(size_t)l * k + i] * P[(size_t)order[j] * k + l];
    M[e] = s;
  }
}

}  // namespace

cudaError_t launch_cholqr_first(const double* W, double* R1, double* M1, int k, int* flag, cudaStream_t s) {
  cholqr_first<<<1, kThreads, 0, s>>>(W, R1, M1, k, flag);
  return cudaGetLastError();
}

cudaError_t launch_cholqr_second(const double* W2, const double* R1, double* work, double* M, double* sigma, int k,
                                 int* flag, cudaStream_t s) {
  if (k > 256) return cudaErrorInvalidValue;
  double* R2 = work;
  double* R2inv = work + (size_t)k * k;
  double* B = work + 2 * (size_t)k * k;
  double* P = work + 3 * (size_t)k * k;
  cholqr_second<<<1, kThreads, 0, s>>>(W2, R1, R2, R2inv, B, P, M, sigma, k, flag, 40);
  return cudaGetLastError();
}

}  // namespace hapod
