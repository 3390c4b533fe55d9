// K2: eigen-decomposition of a node's Gramian G (Sec. 2, Remark
// def:method_of_snapshots: lambda_k, psi_k of G give the POD), one CTA per node.
//
// 1. Rank-revealing factorisation (FP64): diagonally pivoted Cholesky
//    G = L L^T + S, choosing at step k the largest remaining diagonal of the Schur
//    complement S and stopping once trace(S) (the sum of its diagonal, S being PSD)
//    is below min(tol * trace(G), 1e-2 eps^2) (tol * trace(G) without an eps),
//    tol = m 2^-53 (FP64 rotations) or 1e-7 (FP32 rotations), but not below the
//    form's Gram error level floor_rel * trace(G) (the remaining pivots would factor
//    rounding noise).  trace(S) is
//    returned as `resid` and added to every tail of the truncation, so the dropped
//    part is accounted for exactly: no eigenvalue of G exceeds that of L L^T by more
//    than ||S|| <= trace(S).
// 2. One-sided Jacobi (Hestenes) on the r columns of L in precision T: plane
//    rotations from the right make the columns mutually orthogonal, L J = W.  Then
//    L L^T = W W^T, so the eigenvectors of L L^T are u_j = w_j / ||w_j|| (no
//    rotation matrix has to be accumulated); the eigenvalues are taken as FP64
//    Rayleigh quotients u_j^T G u_j with the original G.  Pairs follow the round-robin ("circle") ordering, one warp per
//    pair, all pairs of a step concurrently; a pair is rotated while
//    |w_p . w_q| > tol ||w_p|| ||w_q||, tol = m * unit roundoff of T.
// For the exponentially decaying spectra of snapshot data r is a few tens, so the
// eigensolve costs O(m r^2) per sweep instead of the O(m^3) of a Jacobi sweep on G.
// Output: lambda descending (clamped >= 0, zero beyond r), V (T, m x m) with
// column j = w_j / ||w_j|| for j < r and zero otherwise, perm = sorted order.
#include "hapod_internal.cuh"

namespace hapod {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;

template <typename T>
struct Unit;
template <>
struct Unit<double> {
  static __device__ double eps() { return 1.1102230246251565e-16; }
};
template <>
struct Unit<float> {
  static __device__ float eps() { return 5.9604645e-08f; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Pair k of round t in the circle method on mp (even) players.
__device__ __forceinline__ void rr_pair(int t, int k, int mp, int& p, int& q) {
  const int r = mp - 1;
  if (k == 0) {
    p = t;
    q = r;
  } else {
    p = (t + k) % r;
    q = (t - k + r) % r;
  }
}

// Block-wide argmax of d[i] over unchosen i (ties: lowest index) and the block sum
// of the positive d[i]; every thread receives the results.
__device__ void argmax_block(const double* d, const unsigned char* chosen, int m, int& p, double& dmax, double& dsum,
                             double* red_v, int* red_i, double* red_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double best = -1.0, sum = 0.0;
  int bi = -1;
  for (int i = tid; i < m; i += blockDim.x) {
    if (chosen[i]) continue;
    const double v = d[i];
    if (v > 0.0) sum += v;
    if (v > best) {
      best = v;
      bi = i;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi >= 0 && (bi < 0 || oi < bi))) {
      best = ov;
      bi = oi;
    }
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
  }
  if (lane == 0) {
    red_v[warp] = best;
    red_i[warp] = bi;
    red_s[warp] = sum;
  }
  __syncthreads();
  if (tid == 0) {
    double b = -1.0, s = 0.0;
    int i = -1;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s += red_s[w];
      if (red_v[w] > b || (red_v[w] == b && red_i[w] >= 0 && (i < 0 || red_i[w] < i))) {
        b = red_v[w];
        i = red_i[w];
      }
    }
    red_v[0] = b;
    red_i[0] = i;
    red_s[0] = s;
  }
  __syncthreads();
  p = red_i[0];
  dmax = red_v[0];
  dsum = red_s[0];
  __syncthreads();
}

// One-sided Jacobi sweeps on the r columns (length m) of W in precision U until no
// pair needs a rotation (|w_p . w_q| <= m u ||w_p|| ||w_q||, u the unit roundoff of U)
// or max_sweeps sweeps were made.  Block-wide; returns the sweeps made.
template <typename U>
__device__ int jacobi_sweeps(U* W, int m, int r, int max_sweeps, bool& converged, int* flag_sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rp = r + (r & 1), npairs = rp / 2;
  const U rtol = (U)m * Unit<U>::eps();
  int sweeps = 0;
  converged = (r <= 1);
  while (!converged && sweeps < max_sweeps) {
    ++sweeps;
    if (tid == 0) *flag_sh = 0;
    __syncthreads();
    int rotated = 0;
    for (int t = 0; t < rp - 1; ++t) {
      for (int k = warp; k < npairs; k += kWarps) {
        int p, q;
        rr_pair(t, k, rp, p, q);
        if (p >= r || q >= r) continue;
        U* wp = W + (size_t)p * m;
        U* wq = W + (size_t)q * m;
        U al = 0, be = 0, ga = 0;
        for (int i = lane; i < m; i += 32) {
          const U x = wp[i], y = wq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga == U(0) || !(fabs(ga) > rtol * sqrt(al * be))) continue;
        rotated = 1;
        const U zeta = (be - al) / (U(2) * ga);
        // smaller root of t^2 + 2 zeta t - 1 = 0; 1/(2 zeta) once zeta^2 would overflow
        const U tt = fabs(zeta) > U(1e15) ? U(0.5) / zeta
                                           : (zeta >= U(0) ? U(1) : U(-1)) / (fabs(zeta) + sqrt(U(1) + zeta * zeta));
        const U c = U(1) / sqrt(U(1) + tt * tt);
        const U s = c * tt;
        for (int i = lane; i < m; i += 32) {
          const U x = wp[i], y = wq[i];
          wp[i] = c * x - s * y;
          wq[i] = s * x + c * y;
        }
      }
      __syncthreads();
    }
    if (rotated && lane == 0) *flag_sh = 1;
    __syncthreads();
    converged = (*flag_sh == 0);
    __syncthreads();
  }
  return sweeps;
}

// T: precision of the rotations and of the eigenvectors.
template <typename T>
__global__ void __launch_bounds__(kThreads) chol_jacobi_kernel(const EigJob* __restrict__ jobs, int max_sweeps) {
  typedef T V_t;
  const EigJob J = jobs[blockIdx.x];
  const int m = J.m;
  if (m <= 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* __restrict__ G = J.G;
  double* L = static_cast<double*>(J.A);  // m x m FP64 (first r columns used)
  T* W = static_cast<T*>(J.V);           // m x m in T: rotated columns, then eigenvectors
  NodeResult* res = J.result;
  extern __shared__ double shm[];
  double* d = shm;                                                         // m
  double* rowp = shm + m;                                                  // m (row p of L)
  unsigned char* chosen = reinterpret_cast<unsigned char*>(shm + 2 * m);  // m
  __shared__ double red_v[kWarps], red_s[kWarps];
  __shared__ int red_i[kWarps];
  __shared__ int flag_sh;

  // ---------------- pivoted Cholesky (FP64)
  if (tid == 0) flag_sh = 0;
  __syncthreads();
  for (int i = tid; i < m; i += blockDim.x) {
    const double gi = G[(size_t)i * m + i];
    if (!isfinite(gi)) flag_sh = 1;  // NaN/Inf in a column of X reaches its diagonal entry
    d[i] = gi;
    chosen[i] = 0;
  }
  __syncthreads();
  int p0;
  double dmax0, trace;
  argmax_block(d, chosen, m, p0, dmax0, trace, red_v, red_i, red_s);
  const bool finite = flag_sh == 0 && isfinite(trace) && isfinite(dmax0);
  __syncthreads();
  if (!finite && tid == 0) res->status = HAPOD_ERR_NONFINITE;
  const double tol = (sizeof(V_t) == sizeof(double)) ? (double)m * 1.1102230246251565e-16 : 1e-7;
  const double tr_pos = trace > 0.0 ? trace : 0.0;
  const double stop_round = tol * tr_pos;
  double stop = J.eps2 > 0.0 ? fmin(stop_round, 1e-2 * J.eps2) : stop_round;
  // below the Gram's own error level the remaining pivots would factor rounding noise
  if (J.floor_rel > 0.0) stop = fmax(stop, J.floor_rel * tr_pos);
  int r = 0;
  double resid = finite && trace > 0.0 ? trace : 0.0;
  if (finite && trace > 0.0) {
    for (int k = 0; k < m; ++k) {
      int p;
      double dmax, dsum;
      argmax_block(d, chosen, m, p, dmax, dsum, red_v, red_i, red_s);
      resid = dsum;
      if (p < 0 || !(dmax > 0.0) || dsum <= stop) break;
      for (int j = tid; j < k; j += blockDim.x) rowp[j] = L[(size_t)j * m + p];  // row p of L
      __syncthreads();
      const double piv = sqrt(dmax);
      const double inv = 1.0 / piv;
      for (int i = tid; i < m; i += blockDim.x) {
        double v;
        if (i == p) {
          v = piv;
        } else if (chosen[i]) {
          v = 0.0;
        } else {
          double s = G[(size_t)p * m + i];
          for (int j = 0; j < k; ++j) s -= L[(size_t)j * m + i] * rowp[j];
          v = s * inv;
          d[i] -= v * v;
        }
        L[(size_t)k * m + i] = v;
      }
      __syncthreads();
      if (tid == 0) {
        chosen[p] = 1;
        d[p] = 0.0;
      }
      __syncthreads();
      r = k + 1;
      resid = 0.0;
    }
  }

  // ---------------- one-sided Jacobi on the r columns (precision T)
  for (size_t e = tid; e < (size_t)r * m; e += blockDim.x) W[e] = (T)L[e];
  __syncthreads();
  bool converged = false;
  const int sweeps = jacobi_sweeps<T>(W, m, r, max_sweeps, converged, &flag_sh);
  V_t* U = W;
  for (size_t e = (size_t)r * m + tid; e < (size_t)m * m; e += blockDim.x) U[e] = V_t(0);
  __syncthreads();

  // ---------------- normalised eigenvectors u_j = w_j / ||w_j||, then FP64 Rayleigh
  // quotients lambda_j = u_j^T G u_j against the original G (second order in the
  // eigenvector error, so the rounding of L and of the rotations enters squared)
  for (int j = warp; j < m; j += kWarps) {
    double s = 0.0;
    if (j < r) {
      const V_t* wj = U + (size_t)j * m;
      for (int i = lane; i < m; i += 32) s += (double)wj[i] * (double)wj[i];
      s = warp_sum(s);
    }
    if (j < r && s > 0.0) {
      const double inv = 1.0 / sqrt(s);
      V_t* wj = U + (size_t)j * m;
      for (int i = lane; i < m; i += 32) wj[i] = (V_t)((double)wj[i] * inv);
    }
  }
  __syncthreads();
  for (int j = warp; j < m; j += kWarps) {
    double acc = 0.0;
    if (j < r) {
      const V_t* uj = U + (size_t)j * m;
      for (int i = lane; i < m; i += 32) {
        double gi = 0.0;  // (G u_j)_i; G symmetric, column-major
        for (int l = 0; l < m; ++l) gi = fma(G[(size_t)l * m + i], (double)uj[l], gi);
        acc = fma((double)uj[i], gi, acc);
      }
      acc = warp_sum(acc);
    }
    if (lane == 0) J.lam_tmp[j] = acc;
  }
  __syncthreads();
  for (int j = tid; j < m; j += blockDim.x) {
    const double lj = J.lam_tmp[j];
    int rank = 0;
    for (int i = 0; i < m; ++i) {
      const double li = J.lam_tmp[i];
      rank += (li > lj) || (li == lj && i < j);
    }
    J.lambda[rank] = lj > 0.0 ? lj : 0.0;
    J.perm[rank] = j;
  }
  if (tid == 0) {
    res->sweeps = sweeps;
    res->trace = trace;
    res->rank = r;
    res->resid = resid;
    if (!converged && res->status == HAPOD_OK) res->status = HAPOD_WARN_NOCONVERGE;
  }
}

}  // namespace

int eig_threads() { return kThreads; }

size_t eig_smem_bytes(int m) { return (size_t)m * (2 * sizeof(double) + 1) + 16; }

cudaError_t launch_eig(int mode, const EigJob* jobs_dev, int njobs, int max_m, int max_sweeps, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  const size_t smem = eig_smem_bytes(max_m);
  const void* fn =
      mode == kEigF32 ? (const void*)chol_jacobi_kernel<float> : (const void*)chol_jacobi_kernel<double>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  void* args[] = {(void*)&jobs_dev, (void*)&max_sweeps};
  return cudaLaunchKernel(fn, dim3(njobs), dim3(kThreads), args, smem, s);
}

}  // namespace hapod
