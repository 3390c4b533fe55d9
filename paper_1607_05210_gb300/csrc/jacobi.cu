// K2: eigen-decomposition of a node's Gramian G (Sec. 2, Remark
// def:method_of_snapshots: lambda_k, psi_k of G give the POD).
//
// Method: one-sided cyclic Jacobi applied to the columns of A := G / trace(G).
// Plane rotations from the right orthogonalise the columns, A J = G V with V the
// accumulated rotations; once the columns of G V are mutually orthogonal,
// V^T G^2 V is diagonal, so V diagonalises the PSD matrix G.  The eigenvalues are
// taken as Rayleigh quotients lambda_j = v_j^T (G v_j) accumulated in FP64.
// Pairs follow the round-robin ("circle") ordering: in step t every index is in
// exactly one pair, so the m/2 rotations of a step touch disjoint columns and run
// concurrently, one warp per pair; a sweep is m' - 1 steps (m' = m rounded up to
// even).  A pair is rotated while |a_p.a_q| > tol ||a_p|| ||a_q|| with
// tol = m * unit roundoff of T; columns whose squared norm is below
// (1e-3 u)^2 trace(G)^2, far under the rounding level, are treated as zero.
//
// T = double for the FP64 form; T = float for the mixed form (FP32 rotations on
// the FP64-accumulated Gram; the Rayleigh quotients are still FP64 sums).
//
// Several CTAs may cooperate on one large node (group > 1): they share the pair
// list of each step and meet at a software grid barrier whose spin is bounded
// (~2 s); a timeout sets HAPOD_ERR_TIMEOUT and every CTA returns.  Such groups
// are launched cooperatively so that all their CTAs are co-resident.
#include <cooperative_groups.h>

#include "hapod_internal.cuh"

namespace hapod {
namespace {

constexpr int kThreads = 1024;
constexpr long long kSpinBudget = 4000000000LL;  // clock64 cycles (~2 s)

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

// Group barrier over `nblocks` CTAs: sync[0] = arrival count, sync[1] =
// generation, sync[7] = abort.  Returns false if the wait ran out or another CTA
// aborted; the caller then returns.
__device__ bool group_barrier(unsigned* sync, unsigned nblocks, NodeResult* res) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = sync + 1;
    volatile unsigned* vabort = sync + 7;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(sync, 1u);
    if (arrived == nblocks - 1) {
      sync[0] = 0;
      __threadfence();
      atomicAdd(sync + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (*vabort) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > kSpinBudget) {
          atomicExch(sync + 7, 1u);
          res->status = HAPOD_ERR_TIMEOUT;
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*vabort) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ bool sync_all(int group, unsigned* sync, NodeResult* res) {
  if (group == 1) {
    __syncthreads();
    return true;
  }
  return group_barrier(sync, (unsigned)group, res);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) jacobi_kernel(const EigJob* __restrict__ jobs,
                                                          const int2* __restrict__ block_map, int max_sweeps) {
  const int2 bm = block_map[blockIdx.x];
  const EigJob J = jobs[bm.x];
  const int rank = bm.y, group = J.group, m = J.m;
  if (m <= 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps_blk = blockDim.x >> 5;
  const double* __restrict__ G = J.G;
  T* A = static_cast<T*>(J.A);
  T* V = static_cast<T*>(J.V);
  NodeResult* res = J.result;

  // trace (every CTA computes it; m reads)
  __shared__ double red[32];
  __shared__ int flag_sh;
  double tr = 0.0;
  for (int i = tid; i < m; i += blockDim.x) tr += G[(size_t)i * m + i];
  tr = warp_sum(tr);
  if (lane == 0) red[warp] = tr;
  __syncthreads();
  if (warp == 0) {
    double v = lane < nwarps_blk ? red[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  tr = red[0];
  if (!isfinite(tr) || tr <= 0.0) {
    // NaN/Inf, or G = 0 (a PSD matrix with zero trace): nothing to rotate
    if (rank == 0) {
      for (int i = tid; i < m; i += blockDim.x) {
        J.lambda[i] = 0.0;
        J.perm[i] = i;
      }
      for (size_t e = tid; e < (size_t)m * m; e += blockDim.x) V[e] = (e % (m + 1) == 0) ? T(1) : T(0);
      if (tid == 0) {
        res->sweeps = 0;
        res->trace = tr;
        if (!isfinite(tr)) res->status = HAPOD_ERR_NONFINITE;
      }
    }
    return;
  }
  const double inv = 1.0 / tr;
  {
    const size_t total = (size_t)m * m;
    const size_t stride = (size_t)group * blockDim.x;
    for (size_t e = (size_t)rank * blockDim.x + tid; e < total; e += stride) {
      A[e] = (T)(G[e] * inv);
      V[e] = (e % (m + 1) == 0) ? T(1) : T(0);
    }
  }
  if (!sync_all(group, J.sync, res)) return;

  const int mp = m + (m & 1), npairs = mp / 2;
  const int gwarp = rank * nwarps_blk + warp, nwarps = group * nwarps_blk;
  const T tol = (T)m * Unit<T>::eps();
  const T negligible = T(1e-6) * Unit<T>::eps() * Unit<T>::eps();  // ||A||_F <= trace(A) = 1
  int sweep = 0;
  bool converged = false;
  for (sweep = 1; sweep <= max_sweeps; ++sweep) {
    if (tid == 0) flag_sh = 0;
    if (group > 1 && rank == 0 && tid == 0) J.sync[2 + (sweep + 1) % 3] = 0u;
    __syncthreads();
    int rotated = 0;
    for (int t = 0; t < mp - 1; ++t) {
      for (int k = gwarp; k < npairs; k += nwarps) {
        int p, q;
        rr_pair(t, k, mp, p, q);
        if (p >= m || q >= m) continue;
        T* ap = A + (size_t)p * m;
        T* aq = A + (size_t)q * m;
        T al = 0, be = 0, ga = 0;
        for (int i = lane; i < m; i += 32) {
          const T x = ap[i], y = aq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga == T(0) || al <= negligible || be <= negligible) continue;
        if (fabs(ga) <= tol * sqrt(al * be)) continue;
        rotated = 1;
        const T zeta = (be - al) / (T(2) * ga);
        // smaller root of t^2 + 2 zeta t - 1 = 0; 1/(2 zeta) once zeta^2 would overflow
        const T tt = fabs(zeta) > T(1e15) ? T(0.5) / zeta
                                           : (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + tt * tt);
        const T s = c * tt;
        for (int i = lane; i < m; i += 32) {
          const T x = ap[i], y = aq[i];
          ap[i] = c * x - s * y;
          aq[i] = s * x + c * y;
        }
        T* vp = V + (size_t)p * m;
        T* vq = V + (size_t)q * m;
        for (int i = lane; i < m; i += 32) {
          const T x = vp[i], y = vq[i];
          vp[i] = c * x - s * y;
          vq[i] = s * x + c * y;
        }
      }
      if (!sync_all(group, J.sync, res)) return;
    }
    if (rotated && lane == 0) flag_sh = 1;
    __syncthreads();
    if (group == 1) {
      converged = (flag_sh == 0);
    } else {
      if (tid == 0 && flag_sh) atomicOr(J.sync + 2 + sweep % 3, 1u);
      if (!group_barrier(J.sync, (unsigned)group, res)) return;
      if (tid == 0) flag_sh = ((volatile unsigned*)J.sync)[2 + sweep % 3] != 0u;
      __syncthreads();
      converged = (flag_sh == 0);
    }
    __syncthreads();  // every thread has read flag_sh before the next sweep resets it
    if (converged) break;
  }

  // Rayleigh quotients lambda_j = v_j . (G v_j), FP64 sums, one warp per column
  for (int j = gwarp; j < m; j += nwarps) {
    const T* vj = V + (size_t)j * m;
    const T* aj = A + (size_t)j * m;
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s += (double)vj[i] * (double)aj[i];
    s = warp_sum(s);
    if (lane == 0) J.lam_tmp[j] = s * tr;
  }
  if (!sync_all(group, J.sync, res)) return;
  if (rank != 0) return;
  // rank sort, descending, ties by index
  for (int j = tid; j < m; j += blockDim.x) {
    const double lj = J.lam_tmp[j];
    int r = 0;
    for (int i = 0; i < m; ++i) {
      const double li = J.lam_tmp[i];
      r += (li > lj) || (li == lj && i < j);
    }
    J.lambda[r] = lj > 0.0 ? lj : 0.0;
    J.perm[r] = j;
  }
  if (tid == 0) {
    res->sweeps = converged ? sweep : max_sweeps;
    res->trace = tr;
    if (!converged && res->status == HAPOD_OK) res->status = HAPOD_WARN_NOCONVERGE;
  }
}

}  // namespace

int eig_threads() { return kThreads; }

cudaError_t launch_eig(bool fp64, const EigJob* jobs_dev, const int2* block_map_dev, int num_blocks,
                       bool cooperative, int max_sweeps, cudaStream_t s) {
  if (num_blocks <= 0) return cudaSuccess;
  void* args[] = {(void*)&jobs_dev, (void*)&block_map_dev, (void*)&max_sweeps};
  const void* fn = fp64 ? (const void*)jacobi_kernel<double> : (const void*)jacobi_kernel<float>;
  if (cooperative) return cudaLaunchCooperativeKernel(fn, dim3(num_blocks), dim3(kThreads), args, 0, s);
  return cudaLaunchKernel(fn, dim3(num_blocks), dim3(kThreads), args, 0, s);
}

}  // namespace hapod
