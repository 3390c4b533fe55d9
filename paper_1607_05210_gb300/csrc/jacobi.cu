// K2: eigen-decomposition of a node's Gramian G (Sec. 2, Remark
// def:method_of_snapshots: lambda_k, psi_k of G give the POD) for every node of a
// batch in one cooperative launch, each node spread over several CTAs.
//
// 1. Rank-revealing factorisation: diagonally pivoted Cholesky G = L L^T + S in FP64, stopping once trace(S) is
//    below min(tol trace(G), 1e-2 eps^2), tol = m 2^-53 (FP64 rotations) or 1e-7 (FP32
//    rotations), but not below the form's Gram error level floor_rel trace(G) (the
//    remaining pivots would factor rounding noise).  trace(S) (S is PSD) is returned
//    as `resid` and added to every tail of the truncation, so the dropped part is
//    accounted for exactly: no eigenvalue of G exceeds that of L L^T by more than
//    ||S|| <= trace(S);
// 2. one-sided Jacobi (Hestenes) on the r columns of L in precision T: plane rotations
//    from the right make the columns mutually orthogonal, L J = W, so L L^T = W W^T and
//    the eigenvectors are u_j = w_j / ||w_j|| (no rotation matrix is accumulated);
//    pairs in the round-robin ("circle") order, rotated while
//    |w_p . w_q| > m u ||w_p|| ||w_q||, u the unit roundoff of T.  T is FP64, FP32 or
//    the double-float DF (a pair of FP32 values, hi + lo, about 47 bits: Dekker's
//    exact product via FMA and Knuth's two-sum), which keeps near-FP64 accuracy on the
//    FP32 pipe (GB300 runs FP64 at 1/64 of the FP32 rate); with DF the columns are
//    scaled by a power of two near 1/sqrt(trace G) so that every square stays in the
//    FP32 range, and the rotation angle is formed in FP64 once per pair;
// 3. lambda_j = u_j^T G u_j in FP64 (Rayleigh quotients against the original G: second
//    order in the eigenvector error), sorted descending, clamped >= 0, zero beyond r.
// GB300 executes FP64 at about two fused multiply-adds per clock and SM, so one CTA
// per node leaves the rest of the GPU idle while an O(m r^2) sweep runs.  Here the
// CTAs of a node split every step: the rows of each Cholesky column, the pairs of
// each Jacobi round (one warp per pair), the columns of the Rayleigh quotients.  The
// CTAs of one node meet at a node barrier (global counter and generation word,
// bounded spin) after each Cholesky step and each Jacobi round; a cooperative launch
// keeps every CTA resident, and nodes never wait on one another.  A barrier that
// runs out of its budget raises the node's abort word and error status
// HAPOD_ERR_TIMEOUT; every CTA of the node then leaves.
#include <algorithm>
#include <type_traits>

#include "hapod_internal.cuh"
#include "tc_common.cuh"

namespace hapod {
namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;

// double-float: value hi + lo, |lo| <= ulp(hi) / 2
struct DF {
  float hi, lo;
};

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
template <>
struct Unit<DF> {
  static __device__ double eps() { return 7.105427357601002e-15; }  // 2^-47
};

// FP64 value -> rotation storage, and back.
template <typename T>
__device__ __forceinline__ T to_rot(double v) {
  return (T)v;
}
template <>
__device__ __forceinline__ DF to_rot<DF>(double v) {
  DF r;
  r.hi = __double2float_rn(v);
  r.lo = __double2float_rn(v - (double)r.hi);
  return r;
}
template <typename T>
__device__ __forceinline__ double from_rot(T v) {
  return (double)v;
}
template <>
__device__ __forceinline__ double from_rot<DF>(DF v) {
  return (double)v.hi + (double)v.lo;
}

// s + e = a + b exactly (two-sum, no ordering assumption)
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
  return s;
}
// (S, C) += x y for double-floats: the product hi hi exactly (p + fma residual), the
// cross terms hi lo and lo hi in FP32, lo lo (2^-48 relative) dropped; C collects
// the rounding errors of the running sum S
__device__ __forceinline__ void df_dot_acc(float& S, float& C, DF x, DF y) {
  const float p = x.hi * y.hi;
  float t = fmaf(x.hi, y.hi, -p);
  t = fmaf(x.hi, y.lo, t);
  t = fmaf(x.lo, y.hi, t);
  float e;
  S = two_sum(S, p, e);
  C += e + t;
}
// a x + b y for double-floats, renormalised
__device__ __forceinline__ DF df_lin2(DF a, DF x, DF b, DF y) {
  const float p1 = a.hi * x.hi;
  float e1 = fmaf(a.hi, x.hi, -p1);
  e1 = fmaf(a.hi, x.lo, e1);
  e1 = fmaf(a.lo, x.hi, e1);
  const float p2 = b.hi * y.hi;
  float e2 = fmaf(b.hi, y.hi, -p2);
  e2 = fmaf(b.hi, y.lo, e2);
  e2 = fmaf(b.lo, y.hi, e2);
  float e;
  const float h = two_sum(p1, p2, e);
  const float l = e + (e1 + e2);
  DF r;
  r.hi = h + l;
  r.lo = l - (r.hi - h);
  return r;
}
// warp sum of a running double-float sum (S, C), as FP64
__device__ __forceinline__ double warp_sum_df(float S, float C) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oS = __shfl_xor_sync(0xffffffffu, S, o), oC = __shfl_xor_sync(0xffffffffu, C, o);
    float e;
    S = two_sum(S, oS, e);
    C += oC + e;
  }
  return (double)S + (double)C;
}

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

// Node barrier of the CTAs of one job.  Returns false once the job aborted (a wait
// ran out here or elsewhere).
struct NodeBarrier {
  EigSync* s;
  unsigned ncta;
  unsigned gen;  // generation this CTA waits to leave
  tc::WaitBudget wb;

  __device__ bool sync() {
    __syncthreads();
    __shared__ int ok_sh;
    if (threadIdx.x == 0) {
      int ok = 1;
      volatile unsigned* vgen = &s->gen;
      volatile int* vabort = &s->abort;
      __threadfence();
      const unsigned arrived = atomicAdd(&s->count, 1u) + 1u;
      if (arrived == ncta) {
        atomicExch(&s->count, 0u);
        __threadfence();
        atomicExch(&s->gen, gen + 1u);
      } else {
        const long long t0 = clock64();
        while (*vgen == gen) {
          if (*vabort) {
            ok = 0;
            break;
          }
          if (clock64() - t0 > wb.cycles) {
            atomicExch(&s->abort, 1);
            ok = 0;
            break;
          }
        }
      }
      __threadfence();
      if (*vabort) ok = 0;
      gen += 1u;
      ok_sh = ok;
    }
    __syncthreads();
    const bool ok = ok_sh != 0;
    __syncthreads();
    return ok;
  }
};

// Block-wide argmax of d[i] (ties: lowest index) and sum of the positive d[i];
// chosen pivots hold -inf and take part in neither.  Every thread of the CTA
// receives the results.
__device__ void argmax_block(const double* d, int m, int& p, double& dmax, double& dsum,
                             double* red_v, int* red_i, double* red_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double best = -1.0, sum = 0.0;
  int bi = -1;
  for (int i = tid; i < m; i += blockDim.x) {
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
    for (int w = 0; w < kWarps; ++w) {
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

__device__ __forceinline__ int find_job(const EigJob* jobs, int njobs, int cta) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].cta0 <= cta) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) eig_coop_kernel(const EigJob* __restrict__ jobs, int njobs,
                                                            int max_sweeps, const int* err) {
  const int jb = find_job(jobs, njobs, blockIdx.x);
  const EigJob J = jobs[jb];
  const int c = blockIdx.x - J.cta0;  // this CTA within the job
  const int P = J.ncta;
  const int m = J.m;
  if (m <= 0 || c >= P) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* __restrict__ G = J.G;
  double* L = static_cast<double*>(J.A);  // m x m FP64 (first r columns used)
  T* W = static_cast<T*>(J.V);           // m x m in T: rotated columns, then eigenvectors
  double* d = J.lam_tmp;                  // Schur complement diagonal (even steps), then eigenvalues
  // odd steps of the factorisation read and write a second copy of the diagonal, so
  // that no CTA overwrites entries another CTA of the node is still searching for the
  // pivot of the same step (with one CTA the copy is d itself: the search ends in a
  // CTA barrier before any update); W is free until the rotations start and holds at
  // least m doubles whenever the node has more than one CTA (m > 8)
  double* d_odd = P > 1 ? reinterpret_cast<double*>(W) : d;
  int32_t* perm = J.perm;
  NodeResult* res = J.result;
  extern __shared__ double rowp[];        // row p of L
  __shared__ double red_v[kWarps], red_s[kWarps];
  __shared__ int red_i[kWarps];
  __shared__ int flag_sh;
  NodeBarrier bar{J.sync, (unsigned)P, 0u, tc::wait_budget(err)};
  // rows of this CTA for row-parallel steps
  const int chunk = (m + P - 1) / P;
  const int i0 = c * chunk, i1 = min(m, i0 + chunk);

  // ---------------- pivoted Cholesky (FP64)
  if (tid == 0) flag_sh = 0;
  __syncthreads();
  for (int i = i0 + tid; i < i1; i += blockDim.x) d[i] = G[(size_t)i * m + i];
  // every CTA checks the whole diagonal for non-finite values (NaN/Inf in a column of
  // X reaches its diagonal entry) and forms the same trace
  for (int i = tid; i < m; i += blockDim.x)
    if (!isfinite(G[(size_t)i * m + i])) flag_sh = 1;
  if (!bar.sync()) goto timeout;
  {
    int p0;
    double dmax0, trace;
    argmax_block(d, m, p0, dmax0, trace, red_v, red_i, red_s);
    const bool finite = flag_sh == 0 && isfinite(trace) && isfinite(dmax0);
    if (!finite && c == 0 && tid == 0) res->status = HAPOD_ERR_NONFINITE;
    const double tol = (sizeof(T) == sizeof(double)) ? (double)m * 1.1102230246251565e-16 : 1e-7;
    const double tr_pos = trace > 0.0 ? trace : 0.0;
    const double stop_round = tol * tr_pos;
    double stop = J.eps2 > 0.0 ? fmin(stop_round, 1e-2 * J.eps2) : stop_round;
    if (J.floor_rel > 0.0) stop = fmax(stop, J.floor_rel * tr_pos);
    int r = 0;
    double resid = finite && trace > 0.0 ? trace : 0.0;
    if (finite && trace > 0.0) {
      for (int k = 0; k < m; ++k) {
        int p;
        double dmax, dsum;
        const double* dc = (k & 1) ? d_odd : d;  // this step's diagonal
        double* dn = (k & 1) ? d : d_odd;        // the next step's
        argmax_block(dc, m, p, dmax, dsum, red_v, red_i, red_s);
        resid = dsum;
        if (p < 0 || !(dmax > 0.0) || dsum <= stop) break;
        for (int j = tid; j < k; j += blockDim.x) rowp[j] = L[(size_t)j * m + p];
        __syncthreads();
        const double piv = sqrt(dmax);
        const double inv = 1.0 / piv;
        for (int i = i0 + tid; i < i1; i += blockDim.x) {
          double v;
          const double di = dc[i];
          if (i == p) {
            v = piv;
            dn[i] = -INFINITY;  // chosen
          } else if (di == -INFINITY) {
            v = 0.0;
            dn[i] = -INFINITY;
          } else {
            double s = G[(size_t)p * m + i];
            for (int j = 0; j < k; ++j) s -= L[(size_t)j * m + i] * rowp[j];
            v = s * inv;
            dn[i] = di - v * v;
          }
          L[(size_t)k * m + i] = v;
        }
        r = k + 1;
        resid = 0.0;
        if (!bar.sync()) goto timeout;
      }
    }

    // ---------------- one-sided Jacobi on the r columns (precision T)
    // W held the odd steps' diagonal: every CTA must be done with its last pivot search
    if (P > 1 && !bar.sync()) goto timeout;
    // DF: columns scaled by 2^-e, 2^e near sqrt(trace G) (exact; the eigenvectors and
    // the convergence test do not depend on it)
    const double wscale = std::is_same<T, DF>::value && trace > 0.0 ? ldexp(1.0, -ilogb(sqrt(trace))) : 1.0;
    for (int j = 0; j < r; ++j)
      for (int i = i0 + tid; i < i1; i += blockDim.x) W[(size_t)j * m + i] = to_rot<T>(L[(size_t)j * m + i] * wscale);
    if (!bar.sync()) goto timeout;
    const int rp = r + (r & 1), npairs = rp / 2;
    const int nw = P * kWarps, wg = c * kWarps + warp;
    const auto rtol = m * Unit<T>::eps();
    int sweeps = 0;
    bool converged = (r <= 1);
    volatile int* rot_sweep = &J.sync->rot_sweep;
    while (!converged && sweeps < max_sweeps) {
      ++sweeps;
      for (int t = 0; t < rp - 1; ++t) {
        for (int k = wg; k < npairs; k += nw) {
          int p, q;
          rr_pair(t, k, rp, p, q);
          if (p >= r || q >= r) continue;
          T* wp = W + (size_t)p * m;
          T* wq = W + (size_t)q * m;
          if constexpr (std::is_same<T, DF>::value) {
            float aS = 0.f, aC = 0.f, bS = 0.f, bC = 0.f, gS = 0.f, gC = 0.f;
            for (int i = lane; i < m; i += 32) {
              const DF x = wp[i], y = wq[i];
              df_dot_acc(aS, aC, x, x);
              df_dot_acc(bS, bC, y, y);
              df_dot_acc(gS, gC, x, y);
            }
            const double al = warp_sum_df(aS, aC), be = warp_sum_df(bS, bC), ga = warp_sum_df(gS, gC);
            if (ga == 0.0 || !(fabs(ga) > rtol * sqrt(al * be))) continue;
            if (lane == 0 && *rot_sweep < sweeps) atomicMax(&J.sync->rot_sweep, sweeps);
            const double zeta = (be - al) / (2.0 * ga);
            const double tt = fabs(zeta) > 1e15 ? 0.5 / zeta
                                                : (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double cs = 1.0 / sqrt(1.0 + tt * tt);
            const DF c = to_rot<DF>(cs), sn = to_rot<DF>(cs * tt), msn = to_rot<DF>(-(cs * tt));
            for (int i = lane; i < m; i += 32) {
              const DF x = wp[i], y = wq[i];
              wp[i] = df_lin2(c, x, msn, y);
              wq[i] = df_lin2(sn, x, c, y);
            }
            continue;
          } else {
          T al = 0, be = 0, ga = 0;
          for (int i = lane; i < m; i += 32) {
            const T x = wp[i], y = wq[i];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
          al = warp_sum(al);
          be = warp_sum(be);
          ga = warp_sum(ga);
          if (ga == T(0) || !(fabs(ga) > rtol * sqrt(al * be))) continue;
          if (lane == 0 && *rot_sweep < sweeps) atomicMax(&J.sync->rot_sweep, sweeps);
          const T zeta = (be - al) / (T(2) * ga);
          const T tt = fabs(zeta) > T(1e15) ? T(0.5) / zeta
                                             : (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          const T cs = T(1) / sqrt(T(1) + tt * tt);
          const T sn = cs * tt;
          for (int i = lane; i < m; i += 32) {
            const T x = wp[i], y = wq[i];
            wp[i] = cs * x - sn * y;
            wq[i] = sn * x + cs * y;
          }
          }
        }
        if (!bar.sync()) goto timeout;
      }
      converged = *rot_sweep < sweeps;  // no rotation in this sweep
    }

    // ---------------- u_j = w_j / ||w_j|| and FP64 Rayleigh quotients against G
    // (DF columns become FP64 columns in place: element i of both occupies the same 8 bytes)
    using Out = typename std::conditional<std::is_same<T, DF>::value, double, T>::type;
    for (int j = wg; j < m; j += nw) {
      Out* wj = reinterpret_cast<Out*>(W + (size_t)j * m);
      double acc = 0.0;
      if (j < r) {
        if constexpr (std::is_same<T, DF>::value) {
          const DF* wdf = W + (size_t)j * m;
          for (int i = lane; i < m; i += 32) wj[i] = from_rot(wdf[i]);
          __syncwarp();
        }
        double s = 0.0;
        for (int i = lane; i < m; i += 32) s += (double)wj[i] * (double)wj[i];
        s = warp_sum(s);
        if (s > 0.0) {
          const double inv = 1.0 / sqrt(s);
          for (int i = lane; i < m; i += 32) wj[i] = (Out)((double)wj[i] * inv);
        }
        __syncwarp();
        for (int i = lane; i < m; i += 32) {
          double gi = 0.0;  // (G u_j)_i; G symmetric, column-major
          for (int l = 0; l < m; ++l) gi = fma(G[(size_t)l * m + i], (double)wj[l], gi);
          acc = fma((double)wj[i], gi, acc);
        }
        acc = warp_sum(acc);
      } else {
        for (int i = lane; i < m; i += 32) wj[i] = Out(0);
      }
      if (lane == 0) d[j] = acc;  // d now holds the unsorted eigenvalues
    }
    if (!bar.sync()) goto timeout;
    for (int j = i0 + tid; j < i1; j += blockDim.x) {
      const double lj = d[j];
      int rank = 0;
      for (int i = 0; i < m; ++i) {
        const double li = d[i];
        rank += (li > lj) || (li == lj && i < j);
      }
      J.lambda[rank] = lj > 0.0 ? lj : 0.0;
      perm[rank] = j;  // sorted position -> column of V
    }
    if (c == 0 && tid == 0) {
      res->sweeps = sweeps;
      res->trace = trace;
      res->rank = r;
      res->resid = resid;
      if (!converged && res->status == HAPOD_OK) res->status = HAPOD_WARN_NOCONVERGE;
    }
    return;
  }
timeout:
  if (c == 0 && tid == 0) res->status = HAPOD_ERR_TIMEOUT;
}

}  // namespace

size_t eig_smem_bytes(int m) { return (size_t)std::max(m, 1) * sizeof(double); }

// Per-job CTA counts: one warp per Jacobi pair (m / 8 CTAs of 4 warps, at most 128),
// scaled down to what the GPU keeps resident; jobs beyond that go to further launches.
cudaError_t launch_eig(int mode, EigJob* jobs_host, EigJob* jobs_dev, int njobs, int max_m, int max_sweeps,
                       EigSync* sync_dev, const int* err, cudaStream_t s, HostStage* stage) {
  if (njobs <= 0) return cudaSuccess;
  const void* fn = mode == kEigF32  ? (const void*)eig_coop_kernel<float>
                   : mode == kEigDF ? (const void*)eig_coop_kernel<DF>
                                    : (const void*)eig_coop_kernel<double>;
  const size_t smem = eig_smem_bytes(max_m);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
  if (e != cudaSuccess) return e;
  const int cap = std::max(1, sms * per_sm);
  e = cudaMemsetAsync(sync_dev, 0, sizeof(EigSync) * (size_t)njobs, s);
  if (e != cudaSuccess) return e;
  int j0 = 0;
  while (j0 < njobs) {
    // the jobs of this launch: at most `cap` CTAs, at least one per job
    int j1 = j0;
    int64_t want = 0;
    while (j1 < njobs && want + 1 <= cap && j1 - j0 < cap) {
      want += std::max(1, std::min(128, (jobs_host[j1].m + 7) / 8));
      ++j1;
    }
    const double scale = want > cap ? (double)cap / (double)want : 1.0;
    int total = 0;
    for (int j = j0; j < j1; ++j) {
      EigJob& J = jobs_host[j];
      const int w = std::max(1, std::min(128, (J.m + 7) / 8));
      J.ncta = std::max(1, (int)(w * scale));
      J.cta0 = total;
      J.sync = sync_dev + j;
      total += J.ncta;
    }
    while (total > cap) {  // rounding up to one CTA per job can overshoot
      for (int j = j0; j < j1 && total > cap; ++j)
        if (jobs_host[j].ncta > 1) {
          jobs_host[j].ncta--;
          total--;
        }
      int t = 0;
      for (int j = j0; j < j1; ++j) {
        jobs_host[j].cta0 = t;
        t += jobs_host[j].ncta;
      }
    }
    e = staged_upload(stage, jobs_dev + j0, jobs_host + j0, sizeof(EigJob) * (size_t)(j1 - j0), s);
    if (e != cudaSuccess) return e;
    const EigJob* jd = jobs_dev + j0;
    int nj = j1 - j0;
    void* args[] = {(void*)&jd, (void*)&nj, (void*)&max_sweeps, (void*)&err};
    e = cudaLaunchCooperativeKernel(fn, dim3(total), dim3(kThreads), args, smem, s);
    if (e != cudaSuccess) return e;
    j0 = j1;
  }
  return cudaSuccess;
}

}  // namespace hapod
