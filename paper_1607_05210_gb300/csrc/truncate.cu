// K3: truncation rule of the POD (Sec. 2, Def. truncated POD and Eq. pod_error):
// N = min{N' : sum_{j >= N'} lambda_j <= eps^2}, lambda descending (0-based j,
// inclusive <=), and sigma_j = sqrt(lambda_j) for the kept j < N.  Every tail also
// carries the residual the eigensolver's factorisation left out (result->resid),
// so the rank is never smaller than the complete spectrum requires.
//
// One warp per node.  Lane l owns a contiguous chunk of the eigenvalues; chunk
// sums are Kahan-compensated, a suffix scan over lanes (warp shuffles) gives the
// sum of everything after each chunk, and each lane then walks its chunk from the
// small end.  Since the tail is non-increasing in N', the first qualifying index
// is the warp-wide minimum of the per-lane first qualifying indices.
#include "hapod_internal.cuh"

namespace hapod {
namespace {

__global__ void __launch_bounds__(128) truncate_kernel(const TruncJob* __restrict__ jobs, int njobs) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= njobs) return;
  const TruncJob J = jobs[w];
  const int m = J.m;
  const double resid = J.result->resid;
  const int chunk = (m + 31) / 32;
  const int b = min(m, lane * chunk), e = min(m, b + chunk);
  // Kahan sum of the chunk, smallest first
  double s = 0.0, c = 0.0;
  for (int j = e - 1; j >= b; --j) {
    const double y = J.lambda[j] - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
  }
  // inclusive suffix scan over lanes: after[l] = sum over lanes > l
  double incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double v = __shfl_down_sync(0xffffffffu, incl, o);
    if (lane + o < 32) incl += v;
  }
  const double after = incl - s + resid;
  // walk the chunk: tail(j) = after + sum_{i in [j, e)} lambda_i
  int first = m;  // keep everything unless a shorter prefix qualifies
  double tail_first = resid;
  double run = after, rc = 0.0;
  if (run <= J.eps2 && e > b) {
    first = e;
    tail_first = run;
  }
  for (int j = e - 1; j >= b; --j) {
    const double y = J.lambda[j] - rc;
    const double t = run + y;
    rc = (t - run) - y;
    run = t;
    if (run <= J.eps2) {
      first = j;
      tail_first = run;
    }
  }
  // warp minimum of (first, tail)
  int k = first;
  double tk = tail_first;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int ko = __shfl_xor_sync(0xffffffffu, k, o);
    const double to = __shfl_xor_sync(0xffffffffu, tk, o);
    if (ko < k) {
      k = ko;
      tk = to;
    }
  }
  for (int j = lane; j < k; j += 32) J.sigma[j] = sqrt(J.lambda[j]);
  if (lane == 0) {
    J.result->k = k;
    J.result->tail = tk;
  }
}

}  // namespace

cudaError_t launch_truncate(const TruncJob* jobs_dev, int njobs, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  const int warps_per_block = 4;
  truncate_kernel<<<(njobs + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(jobs_dev, njobs);
  return cudaGetLastError();
}

}  // namespace hapod
