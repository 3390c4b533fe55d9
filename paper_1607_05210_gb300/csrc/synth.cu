// A1, device input generation: snapshots of the travelling-pulse workload that
// stands in for the paper's PDE snapshot data (Sec. 4), written straight into HBM so
// that leaves and stream chunks never pass through the host.  No POD arithmetic.
//
// Column j (global index col0 + j) is the field at time t_j:
//   u(x_i, t_j) = sum_{k=1..32} a_k exp(-nu k^2 t_j) sin(k (x_i - c t_j))
//               + sum_p A_p exp(-d(x_i, x_p + c t_j)^2 / (2 w^2)),
// x_i = 2 pi i / n, d the periodic distance on [0, 2 pi).
// t_j: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC 2011; ten rounds, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key
// increments 0x9E3779B9 / 0xBB67AE85) with key (seed mod 2^32, seed div 2^32) and
// counter (j mod 2^32, j div 2^32, 0, 0) for global column j; the first two output
// words give t_j = (w0 2^21 + (w1 >> 11)) 2^-53, uniform on [0, 1).  Any range of
// columns can therefore be generated independently (stream chunks).
// Arithmetic: t_j, the 64 Fourier coefficients of each column and the pulse
// positions in FP64 (one thread per column); the field itself in FP32 -- sin and cos
// of k x_i from the exactly reduced argument 2 ((k i) mod n) / n, the 64-term sum,
// and each pulse within 9 w (rows from the pulse's nearest grid point, so that the
// distance is formed as an exact integer times h plus a small offset).  The double
// output holds the same FP32 values, so both precisions see identical snapshots.
#include <stdint.h>

#include "hapod_internal.cuh"

namespace hapod {
namespace {

constexpr int kHarmonics = 32;
constexpr int kRowsPerBlock = 256;
constexpr int kColChunk = 32;

__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Per column: t_j, coefficients (sin k x | cos k x) of the advection-diffusion part,
// and per pulse the nearest grid row of its centre and the offset of that row.
struct ColumnInfo {
  float coef[2 * kHarmonics];
  int64_t prow[HAPOD_SYNTH_MAX_PULSES];
  float poff[HAPOD_SYNTH_MAX_PULSES];
};

__global__ void synth_columns_kernel(hapod_synth_params p, int64_t n, int64_t col0, int64_t ncols,
                                     ColumnInfo* __restrict__ info, double* __restrict__ t_out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  const uint64_t col = (uint64_t)(col0 + j);
  uint32_t c[4] = {(uint32_t)col, (uint32_t)(col >> 32), 0u, 0u};
  philox4x32_10(c, (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
  const double t = (double)(((uint64_t)c[0] << 21) | (uint64_t)(c[1] >> 11)) * 0x1.0p-53;
  if (t_out) t_out[j] = t;
  ColumnInfo& I = info[j];
  // sin(k (x - c t)) = sin(k x) cos(k c t) - cos(k x) sin(k c t)
  for (int k = 1; k <= kHarmonics; ++k) {
    const double damp = p.harmonic_amp[k - 1] * exp(-p.nu * (double)k * (double)k * t);
    double s, co;
    sincos((double)k * p.speed * t, &s, &co);
    I.coef[k - 1] = (float)(damp * co);
    I.coef[kHarmonics + k - 1] = (float)(-damp * s);
  }
  const double two_pi = 6.283185307179586476925286766559;
  const double h = two_pi / (double)n;
  for (int q = 0; q < p.num_pulses; ++q) {
    double pos = fmod(p.pulse_centre[q] + p.speed * t, two_pi);
    if (pos < 0.0) pos += two_pi;
    int64_t r = llrint(pos / h);
    const double off = (double)r * h - pos;  // |off| <= h / 2
    r %= n;
    I.prow[q] = r;
    I.poff[q] = (float)off;
  }
}

// One block per 256 rows; every thread one row and all columns.  The pulses that
// reach the block's rows are listed per column chunk in shared memory.
template <typename T>
__global__ void __launch_bounds__(kRowsPerBlock) synth_field_kernel(hapod_synth_params p, int64_t n, int64_t ncols,
                                                                    const ColumnInfo* __restrict__ info,
                                                                    T* __restrict__ X, int64_t ldx) {
  __shared__ float s_coef[kColChunk][2 * kHarmonics];
  __shared__ unsigned long long s_mask[kColChunk];  // pulses that reach the block's rows
  const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
  const int64_t i = r0 + threadIdx.x;
  const bool live = i < n;
  // sin(k x_i), cos(k x_i): sinpi / cospi of 2 ((k i) mod n) / n
  float sv[kHarmonics], cv[kHarmonics];
  int64_t r = 0;  // (k i) mod n, one addition per k
  const double two_over_n = 2.0 / (double)n;
#pragma unroll
  for (int k = 1; k <= kHarmonics; ++k) {
    if (live) {
      r += i;
      if (r >= n) r -= n;
    }
    const float a = (float)((double)r * two_over_n);
    sincospif(a, &sv[k - 1], &cv[k - 1]);
  }
  const double two_pi = 6.283185307179586476925286766559;
  const float h = (float)(two_pi / (double)n);
  const float inv2w2 = (float)(1.0 / (2.0 * p.pulse_width * p.pulse_width));
  const float cut = (float)(9.0 * p.pulse_width);
  // rows within 9 w of a pulse centre, plus one for the offset
  const int64_t reach = (int64_t)ceil(9.0 * p.pulse_width / (two_pi / (double)n)) + 1;
  const int64_t r1 = min(n, r0 + kRowsPerBlock) - 1;  // last row of the block
  for (int64_t j0 = 0; j0 < ncols; j0 += kColChunk) {
    const int nc = (int)min((int64_t)kColChunk, ncols - j0);
    __syncthreads();  // previous chunk done with the shared lists
    for (int e = threadIdx.x; e < nc * 2 * kHarmonics; e += blockDim.x)
      s_coef[e / (2 * kHarmonics)][e % (2 * kHarmonics)] = info[j0 + e / (2 * kHarmonics)].coef[e % (2 * kHarmonics)];
    if (threadIdx.x < kColChunk) s_mask[threadIdx.x] = 0ull;
    __syncthreads();
    // periodic row distance from each pulse row to the block's row interval [r0, r1]
    for (int e = threadIdx.x; e < nc * p.num_pulses; e += blockDim.x) {
      const int jj = e / p.num_pulses, q = e % p.num_pulses;
      const int64_t pr = info[j0 + jj].prow[q];
      int64_t d = 0;
      if (pr < r0) d = min(r0 - pr, pr + n - r1);
      else if (pr > r1) d = min(pr - r1, r0 + n - pr);
      if (d <= reach) atomicOr(&s_mask[jj], 1ull << q);
    }
    __syncthreads();
    if (!live) continue;
    for (int jj = 0; jj < nc; ++jj) {
      float u = 0.f;
#pragma unroll
      for (int k = 0; k < kHarmonics; ++k) u = fmaf(s_coef[jj][k], sv[k], fmaf(s_coef[jj][kHarmonics + k], cv[k], u));
      // pulses in ascending order, so that every column range gives the same bits
      for (unsigned long long mask = s_mask[jj]; mask; mask &= mask - 1ull) {
        const int q = __ffsll((long long)mask) - 1;
        int64_t dr = i - info[j0 + jj].prow[q];  // periodic representative
        if (dr > n / 2) dr -= n;
        else if (dr < -(n / 2)) dr += n;
        if (dr > reach || dr < -reach) continue;
        const float d = fmaf((float)dr, h, info[j0 + jj].poff[q]);
        if (fabsf(d) > cut) continue;
        u = fmaf((float)p.pulse_amp[q], expf(-d * d * inv2w2), u);
      }
      X[(size_t)(j0 + jj) * (size_t)ldx + (size_t)i] = (T)u;
    }
  }
}

}  // namespace
}  // namespace hapod

using namespace hapod;

extern "C" hapod_status hapod_synth_snapshots(const hapod_synth_params* p, int64_t n, int64_t col0, int64_t ncols,
                                              int32_t dtype, void* X, int64_t ldx, double* t_out, void* stream) {
  if (!p || n < 1 || col0 < 0 || ncols < 0 || ldx < n || (dtype != 0 && dtype != 1) || (ncols > 0 && !X) ||
      p->num_pulses < 0 || p->num_pulses > HAPOD_SYNTH_MAX_PULSES || (p->num_pulses > 0 && !(p->pulse_width > 0.0)) ||
      n > ((int64_t)1 << 36)) {
    set_thread_error("hapod_synth_snapshots: invalid argument");
    return HAPOD_ERR_INVALID;
  }
  if (ncols == 0) return HAPOD_OK;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  ColumnInfo* info = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&info), sizeof(ColumnInfo) * (size_t)ncols, s);
  if (e != cudaSuccess) {
    set_thread_error(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HAPOD_ERR_OOM : HAPOD_ERR_CUDA;
  }
  synth_columns_kernel<<<(unsigned)((ncols + 127) / 128), 128, 0, s>>>(*p, n, col0, ncols, info, t_out);
  const unsigned blocks = (unsigned)((n + kRowsPerBlock - 1) / kRowsPerBlock);
  if (dtype == 0)
    synth_field_kernel<float><<<blocks, kRowsPerBlock, 0, s>>>(*p, n, ncols, info, static_cast<float*>(X), ldx);
  else
    synth_field_kernel<double><<<blocks, kRowsPerBlock, 0, s>>>(*p, n, ncols, info, static_cast<double*>(X), ldx);
  e = cudaGetLastError();
  const cudaError_t ef = cudaFreeAsync(info, s);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) {
    set_thread_error(cudaGetErrorString(e));
    return HAPOD_ERR_CUDA;
  }
  return HAPOD_OK;
}
