// hapod_gram_noalloc: the FP64 Gram G = X^T X without any device allocation.
//
// Who needs this: callers that are not allowed to allocate device memory once
// they are running -- for example an application whose own allocator has already
// reserved nearly all of the GPU's memory, or a latency-bound pipeline that must
// not pay for (or synchronise on) cudaMalloc/cudaFree.  hapod_gram takes its
// split-K workspace and work list from a stream-ordered pool; this entry point
// instead keeps the split partials in a fixed array that lives in the library's
// device image (`g_noalloc_scratch`, 32 MiB, held on every GPU that loads the
// library until the process exits) and derives each CTA's work from blockIdx, so
// nothing is allocated per call.
//
// Limits and sharing: the scratch holds kNoallocTiles partial 64 x 64 tiles, so
// the upper triangle of G may have at most kNoallocTiles tiles (m <= 2816); wider
// inputs are rejected with HAPOD_ERR_INVALID.  Every call uses the same scratch:
// each partial tile is written in full before it is read, so nothing has to start
// at zero, but two calls whose kernels overlap on the GPU (different streams
// without ordering) race on it.  The first call on a device looks up the scratch
// address with cudaGetSymbolAddress (once per device, with that device current)
// and keeps it for the life of the process; make that first call before any stream
// capture (a first call inside a capture is rejected with HAPOD_ERR_INVALID).  The
// kept address belongs to the device context that existed at that call: after
// cudaDeviceReset on that device this entry point must not be called again in the
// same process.
#include <algorithm>
#include <mutex>
#include <string>

#include "hapod_internal.cuh"

namespace {

constexpr int kTile = 64;
constexpr int kBK = 32;
constexpr int kNoallocTiles = 1024;                       // partial tiles in the scratch
constexpr int kMinRowsPerSplit = 256;

static __device__ __align__(256) double g_noalloc_scratch[(size_t)kNoallocTiles * kTile * kTile];

struct NoallocJob {
  const double* X;
  double* G;
  double* scratch;
  int64_t ldx;
  int64_t n;
  int64_t rows_per_split;
  int32_t m;
  int32_t tiles;   // tiles per dimension
  int32_t splits;
  int32_t pad;
};

// upper-triangle tile index t -> (ti, tj), ti <= tj, row-major over ti
__device__ __forceinline__ void tile_of(int t, int tiles, int& ti, int& tj) {
  int i = 0, rem = t;
  while (rem >= tiles - i) {
    rem -= tiles - i;
    ++i;
  }
  ti = i;
  tj = i + rem;
}

// block b = tile * splits + split; partial tile b goes to scratch slot b
__global__ void __launch_bounds__(256) noalloc_gram_tiles(const NoallocJob J) {
  const int tile = blockIdx.x / J.splits, sp = blockIdx.x % J.splits;
  int ti, tj;
  tile_of(tile, J.tiles, ti, tj);
  const int64_t r0 = (int64_t)sp * J.rows_per_split;
  const int64_t r1 = min(J.n, r0 + J.rows_per_split);
  const bool diag = (ti == tj);
  __shared__ double As[kBK][kTile + 1];
  __shared__ double Bs[kBK][kTile + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tid & 15, ty = tid >> 4;
  const int i0 = ti * kTile, j0 = tj * kTile;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int64_t rb = r0; rb < r1; rb += kBK) {
    const int64_t r = rb + lane;
    const bool rok = r < r1;
    for (int c = warp; c < kTile; c += 8) {
      const int ci = i0 + c;
      As[lane][c] = (rok && ci < J.m) ? J.X[(size_t)ci * J.ldx + r] : 0.0;
      if (!diag) {
        const int cj = j0 + c;
        Bs[lane][c] = (rok && cj < J.m) ? J.X[(size_t)cj * J.ldx + r] : 0.0;
      }
    }
    __syncthreads();
    const double(*B)[kTile + 1] = diag ? As : Bs;
#pragma unroll 4
    for (int k = 0; k < kBK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[k][ty + 16 * q];
        b[q] = B[k][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
  double* out = J.scratch + (size_t)blockIdx.x * kTile * kTile;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) out[(ty + 16 * p) * kTile + tx + 16 * q] = acc[p][q];
}

// one CTA per tile: sum its splits in order, write both triangles of G
__global__ void __launch_bounds__(256) noalloc_gram_reduce(const NoallocJob J) {
  int ti, tj;
  tile_of(blockIdx.x, J.tiles, ti, tj);
  const double* part = J.scratch + (size_t)blockIdx.x * J.splits * kTile * kTile;
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    double s = 0.0;
    for (int sp = 0; sp < J.splits; ++sp) s += part[(size_t)sp * kTile * kTile + e];
    const int gi = ti * kTile + e / kTile, gj = tj * kTile + e % kTile;
    if (gi < J.m && gj < J.m) {
      J.G[(size_t)gj * J.m + gi] = s;
      J.G[(size_t)gi * J.m + gj] = s;
    }
  }
}

std::mutex g_mu;
double* g_scratch_ptr[64] = {nullptr};  // device address of the scratch, per device ordinal

hapod_status fail(hapod_status st, const std::string& msg) {
  hapod::set_thread_error(msg.c_str());
  return st;
}

}  // namespace

extern "C" {

hapod_status hapod_gram_noalloc(int64_t n, int64_t m, const double* X, int64_t ldx, double* G, void* stream) {
  if (n < 0 || m < 0 || ldx < n || (m > 0 && (!X || !G))) {
    return fail(HAPOD_ERR_INVALID, "hapod_gram_noalloc: invalid argument");
  }
  if (m == 0) return HAPOD_OK;
  const int64_t tiles = (m + kTile - 1) / kTile;
  const int64_t tri = tiles * (tiles + 1) / 2;
  if (tri > kNoallocTiles) {
    return fail(HAPOD_ERR_INVALID, "hapod_gram_noalloc: m exceeds the fixed scratch (at most 2816 columns)");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(HAPOD_ERR_CUDA, std::string("hapod_gram_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  }
  if (dev < 0 || dev >= 64) {
    return fail(HAPOD_ERR_INVALID, "hapod_gram_noalloc: device ordinals of 64 and above are not supported");
  }
  double* scratch;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      // The address lookup may load the library's device image; inside a stream
      // capture that would break the caller's capture, so the set-up call has to
      // come first, outside any capture.
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      e = cudaStreamIsCapturing(s, &cs);
      if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return fail(HAPOD_ERR_INVALID,
                    "hapod_gram_noalloc: the first call on a device must be made outside stream capture "
                    "(it looks up the fixed scratch array's device address)");
      }
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(HAPOD_ERR_CUDA, std::string("hapod_gram_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  NoallocJob J;
  J.X = X;
  J.G = G;
  J.scratch = scratch;
  J.ldx = ldx;
  J.m = (int32_t)m;
  J.tiles = (int32_t)tiles;
  J.pad = 0;
  if (n == 0) {
    e = cudaMemsetAsync(G, 0, sizeof(double) * m * m, s);
  } else {
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>(kNoallocTiles / tri, n / kMinRowsPerSplit));
    int64_t rps = ((n + splits - 1) / splits + kBK - 1) / kBK * kBK;
    splits = (n + rps - 1) / rps;
    J.n = n;
    J.rows_per_split = rps;
    J.splits = (int32_t)splits;
    noalloc_gram_tiles<<<(unsigned)(tri * splits), 256, 0, s>>>(J);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      noalloc_gram_reduce<<<(unsigned)tri, 256, 0, s>>>(J);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) {
    return fail(HAPOD_ERR_CUDA, std::string("hapod_gram_noalloc: launch: ") + cudaGetErrorString(e));
  }
  return HAPOD_OK;
}

}  // extern "C"
