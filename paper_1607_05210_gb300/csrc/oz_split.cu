// Digit slices of FP64 snapshots for the digit-slice FP64 form: the error-free
// splitting of Ozaki, Ogita, Oishi and Rump (2012), "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and its
// applications", specialised to a fixed-point representation per column.
//
// Column j gets the power-of-two bound 2^E_j > max_i |x_ij|.  Every value is
// truncated to the fixed-point integer A = floor(|x| 2^(55 - E_j)) < 2^55 and
// written in balanced base 256 with 7 digits (oz_common.cuh),
//   A = d_1 2^48 + d_2 2^40 + ... + d_7,   d_1 in [0, 128], d_2..d_7 in [-128, 127],
// so x = sign(x) 2^(E_j+1) sum_t d_t 2^(-8 t) up to the dropped tail (< 2^(E_j - 55)).
//
// Layout of a digit block (rows [r0, r0 + rows) of one node):
//   [row group r/8][digit t][column group j/8][j % 8][r % 8]   (fp16)
// i.e. 8 x 8 core matrices of 16-byte rows; one digit plane of one row group is a
// contiguous run of ceil(m / 8) column groups.  Read as columns-by-rows it is the
// K-major no-swizzle UMMA layout of the Gram (K = rows), and consecutive digit
// planes of a block of column groups form one operand of up to 4 digits.
#include <algorithm>

#include "hapod_internal.cuh"
#include "oz_common.cuh"

namespace hapod {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// One block per column: E_j from the largest |x| (compared as bit patterns, which
// orders non-negative doubles; Inf and NaN patterns are above every finite one).
__global__ void __launch_bounds__(kThreads) oz_colmax_kernel(const OzColJob* __restrict__ jobs, int njobs) {
  const int64_t b = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].col_base <= b) lo = mid; else hi = mid - 1;
  }
  const OzColJob J = jobs[lo];
  const int64_t j = b - J.col_base;
  if (j >= J.m) return;
  const unsigned long long* col = reinterpret_cast<const unsigned long long*>(J.X + j * J.ldx);
  uint64_t mx = 0;
  for (int64_t i = threadIdx.x; i < J.n; i += kThreads) {
    const uint64_t a = col[i] & 0x7FFFFFFFFFFFFFFFull;
    mx = a > mx ? a : mx;
  }
  mx = warp_max_u64(mx);
  __shared__ uint64_t red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kThreads / 32; ++w) mx = red[w] > mx ? red[w] : mx;
    int32_t E;
    if (mx >= 0x7FF0000000000000ull) {
      E = kOzNonFinite;
    } else {
      // max in [2^(eb-1023), 2^(eb-1022)) for a normal max; below 2^-1022 otherwise
      const int eb = (int)(mx >> 52);
      E = eb == 0 ? -1022 : eb - 1022;
    }
    J.exps[j] = E;
  }
}

// Tile = 64 rows x 32 columns (8 row groups x 4 column groups) of one digit block.
// Blocks are persistent: each walks the tiles with a stride of the grid and
// prefetches its next FP64 tile (8-byte cp.async, zero-filled outside X) into the
// other half of a double buffer while it converts the current one.  The tile is
// read column by column (each warp 256-byte runs of one column) into shared
// memory, then thread (row group, column) converts 8 consecutive rows of one column
// into one 16-byte core-matrix row per digit; the 32 lanes (32 consecutive columns)
// write one 512-byte segment per digit.
constexpr int kTileRows = 64, kTileCols = 32;
constexpr int kPitch = kTileRows + 1;  // doubles: conflict-free column-wise reads
constexpr int kBlocksPerSM = 4;

__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

struct SplitTile {
  int job;
  int64_t rt;  // 64-row tile
  int c0;      // first column
};

__device__ __forceinline__ SplitTile split_tile(const OzSplitJob* __restrict__ jobs, int njobs, int64_t b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].block_base <= b) lo = mid; else hi = mid - 1;
  }
  const int64_t local = b - jobs[lo].block_base;
  const int ct = (jobs[lo].CGs + 3) / 4;  // column tiles
  SplitTile t;
  t.job = lo;
  t.rt = local / ct;
  t.c0 = (int)(local - t.rt * ct) * kTileCols;
  return t;
}

__device__ __forceinline__ void split_load(double (*tile)[kPitch], const OzSplitJob& J, const SplitTile& t) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = t.rt * kTileRows;
  for (int cc = warp; cc < kTileCols; cc += kThreads / 32) {
    const int j = t.c0 + cc;
    const bool col = j < J.m && J.exps[j] != kOzNonFinite;
    const double* src = J.X + (int64_t)(col ? j : 0) * J.ldx + J.r0;
#pragma unroll
    for (int h = 0; h < kTileRows / 32; ++h) {
      const int64_t r = r0 + lane + 32 * h;
      const bool in = col && r < J.rows;
      cp_async8(&tile[cc][lane + 32 * h], in ? src + r : J.X, in ? 8 : 0);
    }
  }
}

__global__ void __launch_bounds__(kThreads) oz_split_kernel(const OzSplitJob* __restrict__ jobs, int njobs,
                                                            int64_t total_tiles) {
  __shared__ double tile[2][kTileCols][kPitch];
  int64_t b = blockIdx.x;
  SplitTile cur;
  if (b < total_tiles) {
    cur = split_tile(jobs, njobs, b);
    split_load(tile[0], jobs[cur.job], cur);
  }
  cp_async_commit();
  for (int it = 0; b < total_tiles; ++it, b += gridDim.x) {
    const int buf = it & 1;
    const int64_t nb = b + gridDim.x;
    SplitTile nxt;
    if (nb < total_tiles) {
      nxt = split_tile(jobs, njobs, nb);
      split_load(tile[buf ^ 1], jobs[nxt.job], nxt);
    }
    cp_async_commit();
    cp_async_wait_1();  // the current tile's copies have landed (this thread's)
    __syncthreads();    // ... and every thread's
    const OzSplitJob& J = jobs[cur.job];
    const int cc = threadIdx.x & 31;   // column in the tile
    const int rgl = threadIdx.x >> 5;  // row group in the tile
    const int j = cur.c0 + cc;
    const int64_t rg = cur.rt * 8 + rgl;
    if (rg < oz_row_groups(J.rows) && (j >> 3) < J.CGs) {
      const int E = j < J.m ? J.exps[j] : kOzNonFinite;
      uint32_t w[kOzDigits][4];
#pragma unroll
      for (int q = 0; q < kOzDigits; ++q) w[q][0] = w[q][1] = w[q][2] = w[q][3] = 0u;
      if (E != kOzNonFinite) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          uint32_t d[kOzDigits];
          oz_digits2(tile[buf][cc][rgl * 8 + 2 * p], tile[buf][cc][rgl * 8 + 2 * p + 1], E, d);
#pragma unroll
          for (int q = 0; q < kOzDigits; ++q) w[q][p] = d[q];
        }
      }
      uint4* out = reinterpret_cast<uint4*>(J.digits) + ((rg * kOzDigits) * J.CGs + (j >> 3)) * 8 + (j & 7);
#pragma unroll
      for (int q = 0; q < kOzDigits; ++q) out[(size_t)q * J.CGs * 8] = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
    __syncthreads();  // the buffer is refilled two tiles on
    cur = nxt;
  }
}

dim3 grid_for(int64_t blocks) {
  const int64_t gx = blocks < 65535 ? blocks : 65535;
  return dim3((unsigned)gx, (unsigned)((blocks + gx - 1) / gx));
}

}  // namespace

cudaError_t launch_oz_colmax(const OzColJob* jobs_dev, int njobs, int64_t total_cols, cudaStream_t s) {
  if (njobs <= 0 || total_cols <= 0) return cudaSuccess;
  oz_colmax_kernel<<<grid_for(total_cols), kThreads, 0, s>>>(jobs_dev, njobs);
  return cudaGetLastError();
}

int64_t oz_split_blocks(int64_t rows, int32_t CGs) {
  return (oz_row_groups(rows) + 7) / 8 * ((CGs + 3) / 4);
}

cudaError_t launch_oz_split(const OzSplitJob* jobs_dev, int njobs, int64_t total_blocks, cudaStream_t s) {
  if (njobs <= 0 || total_blocks <= 0) return cudaSuccess;
  const int64_t grid = std::min<int64_t>(total_blocks, (int64_t)kNumSMs * kBlocksPerSM);
  oz_split_kernel<<<(unsigned)grid, kThreads, 0, s>>>(jobs_dev, njobs, total_blocks);
  return cudaGetLastError();
}

}  // namespace hapod
