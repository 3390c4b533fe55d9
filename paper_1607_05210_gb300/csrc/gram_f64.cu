// K1, FP64 form: Gramian G = X^T X of the method of snapshots (Sec. 2, Remark
// def:method_of_snapshots), for every node of a batch in one grouped launch.
//
// Work item = one 64 x 64 tile (ti <= tj) of one node's G over one row range
// ("split").  Each CTA streams its row range in 32-row chunks: coalesced column
// reads (a warp reads 32 consecutive rows of one column), FP64 FMAs from shared
// memory into a 4 x 4 register block per thread.  Splits are summed in a fixed
// order by a second kernel, so results are deterministic.  FP64 on GB300 runs at
// ~1/62 of the FP32 rate, so this kernel is bound by the FP64 pipe, not HBM.
#include <algorithm>
#include <vector>

#include "hapod_internal.cuh"

namespace hapod {

void plan_gram(GramJob* jobs, int njobs, int tile, int min_rows_per_split, int target_items, int4** items_out,
               int4** reduce_out, GramPlan* plan, bool split_major, int split_pct) {
  int64_t total_tiles = 0;
  for (int j = 0; j < njobs; ++j) {
    const int t = (jobs[j].m + tile - 1) / tile;
    jobs[j].tiles = t;
    total_tiles += (int64_t)t * (t + 1) / 2;
  }
  // one split count for the batch: `target_items` is the number of CTAs that run at
  // once; choose s minimising (waves of tiles * s items) / s, i.e. the time of the
  // batch when every item costs 1/s, so that no nearly empty last wave is left over
  int64_t max_n = 1;
  for (int j = 0; j < njobs; ++j) max_n = std::max<int64_t>(max_n, jobs[j].n);
  const int64_t s_cap =
      std::max<int64_t>(1, std::min<int64_t>(max_n / std::max(1, min_rows_per_split),
                                             total_tiles > 0 ? 8 * (int64_t)target_items / total_tiles + 1 : 1));
  int64_t splits = 1;
  double best = 1e300;
  for (int64_t s = 1; s <= s_cap && total_tiles > 0; ++s) {
    const double waves = (double)((total_tiles * s + target_items - 1) / target_items);
    const double cost = waves / (double)s;
    if (cost < best * (1.0 - 1e-9)) {
      best = cost;
      splits = s;
    }
  }
  // an autotuned factor on the split count (hapod_autotune), 100 = the rule above
  if (split_pct != 100) splits = std::max<int64_t>(1, splits * split_pct / 100);
  std::vector<int4> items, reduce;
  int64_t item = 0;
  for (int j = 0; j < njobs; ++j) {
    GramJob& J = jobs[j];
    const int64_t max_splits = std::max<int64_t>(1, J.n / std::max(1, min_rows_per_split));
    int64_t s = std::max<int64_t>(1, std::min(splits, max_splits));
    int64_t rps = (J.n + s - 1) / s;
    rps = ((rps + 63) / 64) * 64;  // whole 64-row stages (tensor-core form) / 32-row chunks (FP64)
    s = std::max<int64_t>(1, (J.n + rps - 1) / rps);
    J.splits = (int32_t)s;
    J.rows_per_split = rps;
    J.item_base = item;
    for (int ti = 0; ti < J.tiles; ++ti)
      for (int tj = ti; tj < J.tiles; ++tj) {
        if (s > 1) reduce.push_back(make_int4(j, ti, tj, (int)item));
        for (int sp = 0; sp < s; ++sp) items.push_back(make_int4(j, ti, tj, sp));
        item += s;
      }
  }
  if (split_major) {
    // consecutive items = the tiles of one row range, so that CTAs running together
    // share their column panels through L2 (the partial slot is not the item index)
    std::stable_sort(items.begin(), items.end(), [](const int4& a, const int4& b) { return a.w < b.w; });
  }
  plan->tile = tile;
  plan->num_items = (int)items.size();
  plan->num_reduce = (int)reduce.size();
  plan->partial_bytes = reduce.empty() ? 0 : (size_t)items.size() * tile * tile * sizeof(double);
  int4* it = (int4*)malloc(sizeof(int4) * (items.size() + reduce.size() + 1));
  if (!items.empty()) std::copy(items.begin(), items.end(), it);
  if (!reduce.empty()) std::copy(reduce.begin(), reduce.end(), it + items.size());
  *items_out = it;
  *reduce_out = it + items.size();
}

namespace {

constexpr int kTile = 64;
constexpr int kBK = 32;

__global__ void __launch_bounds__(256) gram_f64_tiles(const GramJob* __restrict__ jobs,
                                                      const int4* __restrict__ items, double* __restrict__ partials) {
  const int4 it = items[blockIdx.x];
  const GramJob J = jobs[it.x];
  const int ti = it.y, tj = it.z, sp = it.w;
  const double* __restrict__ X = static_cast<const double*>(J.X);
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
#pragma unroll 2
    for (int c = warp; c < kTile; c += 8) {
      const int ci = i0 + c;
      As[lane][c] = (rok && ci < J.m) ? X[(size_t)ci * J.ldx + r] : 0.0;
      if (!diag) {
        const int cj = j0 + c;
        Bs[lane][c] = (rok && cj < J.m) ? X[(size_t)cj * J.ldx + r] : 0.0;
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

  if (J.splits == 1) {
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int gi = i0 + ty + 16 * p, gj = j0 + tx + 16 * q;
        if (gi < J.m && gj < J.m) {
          J.G[(size_t)gj * J.m + gi] = acc[p][q];
          J.G[(size_t)gi * J.m + gj] = acc[p][q];
        }
      }
  } else {
    double* out = partials + (size_t)blockIdx.x * kTile * kTile;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) out[(ty + 16 * p) * kTile + tx + 16 * q] = acc[p][q];
  }
}

}  // namespace

// Sum the split partials of one tile in split order and write both triangles.
// Shared by both Gram forms (tile = 64 or 128).  Each tile is spread over
// kReduceChunks CTAs (a contiguous slice of its elements each) so that a tile with
// many splits does not serialise on one SM.
constexpr int kReduceChunks = 16;

template <int TILE>
__global__ void __launch_bounds__(256) gram_reduce(const GramJob* __restrict__ jobs, const int4* __restrict__ reduce,
                                                   const double* __restrict__ partials) {
  const int4 rd = reduce[blockIdx.x / kReduceChunks];
  const int chunk = blockIdx.x % kReduceChunks;
  const GramJob J = jobs[rd.x];
  const int i0 = rd.y * TILE, j0 = rd.z * TILE;
  const bool diag = rd.y == rd.z;
  constexpr int kPer = TILE * TILE / kReduceChunks;
  for (int e = chunk * kPer + threadIdx.x; e < (chunk + 1) * kPer; e += blockDim.x) {
    const int a = e / TILE, b = e % TILE;
    if (diag && a > b) continue;  // one writer per symmetric pair: G stays exactly symmetric
    double s = 0.0;
    for (int sp = 0; sp < J.splits; ++sp) s += partials[((size_t)rd.w + sp) * TILE * TILE + e];
    const int gi = i0 + a, gj = j0 + b;
    if (gi < J.m && gj < J.m) {
      J.G[(size_t)gj * J.m + gi] = s;
      J.G[(size_t)gi * J.m + gj] = s;
    }
  }
}

cudaError_t launch_gram_reduce(int tile, const GramJob* jobs_dev, const int4* reduce_dev, int num_reduce,
                               const double* partials, cudaStream_t s) {
  if (num_reduce <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)num_reduce * kReduceChunks;
  if (tile == 64)
    gram_reduce<64><<<grid, 256, 0, s>>>(jobs_dev, reduce_dev, partials);
  else if (tile == 128)
    gram_reduce<128><<<grid, 256, 0, s>>>(jobs_dev, reduce_dev, partials);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_gram_f64(const GramJob* jobs_dev, const int4* items_dev, int num_items, const int4* reduce_dev,
                            int num_reduce, double* partials, cudaStream_t s) {
  if (num_items > 0) gram_f64_tiles<<<num_items, 256, 0, s>>>(jobs_dev, items_dev, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gram_reduce(kTile, jobs_dev, reduce_dev, num_reduce, partials, s);
}

}  // namespace hapod
