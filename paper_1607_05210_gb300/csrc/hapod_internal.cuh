// Internal declarations shared by the CUDA translation units of libhapod.
// Not part of the public ABI (that is include/hapod.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/hapod.h"

namespace hapod {

constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs (used only as a sizing hint)

// Sets the message hapod_last_error(NULL) returns on the calling thread.
void set_thread_error(const char* msg);

// Per-node result record written by the device, read back once per batch.
struct NodeResult {
  int32_t k;        // kept modes
  int32_t sweeps;   // Jacobi sweeps
  int32_t status;   // hapod_status
  int32_t rank;     // numerical rank found by the pivoted Cholesky
  double tail;      // discarded sum of lambda (including resid)
  double trace;     // trace(G)
  double resid;     // trace of the Schur complement left by the pivoted Cholesky
};

// ---------------------------------------------------------------- Gram (K1)
// One job = one node's Gram matrix.  Work items are (job, ti, tj, split): the
// tile (ti, tj) with ti <= tj of G over the row range of `split`.
struct GramJob {
  const void* X;
  int64_t ldx;
  int64_t n;
  int64_t rows_per_split;
  double* G;        // m x m, ld = m
  int64_t item_base;
  const int32_t* col_exp; // fixed-point form: exponents of the node's columns (launch_fx_colexp)
  int32_t m;
  int32_t tiles;    // tiles per dimension
  int32_t splits;
  int32_t pad;
};

struct GramPlan {
  int tile;             // tile edge (64 FP64, 128 tensor-core)
  int num_items;
  int num_reduce;       // tiles that need a split-K reduction
  size_t partial_bytes; // workspace for split partials
};

// Builds the item list on the host; jobs[] must have X, ldx, n, m, G set.
// Fills tiles, splits, rows_per_split, item_base; items (int4: job, ti, tj, split)
// and reduce list (int4: job, ti, tj, first item) are appended to the vectors.
// With split_major the items are ordered by split first (the partial of item
// (job, ti, tj, split) then lives in slot job.item_base + tile_index * splits + split,
// tile_index the row-major index of (ti, tj) in the upper triangle); otherwise the
// slot is the item's own index.
// split_pct scales the split count (autotuned, 100 = the rule above).
void plan_gram(GramJob* jobs, int njobs, int tile, int min_rows_per_split, int target_items,
               int4** items, int4** reduce, GramPlan* plan, bool split_major = false, int split_pct = 100);

// Sum split partials of each reduce-list tile in split order; both triangles.
cudaError_t launch_gram_reduce(int tile, const GramJob* jobs_dev, const int4* reduce_dev, int num_reduce,
                               const double* partials, cudaStream_t s);
cudaError_t launch_gram_f64(const GramJob* jobs_dev, const int4* items_dev, int num_items, const int4* reduce_dev,
                            int num_reduce, double* partials, cudaStream_t s);
// Mixed form (tcgen05 kind::tf32, hi/lo split); maps_dev[j] is the TMA map of job j's
// X (FP32, box gram_tc_rows_per_stage() rows x 128 columns, 128-byte swizzle);
// items/reduce as for the FP64 form with tile 128, split-major order.
cudaError_t launch_gram_tc(const GramJob* jobs_dev, const CUtensorMap* maps_dev, const int4* items_dev, int num_items,
                           const int4* reduce_dev, int num_reduce, double* partials, int* err_flag, cudaStream_t s);
int gram_tc_rows_per_stage();
// Mixed split-BF16 form (tcgen05 kind::f16 with bf16 pieces): maps as for gram_tc with a
// box of gram_bf3_rows_per_stage() rows x 128 columns, 128-byte swizzle; items/reduce as
// for gram_tc.  err_flag: err[0] timeout flag, err[1] debug wait budget (0 = default).
cudaError_t launch_gram_bf3(const GramJob* jobs_dev, const CUtensorMap* maps_dev, const int4* items_dev,
                            int num_items, const int4* reduce_dev, int num_reduce, double* partials, int* err_flag,
                            cudaStream_t s);
int gram_bf3_rows_per_stage();
// Mixed fixed-point form (exact three-digit products, per-64-row-block exponents):
// 128 x 64 tiles; maps_dev[2 j] / [2 j + 1]: job j's X with boxes of
// gram_fx3_rows_per_stage() rows x gram_fx3_a_cols() / gram_fx3_b_cols() columns
// (128-byte swizzle).  plan_gram_fx3 fills the jobs' tiles, splits, rows_per_split,
// item_base and the item / reduce lists (int4 job, I, J, split).
// split_pct scales the planner's split count (autotuned, 100 = the planner's rule).
void plan_gram_fx3(GramJob* jobs, int njobs, int target_items, std::vector<int4>& items, std::vector<int4>& reduce,
                   size_t* partial_bytes, int split_pct = 100);
cudaError_t launch_gram_fx3(const GramJob* jobs_dev, const CUtensorMap* maps_dev, const int4* items_dev,
                            int num_items, const int4* reduce_dev, int num_reduce, double* partials, int* err_flag,
                            cudaStream_t s);
int gram_fx3_rows_per_stage();
// Exponent markers of the fixed-point form: an all-zero column (block) and a column
// holding Inf / NaN; col_exp arrays start at kFxExpZero.
constexpr int kFxExpZero = -4000;
constexpr int kFxExpBad = 4000;

// X V of the fixed-point form.  V_k digits (modes_fx_vsplit): per mode c the exponent
// F_c (fexp, kpad entries) and six digit planes in the operand layout (vdig,
// fx_vdig_bytes(m, k) bytes); X columns need their exponents (exps, m entries: from
// the Gram's col_exp or launch_fx_colexp).  Modes are tiled fx_mode_tiles(k) x
// fx_mode_width(k) (kpad = their product, at most 128 modes a tile); m at most
// fx_modes_max_m(); for fx_modes_needs_scratch(m) the kernel keeps int32 partial sums
// in Z (n x kpad, leading dimension ldz).
struct FxVSplitJob {
  const double* V;
  int64_t ldv;
  const int32_t* exps;
  uint16_t* vdig;
  int32_t* fexp;
  float2* xscale;  // per column j (padded to whole stages): s1 s2 = 2^(30 - E_j)
  const double* scale;  // k or null: scale of mode c
  float* yscale;        // kpad: FP32 scale of mode c (1 without a scale)
  float* ymul;          // kpad: output factor 2^(F_c - 21) yscale_c (0 zero, NaN bad, -1 not a normal float)
  int32_t m;
  int32_t k;
  int32_t kpad;  // k rounded up to whole mode tiles
  int32_t nt;    // modes per tile (fx_mode_width(k))
};
// Items (row tile, mode tile) of 128 rows x nt modes of one node; maps_dev[j]: X of job j
// (encode_colmajor_f32, box 128 rows x 16 columns, no swizzle).
struct FxModesJob {
  const float* X;
  int64_t ldx;
  const int32_t* exps;
  const float2* xscale;
  const uint16_t* vdig;
  const int32_t* fexp;
  const double* scale;  // k or null
  const float* yscale;  // kpad: FP32 scale of mode c
  const float* ymul;    // kpad: output factor of mode c (see FxVSplitJob)
  float* Y;
  int64_t ldy;
  int32_t* Z;  // fx_modes_needs_scratch(m): int32 partial sums, n x kpad; else null
  int64_t ldz;
  int64_t n;
  int64_t item_base;
  int32_t m;
  int32_t k;
  int32_t row_tiles;
  int32_t mode_tiles;
  int32_t nt;
  int32_t pad;
};
int fx_mode_tiles(int64_t k);
int fx_mode_width(int64_t k);
int64_t fx_modes_max_m();
bool fx_modes_needs_scratch(int64_t m);
size_t fx_vdig_bytes(int64_t m, int64_t k);
size_t fx_xscale_bytes(int64_t m);
cudaError_t launch_fx_colexp(const float* X, int64_t ldx, int64_t n, int64_t m, int* exps, cudaStream_t s);
cudaError_t launch_modes_fx(const FxVSplitJob* vjobs_dev, int njobs, int max_kpad, const FxModesJob* jobs_dev,
                            const CUtensorMap* maps_dev, int64_t total_items, int* err_flag, cudaStream_t s);
int gram_fx3_a_cols();
int gram_fx3_b_cols();
// TMA needs a 16-byte aligned base and a row pitch that is a multiple of 16 bytes.
bool tma_compatible_f32(const void* base, int64_t ld);
bool tma_compatible_f64(const void* base, int64_t ld);
// FP64 column-major map, box box_rows x box_cols, no swizzle, zero fill outside.
bool encode_colmajor_f64(CUtensorMap* out, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                         int box_cols);
bool encode_colmajor_f32(CUtensorMap* out, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                         int box_cols, bool swizzle128);

// ---------------------------------------------------------------- Gram, digit-slice FP64 form
// X (FP64) is represented exactly up to 2^-55 of each column's power-of-two bound
// 2^E_j by 7 balanced base-256 digits per value (Ozaki et al. 2012 error-free
// splitting); digit products are exact in fp16 x fp16 -> FP32 tensor-core arithmetic
// and their level sums (t + u = s <= 8) stay exact integers over kOzKBlock rows.
constexpr int kOzDigits = 7;
constexpr int kOzLevels = 7;                   // s = 2..8
constexpr int kOzKBlock = 128;                 // rows (columns for X V) between exact flushes
constexpr int kOzGroupBytes = kOzDigits * 128; // one 8 x 8 block of all digit planes
constexpr int32_t kOzNonFinite = 0x7FFFFFFF;   // exponent marker of a column holding Inf / NaN

// Column exponents: exps[j] = E_j with max_i |X_ij| < 2^E_j (kOzNonFinite for Inf/NaN).
struct OzColJob {
  const double* X;
  int64_t ldx;
  int64_t n;
  int32_t* exps;
  int64_t col_base;  // first global column index of this job
  int32_t m;
  int32_t pad;
};
cudaError_t launch_oz_colmax(const OzColJob* jobs_dev, int njobs, int64_t total_cols, cudaStream_t s);

// Digit planes of rows [r0, r0 + rows) of X into `digits`, layout
// [row group of 8][digit][column group of 8 (CGs)][column % 8][row % 8] (fp16),
// RG = 2 ceil(rows / 16) row groups, CGs = ceil(m / 8) column groups; rows >= `rows`
// and columns >= m are zero.
struct OzSplitJob {
  const double* X;
  int64_t ldx;
  int64_t r0;
  int64_t rows;
  const int32_t* exps;
  uint16_t* digits;
  int64_t block_base;   // first block of this job (oz_split_blocks(rows, CGs) blocks)
  int32_t m;
  int32_t CGs;
};
int64_t oz_split_blocks(int64_t rows, int32_t CGs);
cudaError_t launch_oz_split(const OzSplitJob* jobs_dev, int njobs, int64_t total_blocks, cudaStream_t s);
__host__ __device__ inline int64_t oz_row_groups(int64_t rows) { return 2 * ((rows + 15) / 16); }
__host__ __device__ inline int32_t oz_col_groups(int64_t m) { return (int32_t)(16 * ((m + 127) / 128)); }
__host__ __device__ inline int32_t oz_stored_groups(int64_t m) { return (int32_t)((m + 7) / 8); }
// Spare bytes after each round's digit buffers (one A block of column groups).  The
// Gram's tensor-map reads zero-fill past the stored column groups and do not reach it.
constexpr size_t kOzDigitSlack = 16 * 128;
// Tensor map of one digit block [RG row groups][7 digits][CGs column groups][64 fp16]
// with a box of 2 row groups x 7 digits x box_groups (<= 16) column groups
// (out-of-range groups read as zero).
bool encode_oz_digits(CUtensorMap* out, const void* base, int32_t CGs, int64_t RG, int box_groups);
constexpr int kOzGramAGroups = 16;  // column groups of a Gram tile's A block (128 columns)
constexpr int kOzGramBGroups = 4;   // column groups of its B block (32 columns)

// Gram of one digit block: items (split, tile) in split-major order; tile (I, J) =
// columns [128 I, 128 I + 128) x [32 J, 32 J + 32), J >= 4 I, 32 J < m.  The item
// writes the entries i, j < m of its FP64 128 x 32 block into partial slot `split`
// (mp x mp, ld mp).  maps[2 k], maps[2 k + 1]: the A and B boxes of job k.
struct OzGramJob {
  const uint16_t* digits;
  const int32_t* exps;
  double* partial;
  int64_t item_base;
  int32_t RG;
  int32_t CGs;
  int32_t m;
  int32_t mp;
  int32_t splits;
  int32_t stages_per_split;  // 16-row stages per split, a multiple of kOzKBlock / 16
  int32_t tiles;
  int32_t pad;
};
int oz_gram_tiles(int32_t m);
cudaError_t launch_gram_oz(const OzGramJob* jobs_dev, const CUtensorMap* maps_dev, int njobs, int64_t total_items,
                           int* err_flag, cudaStream_t s);
// G (m x m, ld m) = sum of `slots` partials (upper triangle, mirrored).
struct OzReduceJob {
  const double* partial;
  double* G;
  int64_t col_base;  // first block of this job (one block per column)
  int32_t slots;
  int32_t m;
  int32_t mp;
  int32_t pad;
};
cudaError_t launch_oz_reduce(const OzReduceJob* jobs_dev, int njobs, int64_t total_cols, cudaStream_t s);

// X V of the digit-slice form: V_k (FP64 m x k, ld ldv) in digits against 2^(F_c - E_j)
// (vdig: [CGp][NG][digit][8][8], fexp: F_c per mode column, NG = kpad / 8).
struct OzVSplitJob {
  const double* V;
  int64_t ldv;
  const int32_t* exps;
  uint16_t* vdig;
  int32_t* fexp;
  int64_t col_base;  // first block (one per padded mode column)
  int32_t m;
  int32_t k;
  int32_t NG;
  int32_t CGp;
};
cudaError_t launch_oz_vsplit(const OzVSplitJob* jobs_dev, int njobs, int64_t total_cols, cudaStream_t s);
// Items (n tile, row tile) of 128 rows x 32 modes of one node; the kernel converts
// X (FP64, ld ldx) to digits itself with the node's column exponents.
struct OzModesJob {
  const double* X;
  int64_t ldx;
  const int32_t* exps;
  const uint16_t* vdig;
  const int32_t* fexp;
  const double* scale;  // k or null
  double* Y;
  int64_t ldy;
  int64_t n;
  int64_t item_base;
  int32_t m;
  int32_t CGp;
  int32_t NG;
  int32_t k;
  int32_t row_tiles;
  int32_t n_tiles;
};
int oz_modes_tile(int k);  // modes per item (32)
// Persistent: min(items, SMs) CTAs walk the items.  maps_dev[j]: TMA map of job j's X
// (encode_colmajor_f64, box 128 rows x 16 columns); X needs tma_compatible_f64.
cudaError_t launch_modes_oz(const OzModesJob* jobs_dev, const CUtensorMap* maps_dev, int njobs, int64_t total_items,
                            int* err_flag, cudaStream_t s);

// ---------------------------------------------------------------- eig (K2)
// Node barrier state of the multi-CTA eigensolver (zeroed before each launch).
struct EigSync {
  unsigned count;   // CTAs arrived at the current barrier
  unsigned gen;     // barrier generation
  int abort;        // a wait of this node ran out
  int rot_sweep;    // last sweep (1-based) in which a pair was rotated
};
struct EigJob {
  const double* G;     // m x m FP64 input (not modified)
  void* A;             // m x m FP64 work: pivoted Cholesky factor L
  void* V;             // m x m work (T): rotated columns, then eigenvectors (unsorted)
  double* lam_tmp;     // m, unsorted eigenvalues
  double* lambda;      // m, sorted descending, clamped >= 0
  int32_t* perm;       // m, sorted position -> column of V
  NodeResult* result;
  double eps2;         // the node's eps^2 (caps the factorisation's stopping residual)
  double floor_rel;    // relative level of the Gram's error: the factorisation stops there at the latest
  int32_t m;
  int32_t cta0;        // first CTA of this job in its launch (set by launch_eig)
  int32_t ncta;        // CTAs of this job (set by launch_eig)
  int32_t pad;
  EigSync* sync;       // node barrier (set by launch_eig)
};
// Rotation precision: FP64 (V in FP64) or FP32 (V in FP32).
constexpr int kEigF64 = 0;
constexpr int kEigF32 = 1;
constexpr int kEigDF = 2;  // double-float rotations (FP32 pairs), FP64 eigenvectors
// Cooperative launches over the jobs, several CTAs per job.  jobs_host is completed
// (cta0, ncta, sync) and copied to jobs_dev (njobs entries); sync_dev: njobs entries.
// err: the bounded-wait flag block (err[1] = debug wait budget) or null.
// Pinned, mapped host arena for the small host-to-device uploads of job tables: the
// bytes are staged here and copied by a kernel instead of a copy engine, so they never
// queue behind large transfers the caller runs on other streams (snapshot uploads).
// Bump-allocated; once full, the stream is synchronised and the arena reused.
struct HostStage {
  uint8_t* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
};
// dst (device) <- src (host), bytes; through `st` when it is set and dst is 16-byte
// aligned, else a plain cudaMemcpyAsync.
cudaError_t staged_upload(HostStage* st, void* dst, const void* src, size_t bytes, cudaStream_t s);
cudaError_t launch_eig(int mode, EigJob* jobs_host, EigJob* jobs_dev, int njobs, int max_m, int max_sweeps,
                       EigSync* sync_dev, const int* err, cudaStream_t s, HostStage* stage = nullptr);
constexpr int kEigMaxM = 13000;  // dynamic shared memory bound of the eigensolver

// C (M x N, ldc) = A (M x K, lda) B (K x N, ldb), column-major FP64 (right vectors).
cudaError_t launch_gemm_nn_f64(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
                               int64_t ldb, double* C, int64_t ldc, cudaStream_t s);

// ---------------------------------------------------------------- truncation (K3)
struct TruncJob {
  const double* lambda;  // m, descending
  double* sigma;         // out: sqrt(lambda_j), j < k
  NodeResult* result;    // out: k, tail
  double eps2;
  int32_t m;
  int32_t pad;
};
cudaError_t launch_truncate(const TruncJob* jobs_dev, int njobs, cudaStream_t s);

// ---------------------------------------------------------------- modes (K4)
// Gather Vk[:, j] = V[:, perm[j]] (FP64), j < k, ld of Vk = m.
struct GatherJob {
  const void* V;       // m x m (T)
  const int32_t* perm;
  double* Vk;
  int32_t m;
  int32_t k;
};
cudaError_t launch_gather(bool fp64_src, const GatherJob* jobs_dev, int njobs, cudaStream_t s);

struct ModesJob {
  const void* X;        // n x m, ld ldx
  const double* Vk;     // m x k, ld ldv
  const double* scale;  // k or null (root: 1 / sigma)
  void* Y;              // n x k, ld ldy
  int64_t ldx;
  int64_t ldv;
  int64_t ldy;
  int64_t n;
  int64_t block_base;   // first block of this job
  int32_t m;
  int32_t k;
  int32_t row_tiles;
  int32_t col_tiles;
};
// FP64 form: tile_cols = modes_f64_tile_cols(max k), row tiles modes_f64_tile_rows(max k).
cudaError_t launch_modes_f64(const ModesJob* jobs_dev, int njobs, int64_t total_blocks, int tile_cols, cudaStream_t s);
int modes_f64_tile_cols(int k);
int modes_f64_tile_rows(int k);
// Mixed form (FP32 in/out): one launch covers jobs whose k fit the mode tile kt
// (kt = modes_mixed_tile_cols(max k)); row tiles are modes_mixed_rows_per_block(max k).
// vec: every job's X, Y bases are 16-byte aligned and ldx, ldy multiples of 4.
cudaError_t launch_modes_mixed(const ModesJob* jobs_dev, int njobs, int64_t total_blocks, int kt, bool vec,
                               cudaStream_t s);
int modes_mixed_tile_cols(int k);
int modes_mixed_rows_per_block(int k);

// ---------------------------------------------------------------- CholQR2 (A6, mixed root)
// R1 = chol(W) (upper, W = Y^T Y), M1 = R1^{-1}; k x k FP64, one CTA.
cudaError_t launch_cholqr_first(const double* W, double* R1, double* M1, int k, int* flag, cudaStream_t s);
// R2 = chol(W2), R = R2 R1 = P S Z^T; M = R2^{-1} P (columns by descending S), sigma = S.
// work: 4 k^2 doubles.  k <= 256.
cudaError_t launch_cholqr_second(const double* W2, const double* R1, double* work, double* M, double* sigma, int k,
                                 int* flag, cudaStream_t s);

}  // namespace hapod
