/*
 * hapod.h -- C ABI of the GB300 (sm_103a) Hierarchical Approximate POD library.
 *
 * Method: Himpe, Leibner, Rave, "Hierarchical Approximate Proper Orthogonal
 * Decomposition" (arXiv 1607.05210).  At every node a of a rooted tree the
 * library computes the truncated POD of the node's input by the method of
 * snapshots -- Gram X^T X, symmetric eigensolve, truncation to the node's
 * tolerance, modes X V -- and passes the singular-value-scaled modes to the
 * parent, level by level up to the root.
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major with a leading dimension (ld >= rows).  A
 *     snapshot matrix X of a node is n x m: one column per snapshot vector.
 *   - "device" pointers are CUDA global-memory addresses of the current device;
 *     "host" pointers are ordinary CPU memory.  The library never takes
 *     ownership of caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it; calls that return results on the host synchronise
 *     that stream.
 *   - Errors are returned, never thrown, and nothing aborts the process.
 *     hapod_last_error() gives a one-line description.  After an HAPOD_ERR_*
 *     from a context call, the context accepts only hapod_node_stats,
 *     hapod_last_error and hapod_destroy.  HAPOD_WARN_* codes are not errors:
 *     the results are produced and the warning is recorded.
 *   - FP64 form (HAPOD_FP64): snapshots are IEEE double; all arithmetic is FP64.
 *     Digit-slice FP64 form (HAPOD_FP64_OZAKI): snapshots and results as in the
 *     FP64 form; the Gram and X V are formed on the fp16 tensor cores from an exact
 *     7-digit balanced base-256 fixed-point representation of each column (relative
 *     to a power-of-two bound 2^E of its largest entry, truncated below 2^(E-55)),
 *     each row's product x_i x_j represented to within 1.26 * 2^(E_i+E_j-53), with
 *     integer-exact accumulation, one FP64 rounding per entry and row split (Gram)
 *     or per 128-column block (X V), and FP64 sums over the splits / blocks.
 *     Mixed TF32 form (HAPOD_MIXED_TF32X3): snapshots are IEEE float; the Gram runs
 *     on the tensor cores as TF32 hi/lo products (x = hi + lo, hi*hi + hi*lo + lo*hi)
 *     accumulated in FP32 over short row chunks and summed in FP64, X V in FP32.
 *     Mixed split-BF16 form (HAPOD_MIXED_BF16X3): snapshots are IEEE float; every
 *     value is split exactly into three bf16 pieces and the Gram and X V are formed
 *     from the six piece products whose levels add to at most 2 (dropped terms below
 *     2^-26 |x_i x_j|), FP32 tensor-core accumulation over 64-row segments summed in
 *     compensated FP32 pairs and FP64; eigensolve with FP64 rotations.
 *     Mixed fixed-point form (HAPOD_MIXED_FX3): snapshots are IEEE float; each
 *     column is scaled by the power of two of its largest |x| (one read of X before
 *     the Gram) and every value rounded to a 32-bit integer written as four balanced
 *     8-bit digits; the thirteen digit pairs of levels 2..6 are summed exactly on the
 *     fp16 tensor cores over 128-row groups and in int64, so the Gram carries only the
 *     representation error (at most 2^-32 of the column maximum per value, unbiased)
 *     and one FP64 rounding per entry and row split.  X V from the same column
 *     exponents and four digits of V: the leading digit pair summed exactly (int32
 *     across groups of 2048 columns), the nine next pairs (weights 2^-8 .. 2^-24 of
 *     it) summed by the tensor cores in FP32, one FP32 rounding per entry; at most
 *     245760 snapshot columns.  Eigensolve with FP64 rotations, FP64 tails, CholQR2
 *     at the root.
 *     Eigensolve, tail sums and truncation use FP64 arithmetic on FP64 data except
 *     where stated.
 */
#ifndef HAPOD_H
#define HAPOD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HAPOD_OK = 0,
  HAPOD_ERR_INVALID = 1,      /* bad argument (null pointer, size, ld, precision) */
  HAPOD_ERR_TREE = 2,         /* not a rooted tree (Sec. 3.1, Def. Rooted Tree) */
  HAPOD_ERR_STATE = 3,        /* call out of order (push to a non-leaf, twice, ...) */
  HAPOD_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  HAPOD_ERR_OOM = 5,          /* device allocation failed */
  HAPOD_ERR_NONFINITE = 6,    /* NaN/Inf in a node's Gram matrix */
  HAPOD_ERR_TIMEOUT = 7,      /* a bounded device-side wait ran out */
  HAPOD_WARN_NOCONVERGE = 8,  /* Jacobi reached its sweep limit */
  HAPOD_WARN_BELOW_FLOOR = 9  /* a kept sigma lies below the form's resolution floor */
} hapod_status;

typedef enum {
  HAPOD_FP64 = 0,           /* double snapshots, FP64 arithmetic everywhere */
  HAPOD_MIXED_TF32X3 = 1,   /* float snapshots, tensor-core (TF32 hi/lo split) Gram, FP32 X V */
  HAPOD_FP64_OZAKI = 2,     /* double snapshots and results; Gram and X V from exact 8-bit
                               digit products on the fp16 tensor cores (error-free splitting
                               of Ozaki et al. 2012, integer-exact accumulation, one final
                               FP64 rounding per entry); eigensolver in FP64 */
  HAPOD_MIXED_BF16X3 = 3,   /* float snapshots; Gram on the tensor cores from the exact
                               three-piece bf16 split x = b1 + b2 + b3 (six products per
                               entry, FP32 accumulation over 64-row segments, compensated
                               sums, FP64 over row splits); Jacobi eigensolve with FP64
                               rotations, FP64 truncation, CholQR2 at the root */
  HAPOD_MIXED_FX3 = 4       /* float snapshots; Gram on the fp16 tensor cores from four
                               balanced 8-bit digits per value, fixed-point per column
                               (thirteen digit pairs, integer-exact sums, int64
                               accumulation, one FP64 rounding per entry and row split);
                               eigensolve, truncation and root as HAPOD_MIXED_BF16X3 */
} hapod_precision;

/*
 * Rooted tree (Sec. 3.1, Def. Rooted Tree): node a's parent is parent[a], the
 * root has parent -1.  Every node is a child of at most one node (Eq.
 * treeonlyoneparent) and reaches the root (Eq. treeconnected); hapod_create
 * checks both.  Leaves are the nodes without children; leaf_cols[a] is
 * |D^-1(a)|, the number of snapshots assigned to leaf a (ignored for inner
 * nodes).  Both arrays are host memory, read during hapod_create only.
 */
typedef struct {
  int32_t num_nodes;
  const int32_t* parent;
  const int64_t* leaf_cols;
} hapod_tree;

/*
 * Tolerances (Sec. 3.3, Thm. cor:hapod_bound).  `eps` is the global l2 target:
 * the result satisfies sum_s ||s - P s||^2 <= eps^2 over all |S| snapshots, i.e.
 * eps* = eps / sqrt(|S|).  Local tolerances: eps(root) = sqrt(|S|) omega eps*,
 * eps(a) = sqrt(|S~_a|) (L_T - 1)^(-1/2) sqrt(1 - omega^2) eps* otherwise, where
 * |S~_a| counts the snapshots below a and L_T is the depth (leaves have level 1).
 * A single-node tree (L_T = 1) gives its root the whole budget eps.
 * eps_override (host, num_nodes entries, or NULL) replaces eps(a) where it is not
 * NaN; 0 makes a pass-through node (Def. truncated POD: POD(S, 0) returns the
 * snapshots with sigma = 1).
 * max_pending_leaves: 0 = process the tree once every leaf has been pushed (or at
 * hapod_result); k > 0 = process as soon as k pushed leaves are waiting, which
 * bounds the device memory held by the library for streamed input (Sec. 3.4).
 * flags: see HAPOD_FLAG_PROFILE below.
 */
typedef struct {
  double eps;
  double omega;
  const double* eps_override;
  int32_t precision;
  int32_t max_pending_leaves;
  int32_t flags;  /* HAPOD_FLAG_* bits */
} hapod_tol;

/* flags: HAPOD_FLAG_PROFILE records CUDA events on the context's stream around
 * every kernel launch so that hapod_profile can report per-step device time.
 * HAPOD_FLAG_RIGHT_VECTORS keeps every node's right singular vectors (its Gram
 * eigenvectors V_N, m_a x N_a FP64 on the device, released at hapod_destroy) and
 * the position of each child's modes in its parent's input, for
 * hapod_result_right. */
#define HAPOD_FLAG_PROFILE 1
#define HAPOD_FLAG_RIGHT_VECTORS 2

typedef struct hapod_ctx hapod_ctx;

/* Per-node record filled by hapod_node_stats. */
typedef struct {
  int64_t m;        /* input columns |S_a| (0 until the node has run) */
  int64_t k;        /* kept modes |HAPOD(a)| (-1 until the node has run) */
  double eps;       /* local tolerance eps(a) */
  double tail_sq;   /* discarded sum of sigma^2 (the local POD error, Eq. pod_error) */
  int32_t level;    /* L_T(a) */
  int32_t sweeps;   /* Jacobi sweeps used (0 for pass-through) */
  int32_t state;    /* 0 waiting, 1 ready, 2 done */
  int32_t status;   /* hapod_status of this node (warnings included) */
} hapod_node_info;

/*
 * hapod_create -- validate the tree, compute levels, |S~_a| and eps(a)
 * (Thm. cor:hapod_bound) and return a context bound to `stream` and the current
 * device.  n_rows is the snapshot length n (dim V).  No device compute.  The
 * context keeps an 8 MiB pinned, device-mapped host buffer through which its small
 * job tables reach the device by a copy kernel (so they never wait behind large
 * transfers the caller queues on other streams); without it (the allocation
 * failed) they are copied with cudaMemcpyAsync.  hapod_destroy frees it.
 * Errors: INVALID (null pointers, n_rows < 1, eps < 0, omega outside [0, 1],
 * unknown precision), TREE, CUDA, OOM.  *out is NULL on error.
 */
hapod_status hapod_create(const hapod_tree* tree, const hapod_tol* tol, int64_t n_rows, void* stream,
                          hapod_ctx** out);

/*
 * hapod_push -- hand leaf `leaf` its snapshots: device matrix n x ncols, leading
 * dimension ld (elements), double for the FP64 forms, float for the mixed form.
 * ncols must equal leaf_cols[leaf].  The caller keeps ownership; the library reads
 * the matrix asynchronously on the context's stream, so it must stay valid and
 * unchanged until that stream has passed the leaf's processing -- guaranteed once
 * hapod_result has returned, or after the push that triggered processing
 * (max_pending_leaves) when the caller synchronises the stream.  May launch work
 * (Def. HAPOD: a node runs once all of its inputs exist).
 * Errors: INVALID, STATE (not a leaf, already pushed, context poisoned), plus any
 * error of the processing it triggers.
 */
hapod_status hapod_push(hapod_ctx* ctx, int32_t leaf, const void* dev_snapshots, int64_t ld, int64_t ncols);

/*
 * hapod_result -- finish every pending node and return HAPOD(root) (Def. HAPOD):
 * *k_out = number of modes; sigma_host (host, k doubles, descending) and
 * dev_modes (device, n x k, leading dimension ld_modes, same element type as the
 * snapshots) receive the singular values and orthonormal modes phi_n when not
 * NULL.  Call once with NULL buffers to learn k, then again with buffers.  For a
 * pass-through root (eps(root) = 0) the modes are the raw inputs and sigma = 1.
 * Synchronises the stream.  Errors: STATE (a leaf was never pushed), INVALID
 * (ld_modes < n with dev_modes set), and processing errors.  A warning from any
 * node is returned if no error occurred.
 */
hapod_status hapod_result(hapod_ctx* ctx, int64_t* k_out, double* sigma_host, void* dev_modes,
                          int64_t ld_modes);

/*
 * hapod_result_right -- the right factor of the HAPOD's low-rank approximation of
 * the snapshot map (Sec. 3.3, Remark "Low-rank approximation of the snapshot
 * mapping"): Lambda~ (|S| x k, orthonormal columns) with
 *   || S - U diag(sigma) Lambda~^T ||_F^2 <= sum over all nodes a of eps(a)^2,
 * U, sigma, k those of hapod_result, S the snapshots as columns.  Rows follow the
 * leaves in increasing node index, each leaf's snapshots in the order pushed.
 * Built as Lambda~_a = diag(Lambda~_c over the children c) Lambda_a from the root
 * down (Def. "Additional notation"), Lambda_a the node's right singular vectors (the
 * identity at pass-through nodes).  W: device, |S| x k FP64, leading dimension
 * ldw >= |S|; rows of leaves that kept no mode are zero.  Requires a context
 * created with HAPOD_FLAG_RIGHT_VECTORS whose hapod_result has returned.  Allocates
 * the intermediate maps (sum over inner nodes of m_a x k doubles) from the library
 * pool; synchronises the stream.  Errors: INVALID (null W with k > 0, ldw < |S|),
 * STATE (flag missing, root not finished, context poisoned), CUDA, OOM.
 */
hapod_status hapod_result_right(hapod_ctx* ctx, double* W, int64_t ldw);

/* Per-step accounting of a context created with HAPOD_FLAG_PROFILE.  Index:
 * 0 Gram, 1 eigensolve, 2 truncation, 3 eigenvector gather, 4 modes, 5 copies
 * (pass-through inputs and parked child outputs), 6 digit conversion of the
 * digit-slice form (column exponents and digit planes of the Gram inputs; its Gram
 * step 0 then counts the tensor-core Gram kernels and the split-sum reduce) and the
 * column-exponent pass of the fixed-point form (4 n m bytes), 7 unused.  ms = summed device time between CUDA events recorded on the context
 * stream around the step's launches; launches = kernel launches; bytes/flops =
 * algorithmic volume of the step as defined by the method (Gram: b n m bytes and
 * n m (m + 1) flops per node; modes: b n (m + k) bytes and 2 n m k flops; b =
 * element size; digit conversion: 22 n m bytes, the FP64 read and the 7 fp16
 * digits written), zero where not defined. */
#define HAPOD_PROFILE_STEPS 8
typedef struct {
  double ms[HAPOD_PROFILE_STEPS];
  int64_t launches[HAPOD_PROFILE_STEPS];
  double bytes[HAPOD_PROFILE_STEPS];
  double flops[HAPOD_PROFILE_STEPS];
} hapod_profile_info;

/* Accumulated profile since hapod_create (zeros without HAPOD_FLAG_PROFILE).
 * Synchronises the context stream.  Errors: INVALID. */
hapod_status hapod_profile(hapod_ctx* ctx, hapod_profile_info* info);

/* Node statistics; valid at any time.  Errors: INVALID (node out of range). */
hapod_status hapod_node_stats(const hapod_ctx* ctx, int32_t node, hapod_node_info* info);

/* One-line description of the last error of ctx (or of the calling thread's last
 * context-free call when ctx is NULL).  Never NULL; owned by the library. */
const char* hapod_last_error(const hapod_ctx* ctx);

/* Free every resource of the context (waits for its stream).  NULL is a no-op.
 * The device memory goes back to the library's stream-ordered pool of the current
 * device, which keeps it cached for the next context (see hapod_trim_pool). */
void hapod_destroy(hapod_ctx* ctx);

/* Return the device memory that the library's pool of the current device keeps
 * cached between calls to the driver (waits for the work queued on `stream`, NULL =
 * legacy default stream).  Memory still in use by a live context stays allocated.
 * Errors: CUDA. */
hapod_status hapod_trim_pool(void* stream);

/* ------------------------------------------------------------------------
 * Single-node steps.  Each runs the same kernels a context uses, on one node,
 * with caller-provided device buffers; workspace is taken from the library's
 * stream-ordered memory pool and returned before the call completes on the
 * stream.  `precision` selects the form as above.
 * ---------------------------------------------------------------------- */

/*
 * hapod_gram -- Gramian G = X^T X of the method of snapshots (Sec. 2, Remark
 * def:method_of_snapshots: G = (s_i, s_j)_{i,j}).  X: device n x m (ld ldx),
 * double (FP64 forms) or float (mixed).  G: device m x m FP64, ld = m, both
 * triangles written; a column holding Inf or NaN makes its row and column of G NaN
 * in the digit-slice form.  Errors: INVALID, CUDA, OOM, TIMEOUT (tensor-core forms:
 * a bounded device-side wait ran out).
 */
hapod_status hapod_gram(int32_t precision, int64_t n, int64_t m, const void* X, int64_t ldx, double* G,
                        void* stream);

/*
 * hapod_eig -- eigen-decomposition G = V diag(lambda) V^T of a symmetric positive
 * semidefinite G (device m x m FP64, ld = m), as needed by the method of snapshots
 * (Sec. 2, Remark def:method_of_snapshots).  A diagonally pivoted Cholesky
 * G = L L^T + S (FP64) stops at the numerical rank r, once trace(S) <= m 2^-53
 * trace(G) (FP64 forms) or 1e-7 trace(G) (mixed form); one-sided Jacobi with
 * round-robin ordering on the r columns of L (FP64 or FP32 rotations) then gives
 * L L^T = W W^T with orthogonal columns w_j: eigenvector u_j = w_j / ||w_j||,
 * eigenvalue lambda_j = u_j^T G u_j in FP64.  lambda: device m doubles, descending,
 * zero beyond r.
 * V: device m x m FP64, ld = m, column j belongs to lambda[j]; columns j >= r are
 * zero.  *sweeps_host (may be NULL) receives the sweep count.  Synchronises the
 * stream.  Returns WARN_NOCONVERGE if the sweep limit was reached, ERR_NONFINITE
 * for NaN/Inf in G, ERR_INVALID for m > 13000.
 */
hapod_status hapod_eig(int32_t precision, int64_t m, const double* G, double* lambda, double* V,
                       int32_t* sweeps_host, void* stream);

/*
 * hapod_truncate -- truncation rule of the POD (Sec. 2, Def. truncated POD, with
 * Eq. pod_error): N = min{N' in 0..m : sum_{j >= N'} lambda_j <= eps^2} (0-based
 * j, inclusive <=) for eigenvalues lambda (device, m doubles, descending,
 * nonnegative).  *N_host and *tail_host (the discarded sum) are host outputs;
 * synchronises the stream.  eps == 0 returns N = m without reading lambda.
 */
hapod_status hapod_truncate(int64_t m, const double* lambda, double eps, int64_t* N_host, double* tail_host,
                            void* stream);

/*
 * hapod_modes -- Y = X V[:, 0:N] diag(scale) (Sec. 2, Remark
 * def:method_of_snapshots: phi_k = lambda_k^{-1/2} sum_i psi_{k,i} s_i; with
 * scale = NULL this is the sigma-scaled mode sigma_k phi_k that Def. HAPOD passes
 * to the parent, with scale_j = 1/sigma_j it is phi_j).  X: device n x m (ld ldx,
 * double or float by precision); V: device m x >= N FP64 (ld ldv); scale: device N
 * doubles or NULL; Y: device n x N (ld ldy), same type as X.  The digit-slice form
 * computes Y from exact digit products (X as for hapod_gram, V column c against a
 * power-of-two bound of max_j 2^E_j |V_jc|), rounds once per entry and 128-column
 * block of X and sums the blocks in FP64; the fixed-point form as described for
 * HAPOD_MIXED_FX3 (m <= 245760, else ERR_INVALID).  Both synchronise the stream and
 * return NaN columns if X or V holds Inf or NaN; TIMEOUT if a bounded device-side
 * wait ran out.
 */
hapod_status hapod_modes(int32_t precision, int64_t n, int64_t m, const void* X, int64_t ldx, const double* V,
                         int64_t ldv, int64_t N, const double* scale, void* Y, int64_t ldy, void* stream);

/*
 * hapod_pod -- POD(S, eps) of one node (Sec. 2, Def. truncated POD): Gram,
 * eigensolve, truncation, scaled modes.  X: device n x m (ld ldx).  Outputs:
 * *N_host; sigma (device, capacity m doubles, first N written, descending);
 * Y (device n x capacity m, ld ldy, first N columns = sigma_j phi_j; for eps == 0
 * Y = X and sigma = 1); *tail_host = discarded sum of sigma^2.  Synchronises the
 * stream.  Errors: INVALID (also m > 13000 with eps > 0: the eigensolver's limit),
 * CUDA, OOM, TIMEOUT, NONFINITE.
 */
hapod_status hapod_pod(int32_t precision, int64_t n, int64_t m, const void* X, int64_t ldx, double eps,
                       int64_t* N_host, double* sigma, void* Y, int64_t ldy, double* tail_host, void* stream);

/* ------------------------------------------------------------------------
 * Input generation (stand-in for the PDE snapshot data of Sec. 4, which is not
 * available): snapshots written directly into device memory, so that leaves and
 * stream chunks (Sec. 3.4, reduced memory) need no host copy.
 */
#define HAPOD_SYNTH_MAX_PULSES 64
typedef struct {
  uint64_t seed;                                 /* Philox4x32-10 key of the snapshot times */
  double nu;                                     /* diffusion coefficient */
  double speed;                                  /* advection speed c */
  double harmonic_amp[32];                       /* a_k of sin(k (x - c t)), k = 1..32 */
  int32_t num_pulses;                            /* 0 .. HAPOD_SYNTH_MAX_PULSES */
  double pulse_width;                            /* w (> 0 when num_pulses > 0) */
  double pulse_centre[HAPOD_SYNTH_MAX_PULSES];   /* x_p at t = 0, in [0, 2 pi) */
  double pulse_amp[HAPOD_SYNTH_MAX_PULSES];      /* A_p */
} hapod_synth_params;

/*
 * hapod_synth_snapshots -- columns col0 .. col0 + ncols - 1 of the travelling-pulse
 * trajectory on the periodic grid x_i = 2 pi i / n, i < n:
 *   X[i, j] = sum_k a_k exp(-nu k^2 t) sin(k (x_i - c t))
 *           + sum_p A_p exp(-d(x_i, x_p + c t)^2 / (2 w^2)),   t = t_{col0 + j},
 * d the periodic distance, pulses beyond 9 w omitted (below 3e-18 A_p).  The time of
 * global column g is the uniform t_g = (w0 2^21 + (w1 >> 11)) 2^-53 from the first
 * two words (w0, w1) of Philox4x32-10 (Salmon et al., SC 2011) with key (seed mod
 * 2^32, seed div 2^32) and counter (g mod 2^32, g div 2^32, 0, 0), so any column
 * range is reproducible on its own.  The field is evaluated in FP32 (the Fourier
 * coefficients, times and pulse positions in FP64); dtype 0 writes float, 1 writes
 * double holding the same FP32 values.  X: device, n x ncols, column-major, leading
 * dimension ldx >= n (elements).  t_out: device, ncols doubles receiving t_g, or
 * NULL.  p: host, read during the call.  Asynchronous on `stream`; allocates a
 * small per-column table (about 1 KB per column) from the stream-ordered default
 * pool and frees it on the stream.  Errors: INVALID (n < 1 or n > 2^36, col0 < 0,
 * ld, dtype, pulse count or width), OOM, CUDA.
 */
hapod_status hapod_synth_snapshots(const hapod_synth_params* p, int64_t n, int64_t col0, int64_t ncols,
                                   int32_t dtype, void* X, int64_t ldx, double* t_out, void* stream);

/*
 * hapod_autotune -- schedule autotuner for the Gram kernels of the FP64, TF32X3,
 * BF16X3 and FX3 forms.  The Gram is split over row ranges ("splits") whose
 * number the library chooses so that the tiles x splits work items fill whole waves
 * of resident CTAs; this call times the Gram of the caller's node X (device, n x m,
 * ld ldx, element type of the form) with the split count scaled by 50, 100, 200 and
 * 400 % (one warm-up and three timed calls each, CUDA events on `stream`) and keeps
 * the fastest factor (a factor other than 100 % must win by 2 %) in a process-wide
 * table keyed by (form, ceil(log2 m), ceil(log2 n)).  Every later Gram of a batch
 * whose widest node falls in that bucket uses the factor (hapod_gram, hapod_pod and
 * contexts alike).  *pct_out (host, may be NULL) receives the factor in percent,
 * ms_out (host, 4 doubles or NULL) the mean times of the four candidates.
 * Allocates an m x m FP64 work matrix from the library pool; synchronises the
 * stream.  Errors: INVALID (other forms, sizes, ld), and those of hapod_gram; on an
 * error the bucket's entry is removed.
 */
hapod_status hapod_autotune(int32_t precision, int64_t n, int64_t m, const void* X, int64_t ldx, int32_t* pct_out,
                            double* ms_out, void* stream);

/* Forget every autotuned factor (the planners' own rule applies again). */
void hapod_autotune_clear(void);

/*
 * hapod_gram_noalloc -- the FP64 Gram G = X^T X of hapod_gram (HAPOD_FP64 form)
 * for callers that must not allocate device memory while they run: for example
 * an application whose own allocator already holds nearly all of the GPU's
 * memory, or a latency-bound pipeline that cannot afford cudaMalloc/cudaFree or
 * the synchronisation they imply.  The paper has no counterpart to this call; it
 * is a property of this library's memory handling only.
 * X: device n x m doubles (ld ldx); G: device m x m doubles, ld = m, both
 * triangles written.  Nothing is allocated per call: split-K partials go to a
 * fixed 32 MiB device array inside the library, held on every GPU that loads the
 * library until the process exits.  Limit: m <= 2816 (the upper triangle of G in
 * 64 x 64 tiles must fit the array); larger m returns HAPOD_ERR_INVALID with a
 * message in hapod_last_error(NULL).  All calls share the array: calls whose
 * work overlaps on the GPU (unordered streams) race on it.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it until the process exits; make that first call
 * before any stream capture (a first call made inside a capture returns
 * HAPOD_ERR_INVALID).  A cudaDeviceReset of that device invalidates the kept
 * address: do not call this entry point again in that process afterwards.
 * Errors: INVALID, CUDA.
 */
hapod_status hapod_gram_noalloc(int64_t n, int64_t m, const double* X, int64_t ldx, double* G, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HAPOD_H */
