/*
 * hapod_oracle.c -- CPU FP64 oracle for the per-node truncated POD of the
 * Hierarchical Approximate POD (Himpe, Leibner, Rave, arXiv 1607.05210).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg use it.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, and where the paper defines it:
 *   oracle_gram   G = X^T X, the Gramian (s_i, s_j) of the method of snapshots
 *                 (Sec. 2, Remark "method of snapshots"); written as the plain sum.
 *   oracle_svd    singular values / left and right singular vectors of the snapshot
 *                 map e_m -> s_m (Sec. 2, Def. POD, Eq. snapshot_map).  Computed as
 *                 a Householder QR X = QR followed by a one-sided (Hestenes) Jacobi
 *                 SVD of R.  This deliberately avoids the Gramian, so that it does
 *                 not inherit the squared condition number the paper's footnote to
 *                 the method-of-snapshots remark warns about, and so that it shares
 *                 nothing with the GPU path, which is Gram + eigensolve.
 *   oracle_pod    POD(S, eps) of Sec. 2, Def. (truncated POD): the first N pairs
 *                 (sigma_n, phi_n) with N the smallest N' such that
 *                 sum_{n > N'} sigma_n^2 <= eps^2 (Schmidt-Eckart-Young-Mirsky
 *                 theorem, Eq. pod_error), and POD(S, 0) = {(1, s)} (no SVD).
 *                 The output Y holds the scaled modes sigma_n * phi_n, which is
 *                 what a HAPOD node passes to its parent (Sec. 3.1, Def. HAPOD).
 *
 * All matrices are column-major with a leading dimension; all arithmetic is
 * IEEE double.  Memory is owned by the caller.  No function here allocates
 * memory that outlives the call.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define COL(A, ld, j) ((A) + (size_t)(j) * (size_t)(ld))

/* G (m x m, ld = m) = X^T X, X is n x m with leading dimension ldx. */
void oracle_gram(int64_t n, int64_t m, const double* X, int64_t ldx, double* G) {
#pragma omp parallel for schedule(dynamic)
  for (int64_t j = 0; j < m; ++j) {
    const double* xj = COL(X, ldx, j);
    for (int64_t i = 0; i <= j; ++i) {
      const double* xi = COL(X, ldx, i);
      double s = 0.0;
      for (int64_t r = 0; r < n; ++r) s += xi[r] * xj[r];
      G[i + j * m] = s;
      G[j + i * m] = s;
    }
  }
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t r = 0; r < n; ++r) s += a[r] * b[r];
  return s;
}

/*
 * Householder QR of A (n x m, in place).  For k < min(n, m) the k-th reflector
 * H_k = I - tau_k v_k v_k^T, v_k = (0,..,0, 1, A[k+1:n, k]) maps the current
 * column k below the diagonal to beta * e_k.  On return the upper triangle of A
 * holds R and the strict lower part holds the reflector tails.
 */
static void householder_qr(int64_t n, int64_t m, double* A, int64_t lda, double* tau) {
  const int64_t kmax = n < m ? n : m;
  for (int64_t k = 0; k < kmax; ++k) {
    double* ak = COL(A, lda, k);
    double xnorm2 = 0.0;
    for (int64_t r = k + 1; r < n; ++r) xnorm2 += ak[r] * ak[r];
    const double x0 = ak[k];
    if (xnorm2 == 0.0) { /* already zero below the diagonal: H_k = I */
      tau[k] = 0.0;
      continue;
    }
    const double beta = -copysign(sqrt(x0 * x0 + xnorm2), x0);
    tau[k] = (beta - x0) / beta;
    const double inv = 1.0 / (x0 - beta);
    for (int64_t r = k + 1; r < n; ++r) ak[r] *= inv;
    ak[k] = beta;
    /* apply H_k to the trailing columns */
#pragma omp parallel for schedule(static)
    for (int64_t j = k + 1; j < m; ++j) {
      double* aj = COL(A, lda, j);
      double w = aj[k];
      for (int64_t r = k + 1; r < n; ++r) w += ak[r] * aj[r];
      w *= tau[k];
      aj[k] -= w;
      for (int64_t r = k + 1; r < n; ++r) aj[r] -= w * ak[r];
    }
  }
}

/* y (length n) <- Q y with Q = H_0 H_1 ... H_{kmax-1} stored in A/tau. */
static void apply_q(int64_t n, int64_t kmax, const double* A, int64_t lda, const double* tau, double* y) {
  for (int64_t k = kmax - 1; k >= 0; --k) {
    if (tau[k] == 0.0) continue;
    const double* ak = COL(A, lda, k);
    double w = y[k];
    for (int64_t r = k + 1; r < n; ++r) w += ak[r] * y[r];
    w *= tau[k];
    y[k] -= w;
    for (int64_t r = k + 1; r < n; ++r) y[r] -= w * ak[r];
  }
}

/*
 * One-sided (Hestenes) Jacobi on the columns of B (k x m): plane rotations from
 * the right make the columns mutually orthogonal, B V = W, and accumulate V
 * (m x m).  Cyclic row-by-row pair order; a pair (p, q) is rotated while
 * |b_p . b_q| > tol * ||b_p|| ||b_q||, tol = m * 2^-53.  A column whose squared
 * norm is below (tol * ||B||_F)^2 is numerically zero and is not rotated (when
 * m > k at least m - k columns must end at zero, and rounding noise at that level
 * cannot be made mutually orthogonal).  Returns the number of sweeps, or -1 if
 * max_sweeps did not suffice.
 */
static int hestenes_jacobi(int64_t k, int64_t m, double* B, int64_t ldb, double* V, int64_t ldv,
                           int max_sweeps) {
  const double tol = (double)m * ldexp(1.0, -53);
  double fro2 = 0.0;
  for (int64_t j = 0; j < m; ++j) fro2 += dot(k, COL(B, ldb, j), COL(B, ldb, j));
  const double negligible = tol * tol * fro2;
  for (int64_t j = 0; j < m; ++j) {
    double* vj = COL(V, ldv, j);
    for (int64_t i = 0; i < m; ++i) vj[i] = (i == j) ? 1.0 : 0.0;
  }
  for (int sweep = 1; sweep <= max_sweeps; ++sweep) {
    int rotated = 0;
    for (int64_t p = 0; p + 1 < m; ++p) {
      for (int64_t q = p + 1; q < m; ++q) {
        double* bp = COL(B, ldb, p);
        double* bq = COL(B, ldb, q);
        const double alpha = dot(k, bp, bp);
        const double beta = dot(k, bq, bq);
        const double gamma = dot(k, bp, bq);
        if (gamma == 0.0 || alpha <= negligible || beta <= negligible) continue;
        if (fabs(gamma) <= tol * sqrt(alpha * beta)) continue;
        rotated = 1;
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double s = c * t;
        for (int64_t r = 0; r < k; ++r) {
          const double x = bp[r], y = bq[r];
          bp[r] = c * x - s * y;
          bq[r] = s * x + c * y;
        }
        double* vp = COL(V, ldv, p);
        double* vq = COL(V, ldv, q);
        for (int64_t r = 0; r < m; ++r) {
          const double x = vp[r], y = vq[r];
          vp[r] = c * x - s * y;
          vq[r] = s * x + c * y;
        }
      }
    }
    if (!rotated) return sweep;
  }
  return -1;
}

/*
 * Thin SVD X = U diag(sigma) V^T of X (n x m, ld ldx), r = min(n, m) triplets,
 * sigma descending.  Outputs (any may be NULL):
 *   sigma  r values
 *   US     n x r, column j = sigma_j * u_j (scaled left singular vectors), ld n
 *   V      m x r right singular vectors, ld m
 * Returns the Jacobi sweep count, -1 on non-convergence, -2 on allocation failure.
 */
int oracle_svd(int64_t n, int64_t m, const double* X, int64_t ldx, double* sigma, double* US, double* V) {
  const int64_t r = n < m ? n : m;
  if (r == 0) return 0;
  double* A = (double*)malloc(sizeof(double) * (size_t)n * (size_t)m);
  double* tau = (double*)malloc(sizeof(double) * (size_t)r);
  double* R = (double*)calloc((size_t)r * (size_t)m, sizeof(double));
  double* W = (double*)malloc(sizeof(double) * (size_t)m * (size_t)m);
  double* nrm = (double*)malloc(sizeof(double) * (size_t)m);
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
  if (!A || !tau || !R || !W || !nrm || !order) {
    free(A); free(tau); free(R); free(W); free(nrm); free(order);
    return -2;
  }
  for (int64_t j = 0; j < m; ++j) memcpy(COL(A, n, j), COL(X, ldx, j), sizeof(double) * (size_t)n);
  householder_qr(n, m, A, n, tau);
  /* R (r x m): upper triangle / trapezoid of the factored A */
  for (int64_t j = 0; j < m; ++j)
    for (int64_t i = 0; i <= j && i < r; ++i) R[i + j * r] = A[i + j * n];
  const int sweeps = hestenes_jacobi(r, m, R, r, W, m, 60);
  /* singular values are the column norms of R W; sort descending (stable) */
  for (int64_t j = 0; j < m; ++j) {
    nrm[j] = sqrt(dot(r, COL(R, r, j), COL(R, r, j)));
    order[j] = j;
  }
  for (int64_t a = 1; a < m; ++a) { /* insertion sort, ties keep index order */
    const int64_t key = order[a];
    int64_t b = a - 1;
    while (b >= 0 && nrm[order[b]] < nrm[key]) {
      order[b + 1] = order[b];
      --b;
    }
    order[b + 1] = key;
  }
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  if (!y) {
    free(A); free(tau); free(R); free(W); free(nrm); free(order);
    return -2;
  }
  for (int64_t j = 0; j < r; ++j) {
    const int64_t src = order[j];
    if (sigma) sigma[j] = nrm[src];
    if (V) memcpy(COL(V, m, j), COL(W, m, src), sizeof(double) * (size_t)m);
    if (US) {
      /* sigma_j u_j = Q [ (R W)_{:,src} ; 0 ] */
      memset(y, 0, sizeof(double) * (size_t)n);
      memcpy(y, COL(R, r, src), sizeof(double) * (size_t)r);
      apply_q(n, r, A, n, tau, y);
      memcpy(COL(US, n, j), y, sizeof(double) * (size_t)n);
    }
  }
  free(y); free(A); free(tau); free(R); free(W); free(nrm); free(order);
  return sweeps;
}

/*
 * Tail sums of squared singular values: tail[N'] = sum_{j >= N'} sigma_j^2 for
 * N' = 0..r (tail[r] = 0), accumulated from the smallest value upward with
 * Kahan compensation.
 */
void oracle_tail_sums(int64_t r, const double* sigma, double* tail) {
  double s = 0.0, c = 0.0;
  tail[r] = 0.0;
  for (int64_t j = r - 1; j >= 0; --j) {
    const double y = sigma[j] * sigma[j] - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
    tail[j] = s;
  }
}

/*
 * POD(S, eps) (Sec. 2, Def. truncated POD) of the snapshots X (n x m, ld ldx).
 *   eps == 0 : no SVD, the snapshots are returned with sigma = 1 (N = m).
 *   eps >  0 : N = min{N' : sum_{j >= N'} sigma_j^2 <= eps^2} (0-based j).
 * Outputs: *N_out; sigma_out (capacity min(n, m), or m when eps == 0);
 * Y_out (n x capacity, ld n): column j = sigma_j * phi_j; *tail_out =
 * sum of the discarded sigma^2.  Returns the SVD's sweep count (>= 0) on
 * success, -1 when the one-sided Jacobi did not converge (no output is then
 * defined) and -2 when an allocation failed.
 */
int oracle_pod(int64_t n, int64_t m, const double* X, int64_t ldx, double eps, int64_t* N_out,
               double* sigma_out, double* Y_out, double* tail_out) {
  if (eps == 0.0) {
    for (int64_t j = 0; j < m; ++j) {
      sigma_out[j] = 1.0;
      memcpy(COL(Y_out, n, j), COL(X, ldx, j), sizeof(double) * (size_t)n);
    }
    *N_out = m;
    *tail_out = 0.0;
    return 0;
  }
  const int64_t r = n < m ? n : m;
  double* tail = (double*)malloc(sizeof(double) * (size_t)(r + 1));
  if (!tail) return -2;
  const int st = oracle_svd(n, m, X, ldx, sigma_out, Y_out, NULL);
  if (st < 0) {  /* an unconverged SVD is not a POD: the caller gets the failure */
    free(tail);
    return st;
  }
  oracle_tail_sums(r, sigma_out, tail);
  int64_t N = r;
  for (int64_t Np = 0; Np <= r; ++Np) {
    if (tail[Np] <= eps * eps) {
      N = Np;
      break;
    }
  }
  *N_out = N;
  *tail_out = tail[N];
  free(tail);
  return st;
}
