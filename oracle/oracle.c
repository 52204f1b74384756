/*
 * oracle.c -- plain, slow CPU oracle for direct TSQR.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * Paper: A. R. Benson, D. F. Gleich, J. Demmel, "Direct QR factorizations
 * for tall-and-skinny matrices in MapReduce architectures" (arXiv:1301.1071).
 *
 * What the oracle computes and why it is the definition:
 *   Direct TSQR (Sec. III-B, the three-step factorisation A = Q R with
 *   Q = diag(Q_1..Q_p) * [Q^2_1; ..; Q^2_p]) reaches, in exact arithmetic,
 *   the thin QR factorisation of A (Sec. I, A = QR, Q m x n with orthonormal
 *   columns, R n x n upper triangular).  For full-rank A that factorisation
 *   is unique once diag(R) > 0 (Sec. II-A: R^T R = A^T A and the Cholesky
 *   factor is unique).  The oracle therefore computes one unblocked
 *   Householder QR of the WHOLE matrix (the textbook method the paper cites
 *   in Sec. III and III-A; no row blocks, no tree), forms Q explicitly by
 *   backward accumulation, and normalises diag(R) to be positive.
 *
 * Householder convention (Sec. III-A only states A <- A - 2 v (A^T v)^T for
 * a unit v; the equivalent scaled form used here):
 *   alpha = x_1, sigma = ||x||_2 (scaled accumulation), beta = -copysign(sigma, alpha),
 *   v = x / (alpha - beta) with v_1 = 1, tau = (beta - alpha) / beta,
 *   H = I - tau v v^T, H x = beta e_1; a zero column gives tau = 0.
 *
 * Floating point: IEEE binary64 for the method; long double only in the
 * independent pins (MGS, Cholesky of A^T A, Jacobi eigen/SVD) and in the
 * checkers, which also use Dot2 compensated sums (Ogita, Rump, Oishi,
 * "Accurate sum and dot product", SIAM J. Sci. Comput. 2005).
 * Build with -ffp-contract=off so that no a*b+c is silently fused.
 *
 * Layout: every matrix argument is dense row-major (A[i*n + j]).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NOT_SPD 6
#define OR_ERR_SINGULAR 7
#define OR_ERR_NOCONV 10

/* Loops over independent columns (or rows) run on several threads when they
 * hold more than this many entries.  Only loops whose iterations compute
 * disjoint results are parallel, each iteration doing exactly the operations
 * of the serial loop, so the bits do not depend on the thread count. */
#define OR_PAR_MIN 65536
#define OR_NMAX_BWD 1024

/* ------------------------------------------------------------------------ */
/* Householder QR (Sec. III-A, textbook method), column-major work copy.     */
/* ------------------------------------------------------------------------ */

/* ||x||_2 with a running scale so that no square over- or underflows. */
static double nrm2_scaled(const double* x, int64_t len) {
  double scale = 0.0, ssq = 1.0;
  for (int64_t i = 0; i < len; ++i) {
    if (x[i] != 0.0) {
      double a = fabs(x[i]);
      if (scale < a) {
        double r = scale / a;
        ssq = 1.0 + ssq * r * r;
        scale = a;
      } else {
        double r = a / scale;
        ssq += r * r;
      }
    }
  }
  return scale * sqrt(ssq);
}

/* Factor the m x n column-major W in place: on return the upper triangle of
 * W holds the unnormalised R, the part below the diagonal holds v_j(2:end),
 * and tau[j] the reflector coefficients. */
static void house_factor_colmajor(double* W, int64_t m, int64_t n, double* tau) {
  for (int64_t j = 0; j < n; ++j) {
    double* x = W + j * m + j;
    int64_t len = m - j;
    double alpha = x[0];
    double sigma = nrm2_scaled(x, len);
    if (sigma == 0.0) {
      tau[j] = 0.0;
      continue;
    }
    double beta = -copysign(sigma, alpha);
    double denom = alpha - beta;
    for (int64_t i = 1; i < len; ++i) x[i] = x[i] / denom;
    tau[j] = (beta - alpha) / beta;
    x[0] = beta;
    /* apply H_j = I - tau v v^T to the trailing columns.  Each column's
       update is the same sequence of operations whichever thread runs it,
       so the result does not depend on the thread count. */
#pragma omp parallel for schedule(static) if (len * (n - j - 1) > OR_PAR_MIN)
    for (int64_t k = j + 1; k < n; ++k) {
      double* y = W + k * m + j;
      double w = y[0];
      for (int64_t i = 1; i < len; ++i) w += x[i] * y[i];
      w *= tau[j];
      y[0] -= w;
      for (int64_t i = 1; i < len; ++i) y[i] -= w * x[i];
    }
  }
}

static double* to_colmajor(const double* A, int64_t m, int64_t n) {
  double* W = (double*)malloc(sizeof(double) * (size_t)(m * n));
  if (!W) return NULL;
#pragma omp parallel for schedule(static) if (m * n > OR_PAR_MIN)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) W[j * m + i] = A[i * n + j];
  return W;
}

/* sign(R_jj) with sign(0) = +1 */
static double diag_sign(double r) { return r < 0.0 ? -1.0 : 1.0; }

/*
 * Thin QR of A (m x n, m >= n >= 1): Q m x n, R n x n upper triangular with
 * diag(R) >= 0.  Sec. I (A = QR) and Sec. III-A (Householder QR).
 * Q = H_1 H_2 ... H_n [I_n; 0] by backward accumulation.
 */
int oracle_householder_qr(const double* A, int64_t m, int64_t n, double* Q, double* R) {
  if (!A || !R || n < 1 || m < n) return OR_ERR_ARG;
  double* W = to_colmajor(A, m, n);
  double* tau = (double*)malloc(sizeof(double) * (size_t)n);
  double* M = Q ? (double*)calloc((size_t)(m * n), sizeof(double)) : NULL;
  if (!W || !tau || (Q && !M)) { free(W); free(tau); free(M); return OR_ERR_ARG; }
  house_factor_colmajor(W, m, n, tau);

  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  for (int64_t j = 0; j < n; ++j) d[j] = diag_sign(W[j * m + j]);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j)
      R[i * n + j] = (j >= i) ? d[i] * W[j * m + i] : 0.0;

  if (Q) {
    /* M (column-major) = [I; 0], then M <- H_j M for j = n..1 */
    for (int64_t j = 0; j < n; ++j) M[j * m + j] = 1.0;
    for (int64_t j = n - 1; j >= 0; --j) {
      if (tau[j] == 0.0) continue;
      const double* v = W + j * m + j; /* v[0] is implicitly 1 */
      int64_t len = m - j;
#pragma omp parallel for schedule(static) if (len * n > OR_PAR_MIN)
      for (int64_t k = 0; k < n; ++k) {
        double* y = M + k * m + j;
        double w = y[0];
        for (int64_t i = 1; i < len; ++i) w += v[i] * y[i];
        w *= tau[j];
        y[0] -= w;
        for (int64_t i = 1; i < len; ++i) y[i] -= w * v[i];
      }
    }
#pragma omp parallel for schedule(static) if (m * n > OR_PAR_MIN)
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) Q[i * n + j] = d[j] * M[j * m + i];
  }
  free(d);
  free(W);
  free(tau);
  free(M);
  return OR_OK;
}

/* R factor only (diag(R) >= 0): the output of indirect TSQR (Sec. II-B);
 * any reduction tree gives this R in exact arithmetic. */
int oracle_householder_r(const double* A, int64_t m, int64_t n, double* R) {
  return oracle_householder_qr(A, m, n, NULL, R);
}

/* ------------------------------------------------------------------------ */
/* Small dense helpers for the comparators (Sec. II).                        */
/* ------------------------------------------------------------------------ */

/* X <- B R^{-1} row by row (R upper triangular): x R = b, forward in j.
 * Sec. II-C, Q = A R^{-1}.  Returns OR_ERR_SINGULAR on a zero pivot. */
int oracle_right_solve_upper(const double* B, int64_t m, int64_t n, const double* R, double* X) {
  for (int64_t j = 0; j < n; ++j)
    if (R[j * n + j] == 0.0) return OR_ERR_SINGULAR;
  for (int64_t i = 0; i < m; ++i) {
    const double* b = B + i * n;
    double* x = X + i * n;
    for (int64_t j = 0; j < n; ++j) {
      double s = b[j];
      for (int64_t k = 0; k < j; ++k) s -= x[k] * R[k * n + j];
      x[j] = s / R[j * n + j];
    }
  }
  return OR_OK;
}

/* Inverse of the upper-triangular n x n R by back substitution on the
 * columns of I (Sec. II-C: "compute the inverse of R and multiply by A").
 * Returns OR_ERR_SINGULAR on a zero pivot. */
int oracle_upper_inverse(const double* R, int64_t n, double* X) {
  for (int64_t j = 0; j < n; ++j)
    if (R[j * n + j] == 0.0) return OR_ERR_SINGULAR;
  for (int64_t c = 0; c < n; ++c)
    for (int64_t i = n - 1; i >= 0; --i) {
      if (i > c) { X[i * n + c] = 0.0; continue; }
      double s = (i == c) ? 1.0 : 0.0;
      for (int64_t k = i + 1; k <= c; ++k) s -= R[i * n + k] * X[k * n + c];
      X[i * n + c] = s / R[i * n + i];
    }
  return OR_OK;
}

/* X = B R^{-1} with R^{-1} formed explicitly (Sec. II-C), row by row. */
static int apply_inverse(const double* B, int64_t m, int64_t n, const double* R, double* X) {
  double* Ri = (double*)malloc(sizeof(double) * (size_t)(n * n));
  int st = oracle_upper_inverse(R, n, Ri);
  if (st == OR_OK)
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t k = 0; k <= j; ++k) s += B[i * n + k] * Ri[k * n + j];
        X[i * n + j] = s;
      }
  free(Ri);
  return st;
}

/* C = A B for n x n row-major matrices. */
static void matmul_nn(const double* A, const double* B, int64_t n, double* C) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double s = 0.0;
      for (int64_t k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
      C[i * n + j] = s;
    }
}

/* Cholesky of the SPD n x n G = R^T R (R upper).  Sec. II-A.  Breakdown
 * (a pivot that is not positive and finite) returns OR_ERR_NOT_SPD. */
static int cholesky_upper(const double* G, int64_t n, double* R) {
  memset(R, 0, sizeof(double) * (size_t)(n * n));
  for (int64_t j = 0; j < n; ++j) {
    double s = G[j * n + j];
    for (int64_t k = 0; k < j; ++k) s -= R[k * n + j] * R[k * n + j];
    if (!(s > 0.0) || !isfinite(s)) return OR_ERR_NOT_SPD;
    double rjj = sqrt(s);
    R[j * n + j] = rjj;
    for (int64_t i = j + 1; i < n; ++i) {
      double t = G[j * n + i];
      for (int64_t k = 0; k < j; ++k) t -= R[k * n + j] * R[k * n + i];
      R[j * n + i] = t / rjj;
    }
  }
  return OR_OK;
}

/* G = A^T A = sum_p A_p^T A_p, summed row by row (Sec. II-A, Alg. 1). */
static void gram(const double* A, int64_t m, int64_t n, double* G) {
  memset(G, 0, sizeof(double) * (size_t)(n * n));
  for (int64_t i = 0; i < m; ++i) {
    const double* a = A + i * n;
    for (int64_t j = 0; j < n; ++j)
      for (int64_t k = 0; k < n; ++k) G[j * n + k] += a[j] * a[k];
  }
}

/*
 * Cholesky QR (Sec. II-A): R = chol(A^T A), Q = A R^{-1} with R^{-1} formed
 * explicitly (Sec. II-C).
 * refine_steps extra passes repeat the same method on the computed Q
 * (iterative refinement, Sec. I): Q <- Q R2^{-1}, R <- R2 R.
 */
int oracle_cholqr(const double* A, int64_t m, int64_t n, int refine_steps, double* Q, double* R) {
  if (!A || !Q || !R || n < 1 || m < n || refine_steps < 0) return OR_ERR_ARG;
  double* G = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* R2 = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* RR = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* Qt = (double*)malloc(sizeof(double) * (size_t)(m * n));
  int st = OR_OK;
  gram(A, m, n, G);
  st = cholesky_upper(G, n, R);
  if (st == OR_OK) st = apply_inverse(A, m, n, R, Q);
  for (int s = 0; s < refine_steps && st == OR_OK; ++s) {
    gram(Q, m, n, G);
    st = cholesky_upper(G, n, R2);
    if (st != OR_OK) break;
    memcpy(Qt, Q, sizeof(double) * (size_t)(m * n));
    st = apply_inverse(Qt, m, n, R2, Q);
    matmul_nn(R2, R, n, RR);
    memcpy(R, RR, sizeof(double) * (size_t)(n * n));
  }
  free(G); free(R2); free(RR); free(Qt);
  return st;
}

/*
 * Indirect TSQR with iterative refinement (Sec. II-B, II-C): R1 = R-factor of
 * A, Q0 = A R1^{-1}; each refinement step repeats it on the computed Q:
 * R2 = R-factor of Q0, Q = Q0 R2^{-1}, R = R2 R1.
 */
int oracle_indirect_refine(const double* A, int64_t m, int64_t n, int refine_steps, double* Q, double* R) {
  if (!A || !Q || !R || n < 1 || m < n || refine_steps < 0) return OR_ERR_ARG;
  double* R2 = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* RR = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* Qt = (double*)malloc(sizeof(double) * (size_t)(m * n));
  int st = oracle_householder_r(A, m, n, R);
  if (st == OR_OK) st = apply_inverse(A, m, n, R, Q);
  for (int s = 0; s < refine_steps && st == OR_OK; ++s) {
    st = oracle_householder_r(Q, m, n, R2);
    if (st != OR_OK) break;
    memcpy(Qt, Q, sizeof(double) * (size_t)(m * n));
    st = apply_inverse(Qt, m, n, R2, Q);
    matmul_nn(R2, R, n, RR);
    memcpy(R, RR, sizeof(double) * (size_t)(n * n));
  }
  free(R2); free(RR); free(Qt);
  return st;
}

/*
 * Adjoint of the thin QR (not in the paper; the differentiation form the
 * build adds): given Q, R and the cotangents dQ (m x n) and dR (n x n,
 * upper triangular), M = R dR^T - dQ^T Q, copyltu(M) = tril(M) + tril(M,-1)^T,
 * dA = (dQ + Q copyltu(M)) R^{-T}.  dQ or dR may be NULL (zero).
 */
int oracle_qr_backward(const double* Q, const double* R, const double* dQ, const double* dR,
                       int64_t m, int64_t n, double* dA) {
  if (!Q || !R || !dA || n < 1 || n > OR_NMAX_BWD || m < n) return OR_ERR_ARG;
  for (int64_t j = 0; j < n; ++j)
    if (R[j * n + j] == 0.0) return OR_ERR_SINGULAR;
  double* M = (double*)calloc((size_t)(n * n), sizeof(double));
  double* C = (double*)malloc(sizeof(double) * (size_t)(n * n));
  if (dR)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t k = 0; k < n; ++k) s += R[i * n + k] * dR[j * n + k];
        M[i * n + j] = s;
      }
  if (dQ) {
    /* (dQ^T Q)_ij = sum over rows r, in increasing r, for every (i, j): the
       rows run in the outer loop and each thread owns whole rows i of the
       sum, so every entry is the same sequence of additions for any thread
       count. */
    double* S = (double*)calloc((size_t)(n * n), sizeof(double));
#pragma omp parallel for schedule(static) if (m * n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t r = 0; r < m; ++r) {
        const double di = dQ[r * n + i];
        for (int64_t j = 0; j < n; ++j) S[i * n + j] += di * Q[r * n + j];
      }
    for (int64_t k = 0; k < n * n; ++k) M[k] -= S[k];
    free(S);
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) C[i * n + j] = (i >= j) ? M[i * n + j] : M[j * n + i];
#pragma omp parallel for schedule(static) if (m * n > OR_PAR_MIN)
  for (int64_t r = 0; r < m; ++r) {
    double b[OR_NMAX_BWD];
    /* b = dQ_r + Q_r C */
    for (int64_t j = 0; j < n; ++j) {
      double s = dQ ? dQ[r * n + j] : 0.0;
      for (int64_t k = 0; k < n; ++k) s += Q[r * n + k] * C[k * n + j];
      b[j] = s;
    }
    /* x R^T = b  <=>  R x^T = b^T: back substitution */
    double* x = dA + r * n;
    for (int64_t j = n - 1; j >= 0; --j) {
      double s = b[j];
      for (int64_t k = j + 1; k < n; ++k) s -= R[j * n + k] * x[k];
      x[j] = s / R[j * n + j];
    }
  }
  free(M); free(C);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Long-double pins and the SVD of R (Sec. III-B, SVD paragraph).            */
/* ------------------------------------------------------------------------ */

/* Cyclic threshold Jacobi eigenvalues of the symmetric n x n S (long double);
 * the eigenvalues are returned unsorted in ev.  A rotation is skipped when
 * |a_pq| is negligible next to the larger diagonal entry; the iteration stops
 * after a sweep without rotations or once the off-diagonal norm is below
 * n * eps * ||S||_F (long-double eps). */
int oracle_sym_eig_ld(const long double* S, int64_t n, long double* ev) {
  long double* a = (long double*)malloc(sizeof(long double) * (size_t)(n * n));
  memcpy(a, S, sizeof(long double) * (size_t)(n * n));
  const long double eps = LDBL_EPSILON;
  int conv = 0;
  for (int sweep = 0; sweep < 100 && !conv; ++sweep) {
    long double off = 0.0L, tot = 0.0L;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        tot += a[i * n + j] * a[i * n + j];
        if (i != j) off += a[i * n + j] * a[i * n + j];
      }
    if (off == 0.0L || off <= (long double)(n * n) * eps * eps * tot) { conv = 1; break; }
    int rotated = 0;
    for (int64_t p = 0; p < n - 1; ++p)
      for (int64_t q = p + 1; q < n; ++q) {
        long double apq = a[p * n + q];
        long double dmax = fabsl(a[p * n + p]) > fabsl(a[q * n + q]) ? fabsl(a[p * n + p]) : fabsl(a[q * n + q]);
        if (apq == 0.0L || fabsl(apq) <= eps * dmax) continue;
        rotated = 1;
        long double theta = (a[q * n + q] - a[p * n + p]) / (2.0L * apq);
        long double t = (theta >= 0 ? 1.0L : -1.0L) / (fabsl(theta) + sqrtl(theta * theta + 1.0L));
        long double c = 1.0L / sqrtl(t * t + 1.0L), s = t * c;
        for (int64_t k = 0; k < n; ++k) { /* columns p, q */
          long double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int64_t k = 0; k < n; ++k) { /* rows p, q */
          long double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
      }
    if (!rotated) conv = 1;
  }
  for (int64_t i = 0; i < n; ++i) ev[i] = a[i * n + i];
  free(a);
  return conv ? OR_OK : OR_ERR_NOCONV;
}

/* Eigenvalues (double) of the symmetric n x n S given in double. */
int oracle_sym_eig(const double* S, int64_t n, double* ev) {
  long double* a = (long double*)malloc(sizeof(long double) * (size_t)(n * n));
  long double* e = (long double*)malloc(sizeof(long double) * (size_t)n);
  for (int64_t i = 0; i < n * n; ++i) a[i] = S[i];
  int st = oracle_sym_eig_ld(a, n, e);
  for (int64_t i = 0; i < n; ++i) ev[i] = (double)e[i];
  free(a); free(e);
  return st;
}

/* Modified Gram-Schmidt with one full re-orthogonalisation pass, in long
 * double (independent pin for the thin QR on tiny inputs). */
int oracle_mgs_ld(const double* A, int64_t m, int64_t n, double* Q, double* R) {
  if (!A || !Q || !R || n < 1 || m < n) return OR_ERR_ARG;
  long double* q = (long double*)malloc(sizeof(long double) * (size_t)(m * n));
  long double* r = (long double*)calloc((size_t)(n * n), sizeof(long double));
  for (int64_t i = 0; i < m * n; ++i) q[i] = A[i];
  for (int64_t j = 0; j < n; ++j) {
    for (int pass = 0; pass < 2; ++pass)
      for (int64_t k = 0; k < j; ++k) {
        long double s = 0.0L;
        for (int64_t i = 0; i < m; ++i) s += q[i * n + k] * q[i * n + j];
        r[k * n + j] += s;
        for (int64_t i = 0; i < m; ++i) q[i * n + j] -= s * q[i * n + k];
      }
    long double nn = 0.0L;
    for (int64_t i = 0; i < m; ++i) nn += q[i * n + j] * q[i * n + j];
    nn = sqrtl(nn);
    if (nn == 0.0L) { free(q); free(r); return OR_ERR_SINGULAR; }
    r[j * n + j] = nn;
    for (int64_t i = 0; i < m; ++i) q[i * n + j] /= nn;
  }
  for (int64_t i = 0; i < m * n; ++i) Q[i] = (double)q[i];
  for (int64_t i = 0; i < n * n; ++i) R[i] = (double)r[i];
  free(q); free(r);
  return OR_OK;
}

/* Cholesky factor (upper, long double) of the long-double Gram A^T A:
 * the unique R of Sec. II-A, used as an independent pin on tiny inputs. */
int oracle_chol_gram_ld(const double* A, int64_t m, int64_t n, double* R) {
  if (!A || !R || n < 1 || m < n) return OR_ERR_ARG;
  long double* G = (long double*)calloc((size_t)(n * n), sizeof(long double));
  long double* L = (long double*)calloc((size_t)(n * n), sizeof(long double));
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j)
      for (int64_t k = 0; k < n; ++k) G[j * n + k] += (long double)A[i * n + j] * (long double)A[i * n + k];
  int st = OR_OK;
  for (int64_t j = 0; j < n && st == OR_OK; ++j) {
    long double s = G[j * n + j];
    for (int64_t k = 0; k < j; ++k) s -= L[k * n + j] * L[k * n + j];
    if (!(s > 0.0L)) { st = OR_ERR_NOT_SPD; break; }
    long double rjj = sqrtl(s);
    L[j * n + j] = rjj;
    for (int64_t i = j + 1; i < n; ++i) {
      long double t = G[j * n + i];
      for (int64_t k = 0; k < j; ++k) t -= L[k * n + j] * L[k * n + i];
      L[j * n + i] = t / rjj;
    }
  }
  for (int64_t i = 0; i < n * n; ++i) R[i] = (double)L[i];
  free(G); free(L);
  return st;
}

/*
 * SVD of the n x n R by one-sided (Hestenes) Jacobi in long double:
 * R = U_R diag(S) V^T, S descending; each (u_j, v_j) pair is flipped so that
 * the largest-|.| entry of v_j is positive (lowest index wins a tie).
 * Sec. III-B, SVD paragraph: R = U Sigma V^T, then A = (Q U) Sigma V^T.
 */
int oracle_jacobi_svd_ld(const double* R, int64_t n, double* U, double* S, double* V) {
  long double* a = (long double*)malloc(sizeof(long double) * (size_t)(n * n)); /* columns rotated */
  long double* v = (long double*)calloc((size_t)(n * n), sizeof(long double));
  for (int64_t i = 0; i < n * n; ++i) a[i] = R[i];
  for (int64_t i = 0; i < n; ++i) v[i * n + i] = 1.0L;
  int conv = 0;
  for (int sweep = 0; sweep < 100 && !conv; ++sweep) {
    conv = 1;
    for (int64_t p = 0; p < n - 1; ++p)
      for (int64_t q = p + 1; q < n; ++q) {
        long double alpha = 0, beta = 0, gamma = 0;
        for (int64_t i = 0; i < n; ++i) {
          alpha += a[i * n + p] * a[i * n + p];
          beta += a[i * n + q] * a[i * n + q];
          gamma += a[i * n + p] * a[i * n + q];
        }
        if (gamma == 0.0L || fabsl(gamma) <= (long double)LDBL_EPSILON * sqrtl(alpha * beta)) continue;
        conv = 0;
        long double zeta = (beta - alpha) / (2.0L * gamma);
        long double t = (zeta >= 0 ? 1.0L : -1.0L) / (fabsl(zeta) + sqrtl(1.0L + zeta * zeta));
        long double c = 1.0L / sqrtl(1.0L + t * t), s = c * t;
        for (int64_t i = 0; i < n; ++i) {
          long double x = a[i * n + p], y = a[i * n + q];
          a[i * n + p] = c * x - s * y;
          a[i * n + q] = s * x + c * y;
          x = v[i * n + p]; y = v[i * n + q];
          v[i * n + p] = c * x - s * y;
          v[i * n + q] = s * x + c * y;
        }
      }
  }
  /* singular values = column norms; sort descending (stable selection) */
  long double* sv = (long double*)malloc(sizeof(long double) * (size_t)n);
  int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t j = 0; j < n; ++j) {
    long double s2 = 0;
    for (int64_t i = 0; i < n; ++i) s2 += a[i * n + j] * a[i * n + j];
    sv[j] = sqrtl(s2);
    ord[j] = j;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j)
      if (sv[ord[j]] > sv[ord[i]]) { int64_t t = ord[i]; ord[i] = ord[j]; ord[j] = t; }
  for (int64_t jj = 0; jj < n; ++jj) {
    int64_t j = ord[jj];
    /* sign: largest-|.| entry of v_j positive, lowest index wins a tie */
    int64_t imax = 0;
    for (int64_t i = 1; i < n; ++i)
      if (fabsl(v[i * n + j]) > fabsl(v[imax * n + j])) imax = i;
    long double sg = v[imax * n + j] < 0 ? -1.0L : 1.0L;
    S[jj] = (double)sv[j];
    for (int64_t i = 0; i < n; ++i) {
      V[i * n + jj] = (double)(sg * v[i * n + j]);
      U[i * n + jj] = sv[j] > 0 ? (double)(sg * a[i * n + j] / sv[j]) : 0.0;
    }
  }
  free(a); free(v); free(sv); free(ord);
  return conv ? OR_OK : OR_ERR_NOCONV;
}

/* SVD of A via the thin QR and the SVD of R (Sec. III-B): A = (Q U_R) S V^T. */
int oracle_svd(const double* A, int64_t m, int64_t n, double* U, double* S, double* V) {
  if (!A || !U || !S || !V || n < 1 || m < n) return OR_ERR_ARG;
  double* Q = (double*)malloc(sizeof(double) * (size_t)(m * n));
  double* R = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* UR = (double*)malloc(sizeof(double) * (size_t)(n * n));
  int st = oracle_householder_qr(A, m, n, Q, R);
  if (st == OR_OK) st = oracle_jacobi_svd_ld(R, n, UR, S, V);
  if (st == OR_OK)
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t k = 0; k < n; ++k) s += Q[i * n + k] * UR[k * n + j];
        U[i * n + j] = s;
      }
  free(Q); free(R); free(UR);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Checkers (Sec. I-B metrics): ||Q^T Q - I||_2, ||A - QR||.                 */
/* Dot2 compensated accumulation (Ogita-Rump-Oishi 2005).                    */
/* ------------------------------------------------------------------------ */

typedef struct { double s, c; } acc2;

static inline void two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}
static inline void acc2_add_prod(acc2* A, double x, double y) {
  double p = x * y;
  double ep = fma(x, y, -p);
  double s, es;
  two_sum(A->s, p, &s, &es);
  A->s = s;
  A->c += es + ep;
}
static inline void acc2_add_acc(acc2* A, acc2 B) {
  double s, es;
  two_sum(A->s, B.s, &s, &es);
  A->s = s;
  A->c += es + B.c;
}

/* Symmetric Gram X^T Y with Dot2 over rows, in ROW CHUNKS combined in a
 * fixed order (deterministic for any thread count).  G is n x n. */
static void gram_dot2(const double* X, const double* Y, int64_t m, int64_t n, double* G) {
  const int64_t chunk = 65536;
  int64_t nch = (m + chunk - 1) / chunk;
  int64_t nn = n * n;
  acc2* part = (acc2*)calloc((size_t)(nch * nn), sizeof(acc2));
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nch; ++c) {
    acc2* P = part + c * nn;
    int64_t r0 = c * chunk, r1 = r0 + chunk < m ? r0 + chunk : m;
    for (int64_t r = r0; r < r1; ++r) {
      const double* x = X + r * n;
      const double* y = Y + r * n;
      for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) acc2_add_prod(&P[i * n + j], x[i], y[j]);
    }
  }
  for (int64_t k = 0; k < nn; ++k) {
    acc2 t = {0.0, 0.0};
    for (int64_t c = 0; c < nch; ++c) acc2_add_acc(&t, part[c * nn + k]);
    G[k] = t.s + t.c;
  }
  free(part);
}

/* ||Q^T Q - I||_2 (largest |eigenvalue| of the symmetric error, long-double
 * Jacobi) and ||Q^T Q - I||_F.  Sec. I-B / Sec. IV metric. */
int oracle_orth_error(const double* Q, int64_t m, int64_t n, double* err2, double* errF) {
  const int64_t chunk = 65536;
  int64_t nch = (m + chunk - 1) / chunk;
  int64_t nn = n * n;
  acc2* part = (acc2*)calloc((size_t)(nch * nn), sizeof(acc2));
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nch; ++c) {
    acc2* P = part + c * nn;
    int64_t r0 = c * chunk, r1 = r0 + chunk < m ? r0 + chunk : m;
    for (int64_t r = r0; r < r1; ++r) {
      const double* q = Q + r * n;
      for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i; j < n; ++j) acc2_add_prod(&P[i * n + j], q[i], q[j]);
    }
  }
  long double* E = (long double*)malloc(sizeof(long double) * (size_t)nn);
  long double* ev = (long double*)malloc(sizeof(long double) * (size_t)n);
  long double f2 = 0.0L;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i; j < n; ++j) {
      acc2 t = {0.0, 0.0};
      for (int64_t c = 0; c < nch; ++c) acc2_add_acc(&t, part[c * nn + i * n + j]);
      long double e = (long double)t.s + (long double)t.c - (i == j ? 1.0L : 0.0L);
      E[i * n + j] = E[j * n + i] = e;
      f2 += (i == j ? 1.0L : 2.0L) * e * e;
    }
  int st = oracle_sym_eig_ld(E, n, ev);
  long double mx = 0.0L;
  for (int64_t i = 0; i < n; ++i) if (fabsl(ev[i]) > mx) mx = fabsl(ev[i]);
  *err2 = (double)mx;
  *errF = (double)sqrtl(f2);
  free(part); free(E); free(ev);
  return st;
}

/* Residual of a factorisation: relF = ||A - Q R||_F / ||A||_F and
 * rel2 = ||A - Q R||_2 / ||R||_2 (the metric of Sec. I-B).  Each residual
 * entry a_ij - sum_k q_ik r_kj is formed with Dot2 (it is far smaller than
 * the terms it cancels); the norms of the residual only need a few correct
 * digits and are summed in plain double per row chunk.  R is n x n (its
 * lower triangle is read as stored).  n <= 512. */
int oracle_residual(const double* A, const double* Q, const double* R, int64_t m, int64_t n,
                    double* relF, double* rel2) {
  if (!A || !Q || !R || n < 1 || n > 512 || m < 1) return OR_ERR_ARG;
  const int64_t chunk = 65536;
  int64_t nch = (m + chunk - 1) / chunk;
  int64_t nn = n * n;
  double* ssE = (double*)calloc((size_t)nch, sizeof(double));
  double* ssA = (double*)calloc((size_t)nch, sizeof(double));
  double* GE = (double*)calloc((size_t)(nch * nn), sizeof(double));
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nch; ++c) {
    int64_t r0 = c * chunk, r1 = r0 + chunk < m ? r0 + chunk : m;
    double* g = GE + c * nn;
    double e[512];
    for (int64_t r = r0; r < r1; ++r) {
      for (int64_t j = 0; j < n; ++j) {
        acc2 t = {A[r * n + j], 0.0};
        for (int64_t k = 0; k < n; ++k) acc2_add_prod(&t, -Q[r * n + k], R[k * n + j]);
        e[j] = t.s + t.c;
        ssE[c] += e[j] * e[j];
        ssA[c] += A[r * n + j] * A[r * n + j];
      }
      for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) g[i * n + j] += e[i] * e[j];
    }
  }
  double sE = 0, sA = 0;
  long double* G = (long double*)calloc((size_t)nn, sizeof(long double));
  for (int64_t c = 0; c < nch; ++c) {
    sE += ssE[c];
    sA += ssA[c];
    for (int64_t k = 0; k < nn; ++k) G[k] += GE[c * nn + k];
  }
  long double* ev = (long double*)malloc(sizeof(long double) * (size_t)n);
  int st = oracle_sym_eig_ld(G, n, ev);
  long double emax = 0;
  for (int64_t i = 0; i < n; ++i) if (ev[i] > emax) emax = ev[i];
  /* ||R||_2^2 = largest eigenvalue of R^T R */
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      long double s = 0;
      for (int64_t k = 0; k < n; ++k) s += (long double)R[k * n + i] * R[k * n + j];
      G[i * n + j] = s;
    }
  int st2 = oracle_sym_eig_ld(G, n, ev);
  long double rmax = 0;
  for (int64_t i = 0; i < n; ++i) if (ev[i] > rmax) rmax = ev[i];
  *relF = sA > 0 ? sqrt(sE / sA) : sqrt(sE);
  *rel2 = rmax > 0 ? (double)sqrtl(emax / rmax) : (double)sqrtl(emax);
  free(ssE); free(ssA); free(GE); free(G); free(ev);
  return st != OR_OK ? st : st2;
}

/* Dot2 Gram X^T Y (n x n), exposed for the tests. */
int oracle_gram_dot2(const double* X, const double* Y, int64_t m, int64_t n, double* G) {
  if (!X || !Y || !G || n < 1 || m < 1) return OR_ERR_ARG;
  gram_dot2(X, Y, m, n, G);
  return OR_OK;
}

/* Threads for the parallel loops (1 = the plain serial oracle). */
int oracle_set_num_threads(int t) {
#ifdef _OPENMP
  if (t < 1) return OR_ERR_ARG;
  omp_set_num_threads(t);
#else
  (void)t;
#endif
  return OR_OK;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
