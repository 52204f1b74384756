/*
 * tsqr.h -- C-ABI of the GB300 (sm_103a) direct-TSQR library.
 *
 * Method: A. R. Benson, D. F. Gleich, J. Demmel, "Direct QR factorizations
 * for tall-and-skinny matrices in MapReduce architectures" (arXiv:1301.1071).
 *
 * Problem statement (Sec. I): A is m x n, full rank, m >> n; the thin QR
 * factorisation is A = Q R with Q m x n (orthonormal columns) and R n x n
 * upper triangular.  This library normalises diag(R) >= 0, which makes the
 * factorisation unique for full-rank A (Sec. II-A).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are dense ROW-MAJOR (the paper's row-wise layout, Sec. III-A):
 *    element (i, j) of A is A[i * lda + j].  Version 1 requires every leading
 *    dimension to equal n and every base pointer to be 16-byte aligned, else
 *    TSQR_ERR_ALIGN is returned.
 *  - All data pointers (A, Q, R, U, S, V, dQ, dR, dA, work) are DEVICE
 *    pointers owned by the caller.  The library allocates no device memory;
 *    it keeps no pointer after a call returns.  Inputs are read-only.
 *  - dtype selects the storage (and compute) type of the tall matrices
 *    (A, Q, U, dQ, dA): TSQR_F64 (IEEE binary64) or TSQR_F32 (binary32).
 *    The small n x n matrices R, V, dR and the singular values S are always
 *    binary64, as are all stacked R factors and the reduction tree (Step 2).
 *  - work / work_bytes: device workspace of at least the size returned by
 *    tsqr_workspace_size() for the same (op, m, n, dtype, opts).  It holds
 *    the device status word, the stacked R factors, the compact-WY T factors
 *    and the Step-2 coefficient blocks.  Its first 256 bytes are the status
 *    header; the rest need no initialisation.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call only enqueues work on it and returns; argument, shape,
 *    alignment and workspace errors are returned synchronously, before any
 *    launch.  Data-dependent errors (NOT_SPD, SINGULAR, NONFINITE, TIMEOUT,
 *    NOCONV) are written to the status word in the workspace: read them with
 *    tsqr_read_status(), or set opts->sync = 1 to have the call synchronise
 *    the stream and return that status.  No kernel traps.
 *  - tsqr_direct, tsqr_svd (and tsqr_direct_static through tsqr_direct),
 *    when the row blocks' T factors cover at least 16 MiB, run the Step-2
 *    tree on an internal stream of the device's highest priority, forked
 *    from `stream` after Step 1 and joined back into it before Step 3 (one
 *    such stream per device, created on the first large call and kept until
 *    the process exits; two events created and released per call).  To the
 *    caller the call is still ordered on `stream` alone: earlier work on it
 *    precedes the call, and later work waits for all of it -- also when the
 *    call returns an error after the fork.
 *  - Calls that share a workspace must be ordered (same stream).
 */
#ifndef TSQR_GB300_H
#define TSQR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSQR_NMAX 100 /* largest supported n */

typedef enum tsqr_status {
  TSQR_OK = 0,
  TSQR_ERR_ARG = 1,       /* null pointer, bad enum/option value */
  TSQR_ERR_SHAPE = 2,     /* n < 1, n > TSQR_NMAX, m < n, m n 8 bytes beyond int64, block_rows or
                             tree_fanout out of range, a workspace size beyond size_t, a block
                             height or a count of row blocks (or of their T slots) beyond
                             2^31 - 1 */
  TSQR_ERR_ALIGN = 3,     /* a leading dimension != n, or a pointer not 16-byte aligned */
  TSQR_ERR_WORKSPACE = 4, /* work == NULL or work_bytes too small */
  TSQR_ERR_CUDA = 5,      /* a CUDA runtime call or launch failed */
  TSQR_ERR_NOT_SPD = 6,   /* device: Cholesky breakdown (cholqr) */
  TSQR_ERR_SINGULAR = 7,  /* device: zero diagonal of R where R^-1 is applied */
  TSQR_ERR_NONFINITE = 8, /* device: NaN or Inf met in an input or a result */
  TSQR_ERR_TIMEOUT = 9,   /* device: a bounded wait on a bulk copy gave up */
  TSQR_ERR_NOCONV = 10    /* device: the Jacobi SVD of R did not converge */
} tsqr_status;

typedef enum tsqr_dtype { TSQR_F64 = 0, TSQR_F32 = 1 } tsqr_dtype;

/* Arithmetic of the tall passes (Step 1 and Step 3).  Only tsqr_direct and
 * tsqr_svd honour it; the Step-2 tree, the SVD of R and all n x n work are
 * binary64 in every mode.
 * NATIVE: the data's type (binary64 for TSQR_F64, binary32 with binary32
 *         accumulation for TSQR_F32).
 * DF64:   TSQR_F64 data only.  Binary64 storage, double-float arithmetic
 *         (pairs of binary32, ~48-bit significand) in Step 1 and Step 3, each
 *         row block scaled by a power of two (exact).  Targets ||Q^TQ - I||
 *         and the residual at the 1e-13 level for kappa up to ~1e15.
 * TF32X3: TSQR_F32 data only.  Step 1 as NATIVE; the Step-3 product
 *         Y_i W_i runs on the tensor cores as 3xTF32 split precision
 *         (Y = Yh + Yl, W = Wh + Wl rounded to TF32; Y W ~ Yh Wh + Yh Wl +
 *         Yl Wh, binary32 accumulation), for every n.
 * AUTO:   the library's choice for the data: TSQR_F32 data takes TF32X3 at
 *         n >= 20 (where it is the faster Step 3) and NATIVE below;
 *         TSQR_F64 data takes OZAKI at n <= 32 and NATIVE above.
 * OZAKI:  TSQR_F64 data only.  Step 1's Householder factorisation and the
 *         tree in binary64; for n <= 32 the two products of the method run on
 *         the tensor cores as error-free split products (Ozaki, Ogita, Oishi,
 *         Rump 2012): the Step-3 product Y_i W_i (each row of Y and column of
 *         W cut into 7 digits of 8 bits, 56 bits, against its largest
 *         exponent) and the Gram entries V^T V of the compact-WY T factors
 *         (8 digits, 64 bits; Step 1 then leaves them out of its column
 *         loop).  The digit products accumulate exactly in binary32
 *         (binary16 operands), are recombined in 64-bit integers and rounded
 *         once to binary64.  Above n = 32, NATIVE. */
typedef enum tsqr_prec {
  TSQR_PREC_NATIVE = 0,
  TSQR_PREC_DF64 = 1,
  TSQR_PREC_TF32X3 = 2,
  TSQR_PREC_AUTO = 3,
  TSQR_PREC_OZAKI = 4
} tsqr_prec;

/* Which computation a workspace is sized for. */
typedef enum tsqr_op {
  TSQR_OP_DIRECT = 0,
  TSQR_OP_SVD = 1,
  TSQR_OP_CHOLQR = 2,
  TSQR_OP_INDIRECT = 3,
  TSQR_OP_BACKWARD = 4,
  TSQR_OP_DIRECT_HOST = 5, /* tsqr_direct_host: its own row-block plan (copy chunks) */
  TSQR_OP_R = 6,           /* tsqr_r */
  TSQR_OP_SVD_VALUES = 7,  /* tsqr_svd_values */
  TSQR_OP_ACCURACY = 8     /* tsqr_accuracy */
} tsqr_op;

typedef struct tsqr_opts {
  int64_t block_rows; /* rows per Step-1 row block; 0 = automatic.  Must be >= n.
                         A block taller than one CTA's register tile is factored
                         by that CTA tile by tile (a flat reduction tree). */
  int32_t tree_fanout; /* R factors merged per Step-2 tree node; 0 = automatic.
                          >= 2; at most what one CTA's shared memory holds
                          (f n (n+1) binary64 values) or 8 (a node over a
                          cluster of f CTAs, one R factor each), else
                          TSQR_ERR_SHAPE.  Automatic: one CTA per node with
                          as many R factors as the binary64 register tile has
                          rows for, where that is at least 4 and 4 fit the
                          CTA; else 8 per node on a cluster. */
  int32_t sync;        /* 1 = synchronise the stream and return the device status */
  /* Optional stage timing (tsqr_direct, tsqr_svd): NULL, or 4 cudaEvent_t
     handles (as void*) recorded on the stream at the start, after Step 1's
     Householder kernel, after Step 2 (the T factors' build, tree up, top QR,
     SVD, tree down) and after Step 3. */
  void* const* stage_events;
  int32_t prec;        /* tsqr_prec (default 0 = NATIVE) */
  int32_t reserved;    /* must be zero */
} tsqr_opts;

/*
 * Workspace bytes needed by `op` for an m x n matrix of `dtype` under `opts`
 * (NULL = defaults).  Host-only; launches nothing.  The workspace holds what
 * the paper's MapReduce passes keep on disk between steps: the stacked R
 * factors of every Step-2 level (Sec. III-B, III-C), the compact-WY T
 * factors and the coefficient blocks Q2 (no call of the paper corresponds).
 * Errors: TSQR_ERR_ARG (NULL bytes, unknown op or dtype, bad opts),
 * TSQR_ERR_SHAPE (as the op's entry point).
 */
tsqr_status tsqr_workspace_size(int32_t op, int64_t m, int64_t n, int32_t dtype,
                                const tsqr_opts* opts, size_t* bytes);

/*
 * Direct TSQR (Sec. III-B, with the recursive Step 2 of Sec. III-C, Alg. 2):
 *   Step 1: each row block A_i (block_rows rows, the last one may be short)
 *           is factored by Householder QR, A_i = Q1_i R_i; Q1_i is kept in
 *           compact-WY form (Y_i written into Q's storage, T_i into work).
 *   Step 2: the stacked R_i (p*n x n, binary64) are factored, recursively
 *           while the stack is taller than one tree node (Alg. 2), giving the
 *           coefficient blocks Q2_i and R.
 *   Step 3: Q_i = Q1_i Q2_i, written over Y_i.
 * In:  A (m x n, dtype, lda == n).  Out: Q (m x n, dtype, ldq == n; may NOT
 * alias A), R (n x n binary64, ldr == n, upper triangular, diag(R) >= 0).
 */
tsqr_status tsqr_direct(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype,
                        void* Q, int64_t ldq, double* R, int64_t ldr,
                        void* work, size_t work_bytes, const tsqr_opts* opts, void* stream);

/*
 * SVD variant (Sec. III-B, SVD paragraph): Step 2 also computes
 * R = U_R diag(S) V^T (one-sided Jacobi in binary64, S descending, each
 * (u_j, v_j) signed so that the largest-|.| entry of v_j is positive) and
 * U_R is folded into the coefficient blocks, so Step 3 writes U = Q U_R
 * directly without writing Q (same data passes as the QR).
 * Out: U (m x n, dtype), S (n, binary64), V (n x n binary64, ldv == n).
 */
tsqr_status tsqr_svd(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype,
                     void* U, int64_t ldu, double* S, double* V, int64_t ldv,
                     void* work, size_t work_bytes, const tsqr_opts* opts, void* stream);

/*
 * R factor only (Sec. II-B, the R-only TSQR reduction; Sec. III-B names it
 * the method of choice when only R or only the singular values are wanted):
 * Steps 1 and 2 of direct TSQR with no Householder vectors, T factors or Q2
 * blocks kept, then the sign normalisation diag(R) >= 0.  A is read once and
 * nothing of size m is written.
 * In:  A (m x n, dtype, lda == n).  Out: R (n x n binary64, ldr == n, upper
 * triangular, diag(R) >= 0) -- the R of tsqr_direct up to rounding.
 * opts->prec: NATIVE or DF64 (FP64 data); TF32X3 only affects Step 3, which
 * this call does not run, and computes as NATIVE.  The workspace is that of
 * TSQR_OP_R (the same size as TSQR_OP_DIRECT).  Errors as tsqr_direct.
 */
tsqr_status tsqr_r(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype,
                   double* R, int64_t ldr,
                   void* work, size_t work_bytes, const tsqr_opts* opts, void* stream);

/*
 * Singular values (and right singular vectors) only (Sec. III-B, SVD
 * paragraph: Steps 1 and 2 plus the SVD of R suffice, with the R-only TSQR):
 * tsqr_r's R, then R = U_R diag(S) V^T by the one-sided Jacobi method of
 * tsqr_svd (S descending, V's columns signed as there).  No U is formed.
 * Out: S (n, binary64), V (n x n binary64, ldv == n), or V == NULL when only
 * S is wanted.  A Jacobi method that does not converge sets TSQR_ERR_NOCONV
 * in the status word.  Workspace: TSQR_OP_SVD_VALUES.
 */
tsqr_status tsqr_svd_values(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype,
                            double* S, double* V, int64_t ldv,
                            void* work, size_t work_bytes, const tsqr_opts* opts, void* stream);

/*
 * Cholesky QR (Sec. II-A; Q = A R^{-1} of Sec. II-C): R = chol(A^T A) with
 * A^T A accumulated in binary64, Q = A R^{-1}.  refine_steps >= 0 extra
 * passes repeat the method on the computed Q (iterative refinement, Sec. I):
 * Q <- Q R2^{-1}, R <- R2 R (binary64).  A Cholesky breakdown sets
 * TSQR_ERR_NOT_SPD in the status word (Q, R are then undefined).
 */
tsqr_status cholqr(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype,
                   void* Q, int64_t ldq, double* R, int64_t ldr, int32_t refine_steps,
                   void* work, size_t work_bytes, const tsqr_opts* opts, void* stream);

/*
 * Indirect TSQR with iterative refinement (Sec. II-B, II-C): R1 from the
 * R-only TSQR of A (Steps 1-2 without Q1/Q2), Q0 = A R1^{-1}; each of the
 * refine_steps passes repeats it on the computed Q: R2 from TSQR(Q0),
 * Q = Q0 R2^{-1}, R = R2 R1 (binary64).  A zero diagonal in R sets
 * TSQR_ERR_SINGULAR.
 */
tsqr_status tsqr_indirect_refine(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype,
                                 void* Q, int64_t ldq, double* R, int64_t ldr, int32_t refine_steps,
                                 void* work, size_t work_bytes, const tsqr_opts* opts, void* stream);

/*
 * Adjoint of the thin QR (not in the paper; the differentiation form):
 *   M = R dR^T - dQ^T Q,  copyltu(M) = tril(M) + tril(M, -1)^T,
 *   dA = (dQ + Q copyltu(M)) R^{-T}.
 * Q (m x n, dtype) and R (n x n binary64) are the saved forward outputs.
 * dQ (m x n, dtype) and dR (n x n binary64; only its upper triangle is read)
 * may each be NULL, meaning zero.  Out: dA (m x n, dtype).  A zero diagonal
 * in R sets TSQR_ERR_SINGULAR.
 */
tsqr_status tsqr_backward(const void* Q, const double* R, const void* dQ, const double* dR,
                          int64_t m, int64_t n, int32_t dtype, void* dA,
                          void* work, size_t work_bytes, const tsqr_opts* opts, void* stream);

/*
 * Direct TSQR without a caller-provided workspace (the paper has no
 * counterpart; this is a deployment convenience).  Same computation,
 * arguments and outputs as tsqr_direct, but the workspace is a fixed array of
 * TSQR_STATIC_WORK_BYTES in device memory owned by the library, so the call
 * allocates nothing.  It is meant for callers that cannot allocate device
 * memory themselves: a host framework that owns all device memory and forbids
 * other allocations, a latency-critical caller that cannot pay for the
 * implicit device synchronisation of cudaMalloc/cudaFree, or plain C code
 * without a device allocator.
 *  - Limit: the problem's tsqr_workspace_size(TSQR_OP_DIRECT, ...) must not
 *    exceed TSQR_STATIC_WORK_BYTES (16 MiB; e.g. about 390,000 rows at
 *    n = 25 in FP64 with the default plan); larger problems get
 *    TSQR_ERR_WORKSPACE before any launch.
 *  - Every GPU that loads the library holds the array until the process exits.
 *  - The first call on each device (with that device current) looks up the
 *    array's device address; make that first call before any stream capture.
 *  - All calls of one process on one device share the one array: calls that
 *    overlap on the GPU (issued on different streams, or from different host
 *    threads) race and give undefined results.  Order them on one stream.
 *    (Each process's CUDA context holds its own copy of the array.)
 *  - The status word lives in the array and is cleared at every call; pass
 *    opts->sync = 1 to get a data-dependent error as the return value.
 */
#define TSQR_STATIC_WORK_BYTES (16u * 1024u * 1024u)
tsqr_status tsqr_direct_static(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype,
                               void* Q, int64_t ldq, double* R, int64_t ldr,
                               const tsqr_opts* opts, void* stream);

/*
 * Direct TSQR from and to HOST memory (Sec. III-B, Alg. 2), with the
 * host<->device copies overlapped with the kernels.  The same computation as
 * tsqr_direct on the device copy of A; the row blocks are taken in chunks of
 * whole waves of CTAs: chunk c's rows of A are copied on `copy_stream` while
 * Step 1 of chunk c - 1 runs on `stream`; after the tree (Step 2), Step 3
 * forms chunk c's rows of Q on `stream` while chunk c - 1's rows are copied
 * back on `copy_stream`.
 *  - A (read-only), Q: HOST, m x n row-major, dtype (leading dimension n).
 *    Page-locked memory lets the copies overlap the kernels; pageable memory
 *    works, with the copies serialised by the runtime.
 *  - R: HOST, n x n binary64, row-major, diag(R) >= 0.
 *  - dbuf: DEVICE, m x n elements of dtype, 16-byte aligned, caller-owned:
 *    holds A's rows, then Y (Step 1), then Q (Step 3), in place.
 *  - work: DEVICE workspace of tsqr_workspace_size(TSQR_OP_DIRECT_HOST, ...)
 *    bytes (its row-block plan differs from tsqr_direct's: the default block
 *    height makes each chunk a whole number of waves).
 *  - stream, copy_stream: two different CUDA streams of the current device.
 *    On return everything is enqueued and `stream` has been made to wait for
 *    the last copy on `copy_stream`: synchronising `stream` (or opts->sync = 1,
 *    which also returns the device status) completes the call.  An error
 *    returned after work was queued on `copy_stream` also leaves `stream`
 *    waiting for it (or, where that cannot be enqueued, the call waits for
 *    `copy_stream` on the host before returning).
 *  - The call creates and releases 2 x chunks + 1 CUDA events (no device
 *    memory); chunks <= 8.
 *  - Errors: as tsqr_direct (TSQR_ERR_ARG also for a NULL pointer or equal
 *    streams).
 */
tsqr_status tsqr_direct_host(const void* A, int64_t m, int64_t n, int32_t dtype, void* Q, double* R,
                             void* dbuf, void* work, size_t work_bytes, const tsqr_opts* opts,
                             void* stream, void* copy_stream);

/*
 * Accuracy of a computed factorisation: the metrics of Sec. I-B,
 * ||Q^T Q - I||_2 and ||A - Q R||_2 / ||R||_2, and ||A - Q R||_F / ||A||_F,
 * with every sum over the m rows accumulated in compensated (double-double)
 * arithmetic -- TwoProduct and TwoSum, Ogita, Rump and Oishi 2005 -- so that
 * the results hold at the 1e-15 level for any m (a plain binary64 sum over
 * m rows errs by about sqrt(m) eps).  The n x n results are left on the
 * device; the 2-norms are the largest |eigenvalue| of the symmetric n x n
 * matrices, taken by the caller.
 * In:  Q (m x n, dtype, ld n); A (m x n, dtype) and R (n x n binary64) both
 *      given or both NULL (orthogonality only).
 * Out: out, DEVICE, 3 n^2 + 2 binary64, row-major:
 *      out[0 .. n^2)        E_hi, out[n^2 .. 2 n^2) E_lo: Q^T Q - I = E_hi + E_lo
 *      out[2 n^2 .. 3 n^2)  F = (A - QR)^T (A - QR)  (zero without A)
 *      out[3 n^2]           ||A - QR||_F^2, out[3 n^2 + 1] ||A||_F^2
 * work: tsqr_workspace_size(TSQR_OP_ACCURACY, m, n, dtype, NULL) bytes.
 * The combination of the per-CTA sums is in a fixed order: the results do
 * not depend on scheduling.  Errors as tsqr_direct.
 */
tsqr_status tsqr_accuracy(const void* A, const void* Q, const double* R, int64_t m, int64_t n, int32_t dtype,
                          double* out, void* work, size_t work_bytes, void* stream);

/*
 * Number of kernel launches one call of `op` makes for this shape and opts
 * (refine_steps applies to TSQR_OP_CHOLQR / TSQR_OP_INDIRECT).  Host-only;
 * a measurement aid with no counterpart in the paper.  Errors as
 * tsqr_workspace_size (TSQR_ERR_ARG also for NULL launches or
 * refine_steps < 0).
 */
tsqr_status tsqr_launch_count(int32_t op, int64_t m, int64_t n, int32_t dtype, const tsqr_opts* opts,
                              int32_t refine_steps, int32_t* launches);

/*
 * The plan a call of `op` would use for this shape and opts (host-only;
 * launches nothing): the row-block partition of Step 1 (Sec. III-B: row
 * blocks of block_rows rows, the last one possibly shorter) and the
 * recursive Step-2 tree (Sec. III-C, Alg. 2: levels of tree_fanout stacked
 * R factors per node until one node remains).
 *   block_rows      rows per Step-1 row block
 *   blocks          number of row blocks (= R factors in the first stack)
 *   tiles_per_block register tiles per block (a taller block is factored
 *                   tile by tile, a flat tree inside the CTA)
 *   tree_levels     Step-2 tree levels (0: a single block, no tree)
 *   tree_fanout     R factors merged per tree node
 *   prec            the tsqr_prec the call computes in (TSQR_PREC_AUTO resolved)
 *   step3_tensor    1 when Step 3 runs on the tensor cores
 */
typedef struct tsqr_plan_info {
  int64_t block_rows;
  int64_t blocks;
  int32_t tiles_per_block;
  int32_t tree_levels;
  int32_t tree_fanout;
  int32_t prec;
  int32_t step3_tensor;
  int32_t reserved;
} tsqr_plan_info;
tsqr_status tsqr_plan_query(int32_t op, int64_t m, int64_t n, int32_t dtype, const tsqr_opts* opts,
                            tsqr_plan_info* info);

/*
 * Synchronises `stream` and returns the device status word of the last call
 * that used `work` (TSQR_OK if it succeeded).  A boundary utility with no
 * counterpart in the paper.  work: that call's workspace (device); stream:
 * the stream the call was issued on.  Returns TSQR_ERR_ARG for a NULL work
 * and TSQR_ERR_CUDA when the read-back or the synchronisation fails.
 */
tsqr_status tsqr_read_status(const void* work, void* stream);

/* Static, human-readable name of a status code (never NULL; an unknown
 * code gives "unknown tsqr_status").  No counterpart in the paper. */
const char* tsqr_status_string(int32_t status);

#ifdef __cplusplus
}
#endif

#endif /* TSQR_GB300_H */
