/* PHSVDS on GB300: C-ABI of the two-stage preconditioned SVD solver.
 *
 * The problem statement follows the paper's C interface (Wu, Romero,
 * Stathopoulos, "PRIMME_SVDS", Sec. 3.4 and Fig. 1): find the k largest or
 * smallest singular triplets (sigma_i, u_i, v_i) of a sparse m x n matrix A so
 * that the triplet residual of Eq. (res),
 *     ||r_i|| = sqrt(||A v_i - sigma_i u_i||^2 + ||A^T u_i - sigma_i v_i||^2),
 * is below tol * ||A||_2.  The method is Algorithm 1 (PHSVDS): a first stage on
 * C = A^T A and, if needed, a second stage on B = [0 A^T; A 0] (Sec. 3.1).
 *
 * All entry points return 0 on success, a negative SVDS_ERR_* code for invalid
 * arguments (detected before any device work) or SVDS_ERR_CUDA for a device
 * error, and SVDS_ERR_MAXIT (> 0) when the matvec or time budget ran out.
 * No function keeps a pointer to caller memory after it returns.
 */
#ifndef PHSVDS_H
#define PHSVDS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define SVDS_OK 0
#define SVDS_ERR_ARG (-1)      /* null pointer or out-of-range scalar argument */
#define SVDS_ERR_SHAPE (-2)    /* m, n, nnz or k inconsistent */
#define SVDS_ERR_CSR (-3)      /* rowptr not monotone, column index unsorted or out of range */
#define SVDS_ERR_VALUE (-4)    /* non-finite matrix value */
#define SVDS_ERR_NOMEM (-5)    /* device or host allocation failed, or workspace too small */
#define SVDS_ERR_CUDA (-6)     /* CUDA runtime error; svds_last_error() has the message */
#define SVDS_ERR_NUMERIC (-7)  /* unrecoverable breakdown in a small dense problem */
#define SVDS_ERR_OPERATOR (-8) /* a caller-supplied operator (svds_create_op) returned non-zero */
#define SVDS_ERR_MAXIT 1       /* budget exhausted: the first *numConverged triplets are valid */

/* ---- enumerations ---- */
#define SVDS_LARGEST 0
#define SVDS_SMALLEST 1

#define SVDS_GDPK 0  /* GD+k (generalised Davidson with +k restarting) */
#define SVDS_JDQMR 1 /* JDQMR: GD+k outer basis, corrections from symmetric QMR on the
                        Jacobi-Davidson correction equation (FP32 inner solves) */
#define SVDS_DYNAMIC 2 /* stage 1 only: GD+k or JDQMR correction chosen per outer iteration
                          from the measured reduction of log ||r|| per second of each
                          (Sec. 3.4: the paper's stage-1 default switches to minimise time) */

#define SVDS_DF64 3  /* FP64-class stage 1 in DOUBLE-FLOAT arithmetic: every long vector is a pair
                        (hi, lo) of floats and every operation an error-free FP32 transformation,
                        unit roundoff about 2^-48 (native FP64 is 2^-53) with the FP32 exponent
                        range (A is scaled by a power of two).  Not IEEE binary64: use
                        SVDS_NATIVE_FP64 for native FP64 arithmetic throughout. */
#define SVDS_FP64 SVDS_DF64 /* older name of SVDS_DF64, kept for source compatibility: it selects
                               DOUBLE-FLOAT arithmetic, not native FP64 */
#define SVDS_FP32 1  /* FP32 first phase of stage 1 (see svds_opts.stage1_precision) */
#define SVDS_NATIVE_FP64 4 /* native FP64 arithmetic everywhere (check mode; slow on GB300) */
#define SVDS_BF16 5  /* as SVDS_FP32, with the values of A (and of the explicit A^T A) stored in
                        bfloat16 wherever the operator is applied in FP32 (FP32 vectors and
                        accumulation); the FP64-class phases use the exact values */

#define SVDS_NORMAL_AUTO 0     /* C = A^T A applied as an explicit sparse matrix when that moves
                                  fewer bytes than A then A^T (estimated from the patterns) */
#define SVDS_NORMAL_TWOPASS 1  /* always A then A^T (Sec. 3.3) */
#define SVDS_NORMAL_EXPLICIT 2 /* always the explicit C (when its pattern can be formed) */

#define SVDS_PRECOND_NONE 0
#define SVDS_PRECOND_JACOBI 1
#define SVDS_PRECOND_LEARNED 2 /* sparse approximate inverse on the pattern of A^T A from the
                                  graph network of phsvds_gnn.h (stage 1, smallest values) */
#define SVDS_PRECOND_BLOCKJACOBI 3 /* block Jacobi on A^T A (Sec. 4): inverses of the diagonal
                                      blocks of precondBlockSize consecutive columns (stage 1,
                                      smallest values) */

/* Sparse matrix in CSR form (0-based).  Column indices must be strictly
 * increasing inside each row and values finite.  When on_device is non-zero
 * the three arrays are CUDA device pointers, otherwise host pointers.  The
 * caller keeps ownership; svds_create copies what it needs. */
typedef struct {
  int64_t m, n, nnz;
  const int32_t *rowptr; /* m + 1 entries, rowptr[0] = 0, rowptr[m] = nnz */
  const int32_t *colidx; /* nnz entries, 0 <= colidx < n */
  const double *vals;    /* nnz entries */
  int on_device;
} svds_csr;

/* Options.  svds_opts_default() fills the paper's defaults (Sec. 3.4):
 * maxBasisSize 15 / minRestartSize 6 for fewer than 10 largest values, else
 * 35 / 14 (raised to k + blockSize and minRestart + 2 blockSize when larger),
 * block size 1, Jacobi preconditioner for the smallest values. */
typedef struct {
  int maxBasisSize;     /* 0 = default */
  int minRestartSize;   /* 0 = default */
  int maxBlockSize;     /* 0 = 1 */
  int method_stage1;    /* SVDS_GDPK (default), SVDS_JDQMR or SVDS_DYNAMIC */
  int method_stage2;    /* SVDS_GDPK (default) or SVDS_JDQMR */
  int stage1_precision; /* SVDS_DF64 (default), SVDS_FP32, SVDS_BF16 or SVDS_NATIVE_FP64 */
  int stage1_polish;    /* with SVDS_FP32: 1 = continue stage 1 in FP64-class arithmetic
                           to the paper's stage-1 criterion before stage 2 (default 1) */
  int precond;          /* SVDS_PRECOND_JACOBI (default), SVDS_PRECOND_NONE, SVDS_PRECOND_LEARNED
                           or SVDS_PRECOND_BLOCKJACOBI */
  double aNorm;         /* ||A||_2 if known, 0 = estimate */
  int64_t maxMatvecs;   /* budget in products with A or A^T (per column), 0 = unlimited */
  double maxSeconds;    /* wall-clock budget, 0 = unlimited */
  uint64_t seed;        /* seed of the random initial block and breakdown replacements */
  int printLevel;       /* 0 silent .. 3 per-iteration lines on stderr */
  int initSize;         /* number of initial right vectors in initV (Sec. 3.4 initSize) */
  const double *initV;  /* host, n x initSize column-major, or NULL */
  void *stream;         /* cudaStream_t to run on, or NULL for the library's own stream */
  int innerMaxIt;       /* JDQMR: inner steps per correction, 0 = 30 */
  double innerRelTol;   /* JDQMR: stop an inner solve when its QMR residual bound falls below
                           this fraction of the right-hand side, 0 = 0.1 */
  int innerPrecision;   /* JDQMR inner solves: SVDS_FP32 (default) or SVDS_DF64 (the FP64-class
                           mode of the outer iteration) */
  const float *precondParams; /* SVDS_PRECOND_LEARNED: host array of phsvds_gnn_num_params()
                                 network parameters (copied by svds_create), or NULL */
  const char *precondModel;   /* SVDS_PRECOND_LEARNED without precondParams: path of a
                                 parameter file written by phsvds_gnn_save */
  int normalOperator;         /* SVDS_NORMAL_AUTO (default), _TWOPASS or _EXPLICIT */
  double relTol;              /* > 0: low-accuracy mode of the condition-number estimate (Sec. 5):
                                 stage 1 stops when ||r^C|| <= relTol |lambda| (or at the floor
                                 10 u ||C||), stage 2 is not run, and numConverged counts the
                                 triplets that meet that relative rule; tol is then unused.
                                 Stage 1 uses GD+k corrections in this mode whatever
                                 method_stage1 says.  0 (default) = the rules of Algorithm 1 */
  int precondBlockSize;       /* SVDS_PRECOND_BLOCKJACOBI: columns per block, 1..64 (0 = 32) */
  int precondStallIts;        /* SVDS_PRECOND_LEARNED: the plain Jacobi preconditioner replaces the
                                 learned M for the rest of stage 1 after this many outer iterations
                                 in which the smallest residual of the corrected block did not fall
                                 below 0.99 of its best since a pair last converged (0 = 50, < 0 =
                                 never).  An M with a non-finite value or a non-positive diagonal is
                                 replaced before the first iteration.  See svds_stats.precond_fallback */
} svds_opts;

/* Performance report (the paper's stats, Sec. 3.4; matvecs count products
 * with A or A^T per column as in the paper's tables). */
typedef struct {
  int64_t matvecs_stage1, matvecs_stage2;
  int64_t matvecs_stage1_lowprec; /* part of matvecs_stage1 done in FP32 */
  int64_t outer_stage1, outer_stage2;
  int64_t restarts, resets;
  int stage2_used;
  double aNorm;               /* ||A|| used in the tolerances */
  double seconds_setup;       /* device setup inside svds_solve (norm estimate, buffers) */
  double seconds_stage1, seconds_stage2, seconds_total;
  int64_t kernel_launches;    /* device kernels launched by this call */
  double seconds_host_eig;    /* host time in the projected eigenproblems */
  double seconds_sync_wait;   /* host time blocked on the device (small results coming back) */
  int64_t host_syncs;         /* device-to-host round trips */
  int64_t inner_steps;        /* JDQMR inner sQMR steps (each applies the operator to the block) */
  double seconds_precond;     /* building the learned (graph of A^T A and network inference) or
                                 block-Jacobi preconditioner */
  int64_t normal_nnz;         /* nonzeros of the explicit C = A^T A, 0 when A then A^T is used */
  double seconds_output;      /* returning the vectors: FP64 conversion, sign convention, copies to U, V */
  int64_t outer_stage1_jdqmr; /* stage-1 outer iterations whose correction came from JDQMR */
  int precond_fallback;       /* 0, or the learned preconditioner was replaced by Jacobi: 1 = M
                                 rejected (non-finite value or non-positive diagonal), 2 = stall */
  double seconds_norm;        /* the ||A|| estimate inside seconds_setup (0 when aNorm was given) */
  int norm_steps;             /* its Arnoldi steps on C */
} svds_stats;

typedef struct svds_handle svds_handle;

/* Fill opts with the defaults above. */
int svds_opts_default(svds_opts *opts);

/* Copy A to the device, build A^T (deterministic transpose), the value formats
 * of every precision mode and the Jacobi diagonals (Sec. 3.3: the operator must
 * apply both A and A^T).  *h receives a new handle owned by the caller. */
int svds_create(svds_handle **h, const svds_csr *A, const svds_opts *opts);

/* Caller-supplied operators (Sec. 3.4: the C and B operators may be given
 * directly instead of the matrix).  The library calls
 *     apply(op, rows, nb, X, ldx, Y, ldy, stream, ctx)
 * with op = SVDS_OP_C for Y = A^T A X (rows = n) or op = SVDS_OP_B for
 * Y = [0 A^T; A 0] X (rows = n + m; the first n rows of a block are its right
 * part, the next m its left part, so Y[0:n] = A^T X[n:n+m] and
 * Y[n:n+m] = A X[0:n]).  X and Y are row-major FP64 device blocks of nb
 * columns with leading dimensions ldx, ldy (elements, >= nb); the function
 * must leave X unchanged and finish writing Y in stream order on `stream` (a
 * cudaStream_t): enqueue its kernels there, or synchronise before returning.
 * A non-zero return stops the solve with SVDS_ERR_OPERATOR.  In the reduced-
 * precision and double-float modes the library converts its blocks to FP64
 * around each call.  The operator is called from the thread that calls
 * svds_solve / svds_condest. */
#define SVDS_OP_C 1
#define SVDS_OP_B 2
typedef int (*svds_apply_fn)(int op, int64_t rows, int nb, const double *X, int64_t ldx, double *Y,
                             int64_t ldy, void *stream, void *ctx);

/* A handle on an m x n matrix given by its operators (m >= n >= 1: the tall
 * orientation, as the library stores a CSR matrix).  diagC: host array of the
 * n diagonal entries of A^T A (copied), needed for SVDS_PRECOND_JACOBI, else
 * NULL.  Options as for svds_create, except that precond is SVDS_PRECOND_NONE
 * or SVDS_PRECOND_JACOBI, stage1_precision is not SVDS_BF16 (there are no
 * matrix values to round) and normalOperator is unused.  The operator's norm
 * must stay within the FP32 exponent range in the double-float and FP32 modes
 * (the library does not rescale it).  ctx is passed through unchanged. */
int svds_create_op(svds_handle **h, int64_t m, int64_t n, svds_apply_fn apply, void *ctx, const double *diagC,
                   const svds_opts *opts);

/* Compute k singular triplets (Algorithm 1).  Outputs are caller-owned host
 * arrays: sigma[k] (descending for SVDS_LARGEST, ascending for SVDS_SMALLEST),
 * U (m x k column-major, ld m), V (n x k column-major, ld n), rnorm[k] (Eq. res,
 * recomputed from the returned vectors).  Each v has its largest-magnitude
 * entry positive.  Any of U, V, rnorm, stats may be NULL.  *numConverged is
 * the number of leading triplets that meet the tolerance. */
int svds_solve(svds_handle *h, int k, int target, double tol, double *sigma, double *U, double *V,
               double *rnorm, int *numConverged, svds_stats *stats);

/* Condition-number estimate (Sec. 5): one largest and one smallest singular
 * value, block size 1, each stage-1 solve stopped when ||r^C|| <= relTol
 * |lambda| (relTol = 0.1 in the paper's experiments: a 10% relative error of
 * the smallest value); the smallest solve uses the largest value as ||A||.
 * Rayleigh-Ritz values bound the spectrum from inside, so *sigma_max <=
 * sigma_1, *sigma_min >= sigma_n and *kappa = *sigma_max / *sigma_min never
 * exceeds the true condition number.  stats: NULL or an array of two (largest,
 * smallest).  The handle's precision and preconditioner apply; both solves
 * use GD+k (see relTol) and block size 1.  Returns the
 * first non-zero status of the two solves (SVDS_ERR_MAXIT: budget exhausted). */
int svds_condest(svds_handle *h, double relTol, double *sigma_max, double *sigma_min, double *kappa,
                 svds_stats *stats);

/* Release the handle and its device memory (NULL is accepted). */
void svds_destroy(svds_handle *h);

/* Static message for an error code. */
const char *svds_strerror(int code);
/* Message of the last SVDS_ERR_CUDA or SVDS_ERR_NUMERIC in this thread (empty if none). */
const char *svds_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PHSVDS_H */
