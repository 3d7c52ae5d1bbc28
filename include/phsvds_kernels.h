/* PHSVDS on GB300: kernel-level C-ABI (per-kernel parity tests, custom drivers).
 *
 * Every entry point works on caller-owned CUDA device memory, enqueues its
 * kernels on `stream` (a cudaStream_t, NULL = legacy default stream) and
 * returns 0, SVDS_ERR_ARG for an invalid argument (checked before any launch)
 * or SVDS_ERR_CUDA on a launch error.  Nothing is allocated: buffers that need
 * scratch take it from the caller (sizes from the *_bytes queries).
 *
 * Precision modes (prec):
 *   1 = F32  : float storage and arithmetic;
 *   2 = DF64 : double-float storage (pairs (hi, lo) of floats, 8 bytes per
 *              element, value hi + lo) and double-float arithmetic (FP64-class);
 *   3 = F64  : double storage and native FP64 arithmetic.
 * Blocks of vectors are row-major: element (r, j) of a block with leading
 * dimension ld is at base[r * ld + j] (in elements of the mode's storage type).
 * Small coefficient matrices are row-major in the mode's coefficient format
 * (float, float pair or double; see phsvds_coef_convert).
 */
#ifndef PHSVDS_KERNELS_H
#define PHSVDS_KERNELS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Y (rows x b, ldy) = A X (cols x b, ldx) for CSR A (the user matvec of the
 * paper's Sec. 3.4; A^T products use the CSR of A^T).  Values: F32 reads v32;
 * DF64 reads v32 (+ v32lo unless it is NULL, meaning every value is a float);
 * F64 reads v64. */
int phsvds_spmm(int prec, int64_t rows, int64_t cols, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                const float *v32, const float *v32lo, const double *v64, const void *X, int64_t ldx, void *Y,
                int64_t ldy, int b, void *stream);

/* Y = A X in the FP32 mode with bfloat16 values of A (v16: the upper 16 bits
 * of FP32 numbers; X, Y FP32 row-major as phsvds_spmm).  Not in the paper: the
 * reduced-precision operator of the mixed-precision stage 1. */
int phsvds_spmm_bf16(int64_t rows, int64_t cols, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                     const uint16_t *v16, const float *X, int64_t ldx, float *Y, int64_t ldy, int b, void *stream);
/* v16 = bfloat16(v32), round to nearest even, for nnz finite device values;
 * flags[0] (device int) |= 1 when some value is not exactly representable. */
int phsvds_to_bf16(int64_t nnz, const float *v32, uint16_t *v16, int *flags, void *stream);

/* The operator apply of a JDQMR inner step fused with its dot products: for a
 * square CSR K (n x n, value arrays as phsvds_spmm), W = K X (X: ld ldx) and,
 * per column j < nb, dots = [x_j^T w_j, q_j^T w_j, x_j^T q_j, q_j^T q_j] with
 * x = E1, q = E2 (row-major n x nb blocks, ld nb); dots: device doubles laid
 * out [4][nb].  nb in {1, 2, 4, 8}; W, E1, E2 and X 16-byte aligned with 16-byte
 * rows when nb * element >= 16 (SVDS_ERR_ARG otherwise).  scratch: device,
 * phsvds_spmm_dots_scratch_bytes(nb) bytes. */
int phsvds_spmm_dots(int prec, int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                     const float *v32, const float *v32lo, const double *v64, int nb, const void *X, int64_t ldx,
                     void *W, const void *E1, const void *E2, double *dots, void *scratch, size_t scratch_bytes,
                     void *stream);
size_t phsvds_spmm_dots_scratch_bytes(int nb);

/* Block-Jacobi preconditioner on C = A^T A (Sec. 4: block Jacobi on A^T A):
 * M = blockdiag((C_II + delta_I I)^-1) over consecutive blocks I of bs columns
 * (the last one ragged), C_II = A_I^T A_I, a zero diagonal entry (empty
 * column) replaced by 1, delta_I = 1e-10 max_r (C_II)_rr; inverted in FP64,
 * symmetrised.  Input: CSR of A^T (n rows = the columns of A, sorted column
 * indices, FP64 values), device.  Output (device, caller-allocated): CSR of M
 * with rowptr (n + 1 entries), colidx and the values in FP64 (v64) and / or
 * FP32 (v32), phsvds_block_jacobi_nnz(n, bs) entries each; either value
 * pointer may be NULL, not both.  1 <= bs <= 64, else SVDS_ERR_ARG. */
int64_t phsvds_block_jacobi_nnz(int64_t n, int bs);
int phsvds_block_jacobi(int64_t n, const int32_t *rowptrT, const int32_t *colidxT, const double *valsT, int bs,
                        int32_t *rowptr, int32_t *colidx, double *v64, float *v32, void *stream);

/* Orthonormalise the block T (L x nb, ld ldt, in place) against the orthonormal
 * basis V (L x g, ld ldv) by the solver's device-side CGS2 + CholQR2 (Sec. 3.2,
 * Sec. 4.4): T <- (I - V V^T)^2 T, then Cholesky-QR twice, the small Cholesky
 * and triangular steps on the device (FP64).  Blocks in the storage of mode
 * prec; 1 <= nb <= 8, 1 <= g, g + nb <= 256.  *status (host, may be NULL) is 0,
 * or nonzero when a Cholesky factor broke down (rank-deficient block; the
 * solver then replaces columns on the host path).  Allocates its own scratch. */
int phsvds_ortho(int prec, int64_t L, const void *V, int64_t ldv, int g, void *T, int64_t ldt, int nb, int *status,
                 void *stream);

/* phsvds_ortho followed, when the device steps report a breakdown (*status
 * nonzero), by the solver's repair (Sec. 3.2 orthogonalisation; the replacement
 * rule of the method's restatement): the block as given is orthonormalised
 * again by host-driven CGS2 + CholQR2 in which a column that keeps at most
 * 1e-10 of its norm after the projection on V, or whose Cholesky pivot within
 * the block keeps at most 1e-14 of its squared norm (a column that depends on
 * the block's earlier columns), is
 * replaced by a seeded N(0, 1) vector (seed) before the block is
 * orthonormalised again.  On return T is orthonormal and orthogonal to V;
 * *replaced (host, may be NULL) is 1 when columns were replaced.  Allocates
 * its own device and pinned host scratch. */
int phsvds_ortho_repair(int prec, int64_t L, const void *V, int64_t ldv, int g, void *T, int64_t ldt, int nb,
                        uint64_t seed, int *status, int *replaced, void *stream);

/* JDQMR inner solve (Sec. 3.4): for each of the nb columns j, block symmetric
 * QMR on the correction equation
 *     (I - x_j x_j^T)(K - eta_j I)(I - x_j x_j^T) t_j = b_j,   t_j orthogonal to x_j,
 * with the projected preconditioner built from dinv (Jacobi diagonal in the
 * mode's storage, or NULL), exactly as inside svds_solve.  K: CSR (n x n, the
 * value arrays of the mode as in phsvds_spmm); X, Bv, T: row-major n x nb
 * device blocks of mode prec (X orthonormal columns, Bv orthogonal to them);
 * eta: host doubles.  Stops a column when its QMR residual bound falls below
 * xi ||b_j|| or after maxit steps; *steps (host, may be NULL) receives the
 * number of steps taken.  nb <= 8.  Allocates and frees its own scratch. */
int phsvds_jd_solve(int prec, int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                    const float *v32, const float *v32lo, const double *v64, int nb, const void *X, const void *Bv,
                    const double *eta, const void *dinv, int maxit, double xi, void *T, int *steps, void *stream);

/* G (p x q row-major doubles, device) = P^T Q over rows [r0, r1) (the Table 3
 * inner products: Rayleigh-Ritz projection V^T W, Gram matrices of CGS and
 * CholQR).  Accumulation is FP64-class in every mode and the reduction order
 * is fixed (deterministic).  p <= 256; any q. */
int phsvds_gram(int prec, int64_t r0, int64_t r1, const void *P, int64_t ldp, int p, const void *Q, int64_t ldq,
                int q, double *G, void *scratch, size_t scratch_bytes, void *stream);
size_t phsvds_gram_scratch_bytes(int p, int q);

/* Out (L x q) = alpha In + P coef (p x q), then Out <- Out Rinv when Rinv is
 * not NULL (q x q upper triangular).  Out may equal P (in-place restart
 * V <- V Z with q <= p) or In. */
int phsvds_combine(int prec, int64_t L, const void *P, int64_t ldp, int p, const void *coef, const void *In,
                   int64_t ldin, int alpha_one, void *Out, int64_t ldout, int q, const void *Rinv, void *stream);

/* Allocation-free variant of phsvds_gram, for callers that cannot allocate
 * device memory (host callbacks, allocator hooks, plug-ins that must not touch
 * their host application's device heap).  The paper has no counterpart: it is
 * an interface convenience of this library.  Its scratch is a fixed device
 * array inside the library (2,490,368 bytes, held on every GPU that loads the
 * library until the process exits), so it serves p <= 64 and q <= 8 and returns
 * SVDS_ERR_ARG beyond that.  It allocates nothing.  Every call resolves the
 * array's device address in the current context (cudaGetSymbolAddress); the
 * first call in a context also loads the library's device code, so make it
 * before any stream capture.  All calls share the one array: calls whose
 * kernels overlap on the GPU (different streams, or different host threads)
 * race on it; serialise them.  Each call overwrites the part of the array it
 * uses, so the previous call's contents do not affect its result. */
int phsvds_gram_noalloc(int prec, int64_t r0, int64_t r1, const void *P, int64_t ldp, int p, const void *Q,
                        int64_t ldq, int q, double *G, void *stream);

/* Fused Ritz vectors and residuals (Sec. 3.3 residual kernel):
 * X = V Y, R = W Y - X diag(theta), norms2[j] = ||R_j||^2 (device doubles).
 * V, W: L x g with leading dimension ldv; X, R: L x nb with leading dimension ldb. */
int phsvds_ritz_residual(int prec, int64_t L, const void *V, const void *W, int64_t ldv, int g, const void *Y,
                         const void *theta, void *X, void *R, int64_t ldb, int nb, double *norms2, void *scratch,
                         size_t scratch_bytes, void *stream);
size_t phsvds_ritz_scratch_bytes(int nb);

/* Conversions between FP64 column-major (src/dst with leading dimension lds/ldd
 * counted in rows) and the mode's row-major storage. */
int phsvds_from_f64(int prec, int64_t L, int nc, const double *src, int64_t lds, void *dst, int64_t ldd, void *stream);
int phsvds_to_f64(int prec, int64_t L, int nc, const void *src, int64_t lds, double *dst, int64_t ldd, void *stream);

/* Deterministic CSR transpose (rows x cols -> cols x rows, indices increasing in
 * each row of the result).  work: phsvds_csr_transpose_work_bytes(cols) bytes. */
int phsvds_csr_transpose(int64_t rows, int64_t cols, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                         const double *vals, int32_t *rowptrT, int32_t *colidxT, double *valsT, void *work,
                         size_t work_bytes, void *stream);
size_t phsvds_csr_transpose_work_bytes(int64_t cols);

/* CSR value formats: v32 = fl32(v), v32lo = fl32(v - v32), v64 = v; *flags |= 1
 * if any v32lo != 0 (flags is a device int). */
int phsvds_csr_values(int64_t nnz, const double *vals, float *v32, float *v32lo, double *v64, int *flags, void *stream);

/* Host: convert doubles to the mode's coefficient format (count elements). */
int phsvds_coef_convert(int prec, const double *src, size_t count, void *dst);

/* Host small dense FP64 problems of the engine (column-major, n <= 512):
 * symmetric eigendecomposition (ascending) and right singular vectors of a
 * square matrix (ascending singular values). */
int phsvds_host_symeig(int n, const double *A, double *w, double *Z);
int phsvds_host_svd(int n, const double *R, double *s, double *Yr);

#ifdef __cplusplus
}
#endif
#endif /* PHSVDS_KERNELS_H */
