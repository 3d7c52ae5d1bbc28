// Host-side launch wrappers of the device kernels (internal C++ interface).
//
// Layout conventions: a "block" of vectors with L rows and c columns is stored
// row-major with leading dimension ld (element (r, j) at ptr[r * ld + j]); all
// long vectors of the solver use this layout, so the b entries of one row that
// a CSR nonzero gathers are contiguous.  Storage element type per mode:
// F32 -> float, DF64 -> float2 (hi, lo), F64 -> double.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace phsvds {

enum Prec { kF32 = 1, kDF64 = 2, kF64 = 3 };

inline size_t elem_bytes(int prec) { return prec == kF32 ? 4 : 8; }

// Column segment of a row-major block: columns [0, nc) of ptr with stride ld.
struct SegV {
  const void* p;
  long long ld;
  int nc;
};

// CSR matrix values in the formats of one mode.
struct CsrDev {
  long long rows = 0, cols = 0, nnz = 0;
  const int* rowptr = nullptr;
  const int* colidx = nullptr;
  const float* v32 = nullptr;     // F32 values (also the hi part of DF64)
  const float* v32lo = nullptr;   // DF64 lo part, nullptr when every value is a float
  const double* v64 = nullptr;    // F64 values
  const uint16_t* v16 = nullptr;  // bfloat16 values: used instead of v32 by the F32 mode when set
};

// Y (rows x b, ldy) = A X (cols x b, ldx).
cudaError_t launch_spmm(int prec, const CsrDev& A, const void* X, long long ldx, void* Y, long long ldy,
                        int b, cudaStream_t st);

// Partial Gram sums: for rows [r0, r1), G = [P0 P1 P2]^T Q (p = sum of nc, q <= 8)
// into `partial` (nblocks x p x q accumulators, 8 bytes each); returns the
// number of blocks used via *nblocks.  `max_blocks` bounds the grid.
cudaError_t launch_gram(int prec, long long r0, long long r1, const SegV* P, int nseg, SegV Q,
                        void* partial, int max_blocks, int* nblocks, cudaStream_t st);
// The TMA-fed Gram of gram_tma.cu (F32 and DF64, p <= 64, q <= 8, 16-byte row
// strides): same contract as launch_gram; cudaErrorNotSupported when its
// preconditions do not hold (the caller then uses the row kernels).
cudaError_t launch_gram_tma(int prec, long long r0, long long r1, const SegV* P, int nseg, SegV Q, void* partial,
                            int max_blocks, int* nblocks, cudaStream_t st);
// TMA-fed basis update for F32/DF64, p <= 64, q <= 32 (R^-1: q <= 8), every
// segment, In, Out and Out2 16-byte aligned with 16-byte-multiple strides:
// same contract as launch_combine; cudaErrorNotSupported when its
// preconditions do not hold (the caller then uses the row kernels).
cudaError_t launch_combine_tma(int prec, long long L, const SegV* P, int nseg, const void* coef, const void* In,
                               long long ldin, int alpha_one, void* Out, long long ldout, int q, const void* Rinv,
                               void* Out2, long long ldout2, cudaStream_t st);
// TMA-fed Ritz vectors and residuals for F32/DF64, g <= 64, nb <= 8, V and W
// 16-byte aligned with 16-byte-multiple strides: same contract as
// launch_ritz_residual; cudaErrorNotSupported when its preconditions do not
// hold (the caller then uses the row kernels).
cudaError_t launch_ritz_tma(int prec, long long L, SegV V, SegV W, int g, const void* Y, const void* theta, void* X,
                            void* R, long long ldb, int nb, const void* dscale, void* T, void* partial,
                            int max_blocks, int* nblocks, cudaStream_t st);
// Sum the partials in fixed order into G (p x q, row-major doubles, device).
cudaError_t launch_gram_reduce(int prec, const void* partial, int nblocks, int pq, double* G, cudaStream_t st);
// Bytes of partial storage that launch_gram may use.
size_t gram_partial_bytes(int max_blocks, int p, int q);
int gram_default_blocks();

// Out[:, 0:q] = alpha * In[:, 0:q] + [P0 P1 P2] * coef  (coef p x q, row-major,
// device, in the mode's coefficient format), then, if Rinv != nullptr,
// Out[r, :] <- Out[r, :] * Rinv (q x q upper triangular, row-major).  Out may
// alias P0 (in-place restart: every CTA stages its rows before writing).  If
// Out2 != nullptr the result is also written there.
cudaError_t launch_combine(int prec, long long L, const SegV* P, int nseg, const void* coef,
                           const void* In, long long ldin, int alpha_one, void* Out, long long ldout, int q,
                           const void* Rinv, void* Out2, long long ldout2, cudaStream_t st);

// Fused Ritz vectors, residuals and residual norms:
//   X = V Y, R = W Y - X diag(theta), norm_partial <- sum_r R^2 per column,
// optionally T = diag(dscale) R (preconditioner) when T != nullptr.
cudaError_t launch_ritz_residual(int prec, long long L, SegV V, SegV W, int g, const void* Y,
                                 const void* theta, void* X, void* R, long long ldb, int nb,
                                 const void* dscale, void* T, void* norm_partial, int max_blocks,
                                 int* nblocks, cudaStream_t st);

// Stage-2 residual of Eq. res from x = [x_v; x_u] and Bx = [A^T x_u; A x_v]:
// per column j, sum over rows of (a_j Bx - c_j x)^2 with (a, c) = (av, cv) for
// rows < n and (au, cu) for rows >= n.  Partials as launch_gram with q = nb.
cudaError_t launch_split_resnorm(int prec, long long L, long long n, const void* X, const void* BX,
                                 long long ldb, int nb, const void* coefs /*4*nb coef*/, void* partial,
                                 int max_blocks, int* nblocks, cudaStream_t st);

// Elementwise T[r, j] = d[r] * R[r, j] (d in storage format).
cudaError_t launch_scale_rows(int prec, long long L, const void* d, const void* R, long long ldr, void* T,
                              long long ldt, int nb, cudaStream_t st);
// Copy columns: Dst[r, 0:nb] = Src[r, 0:nb].
cudaError_t launch_copy_cols(int prec, long long L, const void* Src, long long lds, void* Dst, long long ldd,
                             int nb, cudaStream_t st);
// Seeded N(0,1) fill of a block (splitmix64 counter hash + Box-Muller).
cudaError_t launch_fill_normal(int prec, long long L, void* Dst, long long ldd, int nb, unsigned long long seed,
                               cudaStream_t st);

// Conversions between FP64 column-major (device) and mode storage row-major.
// Row-major blocks in the mode's storage <-> row-major FP64 blocks.
cudaError_t launch_rows_to_f64(int prec, long long L, int nc, const void* src, long long lds, double* dst,
                               long long ldd, cudaStream_t st);
cudaError_t launch_rows_from_f64(int prec, long long L, int nc, const double* src, long long lds, void* dst,
                                 long long ldd, cudaStream_t st);
cudaError_t launch_from_f64_colmajor(int prec, long long L, int nc, const double* src, long long lds, void* dst,
                                     long long ldd, double scale, cudaStream_t st);
cudaError_t launch_to_f64_colmajor(int prec, long long L, int nc, const void* src, long long lds, double* dst,
                                   long long ldd, double scale, cudaStream_t st);
// Convert a coefficient array of doubles to the mode's coefficient format (host side).
size_t coef_bytes(int prec);
void host_coef_convert(int prec, const double* src, size_t count, void* dst);

// ---- setup (CSR) ----
cudaError_t launch_absmax(long long nnz, const double* vals, unsigned long long* out_bits, cudaStream_t st);
// Values: v32 = round(scale * v), v32lo = round(scale * v - v32), v64 = scale * v; flags[0] |= 1 if any lo != 0.
cudaError_t launch_csr_values(long long nnz, const double* vals, double scale, float* v32, float* v32lo,
                              double* v64, int* flags, cudaStream_t st);
// Deterministic transpose: (rowptr, colidx, vals) of an rows x cols CSR to its
// cols x rows CSR with increasing column (= original row) indices per row.
cudaError_t launch_csr_transpose(long long rows, long long cols, long long nnz, const int* rowptr,
                                 const int* colidx, const double* vals, int* rowptrT, int* colidxT,
                                 double* valsT, int* work /* cols + 1 + scan scratch */, cudaStream_t st);
size_t transpose_work_ints(long long cols);
// out[0] = 0, out[i + 1] = in[0] + ... + in[i] (int32), for n counts; work: scan_work_ints(n) ints.
cudaError_t launch_exclusive_scan(long long n, const int* in, int* out, int* work, cudaStream_t st);
size_t scan_work_ints(long long n);
// C = A^T A (n x n) from A (rp, ci, va; sorted rows) and A^T (rpT, ciT, vT; n
// rows): count pass cnt[j] = entries of row j of C (err[0] |= 1 when a row of
// A^T has more than normal_merge_max() entries; its count is 0), then, after
// an exclusive scan into cptr, the fill pass (sorted columns, values
// scale * sum_i a_ij a_ik in FP64).
cudaError_t launch_normal_count(long long n, const int* rpT, const int* ciT, const int* rp, const int* ci, int* cnt,
                                int* err, cudaStream_t st);
cudaError_t launch_normal_fill(long long n, const int* rpT, const int* ciT, const double* vT, const int* rp,
                               const int* ci, const double* va, double scale, const int* cptr, int* cidx,
                               double* cval, cudaStream_t st);
int normal_merge_max();
// FP32 -> bfloat16 (round to nearest even) of n finite values; flags[0] |= 1
// when some value is not exactly representable.
cudaError_t launch_to_bf16(long long n, const float* x, uint16_t* y, int* flags, cudaStream_t st);
// Sign convention of the returned vectors: column j of the column-major block
// X (rows x k, ld) is negated when its largest-magnitude entry in rows
// [r0, r0 + len) (lowest index on ties) is negative.
cudaError_t launch_col_sign(long long rows, long long ld, int k, long long r0, long long len, double* X, double* work,
                            cudaStream_t st);
// doubles of `work` that launch_col_sign needs
size_t col_sign_work_doubles(int k, long long len);
// Out (len x k, column-major, contiguous) = rows [r0, r0 + len) of the columns
// perm[0..k) of the column-major X (ld ldx); perm is a device int array.
cudaError_t launch_gather_cols(long long len, int k, const double* X, long long ldx, long long r0, const int* perm,
                               double* Out, cudaStream_t st);
// out[i] = sum_k vals[k]^2 over row i (FP64).
cudaError_t launch_row_sumsq(long long rows, const int* rowptr, const double* vals, double* out, cudaStream_t st);
// Jacobi scale in storage format: d[r] = 1 / s[r] (1 where s[r] == 0), optionally sqrt'ed first.
cudaError_t launch_make_dscale(int prec, long long L, const double* s, int use_sqrt, void* d, cudaStream_t st);
// CSR validation: sorted, in range, finite values; flags bit 1 = bad index/order, bit 2 = non-finite.
cudaError_t launch_csr_validate(long long rows, long long cols, const int* rowptr, const int* colidx,
                                const double* vals, int* flags, cudaStream_t st);

// Check of a square sparse preconditioner (FP32 values v32, or FP64 v64 when
// v32 is null): flags[0] |= 1 for a non-finite value, |= 2 for a row whose
// diagonal entry is missing or not positive.
cudaError_t launch_precond_check(long long n, const int* rowptr, const int* colidx, const float* v32,
                                 const double* v64, int* flags, cudaStream_t st);

// Small dense steps of the device-side CGS2 + CholQR2 (see kernels.cu).
cudaError_t launch_ortho_small(int stage, int prec, int g, int nb, const double* G, double* work, void* coef,
                               void* rinv, int* status, double drop2, cudaStream_t st);

void kernels_init();

}  // namespace phsvds
