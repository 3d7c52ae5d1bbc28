// Small dense FP64 linear algebra on the host (the projected problems of size
// g <= a few dozen, which the paper keeps replicated and calls negligible,
// Sec. 3.3).  All matrices are column-major with leading dimension n unless
// stated otherwise.
#pragma once
#include <vector>

namespace phsvds {
namespace hla {

// Symmetric eigendecomposition A = Z diag(w) Z^T, w ascending.  Householder
// tridiagonalisation followed by implicit QR steps with Wilkinson shifts
// (Golub & Van Loan, Matrix Computations, Algorithms 8.3.1 and 8.3.3).
// Returns false if the QR iteration does not converge.
bool sym_eig(int n, const double* A, double* w, double* Z);

// Singular value decomposition of a square n x n matrix R by one-sided Jacobi
// rotations (Hestenes 1958): s ascending, Yr the matching right singular vectors.
bool svd_right(int n, const double* R, double* s, double* Yr);

// Upper Cholesky factor G = R^T R; false if G is not numerically positive definite.
bool chol_upper(int n, const double* G, double* R);
// Inverse of an upper triangular matrix.
void tri_inv_upper(int n, const double* R, double* Rinv);

// Orthonormalise the c columns of the n x c matrix Y in place by modified
// Gram-Schmidt applied twice; columns whose norm falls below tol (relative)
// are dropped.  Returns the number of columns kept (packed to the front).
int orth_cols(int n, int c, double* Y, double tol);

// C (m x n) = A^T (k x m)^T * B (k x n): C = A^T B, all column-major.
void gemm_tn(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc);
// C = A B.
void gemm_nn(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc);

}  // namespace hla
}  // namespace phsvds
