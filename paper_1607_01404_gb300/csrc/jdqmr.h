// JDQMR inner solver (symmetric QMR on the projected correction equation),
// internal interface; see jdqmr.cu.
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"

namespace phsvds {

// Per-column state of the block sQMR recurrences (device memory).
struct QmrState {
  double rho, tau, tau0, theta, alpha, beta, gamma, xkx, c1, coefd, coefq;
  int active, upd, k, pad;
};

// Blocks are in the storage of mode prec (F32, DF64 or F64), row-major L x nb
// with leading dimension nb (nb <= 8).  x: Ritz vectors (orthonormal columns),
// b: right-hand sides (orthogonal to x), dinv: Jacobi diagonal K^-1 in the same
// storage, or nullptr; K: a sparse symmetric K^-1 (values in the mode's
// format) applied by SpMM instead of dinv, with u an L x nb work block, or
// nullptr.  partial: >= 2048 * 5 * nb * 8 bytes, dots: >= 5 * nb doubles.
cudaError_t qmr_init(int prec, long long L, int nb, const void* x, const void* b, const void* dinv, const CsrDev* K,
                     void* u, void* kx, void* q, void* r, void* d, void* sol, QmrState* S, void* partial,
                     double* dots, cudaStream_t st);
// One inner step after w = op(q) (the caller applies the operator): updates r,
// d, sol, q and the scalars; eta: per-column shifts (device doubles).  A column
// stops when tau sqrt(k + 1) <= xi tau0 or after maxk steps.
// ready: 0 = this step computes the dots of w = op(q) with x and q; 1 = they
// are in `dots` (qmr_op_dots); 2 = and the first scalar step is done too.
// ticks: >= 3 zeroed device counters that let the producing kernels reduce
// their partial sums and run the scalar steps in their tails (fewer
// launches), or nullptr for separate reduction and scalar launches.
cudaError_t qmr_step(int prec, long long L, int nb, const void* x, const void* w, int ready, unsigned* ticks,
                     const void* kx, const void* dinv, const CsrDev* K, void* u, const double* eta, double xi,
                     int maxk, void* q, void* r, void* d, void* sol, QmrState* S, void* partial, double* dots,
                     cudaStream_t st);
// w = K X for a single CSR operator (K: rows L, X: ld ldx) fused with the four
// dots x^T w, q^T w, x^T q, q^T q of a step, reduced into `dots`; with ticks
// the first scalar step of the step (eta, S) runs in the kernel's tail.
// *ready = 0 (nothing launched: nb or the alignment has no fused form), 1 or 2
// as for qmr_step.
cudaError_t qmr_op_dots(int prec, long long L, int nb, const CsrDev& K, const void* X, long long ldx, void* w,
                        const void* x, const void* q, void* partial, double* dots, unsigned* ticks,
                        const double* eta, QmrState* S, int* ready, cudaStream_t st);
int qmr_step_launches(int nb, bool sparse_k, int ready, bool ticks);
int qmr_init_launches(int nb, bool sparse_k);

// Complete inner solve with its own scratch (the kernel-level entry point):
// see phsvds_jd_solve in phsvds_kernels.h.  Returns 0 or an SVDS_ERR_* code.
int jd_solve(int prec, const CsrDev& K, int nb, const void* X, const void* Bv, const double* eta_host,
             const void* dinv, int maxit, double xi, void* T, int* steps, cudaStream_t st);

// dst[:, j] = scale[j] * src[:, j] with a mode conversion (scale: device doubles).
cudaError_t convert_cols(int src_prec, const void* src, long long lds, int dst_prec, void* dst, long long ldd,
                         long long L, int nc, const double* scale, cudaStream_t st);

}  // namespace phsvds
