/* PHSVDS on GB300: learned sparse-approximate-inverse preconditioner (C-ABI).
 *
 * The paper has no learned component: its preconditioners are user functions
 * (Sec. 3.4, applyPreconditioner) and block Jacobi / AMG in the experiments.
 * This interface adds a small graph network over the sparsity graph of
 * C = A^T A that emits the values of a preconditioner M on that pattern:
 *
 *   graph   : nodes = columns of A, edges = nonzeros of C (symmetric);
 *   inputs  : node features [log c_ii - mean log c, deg_i / max deg],
 *             edge weights e_ij = c_ij / sqrt(c_ii c_jj);
 *   layers  : 4 x (z = h W1 + (E h) W2 + b, h = relu(z)), width 32;
 *   heads   : u = h ws, d = softplus(h wd + bd), delta = d / c_ii,
 *             s_ij = tanh(u_i + u_j + we e_ij + bs);
 *   M       : m_ii = delta_i, m_ij = 0.9 s_ij min(delta_i, delta_j) |e_ij| / max(E_i, E_j)
 *             with E_i = sum_j |e_ij|; symmetric and strictly diagonally
 *             dominant with a positive diagonal, hence SPD;
 *   loss    : a condition-number proxy of the preconditioned operator M C,
 *             which is self-adjoint in the C inner product with Rayleigh
 *             quotient rho(t) = (C t)^T M (C t) / t^T C t.  From start blocks
 *             T0 and X0: T = (M C)^ps T0 (power steps: top of the spectrum of
 *             M C), X = (I - omega M C)^ss X0 with omega = 1 / max rho(T)
 *             (smoothing steps: bottom of the spectrum), and
 *             L = log mean_p rho(t_p) - log mean_q rho(x_q).
 *             The samples follow the current M; the gradient holds them fixed
 *             (at eigenvectors of M C the Rayleigh quotient is stationary).
 *
 * Parameters are a flat float array of phsvds_gnn_num_params() entries in the
 * order W1_0 (2x32), W2_0 (2x32), b_0 (32), W1_l, W2_l (32x32), b_l (32) for
 * l = 1..3, ws (32), wd (32), we, bs, bd; matrices row-major.
 * All entry points return 0 or an SVDS_ERR_* code (phsvds.h).
 */
#ifndef PHSVDS_GNN_H
#define PHSVDS_GNN_H

#include <stdint.h>

#include "phsvds.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct phsvds_gnn phsvds_gnn;

int phsvds_gnn_num_params(void);

/* Seeded initial parameters (host array of phsvds_gnn_num_params() floats):
 * W1_l, W2_l ~ N(0, 2 / (fan_in + 32)), wd ~ N(0, 1/32), ws ~ N(0, 0.01/32),
 * bd = 0.5, bs = 1, every other entry 0 (so the initial M is close to a
 * scaled diagonal plus couplings that follow |e_ij|).  Normal deviates: splitmix64 (Steele, Lea, Flood 2014) feeding
 * the Box-Muller transform. */
int phsvds_gnn_init(uint64_t seed, float *params);

/* Build the graph of C = A^T A on the device (pattern by a k-way merge of the
 * rows of A, deterministic).  A may be on the host or the device. */
int phsvds_gnn_create(phsvds_gnn **g, const svds_csr *A, void *stream);
void phsvds_gnn_destroy(phsvds_gnn *g);
/* Nodes (columns of A) and nonzeros of the pattern of C. */
int phsvds_gnn_shape(const phsvds_gnn *g, int64_t *n, int64_t *nnz);
/* Pattern of C (host arrays of n + 1 and nnz entries). */
int phsvds_gnn_pattern(const phsvds_gnn *g, int32_t *rowptr, int32_t *colidx);

/* Forward pass: values of M on the pattern of C (host array of nnz floats). */
int phsvds_gnn_forward(phsvds_gnn *g, const float *params, float *mvals);

/* Loss and gradient from the start blocks T0 (n x P) and X0 (n x Q), host FP64
 * column-major, 1 <= P, Q <= 8, 0 <= power_steps <= 100, 0 <= smooth_steps <=
 * 1000.  grad: host doubles, phsvds_gnn_num_params(); SVDS_ERR_NUMERIC if a
 * Rayleigh quotient is not positive (a start block in the null space of C). */
int phsvds_gnn_loss_grad(phsvds_gnn *g, const float *params, const double *T0, int P, int power_steps,
                         const double *X0, int Q, int smooth_steps, double *loss, double *grad);

/* Training pairs on the graph: T = S^s Z, with S = I - (2/3) diag(C)^-1 C (s
 * steps of damped Jacobi smoothing of seeded N(0,1) columns Z, which leaves
 * mostly the low end of the spectrum of C), and R = C T.  Host FP64
 * column-major n x P arrays, 1 <= P <= 8, 0 <= s <= 1000. */
int phsvds_gnn_pairs(phsvds_gnn *g, int P, int smooth, uint64_t seed, double *R, double *T);
/* Y = C X for host FP64 column-major n x q blocks, 1 <= q <= 8. */
int phsvds_gnn_apply_c(phsvds_gnn *g, const double *X, int q, double *Y);

/* Parameter files: 8-byte tag "PHSGNN01", int32 count, count float32 values
 * (little-endian).  save writes phsvds_gnn_num_params() values; load reads
 * them into params (SVDS_ERR_ARG for a missing or malformed file). */
int phsvds_gnn_save(const char *path, const float *params);
int phsvds_gnn_load(const char *path, float *params);

/* One Adam step on the device (Kingma & Ba 2015): params, m, v are host
 * arrays of phsvds_gnn_num_params() floats updated in place; step >= 1. */
int phsvds_gnn_adam(phsvds_gnn *g, float *params, const double *grad, float *m, float *v, int step, float lr);

#ifdef __cplusplus
}
#endif
#endif /* PHSVDS_GNN_H */
