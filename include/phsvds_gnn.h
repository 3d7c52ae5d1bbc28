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
 *   M       : m_ii = delta_i, m_ij = 0.9 s_ij min(delta_i, delta_j) / max(deg_i, deg_j),
 *             symmetric and strictly diagonally dominant with a positive
 *             diagonal, hence SPD;
 *   loss    : mean(1 - cos^2(M r_p, t_p)) + 0.5 mean(1 - cos^2(M y_q, x_q)).
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

/* Loss and gradient for training pairs (R, T) (n x P) and (Y, X) (n x Q), host
 * FP64 column-major (Q may be 0).  grad: host doubles, phsvds_gnn_num_params(). */
int phsvds_gnn_loss_grad(phsvds_gnn *g, const float *params, const double *R, const double *T, int P,
                         const double *Y, const double *X, int Q, double *loss, double *grad);

/* One Adam step on the device (Kingma & Ba 2015): params, m, v are host
 * arrays of phsvds_gnn_num_params() floats updated in place; step >= 1. */
int phsvds_gnn_adam(phsvds_gnn *g, float *params, const double *grad, float *m, float *v, int step, float lr);

#ifdef __cplusplus
}
#endif
#endif /* PHSVDS_GNN_H */
