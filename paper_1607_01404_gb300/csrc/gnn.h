// Internal interface of the learned preconditioner for the solver engine.
#pragma once
#include <cuda_runtime.h>

#include "engine.h"
#include "kernels.h"

struct phsvds_gnn;

namespace phsvds {

// Graph of C = A^T A on stream st.  Nodes are the columns of the user's
// matrix when user_orientation is set, else the columns of the device matrix
// (the operator of stage 1).  Without `train` only the forward buffers exist.
int gnn_build(phsvds_gnn** out, const DevMatrix& D, bool user_orientation, bool train, cudaStream_t st);

// Evaluate M for the host parameters and describe it as a CSR operator: *f32
// with float values (F32 and DF64 modes), *f64 with double values when
// f64 != nullptr.  Stream-ordered; M stays valid until the graph is destroyed.
int gnn_precond(phsvds_gnn* g, const float* params, CsrDev* f32, CsrDev* f64);

// Kernels launched on the graph so far.
long long gnn_launches(const phsvds_gnn* g);

}  // namespace phsvds
