// Solver state shared by the C-ABI and the engine.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/phsvds.h"
#include "kernels.h"

namespace phsvds {

// Device copy of A and A^T in every value format (see kernels.h, CsrDev).
struct DevMatrix {
  long long m = 0, n = 0, nnz = 0;  // after an optional transpose so that m >= n
  bool transposed = false;          // true when the user matrix was wide (m < n)
  double scale = 1.0;               // device values = scale * user values (power of two)
  int* rowptr = nullptr;
  int* colidx = nullptr;
  float* v32 = nullptr;
  float* v32lo = nullptr;
  double* v64 = nullptr;
  int* rowptrT = nullptr;
  int* colidxT = nullptr;
  float* v32T = nullptr;
  float* v32loT = nullptr;
  double* v64T = nullptr;
  double* colsq = nullptr;  // diag(A^T A), n
  double* rowsq = nullptr;  // diag(A A^T), m
  bool exact32 = true;      // every scaled value is a float: DF64 SpMM skips the lo part
  // explicit C = A^T A (n x n) of the scaled values, built on demand when one
  // SpMM with it moves fewer bytes than the two passes A then A^T
  long long nnzC = -1;      // -1 not decided yet, 0 not used
  int* rowptrC = nullptr;
  int* colidxC = nullptr;
  float* v32C = nullptr;
  float* v32loC = nullptr;
  double* v64C = nullptr;
  bool exactC = true;
  // bfloat16 copies of the values (built on demand for SVDS_BF16)
  uint16_t* v16 = nullptr;
  uint16_t* v16T = nullptr;
  uint16_t* v16C = nullptr;
  bool exact16 = true;  // every value is a bfloat16 number
  // caller-supplied operators (svds_create_op): no CSR; C and B are applied
  // by the caller's function on row-major FP64 blocks
  svds_apply_fn user = nullptr;
  void* user_ctx = nullptr;
  CsrDev csrC() const {
    CsrDev c;
    c.rows = n;
    c.cols = n;
    c.nnz = nnzC;
    c.rowptr = rowptrC;
    c.colidx = colidxC;
    c.v32 = v32C;
    c.v32lo = exactC ? nullptr : v32loC;
    c.v64 = v64C;
    return c;
  }
  CsrDev csr(bool t) const {
    CsrDev c;
    c.rows = t ? n : m;
    c.cols = t ? m : n;
    c.nnz = nnz;
    c.rowptr = t ? rowptrT : rowptr;
    c.colidx = t ? colidxT : colidx;
    c.v32 = t ? v32T : v32;
    c.v32lo = exact32 ? nullptr : (t ? v32loT : v32lo);
    c.v64 = t ? v64T : v64;
    return c;
  }
};

// Simple device arena: one cudaMalloc, bump allocation, reused across solves.
struct Arena {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  void* take(size_t bytes) {
    size_t off = (used + 255) & ~size_t(255);
    if (off + bytes > cap) return nullptr;
    used = off + bytes;
    return base + off;
  }
};

struct svds_handle_impl;

}  // namespace phsvds

struct svds_handle {
  phsvds::DevMatrix A;
  svds_opts opts;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  // allocations owned by the handle
  std::vector<void*> allocs;
  phsvds::Arena arena;  // per-solve workspace
  void* hpin = nullptr;  // pinned host staging
  size_t hpin_bytes = 0;
  unsigned long long launches = 0;
  std::vector<double> initV;  // copy of the caller's initial guesses (n x initSize)
  std::vector<float> gnn_params;  // learned preconditioner parameters (SVDS_PRECOND_LEARNED)
};

namespace phsvds {
int solve(svds_handle* h, int k, int target, double tol, double* sigma, double* U, double* V, double* rnorm,
          int* numConverged, svds_stats* stats);
void set_last_error(const std::string& s);
int ortho_block(int prec, long long L, const void* V, long long ldv, int g, void* T, long long ldt, int nb,
                int* status, cudaStream_t st, bool repair = false, unsigned long long seed = 0,
                int* replaced = nullptr);
}  // namespace phsvds
