// Block-Jacobi preconditioner on A^T A as a CSR matrix with dense diagonal
// blocks (see bjacobi.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace phsvds {

constexpr int kBjMaxBlock = 64;  // blocks up to 64 columns (a shared-memory FP64 inverse)

// Nonzeros of the block-diagonal CSR for n columns in blocks of bs.
long long bj_nnz(long long n, int bs);
size_t bj_smem_bytes(int bs);

// rowptrT / colidxT / valsT: CSR of A^T (n rows, sorted columns, FP64 values),
// device.  Outputs (device, caller-allocated): rowptr (n + 1), colidx, v32
// and / or v64 (bj_nnz entries; either value array may be null, not both).
cudaError_t launch_bj_build(long long n, int bs, const int* rowptrT, const int* colidxT, const double* valsT,
                            int* rowptr, int* colidx, float* v32, double* v64, cudaStream_t st);

}  // namespace phsvds
