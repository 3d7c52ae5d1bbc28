// Block-Jacobi preconditioner on C = A^T A (the paper's generic preconditioner,
// Sec. 4: block Jacobi on A^T A with blocks of up to 600 columns).
//
// M = blockdiag((C_II + delta_I I)^-1) over consecutive column blocks I of
// size bs (the last one ragged).  C_II = A_I^T A_I is formed from sparse dot
// products of the rows of A^T (the columns of A); a zero diagonal entry (an
// empty column) is replaced by 1, and delta_I = 1e-10 max_r (C_II)_rr keeps
// rank-deficient blocks invertible.  The inverse is taken in FP64 by
// Gauss-Jordan elimination (no pivoting: the shifted block is SPD) in shared
// memory, symmetrised, and written as a CSR matrix with dense bs x bs blocks,
// so that the SpMM kernels apply it like any sparse preconditioner.
#include <cuda_runtime.h>

#include <cstdint>

#include "bjacobi.h"

namespace phsvds {

namespace {

constexpr int kBjThreads = 256;

__global__ void __launch_bounds__(kBjThreads) k_bj_build(long long n, int bs, const int* __restrict__ rpT,
                                                         const int* __restrict__ ciT, const double* __restrict__ vT,
                                                         int* __restrict__ rowptr, int* __restrict__ colidx,
                                                         float* __restrict__ v32, double* __restrict__ v64) {
  extern __shared__ double sm[];
  const long long g0 = (long long)blockIdx.x * bs;
  const int s = (int)((n - g0) < bs ? (n - g0) : bs);
  double* G = sm;           // s x s, row-major
  double* f = sm + s * s;   // column p of the current elimination step
  double* red = f + s;      // scalar scratch
  const int tid = threadIdx.x;
  // C_II by sparse dot products of rows of A^T (sorted column indices)
  for (int e = tid; e < s * s; e += blockDim.x) {
    const int r = e / s, c = e % s;
    if (c < r) continue;
    int a = rpT[g0 + r], ae = rpT[g0 + r + 1];
    int b = rpT[g0 + c], be = rpT[g0 + c + 1];
    double acc = 0.0;
    while (a < ae && b < be) {
      const int ja = ciT[a], jb = ciT[b];
      if (ja == jb) {
        acc = fma(vT[a], vT[b], acc);
        ++a;
        ++b;
      } else if (ja < jb) {
        ++a;
      } else {
        ++b;
      }
    }
    G[r * s + c] = acc;
    G[c * s + r] = acc;
  }
  __syncthreads();
  if (tid == 0) {
    double dmax = 0.0;
    for (int r = 0; r < s; ++r) dmax = fmax(dmax, G[r * s + r]);
    red[0] = 1e-10 * dmax;
  }
  __syncthreads();
  const double delta = red[0];
  for (int r = tid; r < s; r += blockDim.x) {
    if (G[r * s + r] == 0.0) G[r * s + r] = 1.0;
    G[r * s + r] += delta;
  }
  __syncthreads();
  // in-place Gauss-Jordan inversion
  for (int p = 0; p < s; ++p) {
    for (int i = tid; i < s; i += blockDim.x) f[i] = G[i * s + p];
    __syncthreads();
    const double piv = f[p];
    for (int j = tid; j < s; j += blockDim.x) G[p * s + j] = (j == p ? 1.0 : G[p * s + j]) / piv;
    __syncthreads();
    for (int e = tid; e < s * s; e += blockDim.x) {
      const int i = e / s, j = e % s;
      if (i == p) continue;
      G[e] = (j == p ? 0.0 : G[e]) - f[i] * G[p * s + j];
    }
    __syncthreads();
  }
  // symmetrised inverse as CSR rows g0 .. g0 + s - 1 (every earlier block is full)
  const long long base = g0 * bs;
  for (int e = tid; e < s * s; e += blockDim.x) {
    const int r = e / s, c = e % s;
    const double v = 0.5 * (G[r * s + c] + G[c * s + r]);
    const long long k = base + (long long)r * s + c;
    colidx[k] = (int)(g0 + c);
    if (v64) v64[k] = v;
    if (v32) v32[k] = (float)v;
  }
  for (int r = tid; r < s; r += blockDim.x) rowptr[g0 + r] = (int)(base + (long long)r * s);
  if (g0 + s == n && tid == 0) rowptr[n] = (int)(base + (long long)s * s);
}

}  // namespace

long long bj_nnz(long long n, int bs) {
  if (n < 1 || bs < 1) return 0;
  const long long full = n / bs, last = n - full * bs;
  return full * bs * bs + last * last;
}

size_t bj_smem_bytes(int bs) { return (size_t)bs * bs * 8 + (size_t)bs * 8 + 16; }

cudaError_t launch_bj_build(long long n, int bs, const int* rowptrT, const int* colidxT, const double* valsT,
                            int* rowptr, int* colidx, float* v32, double* v64, cudaStream_t st) {
  if (n < 1 || bs < 1 || bs > kBjMaxBlock || !rowptrT || !rowptr || !colidx || (!v32 && !v64))
    return cudaErrorInvalidValue;
  if (bj_nnz(n, bs) > 2147483647LL) return cudaErrorInvalidValue;
  const long long nblk = (n + bs - 1) / bs;
  if (nblk > 2147483647LL) return cudaErrorInvalidValue;
  const size_t smem = bj_smem_bytes(bs);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_bj_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_bj_build<<<(unsigned)nblk, kBjThreads, smem, st>>>(n, bs, rowptrT, colidxT, valsT, rowptr, colidx, v32, v64);
  return cudaGetLastError();
}

}  // namespace phsvds
