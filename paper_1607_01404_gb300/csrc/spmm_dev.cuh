// Device helpers of the CSR SpMM kernels (row-major blocks of NB columns),
// shared by the plain SpMM and the fused SpMM + dot-product kernels.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace phsvds {

// VMODE: 0 float values (F32), 4 bfloat16 values (F32 vectors), 1 float values
// into double-float (DF64, exact
// values), 2 double-float values (DF64), 3 double values (F64).  VEC: the NB
// entries of a row are 16-byte multiples and every row starts on a 16-byte
// boundary, so gathers and stores use 16-byte vector accesses.
template <class P, int NB, bool VEC>
__device__ __forceinline__ void load_xrow(const typename P::S* __restrict__ xr, typename P::A (&v)[NB]) {
  using S = typename P::S;
  if constexpr (VEC) {
    constexpr int W = (int)(NB * sizeof(S) / 16);
    float buf[NB * sizeof(S) / 4];
    const float4* q4 = reinterpret_cast<const float4*>(xr);
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const float4 t = __ldg(q4 + i);
      buf[4 * i] = t.x;
      buf[4 * i + 1] = t.y;
      buf[4 * i + 2] = t.z;
      buf[4 * i + 3] = t.w;
    }
#pragma unroll
    for (int c = 0; c < NB; ++c) v[c] = P::load(reinterpret_cast<const S*>(buf) + c);
  } else {
#pragma unroll
    for (int c = 0; c < NB; ++c) v[c] = P::load(xr + c);
  }
}

template <class P, int NB, int VMODE, bool VEC>
__device__ __forceinline__ void spmm_accum(const int k, const float* __restrict__ v32, const float* __restrict__ v32lo,
                                           const double* __restrict__ v64, const typename P::A (&xv)[NB],
                                           typename P::A (&acc)[NB]) {
  if constexpr (VMODE == 0) {
    const float a = __ldg(v32 + k);
#pragma unroll
    for (int c = 0; c < NB; ++c) acc[c] = fmaf(xv[c], a, acc[c]);
  } else if constexpr (VMODE == 4) {
    // bfloat16 values (the upper 16 bits of an FP32 number; the pointer of the
    // float values carries the 16-bit array in this mode)
    const unsigned short bits = __ldg(reinterpret_cast<const unsigned short*>(v32) + k);
    const float a = __uint_as_float((unsigned)bits << 16);
#pragma unroll
    for (int c = 0; c < NB; ++c) acc[c] = fmaf(xv[c], a, acc[c]);
  } else if constexpr (VMODE == 1) {
    const float a = __ldg(v32 + k);
#pragma unroll
    for (int c = 0; c < NB; ++c) acc[c] = df_fma_f(acc[c], xv[c], a);
  } else if constexpr (VMODE == 2) {
    const df a = {__ldg(v32 + k), __ldg(v32lo + k)};
#pragma unroll
    for (int c = 0; c < NB; ++c) acc[c] = df_fma(acc[c], xv[c], a);
  } else {
    const double a = __ldg(v64 + k);
#pragma unroll
    for (int c = 0; c < NB; ++c) acc[c] = ::fma(xv[c], a, acc[c]);
  }
}

// VEC: 16-byte stores when vst also holds (Y row starts on 16-byte
// boundaries); element stores otherwise.
template <class P, int NB, bool VEC>
__device__ __forceinline__ void store_yrow(typename P::S* yr, const typename P::A (&acc)[NB], bool vst = true) {
  using S = typename P::S;
  if (VEC && vst) {
    constexpr int W = (int)(NB * sizeof(S) / 16);
    float buf[NB * sizeof(S) / 4];
#pragma unroll
    for (int c = 0; c < NB; ++c) P::store(reinterpret_cast<S*>(buf) + c, acc[c]);
    float4* q4 = reinterpret_cast<float4*>(yr);
#pragma unroll
    for (int t = 0; t < W; ++t) q4[t] = make_float4(buf[4 * t], buf[4 * t + 1], buf[4 * t + 2], buf[4 * t + 3]);
  } else {
#pragma unroll
    for (int c = 0; c < NB; ++c) P::store(yr + c, acc[c]);
  }
}

// Gathers in flight per thread: 4 rows of X for FP32 blocks of up to 4
// columns, 2 otherwise (register budget of the wider accumulators).
template <class P, int NB>
__host__ __device__ constexpr int spmm_unroll() {
  return (P::id == kF32 && NB <= 4) ? 4 : 2;
}

// acc += sum_{k0 <= k < k1} a_k X[colidx_k, :], in k order, with U index loads
// and U row gathers issued before their products (memory-level parallelism).
template <class P, int NB, int VMODE, bool VEC, int U>
__device__ __forceinline__ void row_product(int k0, int k1, const int* __restrict__ colidx,
                                            const float* __restrict__ v32, const float* __restrict__ v32lo,
                                            const double* __restrict__ v64, const typename P::S* __restrict__ X,
                                            long long ldx, typename P::A (&acc)[NB]) {
  using A = typename P::A;
  for (int k = k0; k < k1; k += U) {
    int jj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) jj[u] = k + u < k1 ? __ldg(colidx + k + u) : -1;
    A xv[U][NB];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (jj[u] >= 0) load_xrow<P, NB, VEC>(X + (long long)jj[u] * ldx, xv[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (jj[u] >= 0) spmm_accum<P, NB, VMODE, VEC>(k + u, v32, v32lo, v64, xv[u], acc);
  }
}

}  // namespace phsvds
