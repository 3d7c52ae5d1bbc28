// Precision traits and double-float arithmetic shared by the device kernels.
//
// Three storage/arithmetic modes run the same kernels:
//   F32  : float storage, float arithmetic (reduced-precision first phase of
//          stage 1; the Gram matrices of this mode still accumulate the exact
//          products in double-float, so they are FP64-class);
//   DF64 : double-float storage (an unevaluated sum hi + lo of two floats,
//          8 bytes per element like FP64) and double-float arithmetic.  This is
//          the FP64-class mode: GB300's FP64 pipe is ~70x slower than its FP32
//          pipe, so FP64-class accuracy is obtained from error-free FP32
//          transformations instead of DFMA;
//   F64  : native double storage and arithmetic (a check mode).
//
// Error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum
// (Dekker 1971) and TwoProd via a fused multiply-add.  The primitives use the
// _rn intrinsics so that the compiler cannot contract or reassociate them.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <set>
#include <utility>

namespace phsvds {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
// x + y (double-float); low parts added after the TwoSum of the high parts.
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  float t = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, t);
}
__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
// x * y (double-float); the lo*lo term is below the format's precision.
__device__ __forceinline__ df df_mul(df x, df y) {
  df p = two_prod(x.hi, y.hi);
  float t = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
  return fast_two_sum(p.hi, t);
}
// acc + x * y
__device__ __forceinline__ df df_fma(df acc, df x, df y) {
  df p = two_prod(x.hi, y.hi);
  float pl = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
  df s = two_sum(acc.hi, p.hi);
  float t = __fadd_rn(s.lo, __fadd_rn(acc.lo, pl));
  return fast_two_sum(s.hi, t);
}
// acc + x * y for float x, y: the product is exact as a double-float.
__device__ __forceinline__ df df_fma_ff(df acc, float x, float y) {
  df p = two_prod(x, y);
  df s = two_sum(acc.hi, p.hi);
  float t = __fadd_rn(s.lo, __fadd_rn(acc.lo, p.lo));
  return fast_two_sum(s.hi, t);
}
// acc + x * a for double-float x and float a.
__device__ __forceinline__ df df_fma_f(df acc, df x, float a) {
  df p = two_prod(x.hi, a);
  float pl = __fmaf_rn(x.lo, a, p.lo);
  df s = two_sum(acc.hi, p.hi);
  float t = __fadd_rn(s.lo, __fadd_rn(acc.lo, pl));
  return fast_two_sum(s.hi, t);
}

// ---------------------------------------------------------------------------
// Precision policies.  S = storage element, A = arithmetic value, G = Gram
// accumulator (FP64-class in every mode), C = coefficient element.
// ---------------------------------------------------------------------------
struct PF32 {
  using S = float;
  using A = float;
  using G = df;
  using C = float;
  static constexpr int id = 1;
  __device__ static A load(const S* p) { return *p; }
  __device__ static void store(S* p, A v) { *p = v; }
  __device__ static A zero() { return 0.f; }
  __device__ static A fma(A acc, A x, A y) { return fmaf(x, y, acc); }
  __device__ static A fmac(A acc, A x, C c) { return fmaf(x, c, acc); }
  __device__ static A add(A x, A y) { return x + y; }
  __device__ static A sub(A x, A y) { return x - y; }
  __device__ static A mulc(A x, C c) { return x * c; }
  __device__ static G gzero() { return {0.f, 0.f}; }
  __device__ static G gfma(G acc, A x, A y) { return df_fma_ff(acc, x, y); }
  __device__ static G gadd(G a, G b) { return df_add(a, b); }
  __device__ static double gval(G a) { return (double)a.hi + (double)a.lo; }
};

struct PDF64 {
  using S = df;
  using A = df;
  using G = df;
  using C = df;
  static constexpr int id = 2;
  __device__ static A load(const S* p) {
    float2 v = *reinterpret_cast<const float2*>(p);
    return {v.x, v.y};
  }
  __device__ static void store(S* p, A v) { *reinterpret_cast<float2*>(p) = make_float2(v.hi, v.lo); }
  __device__ static A zero() { return {0.f, 0.f}; }
  __device__ static A fma(A acc, A x, A y) { return df_fma(acc, x, y); }
  __device__ static A fmac(A acc, A x, C c) { return df_fma(acc, x, c); }
  __device__ static A add(A x, A y) { return df_add(x, y); }
  __device__ static A sub(A x, A y) { return df_add(x, df_neg(y)); }
  __device__ static A mulc(A x, C c) { return df_mul(x, c); }
  __device__ static G gzero() { return {0.f, 0.f}; }
  __device__ static G gfma(G acc, A x, A y) { return df_fma(acc, x, y); }
  __device__ static G gadd(G a, G b) { return df_add(a, b); }
  __device__ static double gval(G a) { return (double)a.hi + (double)a.lo; }
};

struct PF64 {
  using S = double;
  using A = double;
  using G = double;
  using C = double;
  static constexpr int id = 3;
  __device__ static A load(const S* p) { return *p; }
  __device__ static void store(S* p, A v) { *p = v; }
  __device__ static A zero() { return 0.0; }
  __device__ static A fma(A acc, A x, A y) { return ::fma(x, y, acc); }
  __device__ static A fmac(A acc, A x, C c) { return ::fma(x, c, acc); }
  __device__ static A add(A x, A y) { return x + y; }
  __device__ static A sub(A x, A y) { return x - y; }
  __device__ static A mulc(A x, C c) { return x * c; }
  __device__ static G gzero() { return 0.0; }
  __device__ static G gfma(G acc, A x, A y) { return ::fma(x, y, acc); }
  __device__ static G gadd(G a, G b) { return a + b; }
  __device__ static double gval(G a) { return a; }
};

// Allow `kernel` up to `bytes` of dynamic shared memory on the current device.
// The attribute is per device and per kernel (every template instance is its
// own kernel), so it is set once per (device, kernel); thread safe.
inline cudaError_t smem_optin(const void* kernel, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({dev, kernel})) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.insert({dev, kernel});
  return e;
}

}  // namespace phsvds
