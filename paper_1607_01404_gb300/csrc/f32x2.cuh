// Packed FP32 pairs (sm_100 and later).
//
// One add.f32x2, sub.f32x2, mul.f32x2 or fma.f32x2 instruction applies the
// round-to-nearest operation to both halves of a 64-bit register pair, each
// half rounded exactly as the scalar instruction rounds it.  Kernels whose
// FP32 accumulations are bound by instruction issue pair two independent
// accumulators per instruction with these, without changing a single
// rounding.  Inline PTX fixes the operation (no contraction, no negation left
// to a later pass).
#pragma once
#include <cuda_runtime.h>

namespace phsvds {
namespace x2 {

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {  // a b + c
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {  // a + b
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {  // a - b
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {  // a b
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// Two Dot2 steps (Ogita, Rump and Oishi 2005) at once: hi + lo += x c for
// double-float operands x = xh + xl and c = ch + cl, in the scalar step's
// order: p = x_hi c_hi with its error pe = fma(x_hi, c_hi, -p), the cross
// terms pl = fma(x_hi, c_lo, fma(x_lo, c_hi, pe)), TwoSum(hi, p), then
// lo + (e + pl).  fma has no negated addend here, so the error terms come out
// negated from the negated operand (nch, ncl) = -(ch, cl):
// fma(a, -b, c) = -fma(a, b, -c) exactly in round-to-nearest, and
// lo + (e + pl) = lo + (e - (-pl)).  The results equal the scalar steps' (up
// to the sign of a zero low word).
__device__ __forceinline__ void dot2x2(float2& hi, float2& lo, float2 xh, float2 xl, float2 ch, float2 nch,
                                       float2 ncl) {
  const float2 p = mul2(xh, ch);
  const float2 npe = fma2(xh, nch, p);
  const float2 npl = fma2(xh, ncl, fma2(xl, nch, npe));
  const float2 s = add2(hi, p);
  const float2 bb = sub2(s, hi);
  const float2 e = add2(sub2(hi, sub2(s, bb)), sub2(p, bb));
  hi = s;
  lo = add2(lo, sub2(e, npl));
}

}  // namespace x2
}  // namespace phsvds
