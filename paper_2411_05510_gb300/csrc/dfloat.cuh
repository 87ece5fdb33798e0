// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi) / 2, about 48 significant bits (relative rounding ~2^-46 per
// operation after error accumulation).  The building blocks are the error-free
// transformations of Knuth (two-sum), Dekker (fast two-sum) and the fused product error
// (two-product with fma); addition, multiplication, division and the square root follow
// the double-double algorithms of Hida, Li and Bailey (2001, "Algorithms for quad-double
// precision floating point arithmetic"), written here for FP32 pairs.  They run on the
// FP32 pipes, which issue a warp instruction per clock per SM partition, where this
// part's FP64 pipes take many clocks per warp instruction.
#pragma once

#include <cuda_runtime.h>

namespace ssi {
namespace dfl {

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return make_float2(s, e);
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
  const float s = a + b;
  return make_float2(s, b - (s - a));
}

// p + e = a * b exactly (fused multiply-add)
__device__ __forceinline__ float2 two_prod(float a, float b) {
  const float p = a * b;
  return make_float2(p, fmaf(a, b, -p));
}

__device__ __forceinline__ float2 from_double(double d) {
  const float hi = (float)d;
  return make_float2(hi, (float)(d - (double)hi));
}

__device__ __forceinline__ double to_double(float2 a) { return (double)a.x + (double)a.y; }

__device__ __forceinline__ float2 dneg(float2 a) { return make_float2(-a.x, -a.y); }

// a + b with both error terms carried (the accurate variant: cancellation-safe)
__device__ __forceinline__ float2 dadd(float2 a, float2 b) {
  float2 s = two_sum(a.x, b.x);
  const float2 t = two_sum(a.y, b.y);
  s.y += t.x;
  s = fast_two_sum(s.x, s.y);
  s.y += t.y;
  return fast_two_sum(s.x, s.y);
}

__device__ __forceinline__ float2 dsub(float2 a, float2 b) { return dadd(a, dneg(b)); }

__device__ __forceinline__ float2 dmul(float2 a, float2 b) {
  const float2 p = two_prod(a.x, b.x);
  float e = fmaf(a.x, b.y, p.y);
  e = fmaf(a.y, b.x, e);
  return fast_two_sum(p.x, e);
}

__device__ __forceinline__ float2 dmulf(float2 a, float b) {
  const float2 p = two_prod(a.x, b);
  return fast_two_sum(p.x, fmaf(a.y, b, p.y));
}

// a * 2^e exactly (scaling by a power of two)
__device__ __forceinline__ float2 ldexp2(float2 a, int e) {
  return make_float2(ldexpf(a.x, e), ldexpf(a.y, e));
}

// a / b: three quotient digits, each from the remainder of the previous (long division)
__device__ __forceinline__ float2 ddiv(float2 a, float2 b) {
  const float q1 = a.x / b.x;
  float2 r = dsub(a, dmulf(b, q1));
  const float q2 = r.x / b.x;
  r = dsub(r, dmulf(b, q2));
  const float q3 = r.x / b.x;
  const float2 q = fast_two_sum(q1, q2);
  return dadd(q, make_float2(q3, 0.f));
}

// sqrt(a), a >= 0: one Newton correction of the FP32 root, x + (a - x^2) / (2 x)
__device__ __forceinline__ float2 dsqrt(float2 a) {
  if (!(a.x > 0.f)) return make_float2(0.f, 0.f);
  const float x = sqrtf(a.x);
  const float2 r = dsub(a, two_prod(x, x));
  return fast_two_sum(x, r.x / (2.f * x));
}

__device__ __forceinline__ float absf(float2 a) { return fabsf(a.x); }

}  // namespace dfl
}  // namespace ssi
