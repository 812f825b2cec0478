// Pair-of-floats ("double-float") arithmetic for an FP64-accurate operator on
// the FP32 pipe.
//
// GB300 executes FP64 at about 1/64 of its FP32 rate, so the FP64-accurate
// variant of the cell kernel keeps every intermediate as an unevaluated sum
// hi + lo of two floats (|lo| <= ulp(hi)/2, about 48 significant bits) and
// builds additions and multiply-adds from the classical error-free
// transformations: Knuth's TwoSum, Dekker's FastTwoSum and the FMA-based
// TwoProduct (Dekker 1971; Ogita, Rump & Oishi 2005).  Inputs and outputs stay
// FP64; the split and the final recombination happen at the gather and the
// scatter.
#pragma once
#include <cuda_runtime.h>

namespace feks {

struct ff2 {
  float hi, lo;
};

// Native fused multiply-adds under the same name as the pair-of-floats one, so
// generic kernels call fma() for every arithmetic type.
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }

__host__ __device__ __forceinline__ ff2 ff_make(float h, float l) {
  ff2 r;
  r.hi = h;
  r.lo = l;
  return r;
}

// s + e == a + b exactly (Knuth)
__device__ __forceinline__ ff2 ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return ff_make(s, e);
}

// s + e == a + b exactly when |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ ff2 ff_fast_two_sum(float a, float b) {
  const float s = a + b;
  return ff_make(s, b - (s - a));
}

// p + e == a * b exactly (FMA)
__device__ __forceinline__ ff2 ff_two_prod(float a, float b) {
  const float p = a * b;
  return ff_make(p, fmaf(a, b, -p));
}

__device__ __forceinline__ ff2 operator+(ff2 a, ff2 b) {
  ff2 s = ff_two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return ff_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff2 operator-(ff2 a) { return ff_make(-a.hi, -a.lo); }

__device__ __forceinline__ ff2 operator-(ff2 a, ff2 b) { return a + (-b); }

__device__ __forceinline__ ff2 operator*(ff2 a, ff2 b) {
  ff2 p = ff_two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return ff_fast_two_sum(p.hi, p.lo);
}

// a * b + c
__device__ __forceinline__ ff2 fma(ff2 a, ff2 b, ff2 c) {
  const ff2 p = ff_two_prod(a.hi, b.hi);
  ff2 s = ff_two_sum(p.hi, c.hi);
  s.lo += p.lo + fmaf(a.hi, b.lo, a.lo * b.hi) + c.lo;
  return ff_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff2& operator+=(ff2& a, ff2 b) {
  a = a + b;
  return a;
}

__device__ __forceinline__ ff2& operator*=(ff2& a, ff2 b) {
  a = a * b;
  return a;
}

__device__ __forceinline__ ff2 ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return ff_make(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double ff_to_double(ff2 a) { return (double)a.hi + (double)a.lo; }

// Split of an FP64 value into hi + lo floats with integer operations only (no
// FP64-pipe work): hi keeps the leading 24 significant bits (truncated), lo is
// the remaining 29 bits rounded to a float and scaled by 2^(E-1075).  Exact to
// about 48 bits for |x| in [2^-74, 2^127]; zero maps to (0, 0); anything else
// (tiny, huge, inf, NaN) takes the FP64 conversion route.
__device__ __forceinline__ ff2 ff_split_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned E = (unsigned)(b >> 52) & 0x7FFu;
  if (E - 949u > 201u) {
    if (E == 0u) return ff_make(0.f, 0.f);
    return ff_from_double(x);
  }
  const unsigned sgn = (unsigned)(b >> 63) << 31;
  const unsigned long long M = b & 0xFFFFFFFFFFFFFull;
  const float hi = __uint_as_float(sgn | ((E - 896u) << 23) | (unsigned)(M >> 29));
  const float scale = __uint_as_float(sgn | ((E - 948u) << 23));
  return ff_make(hi, __uint2float_rn((unsigned)(M & 0x1FFFFFFFull)) * scale);
}

// float -> double by bit placement for normal floats (zero and subnormals take
// the conversion instruction)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)f;
  const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

__host__ inline ff2 ff_from_double_host(double x) {
  const float h = (float)x;
  return ff_make(h, (float)(x - (double)h));
}

}  // namespace feks
