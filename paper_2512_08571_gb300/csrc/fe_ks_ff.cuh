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

__host__ inline ff2 ff_from_double_host(double x) {
  const float h = (float)x;
  return ff_make(h, (float)(x - (double)h));
}

}  // namespace feks
