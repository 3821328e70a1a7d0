// Double-float ("df") numbers: an unevaluated sum hi + lo of two float32 values with
// |lo| <= ulp(hi)/2, giving about 48 significand bits.  GB300 issues 64 float32 FMAs for every
// float64 FMA, so the mixed-precision path keeps its MINRES vectors in this format and does the
// per-element arithmetic on the float32 pipes.
//
// Building blocks are the classical error-free transformations: TwoSum (Knuth), FastTwoSum
// (Dekker) and the fused-multiply-add TwoProd; the df operations follow the usual double-double
// constructions (Dekker 1971) with float32 in place of float64.  Compiled without fast-math so
// that the error terms are not optimised away.
#pragma once

#include <cuda_runtime.h>

namespace st {

struct df {
  float hi, lo;
};

// s + e = a + b exactly
__host__ __device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// s + e = a + b exactly when |a| >= |b|
__host__ __device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  e = b - (s - a);
}

// p + e = a * b exactly
__host__ __device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

__host__ __device__ __forceinline__ df df_from_sum(float s, float t) {
  df r;
  fast_two_sum(s, t, r.hi, r.lo);
  return r;
}

__host__ __device__ __forceinline__ df df_add(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  return df_from_sum(s, e);
}

__host__ __device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__host__ __device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// exact difference of two floats as a df
__host__ __device__ __forceinline__ df df_diff(float a, float b) {
  df r;
  two_sum(a, -b, r.hi, r.lo);
  return r;
}

__host__ __device__ __forceinline__ df df_mul(df a, df b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return df_from_sum(p, e);
}

__host__ __device__ __forceinline__ df df_mul_f(df a, float b) {
  float p, e;
  two_prod(a.hi, b, p, e);
  e = fmaf(a.lo, b, e);
  return df_from_sum(p, e);
}

// a*b + c
__host__ __device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }

// running double-float sum (s, t): add p + e, with the high parts added error-free
__host__ __device__ __forceinline__ void dacc_add(float &s, float &t, float p, float e) {
  float ss, err;
  two_sum(s, p, ss, err);
  s = ss;
  t += err + e;
}

// running double-float sum (s, t): add a * b
__host__ __device__ __forceinline__ void dacc_prod(float &s, float &t, df a, df b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  dacc_add(s, t, p, e);
}

__host__ __device__ __forceinline__ df df_of_double(double x) {
  df r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}

__host__ __device__ __forceinline__ double df_to_double(df a) {
  return (double)a.hi + (double)a.lo;
}

}  // namespace st
