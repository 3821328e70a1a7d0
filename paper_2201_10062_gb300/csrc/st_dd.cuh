// "dd": a double-float number (unevaluated sum hi + lo of two float32 values, about 48
// significand bits) with arithmetic operators, so that the transform templates of the
// preconditioner (the Stockham FFT of the spatial DST and the folded time DST) instantiate with it
// as the compute type.  The float64 solve uses it as a second engine for those transforms: GB300
// issues 64 float32 operations for each float64 one, and a double-float addition or product costs
// about ten of them (the error-free transformations of st_df.cuh: TwoSum, FastTwoSum and the FMA
// TwoProd, after Knuth and Dekker), so the double-float transform runs several times faster than
// the float64 one at an accuracy of about 2^-47 per operation.
//
// Conversions from and to float64 use float64 instructions; the preconditioner keeps its
// intermediate vectors in this format between passes so that each element is converted once on
// the way in and once on the way out.
#pragma once

#include <cuda_runtime.h>

#include "st_df.cuh"

namespace st {

struct dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ __forceinline__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // exact split of a float64 value to 48 bits: hi = the nearest float, lo = the nearest float to
  // the remainder
  __host__ __device__ __forceinline__ dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ __forceinline__ explicit dd(int x) : hi((float)x), lo(0.f) {}
  __host__ __device__ __forceinline__ explicit dd(float x) : hi(x), lo(0.f) {}
  __host__ __device__ __forceinline__ explicit operator double() const {
    return (double)hi + (double)lo;
  }
  __host__ __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

__host__ __device__ __forceinline__ dd dd_norm(float s, float t) {
  dd r;
  fast_two_sum(s, t, r.hi, r.lo);
  return r;
}

__host__ __device__ __forceinline__ dd operator+(dd a, dd b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  return dd_norm(s, e);
}

__host__ __device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }

__host__ __device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }

__host__ __device__ __forceinline__ dd operator*(dd a, dd b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return dd_norm(p, e);
}

__host__ __device__ __forceinline__ dd &operator+=(dd &a, dd b) {
  a = a + b;
  return a;
}

__host__ __device__ __forceinline__ dd &operator-=(dd &a, dd b) {
  a = a - b;
  return a;
}

__host__ __device__ __forceinline__ dd &operator*=(dd &a, dd b) {
  a = a * b;
  return a;
}

// a * b + c with the product kept exact until the final normalisation
__host__ __device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  float s, t;
  two_sum(p, c.hi, s, t);
  t += e + c.lo;
  return dd_norm(s, t);
}

// 1/a: float reciprocal refined by one Newton step in double-float
__host__ __device__ __forceinline__ dd operator/(dd a, dd b) {
  const float y0 = 1.0f / b.hi;
  const dd q0(a.hi * y0, 0.f);           // first quotient
  const dd r = a - q0 * b;                // remainder in double-float
  return q0 + dd(r.hi * y0, 0.f);
}

// 1/sqrt(a) for a > 0: float estimate refined by one Newton step in double-float
__host__ __device__ __forceinline__ dd rsqrt_dd(dd a) {
  const float y0 = 1.0f / sqrtf(a.hi);
  // y1 = y0 + y0 (1 - a y0^2) / 2
  const dd y = dd(y0, 0.f);
  const dd r = dd(1.0f, 0.f) - a * (y * y);
  return y + dd(0.5f * y0 * r.hi, 0.f);
}

// Accumulator of a dot product in the compute type of a transform template.  For float64 and
// float32 it is a plain multiply-add.  For double-float the running sum is kept as an unnormalised
// pair (s, t): each product a.hi b.hi is formed exactly (TwoProd), its high part added to s
// error-free (TwoSum) and every low-order term added to t, and the pair is normalised once at the
// end: 12 float32 operations per term instead of 15, with the same 2^-47-level accuracy (the
// compensated dot product of Ogita, Rump and Oishi, 2005).
template <class T>
struct MacAcc {
  T v;
  __device__ __forceinline__ void zero() { v = T(0); }
  __device__ __forceinline__ void add(T a, T b);
  __device__ __forceinline__ T get() const { return v; }
};
template <>
__device__ __forceinline__ void MacAcc<double>::add(double a, double b) { v = ::fma(a, b, v); }
template <>
__device__ __forceinline__ void MacAcc<float>::add(float a, float b) { v = fmaf(a, b, v); }
template <>
struct MacAcc<dd> {
  float s, t;
  __device__ __forceinline__ void zero() { s = t = 0.f; }
  __device__ __forceinline__ void add(dd a, dd b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    float ss, err;
    two_sum(s, p, ss, err);
    s = ss;
    t += err + e;
  }
  __device__ __forceinline__ dd get() const { return dd_norm(s, t); }
};

}  // namespace st
