// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| < ulp(hi), about 48 significant bits with the FP32
// exponent range.  Every operation runs on the FP32 pipe, which on GB300
// issues 64 times as many operations per clock as the FP64 pipe.
//
// Building blocks are the error-free transformations: Knuth's TwoSum (s + e =
// a + b exactly), Dekker's Fast2Sum (the same when |a| >= |b|) and the exact
// product through the FMA (p + e = a * b exactly).  The operations follow the
// double-word algorithms analysed by Joldes, Muller and Popescu (ACM TOMS 44,
// 2017):
//   - addition with one TwoSum on the high parts and the low parts added in
//     FP32: absolute error below about 2u^2 (|a| + |b|), u = 2^-24, the size of
//     the rounding the operands already carry;
//   - product from the exact product of the high parts plus the two cross
//     terms: relative error below about 5u^2;
//   - division and square root: the FP32 result corrected by one step of
//     Newton's iteration on the exact remainder (Dekker 1971; Karp and
//     Markstein 1997).
// The error-free steps use the __f*_rn intrinsics, which the compiler never
// contracts into FMAs or reorders, so the transformations stay exact.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace frgb {

struct __align__(8) dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  // nearest FP32 and the FP32 rounding of the remainder
  __host__ __device__ constexpr dfloat(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr dfloat(int x) : hi((float)x), lo(0.f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

template <typename T>
struct is_dfloat : std::false_type {};
template <>
struct is_dfloat<dfloat> : std::true_type {};

namespace dfl {

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfloat renorm(float s, float e) {
  float h, l;
  fast_two_sum(s, e, h, l);
  return dfloat(h, l);
}

}  // namespace dfl

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  float s, e;
  dfl::two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return dfl::renorm(s, e);
}

__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dfl::renorm(p, e);
}

// a * b + c with one renormalisation (named apart from fma so that it never
// hides the FP64 overloads of the enclosing namespace)
__device__ __forceinline__ dfloat dfma(dfloat a, dfloat b, dfloat c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  dfl::two_sum(p, c.hi, s, t);
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  return dfl::renorm(s, t);
}

// q1 = a.hi / b.hi; the remainder a - q1 b is formed exactly in its leading
// part (q1 b.hi as an exact product, a.hi - q1 b.hi exact by Sterbenz's lemma)
// and divided once more
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const float p = __fmul_rn(q1, b.hi);
  const float pe = __fmaf_rn(q1, b.hi, -p);
  float r = __fsub_rn(__fsub_rn(a.hi, p), pe);
  r = __fadd_rn(r, a.lo);
  r = __fmaf_rn(-q1, b.lo, r);
  const float q2 = __fdiv_rn(r, b.hi);
  return dfl::renorm(q1, q2);
}

__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }

// ordering of normalised values: the high parts decide unless they are equal
__device__ __forceinline__ bool operator>(dfloat a, dfloat b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(dfloat a, dfloat b) { return b > a; }

__device__ __forceinline__ dfloat dabs(dfloat x) { return x.hi < 0.f ? -x : x; }

// s = sqrt(hi) in FP32, then s + (x - s^2) / (2 s) with x - s^2 formed exactly
// in its leading part; zero and negative arguments give sqrt(hi) (0 or NaN)
__device__ __forceinline__ dfloat dsqrt(dfloat x) {
  const float s = __fsqrt_rn(x.hi);
  if (!(x.hi > 0.f)) return dfloat(s, 0.f);
  const float p = __fmul_rn(s, s);
  const float pe = __fmaf_rn(s, s, -p);
  float r = __fsub_rn(__fsub_rn(x.hi, p), pe);
  r = __fadd_rn(r, x.lo);
  const float c = __fdiv_rn(r, __fadd_rn(s, s));
  return dfl::renorm(s, c);
}

// FP64 value to double-float (nearest FP32, then the FP32 rounding of the exact remainder)
__device__ __forceinline__ dfloat to_dfloat(double x) {
  const float h = __double2float_rn(x);
  return dfloat(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double to_double(dfloat x) { return (double)x.hi + (double)x.lo; }

}  // namespace frgb
