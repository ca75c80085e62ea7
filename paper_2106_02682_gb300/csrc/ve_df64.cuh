// ve_df64.cuh -- near-float64 arithmetic on the float32 pipe ("double-float").
//
// A df64 value is the unevaluated sum hi + lo of two float32 numbers with |lo| <= ulp(hi) / 2,
// i.e. a 48-bit significand (relative rounding ~2^-48 = 3.6e-15) with the float32 exponent
// range.  Sums use Knuth's error-free two-sum, products the fma-based two-product, and every
// result is renormalised -- the classical double-word algorithms (Dekker 1971; Hida, Li &
// Bailey's double-double library), written here for float32 words.  On a part whose float64
// rate is ~1/64 of its float32 rate, an eigensolve in df64 runs several times faster than in
// float64 while staying accurate to ~1e-14.
//
// Only what the solver kernels need is provided: construction from / conversion to double,
// + - * and division, comparisons, fabs, and warp shuffles.  Operations are commutative where
// the float64 ones are, so group reductions give the same value in every thread.
#pragma once

#include <cuda_runtime.h>

namespace ve {

// keep the float / double overloads visible next to the df64 ones declared below
using ::fabs;
using ::fmax;
using ::fmin;

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ df64(double x) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
  __device__ __forceinline__ df64(float x) : hi(x), lo(0.f) {}
  __device__ __forceinline__ df64(int x) : hi((float)x), lo(0.f) {}
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

// The error-free transformations below must round every operation on its own: the _rn
// intrinsics are never contracted into fused multiply-adds by the compiler.

// s + e = a + b exactly (Knuth two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly, assuming |a| >= |b| (Dekker fast two-sum)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s1, s2, t1, t2;
  two_sum(a.hi, b.hi, s1, s2);
  two_sum(a.lo, b.lo, t1, t2);
  s2 = __fadd_rn(s2, t1);
  fast_two_sum(s1, s2, s1, s2);
  s2 = __fadd_rn(s2, t2);
  fast_two_sum(s1, s2, s1, s2);
  return df64(s1, s2);
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, t;
  fast_two_sum(p, e, s, t);
  return df64(s, t);
}

__device__ __forceinline__ df64 operator/(df64 a, df64 b) {
  // q1 = a / b in float32, then one correction with the df64 remainder
  const float r = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, r);
  const df64 rem = a - b * df64(q1);
  const float q2 = __fmul_rn(rem.hi, r);
  float s, t;
  fast_two_sum(q1, q2, s, t);
  return df64(s, t);
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

__device__ __forceinline__ bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return !(a < b); }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df64 a, df64 b) { return !(a == b); }

__device__ __forceinline__ df64 fabs(df64 a) { return a.hi < 0.f ? -a : a; }
__device__ __forceinline__ df64 fmin(df64 a, df64 b) { return b < a ? b : a; }

// exact scaling by a power of two
__device__ __forceinline__ df64 ldexp_df(df64 a, float pow2) {
  return df64(__fmul_rn(a.hi, pow2), __fmul_rn(a.lo, pow2));
}

__device__ __forceinline__ df64 shfl_xor(df64 v, int o) {
  return df64(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

}  // namespace ve
