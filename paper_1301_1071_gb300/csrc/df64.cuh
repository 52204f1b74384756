// df64.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo
// of two binary32 numbers with |lo| <= ulp(hi)/2 (about 48 significant bits).
//
// Published methods used: TwoSum (Knuth, TAOCP vol. 2), FastTwoSum (Dekker
// 1971), TwoProduct via a fused multiply-add (the error term of a*b is
// fma(a, b, -a*b)), and the double-word multiply-add of the double-float
// literature (Dekker 1971; Joldes, Muller, Popescu 2017).  The few divisions
// and square roots of the Householder scalars are done in binary64 through
// exact conversions.
//
// On GB300 binary64 FMA runs at ~1.9 per clock per SM, binary32 FMA at ~119;
// a double-float multiply-add costs ~15 binary32 operations and runs ~5x
// faster than a binary64 FMA.  Range is binary32's: callers scale data by
// powers of two (exact) so that magnitudes stay far from under/overflow.
#pragma once

#include <cuda_runtime.h>

namespace tsqr {

// keep the binary64/binary32 overloads visible next to the double-float one
using ::fma;

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df64(int v) : hi(static_cast<float>(v)), lo(0.0f) {}
  // exact split of a binary64 value (its low bits beyond 48 are rounded away)
  __device__ explicit df64(double d) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - static_cast<double>(hi));
  }
  __device__ explicit operator double() const { return static_cast<double>(hi) + static_cast<double>(lo); }
  __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
  const float s = a + b;
  return df64(s, b - (s - a));
}

__device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df64(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ df64 operator+(df64 x, df64 y) {
  df64 s = two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }

__device__ __forceinline__ df64 operator*(df64 x, df64 y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

// a * b + c
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  df64 s = two_sum(p, c.hi);
  s.lo += e + c.lo;
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df64& operator+=(df64& x, df64 y) {
  x = x + y;
  return x;
}

__device__ __forceinline__ df64 operator/(df64 x, df64 y) {
  return df64(static_cast<double>(x) / static_cast<double>(y));
}

__device__ __forceinline__ bool operator==(df64 x, df64 y) { return x.hi == y.hi && x.lo == y.lo; }
__device__ __forceinline__ bool operator!=(df64 x, df64 y) { return !(x == y); }

__device__ __forceinline__ df64 dev_sqrt(df64 x) { return df64(sqrt(static_cast<double>(x))); }
__device__ __forceinline__ df64 dev_copysign(df64 a, df64 b) {
  const bool neg_a = a.hi < 0.0f, neg_b = (b.hi < 0.0f) || (b.hi == 0.0f && signbit(b.hi));
  return neg_a != neg_b ? -a : a;
}
__device__ __forceinline__ df64 dev_abs(df64 a) { return a.hi < 0.0f ? -a : a; }

// butterfly exchange of both words (found by argument-dependent lookup from
// the generic reductions)
__device__ __forceinline__ df64 shfl_xor(df64 v, int o) {
  return df64(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

// exact scaling by 2^e
__device__ __forceinline__ df64 scale2(df64 x, int e) { return df64(ldexpf(x.hi, e), ldexpf(x.lo, e)); }

}  // namespace tsqr
