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

// Dot-product accumulator with deferred normalisation: the running sum is
// hi + lo with hi updated by TwoSum and the rounding errors of both the
// products and the additions collected in lo; normalise once at the end.
// The loop-carried dependency is one binary32 addition per term.
struct df64_acc {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add_prod(df64 x, df64 y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    const float s = hi + p;
    const float bb = s - hi;
    const float t = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += t + e;
  }
  __device__ __forceinline__ df64 value() const { return fast_two_sum(hi, lo); }
};

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

// 2^k as a binary32 for k in [-126, 127]
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// Split of x * 2^-shift into hi + lo (hi = x rounded to 24 bits, lo = the
// remainder rounded to 24 bits) with integer and binary32 operations only --
// no binary64 arithmetic, which is slow on this GPU.  The 53-bit significand
// m of x is rounded to 24 bits (round half to even) by integer arithmetic,
// the remainder m - mh*2^29 (|.| <= 2^28, exact) is converted to binary32 and
// both are scaled by exact powers of two.  Zeros, subnormals, Inf/NaN and
// magnitudes whose parts would leave the binary32 normal range take the
// binary64 path.
__device__ __forceinline__ df64 split_scaled(double x, int shift) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((u >> 52) & 0x7ff) - shift;  // biased exponent of x * 2^-shift
  const int e = E - 1023;                                        // unbiased
  if (((u >> 52) & 0x7ff) == 0 || ((u >> 52) & 0x7ff) == 0x7ff || e > 126 || e - 52 < -126) {
    const double xs = ldexp(x, -shift);
    return df64(xs);
  }
  const unsigned long long m = (u & 0xfffffffffffffull) | (1ull << 52);
  unsigned long long mh = m >> 29;
  const unsigned long long rb = m & ((1ull << 29) - 1);
  if (rb > (1ull << 28) || (rb == (1ull << 28) && (mh & 1ull))) ++mh;  // <= 2^24
  const long long rem = static_cast<long long>(m) - static_cast<long long>(mh << 29);
  float hi = static_cast<float>(static_cast<unsigned int>(mh)) * pow2f(e - 23);
  float lo = static_cast<float>(static_cast<int>(rem)) * pow2f(e - 52);
  if (u >> 63) {
    hi = -hi;
    lo = -lo;
  }
  return df64(hi, lo);
}

// hi + lo rounded to binary64, with integer operations only: both parts'
// significands are added on a common 2^(eh-127-52) grid (hi's significand
// shifted left by 29), the sum is normalised with a count of leading zeros,
// rounded to 53 bits (half to even) and packed.  Falls back to binary64
// addition for zeros, subnormals and non-finite parts.
__device__ __forceinline__ double to_double(df64 v) {
  const unsigned int uh = static_cast<unsigned int>(__float_as_int(v.hi));
  const unsigned int ul = static_cast<unsigned int>(__float_as_int(v.lo));
  const int eh = static_cast<int>((uh >> 23) & 0xff), el = static_cast<int>((ul >> 23) & 0xff);
  if (eh == 0 || eh == 0xff || el == 0xff || (el == 0 && (ul << 1) != 0))
    return static_cast<double>(v.hi) + static_cast<double>(v.lo);
  long long sum = static_cast<long long>((uh & 0x7fffff) | 0x800000) << 29;
  if (uh >> 31) sum = -sum;
  if (el != 0) {
    const int sft = 29 - (eh - el);  // lo's grid relative to hi's 2^-29 grid
    long long sl = static_cast<long long>((ul & 0x7fffff) | 0x800000);
    if (ul >> 31) sl = -sl;
    if (sft >= 0) {
      sum += sl << sft;
    } else if (sft > -48) {
      // keep two guard bits so the final rounding stays correct
      sum = (sum << 2) + (sft + 2 >= 0 ? (sl << (sft + 2)) : (sl >> (-sft - 2)));
      unsigned long long a = static_cast<unsigned long long>(sum < 0 ? -sum : sum);
      const int p = 63 - __clzll(a);
      const int sh = p - 52;  // >= 2 here: shift out guard bits and excess
      unsigned long long mant = a >> sh;
      const unsigned long long rest = a & ((1ull << sh) - 1), halfw = 1ull << (sh - 1);
      if (rest > halfw || (rest == halfw && (mant & 1ull))) ++mant;
      int exp2 = p - 2 + eh - 127 - 52;  // value = 1.f * 2^exp2
      if (mant >> 53) { mant >>= 1; ++exp2; }
      if (exp2 < -1022 || exp2 > 1023) return static_cast<double>(v.hi) + static_cast<double>(v.lo);
      const unsigned long long bits = (static_cast<unsigned long long>(sum < 0) << 63) |
                                      (static_cast<unsigned long long>(exp2 + 1023) << 52) |
                                      (mant & 0xfffffffffffffull);
      return __longlong_as_double(static_cast<long long>(bits));
    }
  }
  unsigned long long a = static_cast<unsigned long long>(sum < 0 ? -sum : sum);
  if (a == 0) return 0.0;
  const int p = 63 - __clzll(a);
  unsigned long long mant;
  int exp2 = p + eh - 127 - 52;  // value = a * 2^(eh-127-52) = 1.f * 2^exp2
  if (p > 52) {
    const int sh = p - 52;
    mant = a >> sh;
    const unsigned long long rest = a & ((1ull << sh) - 1), halfw = 1ull << (sh - 1);
    if (rest > halfw || (rest == halfw && (mant & 1ull))) ++mant;
    if (mant >> 53) { mant >>= 1; ++exp2; }
  } else {
    mant = a << (52 - p);
  }
  if (exp2 < -1022 || exp2 > 1023) return static_cast<double>(v.hi) + static_cast<double>(v.lo);
  const unsigned long long bits = (static_cast<unsigned long long>(sum < 0) << 63) |
                                  (static_cast<unsigned long long>(exp2 + 1023) << 52) |
                                  (mant & 0xfffffffffffffull);
  return __longlong_as_double(static_cast<long long>(bits));
}

}  // namespace tsqr
