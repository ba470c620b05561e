// Pairs of binary32 numbers ("float-float"): a value is hi + lo with
// |lo| <= ulp(hi) / 2, about 48 significant bits, and every operation runs on
// the binary32 pipe.  On GB300 the binary32 pipe issues 64 times as many
// operations per clock as the binary64 pipe, so an elimination in pairs costs
// several times less than one in binary64 while its rounding error stays near
// 2^-46 per operation.
//
// Building blocks, all published error-free transformations:
//   two_sum   Knuth's TwoSum (The Art of Computer Programming, vol. 2,
//             4.2.2): s + e == a + b exactly, six operations.
//   fast_sum  Dekker's Fast2Sum (Numer. Math. 18, 1971): the same when
//             |a| >= |b|, three operations.
//   product   the exact product a*b = p + e with e = fma(a, b, -p).
// Pair addition adds the two low parts to the TwoSum error term and
// renormalises with Fast2Sum (the "sloppy" double-word sum: its error is
// bounded relative to |x| + |y|, which is the quantity the error bounds of
// this library are stated against).  Pair multiplication and multiply-add
// keep the exact product of the high parts and the two cross terms; the
// lo * lo term is below the pair's precision and dropped.
#pragma once

#include <cfloat>

namespace radic {

// The pair type and its arithmetic live in their own namespace and are found
// by argument-dependent lookup, so that they do not hide the binary32 and
// binary64 fma / fabs / fmax overloads inside namespace radic.
namespace pairs {

struct __align__(8) ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit ff(int x) : hi(static_cast<float>(x)), lo(0.0f) {}
  __host__ __device__ constexpr explicit ff(float x) : hi(x), lo(0.0f) {}
  // nearest pair to a binary64 value (exact for values with <= 48
  // significant bits in the normal binary32 range)
  __device__ explicit ff(double x) : hi(static_cast<float>(x)), lo(static_cast<float>(x - static_cast<double>(hi))) {}
  __device__ explicit operator double() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ ff fast_sum(float a, float b) {
  const float s = a + b;
  return ff(s, b - (s - a));
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }

__device__ __forceinline__ ff operator+(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  return fast_sum(s, e);
}

__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_sum(p, e);
}

__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__device__ __forceinline__ ff& operator*=(ff& a, ff b) { return a = a * b; }

// a * b + c with one renormalisation.
__device__ __forceinline__ ff fma(ff a, ff b, ff c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, t;
  two_sum(p, c.hi, s, t);
  t += e + c.lo;
  return fast_sum(s, t);
}

__device__ __forceinline__ ff fabs(ff a) { return a.hi < 0.0f ? -a : a; }

// Magnitude order by the leading parts (ties within one binary32 ulp are
// resolved arbitrarily, which partial pivoting tolerates).
__device__ __forceinline__ bool operator>(ff a, ff b) { return a.hi > b.hi; }
__device__ __forceinline__ bool operator<=(ff a, ff b) { return a.hi <= b.hi; }
__device__ __forceinline__ ff fmax(ff a, ff b) { return (b.hi > a.hi) ? b : a; }

// Reciprocal: binary32 estimate r of 1/a.hi, then one Newton-Raphson step
// r + r (1 - a r) evaluated with the residual 1 - a r formed exactly enough
// in binary32 (a.hi * r is within a few ulps of 1, so 1 - p is exact).
__device__ __forceinline__ ff rcp_t(ff a) {
  if (a.hi == 0.0f) return ff(0.0f, 0.0f);
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a.hi));
  const float p = a.hi * r;
  const float pe = fmaf(a.hi, r, -p);
  const float res = ((1.0f - p) - pe) - a.lo * r;
  return fast_sum(r, r * res);
}

// A pair within 2^-47 of a binary64 value, without the binary64 pipe: the high
// part takes the leading 24 significand bits (truncated), the low part the
// remaining 29 bits rounded once to binary32 (error at most 2^-47 |x|), then
// one Fast2Sum renormalises.  Values outside [2^-70, 2^100] in magnitude (and
// zeros) take the ordinary conversion.
__device__ __forceinline__ ff split_to_pair(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int e = static_cast<int>((b >> 52) & 0x7ffu);
  if (e < 1023 - 70 || e > 1023 + 100) return ff(x);
  const unsigned long long mant = (b & ((1ull << 52) - 1ull)) | (1ull << 52);
  const unsigned int sign = static_cast<unsigned int>(b >> 63) << 31;
  const float hi = __uint_as_float(sign | (static_cast<unsigned int>(e - 1023 + 127) << 23) |
                                   static_cast<unsigned int>((mant >> 29) & 0x7fffffu));
  const float scale = __uint_as_float(static_cast<unsigned int>(e - 1023 - 52 + 127) << 23);
  float lo = __uint2float_rn(static_cast<unsigned int>(mant & ((1ull << 29) - 1ull))) * scale;
  if (sign) lo = -lo;
  return fast_sum(hi, lo);
}

}  // namespace pairs

using pairs::ff;
using pairs::split_to_pair;

// Element conversions used when staging a matrix into shared memory.
template <typename T>
__device__ __forceinline__ T to_elem(double x);
template <>
__device__ __forceinline__ float to_elem<float>(double x) {
  return static_cast<float>(x);
}
template <>
__device__ __forceinline__ double to_elem<double>(double x) {
  return x;
}
template <>
__device__ __forceinline__ ff to_elem<ff>(double x) {
  return ff(x);
}

}  // namespace radic
