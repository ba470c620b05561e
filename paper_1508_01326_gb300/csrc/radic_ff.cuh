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

// Leading product of two pairs with its error term: a.hi b.hi = p + e exactly
// (fma), then the cross terms a.hi b.lo and a.lo b.hi folded into e; the
// lo lo term (below 2^-48 |ab|) is dropped.  |p + e - ab| <= 1.5 2^-46 |ab|.
__device__ __forceinline__ void prod_terms(ff a, ff b, float& p, float& e) {
  p = a.hi * b.hi;
  e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
}

// sum_i a[i] b[i] + c with one renormalisation (N >= 1): the leading parts of
// the products are added by a TwoSum chain (error-free), the error terms,
// the chain's errors and c.lo in binary32, then one Fast2Sum.  With
// S = sum |a_i b_i| + |c| the error is at most
//   (1.5 + N + N (N + 5) / 4 + (N + 5) / 4) 2^-46 S,
// below 2^-43 times (2 S for N = 2, 3 S for N = 3, 7 S for N = 7): the
// per-operation unit BoundTraits<ff>::u times the operation count of the
// chained multiply-adds it replaces.
template <int N, bool kC>
__device__ __forceinline__ ff dot_acc(const ff* a, const ff* b, ff c) {
  float s, lo;
  int i0;
  if constexpr (kC) {
    s = c.hi;
    lo = c.lo;
    i0 = 0;
  } else {
    prod_terms(a[0], b[0], s, lo);
    i0 = 1;
  }
#pragma unroll
  for (int i = i0; i < N; ++i) {
    float p, e, t;
    prod_terms(a[i], b[i], p, e);
    two_sum(s, p, s, t);
    lo += e + t;
  }
  return fast_sum(s, lo);
}

// a b - c d for pairs (2 x 2 determinants and cross-product entries).
__device__ __forceinline__ ff diff_prod(ff a, ff b, ff c, ff d) {
  const ff x[2] = {a, -c}, y[2] = {b, d};
  return dot_acc<2, false>(x, y, ff(0.0f, 0.0f));
}

// The ordinary conversion, kept out of line so that the rare branch of
// split_to_pair costs nothing on the binary64 pipe when it is not taken.
static __device__ __noinline__ ff pair_from_double(double x) { return ff(x); }

// A pair within 2^-47 of a binary64 value, without the binary64 pipe: the high
// part takes the leading 24 significand bits (truncated), the low part the
// remaining 29 bits rounded once to binary32 (error at most 2^-47 |x|), then
// one Fast2Sum renormalises.  Values outside [2^-70, 2^100] in magnitude (and
// zeros) take the ordinary conversion.
__device__ __forceinline__ ff split_to_pair(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int e = static_cast<int>((b >> 52) & 0x7ffu);
  if (__builtin_expect(e < 1023 - 70 || e > 1023 + 100, 0)) return pair_from_double(x);
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

using pairs::diff_prod;
using pairs::dot_acc;
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
