// A-posteriori error bounds of the floating-point paths.
//
// Every floating-point result carries err_bound, an upper bound on
// |computed det_R(A) - exact det_R(A)| for the input as given.  It is built
// from the computation itself (running error analysis), not from a model of
// typical errors:
//
//  * Every quantity of an elimination carries a radius: an upper bound on its
//    distance from the value exact arithmetic would give with the same pivot
//    order (midpoint-radius enclosures).  Radii start at the rounding of the
//    input to the element type and propagate by the enclosure rules
//      |x'y' - xy| <= |x| r_y + |y| r_x + r_x r_y,
//      |a'/p' - a/p| <= (r_a + |a/p| r_p) / (|p| - r_p)   (r_p < |p|),
//      |prod p'_k - prod p_k| <= |prod p_k| (prod (1 + r_k / |p_k|) - 1),
//    plus the rounding of each operation, modelled as
//      fl(a*b + c) = a*b + c + e,  |e| <= u (|a*b| + |c|),
//    u the unit of the arithmetic: binary64 2^-53, binary32 2^-24, pairs of
//    binary32 2^-43 (the pair multiply-add of radic_ff.cuh errs by at most
//    about 19 2^-48 (|a*b| + |c|), its multiplication and addition by less;
//    its dot products with one renormalisation, dot_acc, by less than u
//    times the operation count of the chained form they replace).
//    A multiplier a / p formed with an approximate reciprocal counts as 2
//    (binary64, pairs) or 3 (binary32) roundings.
//  * A pivot whose enclosure reaches zero (r_p >= |p|) cannot be bounded this
//    way: its prefix or minor is flagged (the MIXED and PAIR modes redo it in
//    binary64) or, in binary64, bounded by |computed| + |exact|, with
//    |exact| <= prod_{k<K} (|p_k| + r_k) * prod_j ||(|s_ij| + r_ij)_i||
//    (Hadamard's inequality on the enclosure of the Schur complement S left
//    when pivot K failed; the lane-group LU, whose columns are spread over
//    lanes, takes Hadamard's inequality on the minor's own columns).
//  * The final bound is multiplied by kBoundMargin = 1.02, which covers the
//    binary32 rounding of the radius arithmetic itself.
//  * Prefix sharing (Section 5's runs, factored once per prefix): for the
//    leaves of one prefix the computed value is alpha * det(Z^), alpha the
//    signed product of the prefix pivots and Z^ the D x D matrix of computed
//    Schur-complement columns z^_c.  With |z^_c - z_c| <= r_c and
//    n_c = ||z^_c||_2, multilinearity and Hadamard's inequality give
//      |det Z^ - det Z| <= prod_c (n_c + r_c) - prod_c n_c,
//    and summed over all leaves of the prefix these are symmetric functions
//    of the columns' (n_c, r_c), accumulated in O(1) per column (LeafPoly).
//    r_c is the column's exact radius from the radii of W = -L21 L11^-1 and
//    its own entries (binary64, pairs), or kappa * ||A[:, c]||_2 with kappa
//    from the row norms of W and its radii (binary32: one multiply).
//    The rounding of each leaf determinant adds c_D u prod_c n_c, the radius
//    of alpha adds rel_alpha |term|, and the summation of the prefix's terms
//    adds u_sum * depth * |term| for the longest addition chain.
//  * Lane, block and grid sums of the bounds are taken in binary64 after the
//    per-lane binary32 accumulation, whose relative rounding (at most 2^-24
//    per addition) the margin covers for up to 3e5 prefixes per lane.
//
// Radii are kept in binary32 for every arithmetic (the binary64 fix-up
// kernels keep binary64 radii).  Inputs are scaled by powers of two so that
// every row's largest entry lies in [0.5, 1); a binary32 radius below 2^-126
// is not represented, so the bounds do not cover entries below about 2^-100
// of their row's largest one for binary32 and pairs (such inputs also leave
// the pair format's precision) and below about 2^-70 for binary64; this is
// documented, not detected.
#pragma once

#include <cfloat>
#include <type_traits>

#include "radic_ff.cuh"

namespace radic {

constexpr double kBoundMargin = 1.02;

// A pivot of magnitude ap with radius rp has an enclosure that reaches zero
// (an exact zero pivot with zero radius is exact: its column is singular).
__device__ __forceinline__ bool pivot_unbounded(float ap, float rp) {
  return !(rp < ap) && !(rp == 0.0f && ap == 0.0f);
}
__device__ __forceinline__ bool pivot_unbounded(double ap, double rp) {
  return !(rp < ap) && !(rp == 0.0 && ap == 0.0);
}

template <typename T>
struct BoundTraits;
template <>
struct BoundTraits<double> {
  using R = float;  // radii need few digits; binary32 keeps them off the binary64 pipe and out of spills
  static constexpr float u = 0x1p-53f;
  static constexpr float u_in = 0.0f;  // binary64 input is taken as is
  static constexpr float c_div = 2.0f;
};
template <>
struct BoundTraits<float> {
  using R = float;
  static constexpr float u = 0x1p-24f;
  static constexpr float u_in = 0x1p-24f;  // rounding of binary64 input to binary32
  static constexpr float c_div = 3.0f;
};
template <>
struct BoundTraits<ff> {
  using R = float;
  static constexpr float u = 0x1p-43f;
  static constexpr float u_in = 0x1p-48f;  // binary64 input rounded to about 48 bits
  static constexpr float c_div = 2.0f;
};

template <typename T>
using Rad = typename BoundTraits<T>::R;

// |x| as a radius-type value (pairs: the leading part, inflated by one
// binary32 unit to cover the trailing part).
//
// Binary64: formed on the integer pipe, not by a conversion on the binary64
// pipe (the scarce unit of binary64 work).  The high word of x holds the
// exponent and the leading 20 fraction bits; re-biased to binary32 they give
// |x| truncated to 20 fraction bits, and one unit of the 20th bit more makes
// it an upper bound within 2^-20 relative.  Zero stays zero; magnitudes
// below 2^-126 give 2^-126 and magnitudes beyond binary32's range +inf.
__device__ __forceinline__ float mag(double x) {
  const unsigned int h = static_cast<unsigned int>(__double2hiint(x)) & 0x7fffffffu;
  const unsigned int e = h >> 20;  // biased binary64 exponent
  if (e < 1023u - 126u) return (h | static_cast<unsigned int>(__double2loint(x))) == 0u ? 0.0f : 0x1p-126f;
  if (e > 1023u + 127u) return __int_as_float(0x7f800000);
  return __uint_as_float(((h - ((1023u - 127u) << 20)) << 3) + 8u);
}
__device__ __forceinline__ float mag(float x) { return fabsf(x); }
__device__ __forceinline__ float mag(ff x) { return fabsf(x.hi) * (1.0f + 0x1p-23f); }

// Exact binary64 value of a staged element (pairs: their sum, exact).
__device__ __forceinline__ double as_double(double x) { return x; }
__device__ __forceinline__ double as_double(float x) { return static_cast<double>(x); }
__device__ __forceinline__ double as_double(ff x) { return static_cast<double>(x.hi) + static_cast<double>(x.lo); }

__device__ __forceinline__ double rcp_rad(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_rad(float x) { return __frcp_ru(x); }  // rounded up: radii stay bounds

// Error data of one factored prefix.
template <typename R>
struct PrefixErr {
  R kappa;      // radius of z(x) per unit of ||A[:, x]||_2
  R rel_alpha;  // relative radius of the product of the prefix pivots
  bool bad;     // some pivot's enclosure reaches zero
};

// kappa from W (D x P) and its radii: for row d,
//   |z_d - z^_d| <= sum_j rW_dj |x_j| + (P u + u_in)(|x_Bd| + sum_j |W_dj| |x_j|)
//               <= [||rW_d|| + (P u + u_in)(1 + ||W_d||)] ||x||_2,
// and the D rows together give ||z - z^||_2 <= kappa ||x||_2.
template <typename T, int D, int P>
__device__ __forceinline__ Rad<T> kappa_of(const T (&W)[D][P], const Rad<T> (&rW)[D][P],
                                           float u_in = BoundTraits<T>::u_in) {
  using R = Rad<T>;
  constexpr R kU = BoundTraits<T>::u;
  R k2 = R(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    R w2 = R(0), r2 = R(0);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const R w = mag(W[d][j]);
      w2 += w * w;
      r2 += rW[d][j] * rW[d][j];
    }
    const R kd = sqrt(r2) * (R(1) + u_in) + (R(P) * kU + u_in) * (R(1) + sqrt(w2));
    k2 += kd * kd;
  }
  return sqrt(k2) * R(1.0001);
}

// Symmetric sums over the candidate columns of one prefix, for the bound on
// the leaves (all D-subsets of the columns).  With the generating polynomial
//   prod_c (1 + t (n_c + e r_c)) = sum_{k,j} E[k][j] t^k e^j,
// sum over leaves of prod_c (n_c + r_c) - prod_c n_c is sum_{j >= 1} E[D][j]
// and sum over leaves of prod_c n_c is E[D][0].
template <typename R, int D>
struct LeafPoly {
  R e[D + 1][D + 1];  // e[k][j], j <= k; e[0][0] = 1
  __device__ __forceinline__ LeafPoly() {
#pragma unroll
    for (int k = 0; k <= D; ++k)
#pragma unroll
      for (int j = 0; j <= D; ++j) e[k][j] = R(k == 0 && j == 0 ? 1 : 0);
  }
  __device__ __forceinline__ void add(R n, R r) {
#pragma unroll
    for (int k = D; k >= 1; --k) {
#pragma unroll
      for (int j = k; j >= 0; --j) {
        R v = e[k][j] + n * e[k - 1][j];
        if (j > 0) v += r * e[k - 1][j - 1];
        e[k][j] = v;
      }
    }
  }
  // product with another column set's polynomial (disjoint columns)
  __device__ __forceinline__ void combine(const LeafPoly& o) {
    R c[D + 1][D + 1];
#pragma unroll
    for (int k = 0; k <= D; ++k)
#pragma unroll
      for (int j = 0; j <= D; ++j) {
        R s = R(0);
#pragma unroll
        for (int k1 = 0; k1 <= k; ++k1)
#pragma unroll
          for (int j1 = 0; j1 <= j; ++j1)
            if (j1 <= k1 && j - j1 <= k - k1) s += e[k1][j1] * o.e[k - k1][j - j1];
        c[k][j] = s;
      }
#pragma unroll
    for (int k = 0; k <= D; ++k)
#pragma unroll
      for (int j = 0; j <= D; ++j) e[k][j] = c[k][j];
  }
  __device__ __forceinline__ R perturbation() const {
    R s = R(0);
#pragma unroll
    for (int j = 1; j <= D; ++j) s += e[D][j];
    return s;
  }
  __device__ __forceinline__ R hadamard() const { return e[D][0]; }
};

// Product of polynomials over an aligned group of lp lanes (lp a power of
// two): every lane ends with the polynomial of the whole group's columns.
template <typename R, int D>
__device__ __forceinline__ void group_combine(LeafPoly<R, D>& p, int lp) {
  for (int off = 1; off < lp; off <<= 1) {
    LeafPoly<R, D> o;
#pragma unroll
    for (int k = 0; k <= D; ++k)
#pragma unroll
      for (int j = 0; j <= D; ++j) o.e[k][j] = __shfl_xor_sync(0xffffffffu, p.e[k][j], off);
    p.combine(o);
  }
}

// Rounding of one leaf determinant relative to prod_c ||z_c||: D = 2,
// fma(y0, z1, -(y1 z0)), 2u (|y0 z1| + |y1 z0|) <= 2u ||y|| ||z||; D = 3, the
// cross product (2u per entry) and the dot product (3u), with the permanent
// of |Z| at most sqrt(2) prod ||z_c||: (3 + 2 sqrt 2) u.  Plus u per column
// for the scaling of its first entry by alpha.
template <int D>
__host__ __device__ constexpr float leaf_round_coef() {
  return D == 2 ? 2.0f + 2.0f : 5.83f + 3.0f;
}

// Longest chain of additions a leaf term passes through inside one prefix of
// k candidate columns taken lb at a time: for D = 3 the sum over q1 of one
// (q2, column) pair, then the column sum over q2; for D = 2 the column sum;
// then the block's column sums and the prefix sum over blocks.
__device__ __forceinline__ float leaf_sum_depth(int D, int k, int lb) {
  const float kk = static_cast<float>(k);
  const float inner = (D == 3) ? 2.0f * kk : kk;
  return inner + static_cast<float>(lb * lb + lb) + kk / static_cast<float>(lb) + 2.0f;
}

}  // namespace radic
