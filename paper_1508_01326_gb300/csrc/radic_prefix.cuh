// Prefix-sharing variant of the floating-point path.
//
// All minors whose first m-2 columns form the same ascending prefix
// P = (c_0 < ... < c_{m-3}) share the first m-2 steps of partial-pivot LU:
// those steps only look at the prefix columns.  One thread factors the
// m x (m-2) prefix once (partial pivoting, row exchanges tracked in idx[]),
// and turns every later column x into its 2-entry Schur complement
//     z(x) = x_perm[m-2..m-1] + W x_perm[0..m-3],   W = -L21 L11^{-1},
// so that det(A[:, P + {c, c'}]) = sign * prod(pivots) * det[z(c) z(c')].
// Each leaf minor then costs one 2 x 2 determinant.  These are the same
// elimination steps a per-minor partial-pivot LU performs, shared across the
// lexicographic subtree of P (dictionary order, Definition 2).
//
// Work split: prefixes are grouped by their last column v (every prefix of
// group v has the same k = n-1-v candidate columns and k(k-1)/2 leaves).  A
// warp task is 32 equal runs of consecutive prefixes of one group, one run
// per lane, so all lanes of a warp execute the same control flow; run
// lengths are chosen per group so that tasks have similar cost.
#pragma once

#include <type_traits>

#include "radic_bound.cuh"
#include "radic_ff.cuh"
#include "radic_fp_kernels.cuh"

namespace radic {

// A lane's column buffer of the leaf phase: entry q holds the D
// Schur-complement entries of candidate column q.  Entries of one lane are
// `stride` elements apart (lanes interleaved, so a warp's accesses to the
// same q are contiguous).  D = 2 stores one 2-vector per entry; D = 3 stores
// three planes `plane` elements apart (12 or 24 bytes per entry, no padding).
template <typename T, int D>
struct ZBuf;
template <typename T>
struct ZBuf<T, 2> {
  using V = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
  V* p;
  int stride;
  __device__ ZBuf(void* base, int lane, int stride_, int /*kcap*/) : p(static_cast<V*>(base) + lane), stride(stride_) {}
  __device__ __forceinline__ void get(int q, T (&y)[2]) const {
    const V v = p[q * stride];
    y[0] = v.x;
    y[1] = v.y;
  }
  __device__ __forceinline__ void put(int q, const T (&z)[2]) const {
    V v;
    v.x = z[0];
    v.y = z[1];
    p[q * stride] = v;
  }
};
template <>
struct ZBuf<ff, 2> {  // (x.hi, x.lo, y.hi, y.lo) in one 16-byte vector
  float4* p;
  int stride;
  __device__ ZBuf(void* base, int lane, int stride_, int /*kcap*/)
      : p(static_cast<float4*>(base) + lane), stride(stride_) {}
  __device__ __forceinline__ void get(int q, ff (&y)[2]) const {
    const float4 v = p[q * stride];
    y[0] = ff(v.x, v.y);
    y[1] = ff(v.z, v.w);
  }
  __device__ __forceinline__ void put(int q, const ff (&z)[2]) const {
    p[q * stride] = make_float4(z[0].hi, z[0].lo, z[1].hi, z[1].lo);
  }
};
template <>
struct ZBuf<uint32_t, 2> {  // residues of the exact mode
  uint2* p;
  int stride;
  __device__ ZBuf(void* base, int lane, int stride_, int /*kcap*/)
      : p(static_cast<uint2*>(base) + lane), stride(stride_) {}
  __device__ __forceinline__ void get(int q, uint32_t (&y)[2]) const {
    const uint2 v = p[q * stride];
    y[0] = v.x;
    y[1] = v.y;
  }
  __device__ __forceinline__ void put(int q, const uint32_t (&z)[2]) const { p[q * stride] = make_uint2(z[0], z[1]); }
};
template <typename T>
struct ZBuf<T, 3> {
  T* p;
  int stride, plane;
  __device__ ZBuf(void* base, int lane, int stride_, int kcap)
      : p(static_cast<T*>(base) + lane), stride(stride_), plane(kcap * stride_) {}
  // the buffer of the lane `d` positions away
  __device__ __forceinline__ ZBuf shifted(int d) const {
    ZBuf b = *this;
    b.p += d;
    return b;
  }
  __device__ __forceinline__ void get(int q, T (&y)[3]) const {
    const T* e = p + q * stride;
    y[0] = e[0];
    y[1] = e[plane];
    y[2] = e[2 * plane];
  }
  __device__ __forceinline__ void put(int q, const T (&z)[3]) const {
    T* e = p + q * stride;
    e[0] = z[0];
    e[plane] = z[1];
    e[2 * plane] = z[2];
  }
};

// Bytes of the column buffer for `lanes` lanes with up to kcap entries each.
__host__ __device__ inline size_t zbuf_bytes(int kcap, int lanes, int depth, int elem) {
  return (size_t)kcap * lanes * depth * elem;
}

__host__ __device__ inline size_t prefix_smem_bytes(int n, int m, int cs, int elem, int threads, int depth,
                                                    bool dbl = false) {
  const int kmax = n - m + depth;  // largest number of candidate columns
  return fp_smem_bytes(n, m, cs, elem, threads, dbl) + zbuf_bytes(kmax, threads, depth, elem);
}

// Rank of an ascending 0-based combination in dictionary order (the inverse of
// unrank): C(n,m) - 1 - sum_i C(n-1-c_i, m-i).
__device__ __forceinline__ unsigned long long rank_part(const uint64_t* binom, int bstride, int n, int c, int k) {
  return binom[(n - 1 - c) * bstride + k];
}

// Factor the m x P prefix (P = m - D) with partial pivoting.  Outputs the row
// order idx[], W = -L21 L11^{-1} (D x P), the product of pivots, the largest
// pivot magnitude and the parity of the row permutation.
template <typename T, int M, int D, int CS>
__device__ __forceinline__ void prefix_factor(const T* __restrict__ As, const int (&c)[M - D], T (&W)[D][M - D],
                                              int (&idx)[M], T& prod, T& gmax, bool& neg) {
  constexpr int P = M - D;
  T a[M][P];
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const T* col = As + c[j] * CS;
#pragma unroll
    for (int i = 0; i < M; ++i) a[i][j] = col[i];
  }
#pragma unroll
  for (int i = 0; i < M; ++i) idx[i] = i;
  neg = false;
  prod = T(1);
  gmax = T(0);
#pragma unroll
  for (int k = 0; k < P; ++k) {
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      const bool sw = abs_greater(a[i][k], a[k][k]);
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const T x = a[k][j], y = a[i][j];
        a[k][j] = sw ? y : x;
        a[i][j] = sw ? x : y;
      }
      const int ik = idx[k], ii = idx[i];
      idx[k] = sw ? ii : ik;
      idx[i] = sw ? ik : ii;
      neg ^= sw;
    }
    const T piv = a[k][k];
    const T r = rcp_t(piv);
    prod *= piv;
    gmax = fmax(gmax, fabs(piv));
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      const T l = a[i][k] * r;
      a[i][k] = l;
#pragma unroll
      for (int j = k + 1; j < P; ++j) a[i][j] = fma(-l, a[k][j], a[i][j]);
    }
  }
  // W = -L21 L11^{-1}: w_j = -l21_j - sum_{i > j} w_i L11[i][j], j descending.
#pragma unroll
  for (int rr = 0; rr < D; ++rr) {
#pragma unroll
    for (int j = P - 1; j >= 0; --j) {
      T s = -a[P + rr][j];
#pragma unroll
      for (int i = j + 1; i < P; ++i) s = fma(-W[rr][i], a[i][j], s);
      W[rr][j] = s;
    }
  }
}

// A staged entry in the compute type T (pairs widen exactly to binary64).
template <typename T, typename S>
__device__ __forceinline__ T widen(const S& x) {
  if constexpr (std::is_same<T, double>::value && std::is_same<S, ff>::value)
    return static_cast<double>(x.hi) + static_cast<double>(x.lo);
  else
    return x;
}

// prefix_factor with running error radii (radic_bound.cuh): the same
// elimination, plus rW, the radii of W, the relative radius of the pivot
// product and the pivot condition.  The matrix is staged in type S and
// factored in type T (the pair tier factors its prefixes in binary64 from
// the pair-staged matrix); radii start at S's input rounding.
template <typename T, int M, int D, int CS, typename S = T>
__device__ __forceinline__ void prefix_factor_b(const S* __restrict__ As, const int (&c)[M - D], T (&W)[D][M - D],
                                                Rad<T> (&rW)[D][M - D], int (&idx)[M], T& prod, T& gmax, bool& neg,
                                                Rad<T>& rel_alpha, bool& bad,
                                                float uin = BoundTraits<S>::u_in) {
  using R = Rad<T>;
  using B = BoundTraits<T>;
  constexpr int P = M - D;
  T a[M][P];
  R ra[M][P];
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const S* col = As + c[j] * CS;
#pragma unroll
    for (int i = 0; i < M; ++i) {
      a[i][j] = widen<T>(col[i]);
      ra[i][j] = R(uin) * mag(a[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < M; ++i) idx[i] = i;
  neg = false;
  prod = T(1);
  gmax = T(0);
  R rel = R(0);
  bad = false;
#pragma unroll
  for (int k = 0; k < P; ++k) {
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      const bool sw = abs_greater(a[i][k], a[k][k]);
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const T x = a[k][j], y = a[i][j];
        a[k][j] = sw ? y : x;
        a[i][j] = sw ? x : y;
        const R rx = ra[k][j], ry = ra[i][j];
        ra[k][j] = sw ? ry : rx;
        ra[i][j] = sw ? rx : ry;
      }
      const int ik = idx[k], ii = idx[i];
      idx[k] = sw ? ii : ik;
      idx[i] = sw ? ik : ii;
      neg ^= sw;
    }
    const T piv = a[k][k];
    const R ap = mag(piv), rp = ra[k][k];
    bad |= pivot_unbounded(ap, rp);
    const R ipm = ap > R(0) ? rcp_rad(ap) : R(0);                  // 1 / |p|
    const R ipd = ap > rp ? rcp_rad(__fsub_rd(ap, rp)) : R(0);     // 1 / (|p| - r_p)
    rel = fmaf(R(1) + rel, rp * ipm, rel);
    const T r = rcp_t(piv);
    prod *= piv;
    gmax = fmax(gmax, fabs(piv));
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      const T l = a[i][k] * r;
      const R al = mag(l);
      const R rl = (ra[i][k] + al * rp) * ipd + B::c_div * B::u * al;
      a[i][k] = l;
      ra[i][k] = rl;
#pragma unroll
      for (int j = k + 1; j < P; ++j) {
        const T x = a[k][j];
        const R ax = mag(x), old = mag(a[i][j]);
        a[i][j] = fma(-l, x, a[i][j]);
        ra[i][j] += al * ra[k][j] + (ax + ra[k][j]) * rl + B::u * (al * ax + old);
      }
    }
  }
  rel_alpha = fmaf(R(1) + rel, R(P > 1 ? P - 1 : 0) * B::u * R(1.01), rel);
#pragma unroll
  for (int rr = 0; rr < D; ++rr) {
#pragma unroll
    for (int j = P - 1; j >= 0; --j) {
      T s = -a[P + rr][j];
      R rs = ra[P + rr][j], ms = mag(s);
#pragma unroll
      for (int i = j + 1; i < P; ++i) {
        const R aw = mag(W[rr][i]), aa = mag(a[i][j]);
        s = fma(-W[rr][i], a[i][j], s);
        rs += rW[rr][i] * (aa + ra[i][j]) + aw * ra[i][j];
        ms += aw * aa;
      }
      W[rr][j] = s;
      rW[rr][j] = rs + R(P - 1 - j) * B::u * ms;
    }
  }
}

// Schur complement (D entries) of column `col`, rows read in the order idx[].
template <typename T, int M, int D, typename S = T>
__device__ __forceinline__ void prefix_column(const S* __restrict__ col, const T (&W)[D][M - D], const int (&idx)[M],
                                              T (&z)[D]) {
  constexpr int P = M - D;
  T x[M];
#pragma unroll
  for (int s = 0; s < M; ++s) x[s] = widen<T>(col[idx[s]]);
#pragma unroll
  for (int d = 0; d < D; ++d) z[d] = x[P + d];
#pragma unroll
  for (int j = 0; j < P; ++j) {
#pragma unroll
    for (int d = 0; d < D; ++d) z[d] = fma(W[d][j], x[j], z[d]);
  }
}

// Accumulators of one lane: binary64 two-sum for binary64, float-float
// flushed per prefix for binary32.
template <typename T>
struct PrefixAcc;
// Every variant also sums the error bounds of the prefixes it keeps (bnd,
// radic_bound.cuh); a dropped prefix's bound is dropped with its terms.
template <>
struct PrefixAcc<double> {
  Dd acc;
  double abs_sum = 0.0;
  double bnd = 0.0;
  __device__ __forceinline__ void add_column(double s, double a) {
    acc.add(s);
    abs_sum += a;
  }
  __device__ __forceinline__ void add_bound(double b) { bnd += b; }
  __device__ __forceinline__ void end_prefix() {}
  __device__ __forceinline__ void finish() {}
};
template <>
struct PrefixAcc<float> {
  // per prefix: float-float sums; per thread: float-float totals, converted
  // to binary64 once at the end (keeps the binary64 pipe free)
  Ff pre, tot, tot_abs;
  float pre_abs = 0.0f;
  float pre_bnd = 0.0f, bnd = 0.0f;
  Dd acc;
  double abs_sum = 0.0;
  __device__ __forceinline__ void add_column(float s, float a) {
    pre.add(s);
    pre_abs += a;
  }
  __device__ __forceinline__ void add_bound(float b) { pre_bnd += b; }
  __device__ __forceinline__ void end_prefix() {
    tot.merge(pre);
    tot_abs.add(pre_abs);
    bnd += pre_bnd;
    pre = Ff();
    pre_abs = 0.0f;
    pre_bnd = 0.0f;
  }
  __device__ __forceinline__ void drop_prefix() {
    pre = Ff();
    pre_abs = 0.0f;
    pre_bnd = 0.0f;
  }
  __device__ __forceinline__ void finish() {
    acc.add(static_cast<double>(tot.hi));
    acc.add(static_cast<double>(tot.lo));
    abs_sum = static_cast<double>(tot_abs.hi) + static_cast<double>(tot_abs.lo);
  }
};

template <>
struct PrefixAcc<ff> {
  // per prefix: pair sums; per thread: a pair total of the prefix sums (the
  // binary64 pipe stays free) whose additions are bounded by running error
  // analysis: each errs by at most 2^-46 (|total| + |prefix sum|), and run
  // sums those magnitudes; binary32 pairs for |terms|
  ff pre = ff(0.0f, 0.0f);
  float pre_abs = 0.0f;
  float pre_bnd = 0.0f, bnd = 0.0f;
  ff tot = ff(0.0f, 0.0f);
  float run = 0.0f;
  Ff tot_abs;
  Dd acc;
  double abs_sum = 0.0;
  __device__ __forceinline__ void add_column(ff s, ff a) {
    pre += s;
    pre_abs += a.hi;
  }
  __device__ __forceinline__ void add_bound(float b) { pre_bnd += b; }
  __device__ __forceinline__ void end_prefix() {
    tot += pre;
    run += fabsf(tot.hi) + fabsf(pre.hi);
    tot_abs.add(pre_abs);
    bnd += pre_bnd;
    pre = ff(0.0f, 0.0f);
    pre_abs = 0.0f;
    pre_bnd = 0.0f;
  }
  __device__ __forceinline__ void drop_prefix() {
    pre = ff(0.0f, 0.0f);
    pre_abs = 0.0f;
    pre_bnd = 0.0f;
  }
  __device__ __forceinline__ void finish() {
    acc.add(static_cast<double>(tot.hi));
    acc.add(static_cast<double>(tot.lo));
    // 2^-43 covers the 2^-46 per addition, the binary32 magnitudes of the
    // pairs and the binary32 sum `run` itself
    bnd += 0x1p-43f * run;
    abs_sum = static_cast<double>(tot_abs.hi) + static_cast<double>(tot_abs.lo);
  }
};

// Where per-leaf terms go (terms output of the parity tests); unused otherwise.
struct TermsSink {
  double* terms;
  unsigned long long q0, count, qtot;
  int escale;
};

// Columns per step of the blocked leaf phase: every buffer entry loaded from
// shared memory serves kLeafBlock leaves (fewer loads per leaf, kLeafBlock
// independent sums in flight).  Binary64 keeps one column per step: its
// leaves are bound by the binary64 pipe, and wider blocks only cost registers.
// Pairs too (measured on the batched m = 9 and 10 pair kernels: one column
// per step 1-2% faster than two, three 7% slower): their kernels are bound
// by dependency latency at 255 registers.
#ifndef RADIC_LEAF_BLOCK_F32
#define RADIC_LEAF_BLOCK_F32 4
#endif
#ifndef RADIC_LEAF_BLOCK_F64
#define RADIC_LEAF_BLOCK_F64 1
#endif
#ifndef RADIC_LEAF_BLOCK_FF
#define RADIC_LEAF_BLOCK_FF 1
#endif
template <typename T>
__host__ __device__ constexpr int leaf_block() {
  return std::is_same<T, ff>::value ? RADIC_LEAF_BLOCK_FF
                                    : (sizeof(T) == 4 ? RADIC_LEAF_BLOCK_F32 : RADIC_LEAF_BLOCK_F64);
}

template <typename T>
__device__ __forceinline__ void leaf_add(T d, T& s, T& a) {
  s += d;
  a += fabs(d);
}
// Pairs: the magnitude sum only bounds errors, so it is kept in binary32.
__device__ __forceinline__ void leaf_add(ff d, ff& s, ff& a) {
  s += d;
  a.hi += fabsf(d.hi);
}

// 2 x 2 and 3 x 3 leaf determinants of Schur-complement columns.
template <typename T>
__device__ __forceinline__ T det2(const T (&x)[2], const T (&y)[2]) {
  return fma(x[0], y[1], -(x[1] * y[0]));
}
template <typename T>
__device__ __forceinline__ void cross3(const T (&x)[3], const T (&y)[3], T (&w)[3]) {
  w[0] = fma(x[1], y[2], -(x[2] * y[1]));
  w[1] = fma(x[2], y[0], -(x[0] * y[2]));
  w[2] = fma(x[0], y[1], -(x[1] * y[0]));
}
template <typename T>
__device__ __forceinline__ T dot3(const T (&x)[3], const T (&w)[3]) {
  return fma(x[0], w[0], fma(x[1], w[1], x[2] * w[2]));
}
// Pairs: one renormalisation per determinant or entry (radic_ff.cuh dot_acc),
// within the rounding the chained form is bounded by.
__device__ __forceinline__ ff det2(const ff (&x)[2], const ff (&y)[2]) { return diff_prod(x[0], y[1], x[1], y[0]); }
__device__ __forceinline__ void cross3(const ff (&x)[3], const ff (&y)[3], ff (&w)[3]) {
  w[0] = diff_prod(x[1], y[2], x[2], y[1]);
  w[1] = diff_prod(x[2], y[0], x[0], y[2]);
  w[2] = diff_prod(x[0], y[1], x[1], y[0]);
}
__device__ __forceinline__ ff dot3(const ff (&x)[3], const ff (&w)[3]) {
  return dot_acc<3, false>(x, w, ff(0.0f, 0.0f));
}

// Error-bound state of one prefix's leaf phase (radic_bound.cuh): the
// symmetric sums of the candidate columns' (||z^||, radius) and the lane's
// sum of |terms| of the prefix.  With kOn = false it does nothing.
template <typename T, int D, int P, bool kOn>
struct LeafBound {
  using R = Rad<T>;
  // binary64 and pairs: the exact per-column radius; binary32 (whose bound
  // only has to meet 1e-4 targets): kappa times the column's norm, one
  // multiply per column
  static constexpr bool kExact = kOn && !std::is_same<T, float>::value;
  R cW[kExact ? D : 1][kExact ? P : 1];  // rW (1 + u_in) + cround |W|: the radius weight of |x_j| in entry d
  R cround;                              // P u + u_in: rounding of a Schur-complement entry per unit of its terms
  R uin;
  R kappa;                               // binary32: radius of z(x) per unit of ||x||_2 (kappa_of)
  LeafPoly<R, D> poly;
  R pabs;
  template <typename W_t>
  __device__ __forceinline__ LeafBound(const W_t& W, const R (*rw)[P], R uin_) : uin(uin_), pabs(R(0)) {
    if constexpr (kExact) {
      cround = R(P) * R(BoundTraits<T>::u) + uin_;
#pragma unroll
      for (int d = 0; d < D; ++d)
#pragma unroll
        for (int j = 0; j < P; ++j) cW[d][j] = fmaf(cround, mag(W[d][j]), rw[d][j] * (R(1) + uin_)) * R(1.0000002);
    } else if constexpr (kOn) {
      kappa = kappa_of<T, D, P>(W, *reinterpret_cast<const R(*)[D][P]>(rw), uin_);
    }
  }
  // z: the column's computed Schur complement (before its sign and alpha),
  // ax: the magnitudes of its column entries in the prefix's row order.
  // |z_d - z^_d| <= sum_j rW_dj |x_j| + (P u + u_in)(|x_Bd| + sum_j |W_dj| |x_j|)
  //              = cround |x_Bd| + sum_j cW_dj |x_j|
  __device__ __forceinline__ void column(const T (&z)[D], const R (&ax)[P + D]) {
    if constexpr (kExact) {
      R n2 = R(0), r2 = R(0);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const R a = mag(z[d]);
        n2 += a * a;
        R rz = cround * ax[P + d];
#pragma unroll
        for (int j = 0; j < P; ++j) rz = fmaf(cW[d][j], ax[j], rz);
        r2 += rz * rz;
      }
      poly.add(sqrt(n2) * R(1.0000005), sqrt(r2) * R(1.000002));
    } else if constexpr (kOn) {
      R n2 = R(0), x2 = R(0);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const R a = mag(z[d]);
        n2 += a * a;
      }
#pragma unroll
      for (int s = 0; s < P + D; ++s) x2 += ax[s] * ax[s];
      poly.add(sqrt(n2) * R(1.0000005), kappa * sqrt(x2) * R(1.000002));
    }
  }
  __device__ __forceinline__ void term_abs(const T& babs) {
    if constexpr (kOn) pabs += mag(babs);
  }
};

// Schur complement of candidate column `col`, with the sign of its index
// parity and (first entry) the prefix scale alpha folded in; updates zmax.
template <typename T, int M, int D, int CS, bool kB>
__device__ __forceinline__ void leaf_column(const T* __restrict__ As, int col, const T (&W)[D][M - D],
                                            const int (&idx)[M], T alpha, T (&z)[D], T& zmax,
                                            LeafBound<T, D, M - D, kB>& lb) {
  constexpr int P = M - D;
  const T* cp = As + col * CS;
  T x[M];
#pragma unroll
  for (int s = 0; s < M; ++s) x[s] = cp[idx[s]];
  if constexpr (std::is_same<T, ff>::value) {
#pragma unroll
    for (int d = 0; d < D; ++d) z[d] = dot_acc<P, true>(W[d], x, x[P + d]);
  } else {
#pragma unroll
    for (int d = 0; d < D; ++d) z[d] = x[P + d];
#pragma unroll
    for (int j = 0; j < P; ++j) {
#pragma unroll
      for (int d = 0; d < D; ++d) z[d] = fma(W[d][j], x[j], z[d]);
    }
  }
  if constexpr (kB) {
    Rad<T> ax[M];
#pragma unroll
    for (int s = 0; s < M; ++s) ax[s] = mag(x[s]);
    lb.column(z, ax);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    zmax = fmax(zmax, fabs(z[d]));
    if (col & 1) z[d] = -z[d];
  }
  z[0] *= alpha;
}

// Leaf phase of one prefix without per-leaf output: the k later columns are
// taken LB at a time (q, q+1, ...).  For each block, the leaves whose other
// D-1 columns lie before the block read those columns' z from the buffer
// once for the whole block; leaves with two or three columns inside the
// block are formed from registers.  Leaf sums are kept per column, and a
// block's column sums are added together to acc in block order.  Columns
// past k in the last block are zero, and so are their leaves.  When `lp`
// lanes share the prefix, lane `sub` takes the leaves whose second-to-last
// column from the buffer is congruent to sub modulo lp (and sub 0 those
// inside a block).
//
// kCoop: the buffer already holds every column's z (written by the lanes
// sharing the prefix, see prefix_leaves); the block's columns are read from
// it instead of being reduced here.
template <typename T, int M, int D, int CS, bool kCoop, bool kB>
__device__ __forceinline__ void prefix_leaves_blocked(const T* __restrict__ As, int v, int k, const T (&W)[D][M - D],
                                                      const int (&idx)[M], T alpha, const ZBuf<T, D>& zb, bool act,
                                                      int sub, int lp, PrefixAcc<T>& acc, T& zmax,
                                                      LeafBound<T, D, M - D, kB>& lb) {
  constexpr int LB = leaf_block<T>();
  for (int q = 0; q < k; q += LB) {
    T z[LB][D];
#pragma unroll
    for (int b = 0; b < LB; ++b) {
      if (q + b < k) {  // the same k in every lane of a warp
        if constexpr (kCoop) {
          zb.get(q + b, z[b]);
        } else {
          leaf_column<T, M, D, CS>(As, v + 1 + q + b, W, idx, alpha, z[b], zmax, lb);
        }
      } else {
#pragma unroll
        for (int d = 0; d < D; ++d) z[b][d] = T(0);
      }
    }
    T cs[LB], ca[LB];
#pragma unroll
    for (int b = 0; b < LB; ++b) cs[b] = ca[b] = T(0);
    if constexpr (D == 2) {
      // (q2, q + b), q2 < q
#pragma unroll 2
      for (int q2 = sub; q2 < q; q2 += lp) {
        T y[2];
        zb.get(q2, y);
#pragma unroll
        for (int b = 0; b < LB; ++b) leaf_add(det2(y, z[b]), cs[b], ca[b]);
      }
      // (q + b2, q + b), b2 < b
      if (sub == 0) {
#pragma unroll
        for (int b = 1; b < LB; ++b) {
#pragma unroll
          for (int b2 = 0; b2 < b; ++b2) leaf_add(det2(z[b2], z[b]), cs[b], ca[b]);
        }
      }
    } else {
      // (q1, q2, q + b), q1 < q2 < q: y1 . (y2 x z_b); q2 = 0 has no q1.
      // The leaves of one (q2, b) are summed apart and then added to the
      // column sum, so that no term passes through more than about 2k
      // additions (the summation part of the error bound).
      for (int q2 = (sub == 0 ? lp : sub); q2 < q; q2 += lp) {
        T y2[3];
        zb.get(q2, y2);
        T w[LB][3], s2[LB];
#pragma unroll
        for (int b = 0; b < LB; ++b) {
          cross3(y2, z[b], w[b]);
          s2[b] = T(0);
        }
#pragma unroll 2
        for (int q1 = 0; q1 < q2; ++q1) {
          T y1[3];
          zb.get(q1, y1);
#pragma unroll
          for (int b = 0; b < LB; ++b) leaf_add(dot3(y1, w[b]), s2[b], ca[b]);
        }
#pragma unroll
        for (int b = 0; b < LB; ++b) cs[b] += s2[b];
      }
      if constexpr (LB > 1) {
        // (q1, q + b2, q + b), q1 < q, b2 < b: y1 . (z_b2 x z_b); pair
        // (b2, b) is entry b(b-1)/2 + b2 of w
        T w[LB * (LB - 1) / 2][3];
#pragma unroll
        for (int b = 1; b < LB; ++b) {
#pragma unroll
          for (int b2 = 0; b2 < b; ++b2) cross3(z[b2], z[b], w[b * (b - 1) / 2 + b2]);
        }
#pragma unroll 2
        for (int q1 = sub; q1 < q; q1 += lp) {
          T y1[3];
          zb.get(q1, y1);
#pragma unroll
          for (int b = 1; b < LB; ++b) {
#pragma unroll
            for (int b2 = 0; b2 < b; ++b2) leaf_add(dot3(y1, w[b * (b - 1) / 2 + b2]), cs[b], ca[b]);
          }
        }
        // (q + b1, q + b2, q + b), b1 < b2 < b
        if (sub == 0) {
#pragma unroll
          for (int b = 2; b < LB; ++b) {
#pragma unroll
            for (int b2 = 1; b2 < b; ++b2) {
#pragma unroll
              for (int b1 = 0; b1 < b2; ++b1) leaf_add(dot3(z[b1], w[b * (b - 1) / 2 + b2]), cs[b], ca[b]);
            }
          }
        }
      }
    }
    // the block's column sums (columns past k hold zeros) enter the
    // prefix sum together
    T bsum = cs[0], babs = ca[0];
#pragma unroll
    for (int b = 1; b < LB; ++b) {
      bsum += cs[b];
      babs += ca[b];
    }
    if (act) {
      acc.add_column(bsum, babs);
      lb.term_abs(babs);
    }
    if constexpr (!kCoop) {
#pragma unroll
      for (int b = 0; b < LB; ++b) {
        if (q + b < k) zb.put(q + b, z[b]);
      }
    }
  }
}

// Largest value over the aligned group of lp lanes (lp a power of two).
__device__ __forceinline__ float group_max(float x, int lp) {
  for (int off = 1; off < lp; off <<= 1) x = fmaxf(x, __shfl_xor_sync(kFull, x, off));
  return x;
}
__device__ __forceinline__ double group_max(double x, int lp) {
  for (int off = 1; off < lp; off <<= 1) x = fmax(x, __shfl_xor_sync(kFull, x, off));
  return x;
}
__device__ __forceinline__ ff group_max(ff x, int lp) {
  for (int off = 1; off < lp; off <<= 1) {
    const ff o(__shfl_xor_sync(kFull, x.hi, off), __shfl_xor_sync(kFull, x.lo, off));
    x = fmax(x, o);
  }
  return x;
}

// Leaf phase with per-leaf output (terms of the parity tests): one column at
// a time, every leaf's dictionary-order rank computed and its term stored
// when it falls in the requested window.
template <typename T, int M, int D, int CS>
__device__ __forceinline__ void prefix_leaves_terms(const T* __restrict__ As, const uint64_t* binom, int n, int v,
                                                    int k, const T (&W)[D][M - D], const int (&idx)[M], T alpha,
                                                    unsigned long long rank_prefix, const ZBuf<T, D>& zb, bool act,
                                                    int sub, int lp, PrefixAcc<T>& acc, T& zmax,
                                                    const TermsSink& ts, bool nan_out = false) {
  const int bs = M + 1;
  auto emit = [&](T d, unsigned long long rk) {
    rk = ts.qtot - 1 - rk;
    if (act && rk >= ts.q0 && rk < ts.q0 + ts.count)
      ts.terms[rk - ts.q0] = nan_out ? __longlong_as_double(0x7ff8000000000000ll) : ldexp(static_cast<double>(d), ts.escale);
  };
  for (int q = 0; q < k; ++q) {
    const int col = v + 1 + q;
    T z[D];
    LeafBound<T, D, M - D, false> nob(W, nullptr, Rad<T>(0));
    leaf_column<T, M, D, CS>(As, col, W, idx, alpha, z, zmax, nob);
    const unsigned long long rk_col = rank_prefix + rank_part(binom, bs, n, col, 1);
    T colsum = T(0), colabs = T(0);
    if constexpr (D == 2) {
      for (int q2 = sub; q2 < q; q2 += lp) {
        T y[2];
        zb.get(q2, y);
        const T d = det2(y, z);
        emit(d, rk_col + rank_part(binom, bs, n, v + 1 + q2, 2));
        leaf_add(d, colsum, colabs);
      }
    } else {
      for (int q2 = sub; q2 < q; q2 += lp) {
        T y2[3], w[3];
        zb.get(q2, y2);
        cross3(y2, z, w);
        const unsigned long long rk2 = rk_col + rank_part(binom, bs, n, v + 1 + q2, 2);
        for (int q1 = 0; q1 < q2; ++q1) {
          T y1[3];
          zb.get(q1, y1);
          const T d = dot3(y1, w);
          emit(d, rk2 + rank_part(binom, bs, n, v + 1 + q1, 3));
          leaf_add(d, colsum, colabs);
        }
      }
    }
    zb.put(q, z);
    if (act) acc.add_column(colsum, colabs);
  }
}

// Leaf phase of one factored prefix c[0..m-D-1] (last column v): reduces
// every later column to its D-entry Schur complement and forms the D x D
// leaf determinants with the sign of Eq. (1), adding them to acc.pre (the
// caller commits or drops them).  D = 2: det = z1[0] z2[1] - z1[1] z2[0].
// D = 3: det = z1 . (z2 x z3), the cross product formed once per pair.
// `zb` is this lane's column buffer.  Returns the growth flag of the mixed
// mode: largest prefix pivot, or 2^(D-1) max|z| (a bound for the last D
// pivots under partial pivoting), above `thr`, or a non-finite scale.
// Binary64 slow path for a prefix whose enclosure reached zero (a pivot
// indistinguishable from zero): every minor of its subtree is factored on its
// own (lu_det_local: partial pivoting over the whole minor, with its own
// bound).  This lane takes the minors whose middle leaf column (D = 3) or
// first leaf column (D = 2), counted from v+1, is congruent to sub mod lp.
template <int M, int D, int CS>
__device__ __noinline__ void prefix_minors_f64(const double* __restrict__ As, const int (&c)[M - D], int v, int n,
                                               int sub, int lp, PrefixAcc<double>& acc) {
  constexpr int P = M - D;
  const int k = n - 1 - v;
  if (k < D) return;
  int cols[M];
#pragma unroll
  for (int j = 0; j < P; ++j) cols[j] = c[j];
  int q[D];
#pragma unroll
  for (int d = 0; d < D; ++d) q[d] = d;
  for (;;) {
    const int key = (D == 3) ? q[1] : q[0];
    if (key % lp == sub) {
#pragma unroll
      for (int d = 0; d < D; ++d) cols[P + d] = v + 1 + q[d];
      double a[M * M], b;
      for (int j = 0; j < M; ++j)
        for (int i = 0; i < M; ++i) a[i * M + j] = As[cols[j] * CS + i];
      double det = lu_det_local<M>(a, M, &b);
      if (sign_negative<M>(cols)) det = -det;
      acc.add_column(det, fabs(det));
      acc.add_bound(b);
    }
    int pos = D - 1;
    while (pos >= 0 && q[pos] == k - D + pos) --pos;
    if (pos < 0) break;
    ++q[pos];
    for (int j = pos + 1; j < D; ++j) q[j] = q[j - 1] + 1;
  }
}

template <typename T, int M, int D, int CS, bool kTerms, bool kRedo = true>
__device__ __forceinline__ bool prefix_leaves(const T* __restrict__ As, const uint64_t* binom, int n, int v,
                                              const int (&c)[M - D], const T (&W)[D][M - D], const int (&idx)[M],
                                              T prod, T gmax, bool neg, const ZBuf<T, D>& zb, T thr, bool act,
                                              int sub, int lp, PrefixAcc<T>& acc, const TermsSink& ts,
                                              const PrefixErr<Rad<T>>& pe = PrefixErr<Rad<T>>{},
                                              const Rad<T> (*rW)[M - D] = nullptr, float uin = 0.0f) {
  using R = Rad<T>;
  using B = BoundTraits<T>;
  constexpr bool kB = !kTerms;
  constexpr int P = M - D;
  // parity of r = M(M+1)/2, of the prefix columns' share of s, and of the D
  // leaf columns' "+1" terms; the leaf columns' own parities are folded in
  // per column
  int sp = M * (M + 1) / 2 + D;
#pragma unroll
  for (int j = 0; j < P; ++j) sp += c[j] + 1;
  const T alpha = ((sp & 1) != neg) ? -prod : prod;
  T zmax = T(0);
  const int k = n - 1 - v;
  LeafBound<T, D, P, kB> lb(W, rW, uin);
  // binary64 without a redo pass: a prefix whose enclosure failed takes the
  // per-minor slow path after the warp's leaf phase (its leaves there are
  // formed but not added)
  constexpr bool kSlow = kB && !kRedo && std::is_same<T, double>::value;
  const bool slow = kSlow && pe.bad;
  const bool act_in = act;
  act = act && !slow;
  if constexpr (kTerms) {
    unsigned long long rank_prefix = 0;
#pragma unroll
    for (int j = 0; j < P; ++j) rank_prefix += rank_part(binom, M + 1, n, c[j], M - j);
    // modes that redo flagged prefixes mark every term of one with NaN: the
    // growth flag needs max |z| over all of the prefix's columns first
    bool nan_out = false;
    if constexpr (kRedo) {
      T zm = T(0);
      for (int q = 0; q < k; ++q) {
        T z[D];
        LeafBound<T, D, P, false> nob(W, nullptr, R(0));
        leaf_column<T, M, D, CS>(As, v + 1 + q, W, idx, alpha, z, zm, nob);
      }
      nan_out = !(gmax <= thr) || !((D == 2 ? T(2) : T(4)) * zm <= thr) || !(fabs(alpha) <= static_cast<T>(FLT_MAX));
    }
    prefix_leaves_terms<T, M, D, CS>(As, binom, n, v, k, W, idx, alpha, rank_prefix, zb, act, sub, lp, acc, zmax,
                                     ts, nan_out);
  } else {
    if constexpr (D == 3) {
      // Two phases.  The lp lanes sharing the prefix split its column
      // reductions: lane `sub` reduces the columns q = sub (mod lp) into the
      // group's buffer (the slots of the group's first lane); then each lane
      // forms its share of the leaves from all of them (W and the row order
      // are no longer live there).  Every lane ends with the group's largest
      // |z| for the growth flag, and the symmetric sums of the bound over all
      // of the group's columns.
      const ZBuf<T, D> zg = zb.shifted(-sub);
      for (int q = sub; q < k; q += lp) {
        T z[D];
        leaf_column<T, M, D, CS>(As, v + 1 + q, W, idx, alpha, z, zmax, lb);
        zg.put(q, z);
      }
      zmax = group_max(zmax, lp);
      group_combine(lb.poly, lp);
      __syncwarp();
      prefix_leaves_blocked<T, M, D, CS, true>(As, v, k, W, idx, alpha, zg, act, sub, lp, acc, zmax, lb);
      __syncwarp();  // the buffer is rewritten by the group's next prefix
    } else {
      prefix_leaves_blocked<T, M, D, CS, false>(As, v, k, W, idx, alpha, zb, act, sub, lp, acc, zmax, lb);
    }
  }
  bool bad = false;
  if constexpr (kB) {
    // this lane's share of the prefix's bound (radic_bound.cuh)
    R b = (pe.rel_alpha + B::u * leaf_sum_depth(D, k, leaf_block<T>())) * lb.pabs;
    if (sub == 0)
      b += mag(alpha) * (R(1) + pe.rel_alpha) *
           (lb.poly.perturbation() + R(leaf_round_coef<D>()) * B::u * lb.poly.hadamard());
    if (act) acc.add_bound(b);
    if constexpr (kSlow) {
      if (slow && act_in) prefix_minors_f64<M, D, CS>(As, c, v, n, sub, lp, acc);
    } else if (pe.bad) {
      bad = true;  // the caller redoes the prefix in binary64
    }
  }
  const T growth_bound = (D == 2 ? T(2) : T(4)) * zmax;
  return bad || !(gmax <= thr) || !(growth_bound <= thr) || !(fabs(alpha) <= static_cast<T>(FLT_MAX));
}

// Pairs of binary32 factor their prefixes in binary64 (the FP64 pipe, a
// small share of the work once amortised over the leaves): its radii are
// those of binary64 arithmetic, far below what the same elimination in pairs
// would carry, and the conversion of W, the pivot product and the growth
// measure to pairs (split_to_pair, on the integer and binary32 pipes) adds
// 2^-47 relative.
template <int D, int P>
__device__ __forceinline__ void prefix_to_pairs(const double (&Wd)[D][P], float (&rW)[D][P], double prodd, double gmaxd,
                                                float& rel, ff (&W)[D][P], ff& prod, ff& gmax) {
#pragma unroll
  for (int d = 0; d < D; ++d)
#pragma unroll
    for (int j = 0; j < P; ++j) {
      W[d][j] = split_to_pair(Wd[d][j]);
      rW[d][j] += 0x1p-47f * mag(W[d][j]);
    }
  prod = split_to_pair(prodd);
  gmax = split_to_pair(gmaxd);
  rel = fmaf(1.0f + rel, 0x1p-47f, rel);
}

// Processes one prefix c[0..m-D-1] (last column v): factors it, then its
// leaves (prefix_leaves).
template <typename T, int M, int D, int CS, bool kTerms, bool kRedo = true>
__device__ __forceinline__ bool prefix_one(const T* __restrict__ As, const uint64_t* binom, int n, int v,
                                           const int (&c)[M - D], const ZBuf<T, D>& zb, T thr, bool act, int sub,
                                           int lp, PrefixAcc<T>& acc, const TermsSink& ts,
                                           float uin = BoundTraits<T>::u_in,
                                           const double* As64 = nullptr) {
  constexpr int P = M - D;
  T W[D][P];
  int idx[M];
  T prod, gmax;
  bool neg;
  if constexpr (kTerms) {
    prefix_factor<T, M, D, CS>(As, c, W, idx, prod, gmax, neg);
    return prefix_leaves<T, M, D, CS, kTerms, kRedo>(As, binom, n, v, c, W, idx, prod, gmax, neg, zb, thr, act, sub,
                                                     lp, acc, ts);
  } else {
    Rad<T> rW[D][P];
    PrefixErr<Rad<T>> pe;
    if constexpr (std::is_same<T, ff>::value) {
      double Wd[D][P], prodd, gmaxd;
      prefix_factor_b<double, M, D, ColStride<double, M>::value, double>(As64, c, Wd, rW, idx, prodd, gmaxd, neg,
                                                                          pe.rel_alpha, pe.bad, uin);
      prefix_to_pairs<D, P>(Wd, rW, prodd, gmaxd, pe.rel_alpha, W, prod, gmax);
    } else {
      prefix_factor_b<T, M, D, CS>(As, c, W, rW, idx, prod, gmax, neg, pe.rel_alpha, pe.bad, uin);
    }
    pe.kappa = 0.0f;
    return prefix_leaves<T, M, D, CS, kTerms, kRedo>(As, binom, n, v, c, W, idx, prod, gmax, neg, zb, thr, act, sub,
                                                     lp, acc, ts, pe, rW, uin);
  }
}

// Head sharing: the prefixes whose first H = m-D-1 columns (the head) agree
// share those H elimination steps.  The head is factored once with
// prefix_factor at depth D+1 (W1 = -L21 L11^{-1} for the D+1 rows left);
// appending the prefix's last column v then costs one more elimination step:
// s = the D+1 Schur-complement entries of column v, partial pivoting among
// them by the same compare-and-swap rule, and with l_d = s_{d+1} / s_0
//   W[d][j] = W1[d+1][j] - l_d W1[0][j]  (j < H),   W[d][H] = -l_d.
// Same pivots and elimination steps as factoring the prefix from scratch.
template <typename T, int M, int D, int CS>
__device__ __forceinline__ void prefix_extend(const T* __restrict__ As, int v, const T (&W1)[D + 1][M - D - 1],
                                              const int (&idx1)[M], T prod1, T gmax1, bool neg1, T (&W)[D][M - D],
                                              int (&idx)[M], T& prod, T& gmax, bool& neg) {
  constexpr int H = M - D - 1;
  T s[D + 1];
  prefix_column<T, M, D + 1>(As + v * CS, W1, idx1, s);
  T Wr[D + 1][H];
  int ir[D + 1];
#pragma unroll
  for (int r = 0; r <= D; ++r) {
    ir[r] = idx1[H + r];
#pragma unroll
    for (int j = 0; j < H; ++j) Wr[r][j] = W1[r][j];
  }
  bool ng = neg1;
#pragma unroll
  for (int r = 1; r <= D; ++r) {
    const bool sw = abs_greater(s[r], s[0]);
    const T a0 = s[0], ar = s[r];
    s[0] = sw ? ar : a0;
    s[r] = sw ? a0 : ar;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const T x = Wr[0][j], y = Wr[r][j];
      Wr[0][j] = sw ? y : x;
      Wr[r][j] = sw ? x : y;
    }
    const int i0 = ir[0], irr = ir[r];
    ir[0] = sw ? irr : i0;
    ir[r] = sw ? i0 : irr;
    ng ^= sw;
  }
  const T piv = s[0];
  const T rr = rcp_t(piv);
  prod = prod1 * piv;
  gmax = fmax(gmax1, fabs(piv));
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const T l = s[d + 1] * rr;
#pragma unroll
    for (int j = 0; j < H; ++j) W[d][j] = fma(-l, Wr[0][j], Wr[d + 1][j]);
    W[d][H] = -l;
  }
#pragma unroll
  for (int j = 0; j < H; ++j) idx[j] = idx1[j];
#pragma unroll
  for (int r = 0; r <= D; ++r) idx[H + r] = ir[r];
  neg = ng;
}

// Radii of the D+1 Schur-complement entries of any column x against a
// factored head (W1, rW1): |s_r - s^_r| <= k1[r] ||x||_2 (kappa_of, per row;
// S: the staging type of x).
template <typename T, int Dp1, int H, typename S = T>
__device__ __forceinline__ void head_kappas(const T (&W1)[Dp1][H], const Rad<T> (&rW1)[Dp1][H], Rad<T> (&k1)[Dp1],
                                            float uin = BoundTraits<S>::u_in) {
  using R = Rad<T>;
  constexpr R kU = BoundTraits<T>::u;
  const R kUin = uin;
#pragma unroll
  for (int r = 0; r < Dp1; ++r) {
    R w2 = R(0), r2 = R(0);
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const R w = mag(W1[r][j]);
      w2 += w * w;
      r2 += rW1[r][j] * rW1[r][j];
    }
    k1[r] = (sqrt(r2) * (R(1) + kUin) + (R(H) * kU + kUin) * (R(1) + sqrt(w2))) * R(1.0001);
  }
}

// prefix_extend with running error radii: the elimination step that appends
// column v to a factored head, with the radii of W, of the pivot product and
// the pivot condition.  k1: head_kappas of the head; xnorm = ||A[:, v]||_2.
template <typename T, int M, int D, int CS, typename S = T>
__device__ __forceinline__ void prefix_extend_b(const S* __restrict__ As, int v, Rad<T> xnorm,
                                                const T (&W1)[D + 1][M - D - 1],
                                                const Rad<T> (&rW1)[D + 1][M - D - 1], const Rad<T> (&k1)[D + 1],
                                                const int (&idx1)[M], T prod1, T gmax1, bool neg1, Rad<T> rel1,
                                                bool bad1, T (&W)[D][M - D], Rad<T> (&rW)[D][M - D], int (&idx)[M],
                                                T& prod, T& gmax, bool& neg, Rad<T>& rel_alpha, bool& bad) {
  using R = Rad<T>;
  using B = BoundTraits<T>;
  constexpr int H = M - D - 1;
  T s[D + 1];
  prefix_column<T, M, D + 1, S>(As + v * CS, W1, idx1, s);
  R rs[D + 1];
#pragma unroll
  for (int r = 0; r <= D; ++r) rs[r] = k1[r] * xnorm;
  T Wr[D + 1][H];
  R rWr[D + 1][H];
  int ir[D + 1];
#pragma unroll
  for (int r = 0; r <= D; ++r) {
    ir[r] = idx1[H + r];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      Wr[r][j] = W1[r][j];
      rWr[r][j] = rW1[r][j];
    }
  }
  bool ng = neg1;
#pragma unroll
  for (int r = 1; r <= D; ++r) {
    const bool sw = abs_greater(s[r], s[0]);
    const T a0 = s[0], ar = s[r];
    s[0] = sw ? ar : a0;
    s[r] = sw ? a0 : ar;
    const R q0 = rs[0], qr = rs[r];
    rs[0] = sw ? qr : q0;
    rs[r] = sw ? q0 : qr;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const T x = Wr[0][j], y = Wr[r][j];
      Wr[0][j] = sw ? y : x;
      Wr[r][j] = sw ? x : y;
      const R rx = rWr[0][j], ry = rWr[r][j];
      rWr[0][j] = sw ? ry : rx;
      rWr[r][j] = sw ? rx : ry;
    }
    const int i0 = ir[0], irr = ir[r];
    ir[0] = sw ? irr : i0;
    ir[r] = sw ? i0 : irr;
    ng ^= sw;
  }
  const T piv = s[0];
  const R ap = mag(piv), rp = rs[0];
  bad = bad1 || pivot_unbounded(ap, rp);
  const R ipm = ap > R(0) ? rcp_rad(ap) : R(0);
  const R ipd = ap > rp ? rcp_rad(__fsub_rd(ap, rp)) : R(0);
  rel_alpha = fmaf(R(1) + rel1, fmaf(R(1) + rp * ipm, B::u * R(1.01), rp * ipm), rel1);
  const T rr = rcp_t(piv);
  prod = prod1 * piv;
  gmax = fmax(gmax1, fabs(piv));
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const T l = s[d + 1] * rr;
    const R al = mag(l);
    const R rl = (rs[d + 1] + al * rp) * ipd + B::c_div * B::u * al;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const R aw0 = mag(Wr[0][j]), awd = mag(Wr[d + 1][j]);
      W[d][j] = fma(-l, Wr[0][j], Wr[d + 1][j]);
      rW[d][j] = rWr[d + 1][j] + al * rWr[0][j] + (aw0 + rWr[0][j]) * rl + B::u * (al * aw0 + awd);
    }
    W[d][H] = -l;
    rW[d][H] = rl;
  }
#pragma unroll
  for (int j = 0; j < H; ++j) idx[j] = idx1[j];
#pragma unroll
  for (int r = 0; r <= D; ++r) idx[H + r] = ir[r];
  neg = ng;
}

// prefix_extend_b for pairs of binary32 from a binary64 head: the Schur
// complement s of column v, the pivot and the multipliers l are formed in
// binary64 (their radii are divided by the pivot, so they need its
// precision); the update W[d][j] = W1[d+1][j] - l_d W1[0][j] runs in pairs on
// the binary32 pipe, on the pairs nearest to W1 and l (split_to_pair, 2^-47
// relative, added to their radii), with the pair rounding of BoundTraits<ff>.
template <int M, int D, int CS>
__device__ __forceinline__ void prefix_extend_pair(const double* __restrict__ As, int v, float xnorm,
                                                   const double (&W1)[D + 1][M - D - 1],
                                                   const float (&rW1)[D + 1][M - D - 1], const float (&k1)[D + 1],
                                                   const int (&idx1)[M], double prod1, double gmax1, bool neg1,
                                                   float rel1, bool bad1, ff (&W)[D][M - D], float (&rW)[D][M - D],
                                                   int (&idx)[M], ff& prod, ff& gmax, bool& neg, float& rel_alpha,
                                                   bool& bad) {
  using B64 = BoundTraits<double>;
  using BP = BoundTraits<ff>;
  constexpr int H = M - D - 1;
  constexpr float kSplit = 0x1p-47f;
  double s[D + 1];
  prefix_column<double, M, D + 1, double>(As + v * CS, W1, idx1, s);
  float rs[D + 1];
#pragma unroll
  for (int r = 0; r <= D; ++r) rs[r] = k1[r] * xnorm;
  double Wr[D + 1][H];
  float rWr[D + 1][H];
  int ir[D + 1];
#pragma unroll
  for (int r = 0; r <= D; ++r) {
    ir[r] = idx1[H + r];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      Wr[r][j] = W1[r][j];
      rWr[r][j] = rW1[r][j];
    }
  }
  bool ng = neg1;
#pragma unroll
  for (int r = 1; r <= D; ++r) {
    const bool sw = abs_greater(s[r], s[0]);
    const double a0 = s[0], ar = s[r];
    s[0] = sw ? ar : a0;
    s[r] = sw ? a0 : ar;
    const float q0 = rs[0], qr = rs[r];
    rs[0] = sw ? qr : q0;
    rs[r] = sw ? q0 : qr;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const double x = Wr[0][j], y = Wr[r][j];
      Wr[0][j] = sw ? y : x;
      Wr[r][j] = sw ? x : y;
      const float rx = rWr[0][j], ry = rWr[r][j];
      rWr[0][j] = sw ? ry : rx;
      rWr[r][j] = sw ? rx : ry;
    }
    const int i0 = ir[0], irr = ir[r];
    ir[0] = sw ? irr : i0;
    ir[r] = sw ? i0 : irr;
    ng ^= sw;
  }
  const double piv = s[0];
  const float ap = mag(piv), rp = rs[0];
  bad = bad1 || pivot_unbounded(ap, rp);
  const float ipm = ap > 0.0f ? rcp_rad(ap) : 0.0f;
  const float ipd = ap > rp ? rcp_rad(__fsub_rd(ap, rp)) : 0.0f;
  rel_alpha = fmaf(1.0f + rel1, fmaf(1.0f + rp * ipm, B64::u * 1.01f, rp * ipm), rel1);
  const double rr = rcp_t(piv);
  prod = split_to_pair(prod1 * piv);
  gmax = split_to_pair(fmax(gmax1, fabs(piv)));
  rel_alpha = fmaf(1.0f + rel_alpha, kSplit, rel_alpha);
  // the pivot row in pairs, shared by the D updates
  ff w0[H];
  float aw0[H], rw0[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    w0[j] = split_to_pair(Wr[0][j]);
    aw0[j] = mag(w0[j]);
    rw0[j] = fmaf(kSplit, aw0[j], rWr[0][j]);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const ff lp = split_to_pair(s[d + 1] * rr);
    const float al = mag(lp);
    const float rl = (rs[d + 1] + al * rp) * ipd + (B64::c_div * B64::u + kSplit) * al;
    const ff nl = -lp;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const ff wd = split_to_pair(Wr[d + 1][j]);
      const float awd = mag(wd);
      W[d][j] = fma(nl, w0[j], wd);
      rW[d][j] = fmaf(kSplit, awd, rWr[d + 1][j]) + al * rw0[j] + (aw0[j] + rw0[j]) * rl + BP::u * (al * aw0[j] + awd);
    }
    W[d][H] = nl;
    rW[d][H] = rl;
  }
#pragma unroll
  for (int j = 0; j < H; ++j) idx[j] = idx1[j];
#pragma unroll
  for (int r = 0; r <= D; ++r) idx[H + r] = ir[r];
  neg = ng;
}

// ---------------------------------------------------------------------------
// Single-matrix prefix kernel.
// ---------------------------------------------------------------------------
// Minimum resident blocks per SM the compiler must allow for (register cap)
// of the binary32 and pair prefix kernels.  Binary32: three blocks of 128
// threads (168 registers, a few spilled bytes) rather than the 254 registers
// the error-bound code takes unconstrained, which leave room for two.
#ifndef RADIC_PREFIX_MIN_BLOCKS_F32
#define RADIC_PREFIX_MIN_BLOCKS_F32 3
#endif
#ifndef RADIC_PREFIX_MIN_BLOCKS_FF
#define RADIC_PREFIX_MIN_BLOCKS_FF 1
#endif
template <typename T>
__host__ __device__ constexpr int prefix_min_blocks() {
  return std::is_same<T, float>::value ? RADIC_PREFIX_MIN_BLOCKS_F32
                                       : (std::is_same<T, ff>::value ? RADIC_PREFIX_MIN_BLOCKS_FF : 1);
}

template <typename T, int M, int D, bool kMixed, bool kTerms>
__global__ void __launch_bounds__(128, prefix_min_blocks<T>()) k_fp_prefix(SingleArgs a, PrefixTable tab) {
  static_assert(M > D, "the prefix needs at least one column");
  constexpr int P = M - D;
  constexpr int CS = ColStride<T, M>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n;
  FpSmem<T> sm(smem_raw, n, M, CS);
  const ZBuf<T, D> zb(smem_raw + fp_smem_bytes(n, M, CS, sizeof(T), blockDim.x, std::is_same<T, ff>::value),
                      threadIdx.x, blockDim.x, n - M + D);
  build_binom(sm.binom, n, M);
  bool exact_in;
  const int escale = stage_scaled<T>(a.A, a.dtype, M, n, a.lda, sm.As, CS, sm.row_exp, &exact_in);
  const float uin = exact_in ? 0.0f : static_cast<float>(BoundTraits<T>::u_in);
  if constexpr (!kTerms && std::is_same<T, ff>::value) {
    stage_double_copy(sm.As, CS, M, n, sm.As64, ColStride<double, M>::value, threadIdx.x, blockDim.x);
    __syncthreads();
  }

  const int lane = threadIdx.x & 31;
  const unsigned long long gwarp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * blockDim.x / 32;
  const T thr = static_cast<T>(a.growth);
  const int bs = M + 1;  // binomial table stride

  PrefixAcc<T> acc;
  int fcnt = 0;
  unsigned long long* flist = nullptr;
  if constexpr (kMixed && !kTerms) flist = a.flag_ranks + gwarp * (unsigned long long)a.flag_cap;
  TermsSink ts{static_cast<double*>(a.terms), a.q0, a.count, sm.binom[n * bs + M], escale};

  // Tasks are numbered heaviest group first (ascending v: the most candidate
  // columns).  A warp's first task is its own index; each later one comes
  // from a counter in the workspace header, fetched while the current task
  // runs, so that warps that drew light tasks take more of them.  The
  // per-term launches (no workspace) and deterministic plans stride by the
  // number of warps instead.
  // A warp's task numbers only grow, so its group search resumes where the
  // previous task's ended.
  unsigned long long t = gwarp;
  int v = tab.v_lo;
  while (t < tab.total_tasks) {
    unsigned long long t_next = t + nwarps;
    if constexpr (!kTerms) {
      if (tab.dynamic && lane == 0) t_next = nwarps + atomicAdd(&a.hdr->next_task, 1ull);
    }
    while (v < tab.v_hi && t >= tab.task_start[v + 1]) ++v;
    const unsigned long long runlen = tab.run[v], cnt = tab.count[v];
    // lanes [grp * lp, grp * lp + lp) share each prefix of one run
    const int lp = tab.lanes[v], grp = lane / lp, sub = lane - grp * lp;
    const unsigned long long groups = 32 / lp;
    const unsigned long long r0 = (t - tab.task_start[v]) * groups * runlen + (unsigned long long)grp * runlen;
    const unsigned long long r1 = min(r0 + runlen, cnt);
    constexpr int H = P > 1 ? P - 1 : 1;
    int head[H];  // first P-1 prefix columns, a (P-1)-subset of {0..v-1}
    if constexpr (P > 1) unrank<P - 1>(r0 < cnt ? r0 : 0ull, v, sm.binom, bs, head);
    for (unsigned long long it = 0; it < runlen; ++it) {
      const bool act = r0 + it < r1;
      int c[P];
#pragma unroll
      for (int j = 0; j < P - 1; ++j) c[j] = head[j];
      c[P - 1] = v;
      const bool flag = prefix_one<T, M, D, CS, kTerms, kMixed>(sm.As, sm.binom, n, v, c, zb, thr, act, sub, lp, acc,
                                                                 ts, uin, sm.As64);
      if constexpr (kMixed && !kTerms) {
        if (act && flag) acc.drop_prefix();  // its leaves are recomputed in binary64
        // every lane of the group drops its share; the first one records the prefix
        const unsigned fm = __ballot_sync(kFull, act && flag && sub == 0);
        if (fm) {
          if (act && flag && sub == 0) {
            const int pos = fcnt + __popc(fm & ((1u << lane) - 1u));
            // record the prefix by its rank among all P-subsets of {0..n-1}
            unsigned long long rp = sm.binom[n * bs + P] - 1;
#pragma unroll
            for (int j = 0; j < P; ++j) rp -= rank_part(sm.binom, bs, n, c[j], P - j);
            if (pos < a.flag_cap) flist[pos] = rp;
          }
          fcnt += __popc(fm);
        }
      }
      acc.end_prefix();
      if constexpr (P > 1) {
        if (r0 + it + 1 < r1) successor<P - 1>(head, v);
      }
    }
    t = (kTerms || !tab.dynamic) ? t_next : __shfl_sync(kFull, t_next, 0);
  }
  if constexpr (!kTerms) {
    long long fl = 0;
    if constexpr (kMixed) {
      if (lane == 0) {
        a.flag_count[gwarp] = fcnt;
        if (fcnt > a.flag_cap) atomicOr(&a.hdr->overflow, 1);
        fl = fcnt;
      }
    }
    if constexpr (std::is_same<T, float>::value) {
      double bnd = static_cast<double>(acc.bnd);
      block_reduce_ff(acc.tot, acc.tot_abs, fl, bnd, sm.scratch);
      if (threadIdx.x == 0)
        reinterpret_cast<FfPartial*>(a.partials)[blockIdx.x] =
            FfPartial{acc.tot.hi, acc.tot.lo, acc.tot_abs.hi, acc.tot_abs.lo, fl, bnd, {0, 0}};
      finish_ff_main(a, sm.scratch, escale, M);
    } else {
      acc.finish();
      Dd d = acc.acc;
      double ab = acc.abs_sum;
      double bnd = static_cast<double>(acc.bnd);
      block_reduce_dd(d, ab, fl, bnd, sm.scratch);
      if (threadIdx.x == 0) a.partials[blockIdx.x] = FpPartial{d.hi, d.lo, ab, fl, bnd, 0.0};
      finish_fp_main<kMixed>(a, sm.scratch, escale, M, tier_of<T, kMixed>());
    }
  }
}

}  // namespace radic
