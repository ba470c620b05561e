// Device building blocks shared by the Radic-determinant kernels (sm_103a).
//
// Notation follows arXiv 1508.01326: an m x n matrix A, column sequences
// J = (j1 < ... < jm) numbered 0 .. C(n,m)-1 in dictionary order (Definition
// 2), the sign (-1)^(r+s) of Eq. (1), and the binomial table of Section 4.
// All column indices here are 0-based.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <type_traits>

#include "radic_internal.h"
#include "radic_bound.cuh"
#include "radic_ff.cuh"

namespace radic {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Binomial table (Section 4, Table 1 / Fig. 1): C(v, k) for 0 <= v, k <= 64.
// The table is generated at compile time by the Pascal recurrence (every
// entry is the sum of the two entries above it) and lives in global memory
// (read-only): the lanes of a warp read different entries, which the constant
// cache would serialise.  Each block copies the (n+1) x (kmax+1) part it needs
// into shared memory as binom[v * (kmax + 1) + k] with one barrier.
// ---------------------------------------------------------------------------
struct BinomConst {
  unsigned long long v[kMaxN + 1][kMaxN + 1];
};

constexpr BinomConst make_binom_const() {
  BinomConst t{};
  for (int v = 0; v <= kMaxN; ++v) {
    t.v[v][0] = 1ull;
    for (int k = 1; k <= kMaxN; ++k) t.v[v][k] = (v == 0) ? 0ull : t.v[v - 1][k - 1] + t.v[v - 1][k];
  }
  return t;
}

static __device__ const BinomConst c_binom = make_binom_const();

__device__ inline void build_binom(uint64_t* binom, int n, int kmax) {
  const int stride = kmax + 1;
  for (int idx = threadIdx.x; idx < (n + 1) * stride; idx += blockDim.x) {
    const int v = idx / stride, k = idx - v * stride;
    binom[idx] = __ldg(&c_binom.v[v][k]);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Unranking.  The paper's "combinatorial addition" (Section 4) walks left in
// the Pascal table; the same map is reached in closed form through the
// combinatorial number system: with r = C(n,m) - 1 - q, position i takes the
// largest v with C(v, m-i) <= r, sets j_i = n - 1 - v and subtracts C(v, m-i).
// ---------------------------------------------------------------------------
// k! in binary32 (exact up to k = 13; k <= 34 stays finite).
__host__ __device__ constexpr float fact_f(int k) {
  float f = 1.0f;
  for (int j = 2; j <= k; ++j) f *= static_cast<float>(j);
  return f;
}

// Largest w <= v - 1 with C(w, k) <= r.  The search starts at the estimate
// w ~ (k! r)^(1/k) + (k-1)/2 (from C(w, k) ~ (w - (k-1)/2)^k / k!, which the
// AM-GM inequality shows is an upper bound) and then steps through the
// table to the exact value, so that the estimate only sets the number of
// steps (usually none or one) and never the result.  *b receives C(w, k).
template <int K>
__device__ __forceinline__ int unrank_pos(uint64_t r, int v, const uint64_t* binom, int bstride, uint64_t* b) {
  const float x = exp2f((__log2f(static_cast<float>(r)) + __log2f(fact_f(K))) * (1.0f / K)) + 0.5f * (K - 1);
  int w = static_cast<int>(fminf(x, static_cast<float>(v - 1)));  // r = 0 gives (k-1)/2
  w = max(w, K - 1);
  // both neighbours of the estimate in one round trip
  uint64_t bw = binom[w * bstride + K];
  uint64_t b1 = (w + 1 < v) ? binom[(w + 1) * bstride + K] : 0ull;
  if (bw > r) {
    do {  // C(k-1, k) = 0 ends this
      --w;
      bw = binom[w * bstride + K];
    } while (bw > r);
  } else {
    while (w + 1 < v && b1 <= r) {
      ++w;
      bw = b1;
      if (w + 1 < v) b1 = binom[(w + 1) * bstride + K];
    }
  }
  *b = bw;
  return w;
}

template <int M, int I = 0>
__device__ __forceinline__ void unrank_from(uint64_t r, int v, int n, const uint64_t* binom, int bstride,
                                            int (&c)[M]) {
  if constexpr (I < M) {
    uint64_t b;
    const int w = unrank_pos<M - I>(r, v, binom, bstride, &b);
    c[I] = n - 1 - w;
    unrank_from<M, I + 1>(r - b, w, n, binom, bstride, c);
  }
}

template <int M>
__device__ __forceinline__ void unrank(uint64_t q, int n, const uint64_t* binom, int bstride,
                                       int (&c)[M]) {
  unrank_from<M>(binom[n * bstride + M] - 1 - q, n, n, binom, bstride, c);
}

// Dynamic-m form for the group mapping (c has capacity G >= m).
template <int G>
__device__ __forceinline__ void unrank_dyn(uint64_t q, int n, int m, const uint64_t* binom,
                                           int bstride, int (&c)[G]) {
  uint64_t r = binom[n * bstride + m] - 1 - q;
  int v = n;
#pragma unroll
  for (int i = 0; i < G; ++i) {
    if (i < m) {
      const int k = m - i;
      int w = v - 1;
      uint64_t b = binom[w * bstride + k];
      while (b > r) {
        --w;
        b = binom[w * bstride + k];
      }
      c[i] = n - 1 - w;
      r -= b;
      v = w;
    }
  }
}

// Dictionary successor (Section 5, "dictionary sequence"): the rightmost
// position below its maximum n-m+i moves up by one and the positions after it
// follow consecutively.  Must not be called on the last sequence.
template <int M>
__device__ __forceinline__ void successor(int (&c)[M], int n) {
  int pos = 0;
#pragma unroll
  for (int t = 0; t < M; ++t)
    if (c[t] < n - M + t) pos = t;
#pragma unroll
  for (int t = 0; t < M; ++t) {
    if (t == pos) c[t] += 1;
    if (t > 0 && t > pos) c[t] = c[t - 1] + 1;
  }
}

template <int G>
__device__ __forceinline__ void successor_dyn(int (&c)[G], int n, int m) {
  int pos = 0;
#pragma unroll
  for (int t = 0; t < G; ++t)
    if (t < m && c[t] < n - m + t) pos = t;
#pragma unroll
  for (int t = 0; t < G; ++t) {
    if (t == pos) c[t] += 1;
    if (t > 0 && t > pos && t < m) c[t] = c[t - 1] + 1;
  }
}

// (-1)^(r+s) of Eq. (1): r = m(m+1)/2 and s = sum of the 1-based indices,
// i.e. sum(c_i + 1).  Returns true when the sign is negative.
template <int M>
__device__ __forceinline__ bool sign_negative(const int (&c)[M]) {
  int s = M * (M + 1) / 2 + M;
#pragma unroll
  for (int t = 0; t < M; ++t) s += c[t];
  return s & 1;
}

template <int G>
__device__ __forceinline__ bool sign_negative_dyn(const int (&c)[G], int m) {
  int s = m * (m + 1) / 2 + m;
#pragma unroll
  for (int t = 0; t < G; ++t)
    if (t < m) s += c[t];
  return s & 1;
}

// ---------------------------------------------------------------------------
// Reciprocals; a zero pivot gives 0 so that the elimination of an all-zero
// column stays finite.  Binary64: the hardware approximation refined by two
// Newton-Raphson iterations x <- x + x (1 - d x) (quadratic convergence).
// Binary32: the hardware approximation alone, not refined (the PTX ISA
// states at most one unit in the last place for rcp.approx.f32); the error
// bounds of the binary32 path count a multiplier formed with it as three
// binary32 roundings.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_f32(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return d == 0.0f ? 0.0f : r;
}

__device__ __forceinline__ double rcp_f64(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  return d == 0.0 ? 0.0 : r;
}

__device__ __forceinline__ float rcp_t(float d) { return rcp_f32(d); }
__device__ __forceinline__ double rcp_t(double d) { return rcp_f64(d); }

// Magnitude keys for pivot comparisons that stay off the FP64 pipe: the high
// word of |x| orders binary64 magnitudes up to ties within 2^-20.
__device__ __forceinline__ uint32_t mag_key(double x) {
  return static_cast<uint32_t>(__double2hiint(x)) & 0x7fffffffu;
}
__device__ __forceinline__ uint32_t mag_key(float x) { return __float_as_uint(x) & 0x7fffffffu; }

// |a| > |b| for pivot selection: binary64 by the magnitude keys, binary32
// directly, pairs by their leading parts.
__device__ __forceinline__ bool abs_greater(double a, double b) { return mag_key(a) > mag_key(b); }
__device__ __forceinline__ bool abs_greater(float a, float b) { return fabsf(a) > fabsf(b); }
__device__ __forceinline__ bool abs_greater(ff a, ff b) { return fabsf(a.hi) > fabsf(b.hi); }

// ---------------------------------------------------------------------------
// Partial-pivot LU of one m x m minor held in registers (thread mapping).
// Row exchanges are branch-free compare-and-swap steps that bubble the
// largest remaining |a_ik| into row k.  Returns det; `gmax` receives the
// largest pivot magnitude (growth check of the MIXED mode).
// ---------------------------------------------------------------------------
template <typename T, int M>
__device__ __forceinline__ T lu_det(T (&a)[M][M], T& gmax) {
  T det = T(1);
  bool neg = false;
  gmax = T(0);
#pragma unroll
  for (int k = 0; k < M - 1; ++k) {
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      const bool sw = mag_key(a[i][k]) > mag_key(a[k][k]);
#pragma unroll
      for (int j = k; j < M; ++j) {
        const T x = a[k][j], y = a[i][j];
        a[k][j] = sw ? y : x;
        a[i][j] = sw ? x : y;
      }
      neg ^= sw;
    }
    const T piv = a[k][k];
    T r;
    if constexpr (sizeof(T) == 8) r = rcp_f64(piv);
    else r = rcp_f32(piv);
    det *= piv;
    gmax = fmax(gmax, fabs(piv));
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      const T l = a[i][k] * r;
#pragma unroll
      for (int j = k + 1; j < M; ++j) a[i][j] = fma(-l, a[k][j], a[i][j]);
    }
  }
  det *= a[M - 1][M - 1];
  gmax = fmax(gmax, fabs(a[M - 1][M - 1]));
  return neg ? -det : det;
}

// lu_det with running error radii (radic_bound.cuh), kept in binary32 for
// both element types (registers: one radius per entry).  Returns the
// determinant; bnd receives an upper bound on its error and bad whether a
// pivot's enclosure reached zero (then bnd is not valid and the caller
// falls back to Hadamard's inequality or to binary64).  Binary32 radii do
// not represent values below 2^-126: for binary64 minors the bound does not
// cover entries below about 2^-70 of their row's largest one.
template <typename T, int M>
__device__ __forceinline__ T lu_det_b(T (&a)[M][M], T& gmax, float& bnd, bool& bad,
                                      float u_in = static_cast<float>(BoundTraits<T>::u_in)) {
  constexpr float u = static_cast<float>(BoundTraits<T>::u);
  constexpr float c_div = static_cast<float>(BoundTraits<T>::c_div);
  float ra[M][M];
#pragma unroll
  for (int i = 0; i < M; ++i)
#pragma unroll
    for (int j = 0; j < M; ++j) ra[i][j] = u_in * mag(a[i][j]);
  T det = T(1);
  bool neg = false;
  float rel = 0.0f;
  float hs = 0.0f;  // binary64: bound on |det| from the step where a pivot failed
  bad = false;
  gmax = T(0);
#pragma unroll
  for (int k = 0; k < M; ++k) {
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      const bool sw = mag_key(a[i][k]) > mag_key(a[k][k]);
#pragma unroll
      for (int j = k; j < M; ++j) {
        const T x = a[k][j], y = a[i][j];
        a[k][j] = sw ? y : x;
        a[i][j] = sw ? x : y;
        const float rx = ra[k][j], ry = ra[i][j];
        ra[k][j] = sw ? ry : rx;
        ra[i][j] = sw ? rx : ry;
      }
      neg ^= sw;
    }
    const T piv = a[k][k];
    const float ap = mag(piv), rp = ra[k][k];
    const float ipm = ap > 0.0f ? __frcp_ru(ap) : 0.0f;        // 1 / |p|
    const float ipd = ap > rp ? __frcp_ru(__fsub_rd(ap, rp)) : 0.0f;  // 1 / (|p| - r_p)
    if constexpr (sizeof(T) == 8) {
      if (k < M - 1 && !bad && pivot_unbounded(ap, rp)) {
        // det = prod_{kk<k} p_kk det(S), S the remaining Schur complement
        // with entries in [|s| - r, |s| + r]: Hadamard's inequality on the
        // enclosure of S (the factor covers the binary32 roundings here)
        float h = 1.0f + static_cast<float>(M * M + 4 * M) * 0x1p-23f;
#pragma unroll
        for (int kk = 0; kk < k; ++kk) h *= mag(a[kk][kk]) + ra[kk][kk];
#pragma unroll
        for (int j = k; j < M; ++j) {
          float c2 = 0.0f;
#pragma unroll
          for (int i = k; i < M; ++i) {
            const float e = mag(a[i][j]) + ra[i][j];
            c2 = fmaf(e, e, c2);
          }
          h *= sqrtf(c2);
        }
        hs = h;
      }
    }
    det *= piv;
    gmax = fmax(gmax, fabs(piv));
    if (k == M - 1) {
      if (bad) break;
      // the last pivot divides nothing: a singular minor is bounded by
      // prod (|p_k| + r_k) instead
      if (pivot_unbounded(ap, rp) || ap == 0.0f) {
        float pr = 1.0f;
#pragma unroll
        for (int kk = 0; kk < M - 1; ++kk) pr *= mag(a[kk][kk]) + ra[kk][kk];
        bnd = pr * (ap + rp) * (1.0f + static_cast<float>(M) * u) * 1.0000002f + static_cast<float>(M) * u *
              mag(det);
        return neg ? -det : det;
      }
      rel = fmaf(1.0f + rel, rp * ipm, rel);
      break;
    }
    bad |= pivot_unbounded(ap, rp);
    rel = fmaf(1.0f + rel, rp * ipm, rel);
    T r;
    if constexpr (sizeof(T) == 8) r = rcp_f64(piv);
    else r = rcp_f32(piv);
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      const T l = a[i][k] * r;
      const float al = mag(l);
      const float rl = (ra[i][k] + al * rp) * ipd + c_div * u * al;
#pragma unroll
      for (int j = k + 1; j < M; ++j) {
        const float ax = mag(a[k][j]), old = mag(a[i][j]);
        a[i][j] = fma(-l, a[k][j], a[i][j]);
        ra[i][j] += al * ra[k][j] + (ax + ra[k][j]) * rl + u * (al * ax + old);
      }
    }
  }
  rel = fmaf(1.0f + rel, static_cast<float>(M - 1) * u * 1.01f, rel);
  bnd = rel * mag(det) * 1.0000001f;
  // a failed pivot: |computed - exact| <= |computed| + |exact|, the latter
  // bounded above (binary64 only; the other arithmetics flag the minor)
  if (sizeof(T) == 8 && bad) bnd = mag(det) * 1.0000002f + hs;
  return neg ? -det : det;
}

// Partial-pivot LU of an m x m row-major binary64 matrix in local memory
// (m <= MC; the slow paths: binary64 redo of flagged minors, minors of a
// prefix whose enclosure failed), with running error radii in binary64
// (radic_bound.cuh; exact division, so a multiplier counts one rounding).
// *bnd receives an upper bound on the error of the determinant.  The last
// pivot divides nothing, so its enclosure may reach zero (a singular minor):
// then the product bound prod (|p_k| + r_k) is used.  When an earlier pivot
// p_K's enclosure reaches zero, det = prod_{k<K} p_k det(S) with S the
// remaining Schur complement, so |det| <= prod_{k<K} (|p_k| + r_k) times
// Hadamard's bound of S's enclosure, prod_j ||(|s_j| + r_j)||, and the error
// is at most that plus |computed det|.
template <int MC>
__device__ double lu_det_local(double (&a)[MC * MC], int m, double* bnd) {
  constexpr double u = 0x1p-53;
  double ra[MC * MC];
  for (int i = 0; i < m * MC; ++i) ra[i] = 0.0;
  double det = 1.0, rel = 0.0, pa = 1.0, pr = 1.0;  // pa = prod |p_k|, pr = prod (|p_k| + r_k)
  double hs = 0.0;                                   // bound on |det| once a pivot failed
  bool neg = false, bad = false, last_open = false;
  for (int k = 0; k < m; ++k) {
    int p = k;
    double best = fabs(a[k * MC + k]);
    for (int i = k + 1; i < m; ++i) {
      const double v = fabs(a[i * MC + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    if (p != k) {
      for (int j = 0; j < m; ++j) {
        const double t = a[k * MC + j];
        a[k * MC + j] = a[p * MC + j];
        a[p * MC + j] = t;
        const double tr = ra[k * MC + j];
        ra[k * MC + j] = ra[p * MC + j];
        ra[p * MC + j] = tr;
      }
      neg = !neg;
    }
    const double piv = a[k * MC + k], ap = fabs(piv), rp = ra[k * MC + k];
    if (k < m - 1 && !bad && pivot_unbounded(ap, rp)) {
      // Hadamard's bound of the remaining Schur complement's enclosure
      hs = pr;
      for (int j = k; j < m; ++j) {
        double c2 = 0.0;
        for (int i = k; i < m; ++i) {
          const double e = fabs(a[i * MC + j]) + ra[i * MC + j];
          c2 += e * e;
        }
        hs *= sqrt(c2) * (1.0 + 0x1p-50);
      }
      bad = true;
    }
    det *= piv;
    pa *= ap;
    pr *= ap + rp;
    if (k == m - 1) {
      last_open = pivot_unbounded(ap, rp);
      if (!last_open && ap > 0.0) rel = (1.0 + rel) * (rp / ap) + rel;
      break;
    }
    if (piv == 0.0) {  // an exactly zero column below the diagonal: singular
      det = 0.0;
      break;
    }
    rel = (1.0 + rel) * (rp / ap) + rel;
    const double ipd = bad ? 0.0 : 1.0 / (ap - rp);  // radii are not used once bad
    for (int i = k + 1; i < m; ++i) {
      const double l = a[i * MC + k] / piv, al = fabs(l);
      const double rl = (ra[i * MC + k] + al * rp) * ipd + u * al;
      for (int j = k + 1; j < m; ++j) {
        const double x = a[k * MC + j], ax = fabs(x), old = fabs(a[i * MC + j]);
        a[i * MC + j] = fma(-l, x, a[i * MC + j]);
        ra[i * MC + j] += al * ra[k * MC + j] + (ax + ra[k * MC + j]) * rl + u * (al * ax + old);
      }
    }
  }
  const double rnd = (m - 1) * u * 1.01;  // rounding of the product of pivots
  if (bad) {
    *bnd = (fabs(det) + hs) * (1.0 + 0x1p-50);
  } else if (last_open) {
    *bnd = (pr * (1.0 + rnd) + fabs(det) * rnd) * (1.0 + 0x1p-50);
  } else {
    *bnd = ((1.0 + rel) * (1.0 + rnd) - 1.0) * fabs(det) * (1.0 + 0x1p-50);
  }
  (void)pa;
  return neg ? -det : det;
}

// Gather the minor A[:, c] from the column-major shared copy (column j of A
// at As + j * CS, CS = padded column stride) into registers.
template <typename T, int M, int CS>
__device__ __forceinline__ void gather(const T* __restrict__ As, const int (&c)[M], T (&a)[M][M]) {
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const T* col = As + c[j] * CS;
    if constexpr (sizeof(T) == 4 && CS % 4 == 0) {
#pragma unroll
      for (int i = 0; i < M; i += 4) {
        const float4 v = *reinterpret_cast<const float4*>(col + i);
        a[i][j] = v.x;
        if (i + 1 < M) a[i + 1][j] = v.y;
        if (i + 2 < M) a[i + 2][j] = v.z;
        if (i + 3 < M) a[i + 3][j] = v.w;
      }
    } else if constexpr (sizeof(T) == 8 && CS % 2 == 0) {
#pragma unroll
      for (int i = 0; i < M; i += 2) {
        const double2 v = *reinterpret_cast<const double2*>(col + i);
        a[i][j] = v.x;
        if (i + 1 < M) a[i + 1][j] = v.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < M; ++i) a[i][j] = col[i];
    }
  }
}

template <typename T, int M>
struct ColStride {
  static constexpr int value = (sizeof(T) == 8) ? ((M + 1) / 2) * 2 : ((M + 3) / 4) * 4;
};

// ---------------------------------------------------------------------------
// Compensated sums
// ---------------------------------------------------------------------------
struct Dd {  // binary64 value + error term (Knuth two-sum)
  double hi = 0.0, lo = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double s = hi + x;
    const double bp = s - hi;
    const double err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
  }
  __device__ __forceinline__ void merge(const Dd& o) {
    add(o.hi);
    lo += o.lo;
  }
};

struct Ff {  // binary32 value + error term, flushed to Dd per run of ranks
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
  }
  // adds another float-float value (two-sum of the leading parts, then
  // renormalisation), keeping about twice binary32 precision
  __device__ __forceinline__ void merge(const Ff& o) {
    const float s = hi + o.hi;
    const float bp = s - hi;
    float err = (hi - (s - bp)) + (o.hi - bp);
    err += lo + o.lo;
    hi = s + err;
    lo = err - (hi - s);
  }
};

__device__ __forceinline__ double shfl_xor_d(double x, int off) {
  return __shfl_xor_sync(kFull, x, off);
}

// Fixed-order warp reduction of float-float lane totals (value and magnitude
// sum) on the binary32 pipe; the warp total is valid in every lane.
__device__ __forceinline__ void warp_reduce_ff(Ff& t, Ff& ta) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Ff o, oa;
    o.hi = __shfl_xor_sync(kFull, t.hi, off);
    o.lo = __shfl_xor_sync(kFull, t.lo, off);
    oa.hi = __shfl_xor_sync(kFull, ta.hi, off);
    oa.lo = __shfl_xor_sync(kFull, ta.lo, off);
    t.merge(o);
    ta.merge(oa);
  }
}

// Block-wide fixed-order reduction of float-float lane totals, a count and
// the lanes' error bounds (binary64), the totals entirely on the binary32
// pipe (binary64 runs at 1/64 of its rate): warp trees, then the warps'
// totals in warp order.  The result is valid in thread 0.  `scratch` holds
// kScratchWords * (blockDim.x / 32) binary64 words.
constexpr int kScratchWords = 5;
__device__ inline void block_reduce_ff(Ff& t, Ff& ta, long long& count, double& bnd, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  warp_reduce_ff(t, ta);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    count += __shfl_xor_sync(kFull, count, off);
    bnd += shfl_xor_d(bnd, off);
  }
  double* ws = scratch + kScratchWords * warp;
  float* fs = reinterpret_cast<float*>(ws);
  __syncthreads();
  if (lane == 0) {
    fs[0] = t.hi;
    fs[1] = t.lo;
    fs[2] = ta.hi;
    fs[3] = ta.lo;
    ws[2] = __longlong_as_double(count);
    ws[3] = bnd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Ff s, sa;
    long long cnt = 0;
    double b = 0.0;
    for (int w = 0; w < nw; ++w) {
      const double* wv = scratch + kScratchWords * w;
      const float* fv = reinterpret_cast<const float*>(wv);
      s.merge(Ff{fv[0], fv[1]});
      sa.merge(Ff{fv[2], fv[3]});
      cnt += __double_as_longlong(wv[2]);
      b += wv[3];
    }
    t = s;
    ta = sa;
    count = cnt;
    bnd = b;
  }
}

// Block-wide reduction of (hi, lo, abs, count, bound) in a fixed order; the
// result is valid in thread 0.  `scratch` holds kScratchWords *
// (blockDim.x / 32) words.
__device__ inline void block_reduce_dd(Dd& acc, double& abs_sum, long long& count, double& bnd, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Dd o;
    o.hi = shfl_xor_d(acc.hi, off);
    o.lo = shfl_xor_d(acc.lo, off);
    acc.merge(o);
    abs_sum += shfl_xor_d(abs_sum, off);
    count += __shfl_xor_sync(kFull, count, off);
    bnd += shfl_xor_d(bnd, off);
  }
  double* ws = scratch + kScratchWords * warp;
  __syncthreads();
  if (lane == 0) {
    ws[0] = acc.hi;
    ws[1] = acc.lo;
    ws[2] = abs_sum;
    ws[3] = __longlong_as_double(count);
    ws[4] = bnd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Dd t;
    double ab = 0.0, b = 0.0;
    long long cnt = 0;
    for (int w = 0; w < nw; ++w) {
      const double* wv = scratch + kScratchWords * w;
      Dd o;
      o.hi = wv[0];
      o.lo = wv[1];
      t.merge(o);
      ab += wv[2];
      cnt += __double_as_longlong(wv[3]);
      b += wv[4];
    }
    acc = t;
    abs_sum = ab;
    count = cnt;
    bnd = b;
  }
}

// ---------------------------------------------------------------------------
// Staging of A into shared memory (column-major, padded column stride CS),
// with every row scaled by a power of two so that its largest magnitude lies
// in [0.5, 1).  Row scaling multiplies det_R by the same power of two (each
// minor is linear in every row), which the finaliser restores exactly.
// Returns, in every thread, the total exponent sum_i e_i.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double load_elem(const void* A, int dtype, long long idx) {
  switch (dtype) {
    case kI8: return static_cast<double>(static_cast<const int8_t*>(A)[idx]);
    case kI32: return static_cast<double>(static_cast<const int32_t*>(A)[idx]);
    case kF32: return static_cast<double>(static_cast<const float*>(A)[idx]);
    default: return static_cast<const double*>(A)[idx];
  }
}

// Row scaling by powers of two with integer operations on the binary64 bits
// (binary64 arithmetic runs at 1/64 of the binary32 rate on this GPU, and
// ldexp/frexp take several binary64 operations each).  hi_abs orders
// magnitudes by the exponent and leading mantissa bits, which is all the
// exponent of the largest entry needs.
__device__ __forceinline__ uint32_t hi_abs(double x) {
  return static_cast<uint32_t>(__double2hiint(x)) & 0x7fffffffu;
}

// x * 2^-e, exact: one multiply by a power of two built from its bits when
// 2^-e is a normal binary64 number, ldexp otherwise.
__device__ __forceinline__ double scale_pow2(double x, int e) {
  if (e >= -1022 && e <= 1022) return x * __hiloint2double((1023 - e) << 20, 0);
  return ldexp(x, -e);
}

// Exponent e with |x| * 2^-e in [0.5, 1) for the row maximum x whose hi_abs
// is h, from the bits alone (0 for a zero, infinite or NaN maximum, as
// frexp's convention).  A subnormal maximum takes the position of the leading
// bit of its high word: bit b there has the value 2^(b - 1042).
__device__ __forceinline__ int row_exponent_bits(uint32_t h) {
  const int be = static_cast<int>(h >> 20);
  if (h == 0u || be == 0x7ff) return 0;
  if (be == 0) return (32 - __clz(static_cast<int>(h))) - 1042;
  return be - 1022;
}

template <typename T>
__device__ inline int stage_scaled(const void* A, int dtype, int m, int n, long long lda, T* As, int cs,
                                   int* row_exp /* smem, m ints */, bool* exact = nullptr) {
  // exact (optional, valid in every thread): every staged entry equals its
  // scaled input (no rounding to T), so the error bounds start from radius 0
  bool ex = true;
  // 1. row maxima as hi_abs keys, by shared-memory atomics over all entries
  //    at once; the first kKeep entries of every thread stay in registers
  constexpr int kKeep = 4;
  unsigned* row_h = reinterpret_cast<unsigned*>(row_exp);
  for (int i = threadIdx.x; i < m; i += blockDim.x) row_h[i] = 0u;
  __syncthreads();
  const int mn = m * n;
  double keep[kKeep];
#pragma unroll
  for (int k = 0; k < kKeep; ++k) {
    const int idx = threadIdx.x + k * blockDim.x;
    keep[k] = 0.0;
    if (idx < mn) {
      const int i = idx / n, j = idx - i * n;
      keep[k] = load_elem(A, dtype, (long long)i * lda + j);
      atomicMax(&row_h[i], hi_abs(keep[k]));
    }
  }
  for (int idx = threadIdx.x + kKeep * blockDim.x; idx < mn; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    atomicMax(&row_h[i], hi_abs(load_elem(A, dtype, (long long)i * lda + j)));
  }
  __syncthreads();
  // 2. scaled copy (exact power-of-two scaling) into the column-major shared
  //    copy, padding rows zeroed for vector loads
#pragma unroll
  for (int k = 0; k < kKeep; ++k) {
    const int idx = threadIdx.x + k * blockDim.x;
    if (idx < mn) {
      const int i = idx / n, j = idx - i * n;
      const double x = scale_pow2(keep[k], row_exponent_bits(row_h[i]));
      const T t = to_elem<T>(x);
      As[j * cs + i] = t;
      ex &= as_double(t) == x;
    }
  }
  for (int idx = threadIdx.x + kKeep * blockDim.x; idx < mn; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    const double x = scale_pow2(load_elem(A, dtype, (long long)i * lda + j), row_exponent_bits(row_h[i]));
    const T t = to_elem<T>(x);
    As[j * cs + i] = t;
    ex &= as_double(t) == x;
  }
  for (int idx = threadIdx.x; idx < (cs - m) * n; idx += blockDim.x) {
    const int j = idx / (cs - m), i = m + (idx - j * (cs - m));
    As[j * cs + i] = T(0);
  }
  const int all_exact = __syncthreads_and(ex ? 1 : 0);
  if (exact) *exact = all_exact != 0;
  int tot = 0;
  for (int i = 0; i < m; ++i) tot += row_exponent_bits(row_h[i]);
  return tot;
}

// Last-block finalisation: every block stores its partial, and the block that
// takes the last ticket sums all partials in block order.  Returns true in the
// last block (all its threads), which then holds the totals in thread 0.
__device__ inline bool last_block(unsigned int* ticket) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

}  // namespace radic
