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

#include "radic_fp_kernels.cuh"

namespace radic {

__host__ __device__ inline size_t prefix_smem_bytes(int n, int m, int cs, int elem, int threads) {
  const int kmax = n - m + 2;  // largest number of candidate columns
  size_t off = fp_smem_bytes(n, m, cs, elem, threads);
  off += (size_t)kmax * threads * 2 * elem;
  return off;
}

// Rank of an ascending 0-based combination in dictionary order (the inverse of
// unrank): C(n,m) - 1 - sum_i C(n-1-c_i, m-i).
__device__ __forceinline__ unsigned long long rank_part(const uint64_t* binom, int bstride, int n, int c, int k) {
  return binom[(n - 1 - c) * bstride + k];
}

// Factor the m x (m-2) prefix with partial pivoting.  Outputs the row order
// idx[], W (2 x (m-2)), the product of pivots, the largest pivot magnitude and
// the parity of the row permutation.
template <typename T, int M, int CS>
__device__ __forceinline__ void prefix_factor(const T* __restrict__ As, const int (&c)[M - 2], T (&W)[2][M - 2],
                                              int (&idx)[M], T& prod, T& gmax, bool& neg) {
  constexpr int P = M - 2;
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
      const bool sw = fabs(a[i][k]) > fabs(a[k][k]);
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
    T r;
    if constexpr (sizeof(T) == 8) r = rcp_f64(piv);
    else r = rcp_f32(piv);
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
  for (int rr = 0; rr < 2; ++rr) {
#pragma unroll
    for (int j = P - 1; j >= 0; --j) {
      T s = -a[P + rr][j];
#pragma unroll
      for (int i = j + 1; i < P; ++i) s = fma(-W[rr][i], a[i][j], s);
      W[rr][j] = s;
    }
  }
}

// Schur complement of column `col` (rows read in the pivoted order idx[]).
template <typename T, int M>
__device__ __forceinline__ void prefix_column(const T* __restrict__ col, const T (&W)[2][M - 2], const int (&idx)[M],
                                              T& z0, T& z1) {
  constexpr int P = M - 2;
  T x[M];
#pragma unroll
  for (int s = 0; s < M; ++s) x[s] = col[idx[s]];
  z0 = x[P];
  z1 = x[P + 1];
#pragma unroll
  for (int j = 0; j < P; ++j) {
    z0 = fma(W[0][j], x[j], z0);
    z1 = fma(W[1][j], x[j], z1);
  }
}

// Accumulators of one lane: binary64 two-sum for binary64, float-float
// flushed per prefix for binary32.
template <typename T>
struct PrefixAcc;
template <>
struct PrefixAcc<double> {
  Dd acc;
  double abs_sum = 0.0;
  __device__ __forceinline__ void add_column(double s, double a) {
    acc.add(s);
    abs_sum += a;
  }
  __device__ __forceinline__ void end_prefix() {}
  __device__ __forceinline__ void finish() {}
};
template <>
struct PrefixAcc<float> {
  // per prefix: float-float sums; per thread: float-float totals, converted
  // to binary64 once at the end (keeps the binary64 pipe free)
  Ff pre, tot, tot_abs;
  float pre_abs = 0.0f;
  Dd acc;
  double abs_sum = 0.0;
  __device__ __forceinline__ void add_column(float s, float a) {
    pre.add(s);
    pre_abs += a;
  }
  __device__ __forceinline__ void end_prefix() {
    tot.merge(pre);
    tot_abs.add(pre_abs);
    pre = Ff();
    pre_abs = 0.0f;
  }
  __device__ __forceinline__ void drop_prefix() {
    pre = Ff();
    pre_abs = 0.0f;
  }
  __device__ __forceinline__ void finish() {
    acc.add(static_cast<double>(tot.hi));
    acc.add(static_cast<double>(tot.lo));
    abs_sum = static_cast<double>(tot_abs.hi) + static_cast<double>(tot_abs.lo);
  }
};

// Two-entry vector type of T.
template <typename T>
struct Pair2 {
  using type = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
};

// Where per-leaf terms go (terms output of the parity tests); unused otherwise.
struct TermsSink {
  double* terms;
  unsigned long long q0, count, qtot;
  int escale;
};

// Processes one prefix c[0..m-3] (last column v): factors it, reduces every
// later column to its Schur complement, forms the 2 x 2 leaf determinants
// with the sign of Eq. (1) and adds them to acc.pre (the caller commits or
// drops them).  `zb` is this lane's slot of the column buffer, `zstride` the
// distance between consecutive columns.  Returns the growth flag of the mixed
// mode: largest prefix pivot, or twice the largest Schur entry (a bound for
// the last two pivots), above `thr`, or a non-finite scale.
template <typename T, int M, int CS, bool kTerms>
__device__ __forceinline__ bool prefix_one(const T* __restrict__ As, const uint64_t* binom, int n, int v,
                                           const int (&c)[M - 2], typename Pair2<T>::type* zb, int zstride, T thr,
                                           bool act, PrefixAcc<T>& acc, const TermsSink& ts) {
  constexpr int P = M - 2;
  using T2 = typename Pair2<T>::type;
  const int bs = M + 1;
  T W[2][P];
  int idx[M];
  T prod, gmax;
  bool neg;
  prefix_factor<T, M, CS>(As, c, W, idx, prod, gmax, neg);
  // parity of r = M(M+1)/2, of the prefix columns' share of s, and of the two
  // leaf columns' "+1" terms; the leaf columns' own parities are folded in below
  int sp = M * (M + 1) / 2 + 2;
#pragma unroll
  for (int j = 0; j < P; ++j) sp += c[j] + 1;
  const T alpha = ((sp & 1) != neg) ? -prod : prod;
  unsigned long long rank_prefix = 0;
  if constexpr (kTerms) {
#pragma unroll
    for (int j = 0; j < P; ++j) rank_prefix += rank_part(binom, bs, n, c[j], M - j);
  }
  T zmax = T(0);
  const int k = n - 1 - v;
  for (int q = 0; q < k; ++q) {
    const int col = v + 1 + q;
    T z0, z1;
    prefix_column<T, M>(As + col * CS, W, idx, z0, z1);
    zmax = fmax(zmax, fmax(fabs(z0), fabs(z1)));
    if (col & 1) {
      z0 = -z0;
      z1 = -z1;
    }
    z0 *= alpha;
    T colsum = T(0), colabs = T(0);
    const T2* yp = zb;
#pragma unroll 4
    for (int q2 = 0; q2 < q; ++q2, yp += zstride) {
      const T2 y = *yp;
      const T d = fma(y.x, z1, -(y.y * z0));
      if constexpr (kTerms) {
        const int c2 = v + 1 + q2;
        const unsigned long long rk =
            ts.qtot - 1 - (rank_prefix + rank_part(binom, bs, n, c2, 2) + rank_part(binom, bs, n, col, 1));
        if (act && rk >= ts.q0 && rk < ts.q0 + ts.count) ts.terms[rk - ts.q0] = ldexp(static_cast<double>(d), ts.escale);
      }
      colsum += d;
      colabs += fabs(d);
    }
    T2 zz;
    zz.x = z0;
    zz.y = z1;
    zb[q * zstride] = zz;
    if (act) acc.add_column(colsum, colabs);
  }
  return !(gmax <= thr) || !(2 * zmax <= thr) || !(fabs(alpha) <= static_cast<T>(FLT_MAX));
}

// ---------------------------------------------------------------------------
// Single-matrix prefix kernel.
// ---------------------------------------------------------------------------
template <typename T, int M, bool kMixed, bool kTerms>
__global__ void __launch_bounds__(128) k_fp_prefix(SingleArgs a, PrefixTable tab) {
  static_assert(M >= 3, "prefix sharing needs m >= 3");
  constexpr int P = M - 2;
  constexpr int CS = ColStride<T, M>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n;
  FpSmem<T> sm(smem_raw, n, M, CS);
  T* zbuf = reinterpret_cast<T*>(smem_raw + fp_smem_bytes(n, M, CS, sizeof(T), blockDim.x));
  build_binom(sm.binom, n, M);
  const int escale = stage_scaled<T>(a.A, a.dtype, M, n, a.lda, sm.As, CS, sm.row_exp);

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

  for (unsigned long long t = gwarp; t < tab.total_tasks; t += nwarps) {
    int v = tab.v_lo;
    while (v < tab.v_hi && t >= tab.task_start[v + 1]) ++v;
    const unsigned long long runlen = tab.run[v], cnt = tab.count[v];
    const unsigned long long r0 = (t - tab.task_start[v]) * 32ull * runlen + (unsigned long long)lane * runlen;
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
      using T2 = typename Pair2<T>::type;
      T2* zb = reinterpret_cast<T2*>(zbuf) + threadIdx.x;  // column q at zb[q * blockDim.x]
      const bool flag = prefix_one<T, M, CS, kTerms>(sm.As, sm.binom, n, v, c, zb, blockDim.x, thr, act, acc, ts);
      if constexpr (kMixed && !kTerms) {
        if (act && flag) acc.drop_prefix();  // its leaves are recomputed in binary64
        const unsigned fm = __ballot_sync(kFull, act && flag);
        if (fm) {
          if (act && flag) {
            const int pos = fcnt + __popc(fm & ((1u << lane) - 1u));
            // record the prefix by its rank among all (m-2)-subsets of {0..n-1}
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
    acc.finish();
    Dd d = acc.acc;
    double ab = acc.abs_sum;
    block_reduce_dd(d, ab, fl, sm.scratch);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = FpPartial{d.hi, d.lo, ab, fl};
    finish_fp_main<kMixed>(a, sm.scratch, escale, M);
  }
}

}  // namespace radic
