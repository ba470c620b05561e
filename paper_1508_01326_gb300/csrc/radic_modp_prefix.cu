// Exact path, prefix mapping: the minors of one (m-D)-column prefix share
// its non-dividing elimination mod p (see the comment of k_modp_prefix).
#include "radic_modp.cuh"

namespace radic {

namespace {
// ---------------------------------------------------------------------------
// Prefix mapping (3 <= m = M <= 12): the minors whose first m-D columns form
// one ascending prefix share the first m-D elimination steps.
//
// Non-dividing elimination of the m x P prefix (P = m - D) mod p: step k
// takes the first row at or below k with a nonzero entry in column k
// (compare-and-swap), then a_ij <- pi_k a_ij - a_ik a_kj for i, j > k, with
// pi_k the current pivot; the multipliers a_ik stay in place and move with
// their rows.  The same steps applied to a later column x, its rows taken in
// the final order, leave s z(x) in rows P..m-1, where z(x) is the Schur
// complement of x and s = prod_k pi_k.  The true pivots t_k satisfy
// pi_k = t_k prod_{j<k} pi_j, so every leaf minor of the prefix is
//   det = +- prod_k t_k det(Z) = +- det(s Z) / (s^(D-1) prod_k prod_{j<k} pi_j),
// one denominator for the whole subtree: each lane keeps its sum as one
// fraction and inverts once at the end.  A prefix singular mod p has a zero
// pivot after the search, s = 0, and all its minors are 0 mod p.
// ---------------------------------------------------------------------------
template <int M, int D, int CS>
__device__ __forceinline__ void modp_prefix_factor(const uint32_t* __restrict__ As, const int (&c)[M - D],
                                                   const Mont& mp, uint32_t (&a)[M][M - D], int (&idx)[M],
                                                   uint32_t (&piv)[M - D], bool& neg, uint32_t& den) {
  constexpr int P = M - D;
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const uint32_t* col = As + c[j] * CS;
#pragma unroll
    for (int i = 0; i < M; i += 4) {
      const uint4 v = *reinterpret_cast<const uint4*>(col + i);
      a[i][j] = v.x;
      if (i + 1 < M) a[i + 1][j] = v.y;
      if (i + 2 < M) a[i + 2][j] = v.z;
      if (i + 3 < M) a[i + 3][j] = v.w;
    }
  }
#pragma unroll
  for (int i = 0; i < M; ++i) idx[i] = i;
  neg = false;
#pragma unroll
  for (int k = 0; k < P; ++k) {
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      const bool sw = (a[k][k] == 0u) && (a[i][k] != 0u);
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const uint32_t x = a[k][j], y = a[i][j];
        a[k][j] = sw ? y : x;
        a[i][j] = sw ? x : y;
      }
      const int ik = idx[k], ii = idx[i];
      idx[k] = sw ? ii : ik;
      idx[i] = sw ? ik : ii;
      neg ^= sw;
    }
    piv[k] = a[k][k];
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
#pragma unroll
      for (int j = k + 1; j < P; ++j) a[i][j] = ff_update(piv[k], a[i][j], a[i][k], a[k][j], mp);
    }
  }
  uint32_t q = mp.one, dp = mp.one;  // q: prod_{j<k} pi_j
#pragma unroll
  for (int k = 0; k < P; ++k) {
    dp = mmul(dp, q, mp);
    q = mmul(q, piv[k], mp);
  }
#pragma unroll
  for (int d = 1; d < D; ++d) dp = mmul(dp, q, mp);
  den = dp;
}

// s z(x) of the later column `col` (rows in the final order), with the sign
// of the column's index parity folded in.
template <int M, int D>
__device__ __forceinline__ void modp_prefix_column(const uint32_t* __restrict__ colp, int col,
                                                   const uint32_t (&a)[M][M - D], const int (&idx)[M],
                                                   const uint32_t (&piv)[M - D], const Mont& mp,
                                                   uint32_t (&z)[D]) {
  constexpr int P = M - D;
  uint32_t x[M];
#pragma unroll
  for (int s = 0; s < M; ++s) x[s] = colp[idx[s]];
#pragma unroll
  for (int k = 0; k < P; ++k) {
#pragma unroll
    for (int i = k + 1; i < M; ++i) x[i] = ff_update(piv[k], x[i], a[i][k], x[k], mp);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) z[d] = (col & 1) ? neg_mod(x[P + d], mp.p) : x[P + d];
}

// Leaf determinants (Montgomery form).  Each redc input stays below p 2^32.
__device__ __forceinline__ uint32_t modp_det2(const uint32_t (&y)[2], const uint32_t (&z)[2], const Mont& mp) {
  return ff_update(y[0], z[1], y[1], z[0], mp);  // y0 z1 - y1 z0
}
__device__ __forceinline__ void modp_cross(const uint32_t (&y)[3], const uint32_t (&z)[3], const Mont& mp,
                                           uint32_t (&w)[3]) {
  w[0] = ff_update(y[1], z[2], y[2], z[1], mp);
  w[1] = ff_update(y[2], z[0], y[0], z[2], mp);
  w[2] = ff_update(y[0], z[1], y[1], z[0], mp);
}
__device__ __forceinline__ uint32_t modp_dot(const uint32_t (&y)[3], const uint32_t (&w)[3], const Mont& mp) {
  const uint64_t t = static_cast<uint64_t>(y[0]) * w[0] + static_cast<uint64_t>(y[1]) * w[1];
  return add_mod(redc(t, mp.p, mp.pinv), mmul(y[2], w[2], mp), mp.p);
}

// Sum (Montgomery form) of a lane's share of the leaves of one prefix, one
// candidate column at a time; lane `sub` of `lp` takes the leaves whose
// second-to-last column index is congruent to sub.  Leaf values are added as
// integers and reduced once per column (fewer than 2^31 addends of < p).
// With a terms sink, each leaf's signed term (times inv_den) is stored.
template <int M, int D, bool kTerms>
__device__ __forceinline__ uint32_t modp_prefix_leaves(const uint32_t* __restrict__ As, int cs, const uint64_t* binom,
                                                       int n, int v, const uint32_t (&a)[M][M - D],
                                                       const int (&idx)[M], const uint32_t (&piv)[M - D],
                                                       const Mont& mp, const ZBuf<uint32_t, D>& zb, int sub, int lp,
                                                       bool negp, uint32_t inv_den,
                                                       unsigned long long rank_prefix, const TermsSink& ts,
                                                       uint32_t* terms, bool act) {
  const int k = n - 1 - v, bs = M + 1;
  uint32_t S = 0u;
  for (int q = 0; q < k; ++q) {
    const int col = v + 1 + q;
    uint32_t z[D];
    modp_prefix_column<M, D>(As + col * cs, col, a, idx, piv, mp, z);
    uint64_t csum = 0;
    const unsigned long long rk_col = rank_prefix + rank_part(binom, bs, n, col, 1);
    if constexpr (D == 2) {
      for (int q2 = sub; q2 < q; q2 += lp) {
        uint32_t y[2];
        zb.get(q2, y);
        const uint32_t d = modp_det2(y, z, mp);
        csum += d;
        if constexpr (kTerms) {
          const unsigned long long rk = ts.qtot - 1 - (rk_col + rank_part(binom, bs, n, v + 1 + q2, 2));
          if (act && rk >= ts.q0 && rk < ts.q0 + ts.count) {
            uint32_t t = redc(mmul(d, inv_den, mp), mp.p, mp.pinv);
            terms[rk - ts.q0] = negp ? neg_mod(t, mp.p) : t;
          }
        }
      }
    } else {
      for (int q2 = sub; q2 < q; q2 += lp) {
        uint32_t y2[3], w[3];
        zb.get(q2, y2);
        modp_cross(y2, z, mp, w);
        const unsigned long long rk2 = rk_col + rank_part(binom, bs, n, v + 1 + q2, 2);
#pragma unroll 2
        for (int q1 = 0; q1 < q2; ++q1) {
          uint32_t y1[3];
          zb.get(q1, y1);
          const uint32_t d = modp_dot(y1, w, mp);
          csum += d;
          if constexpr (kTerms) {
            const unsigned long long rk = ts.qtot - 1 - (rk2 + rank_part(binom, bs, n, v + 1 + q1, 3));
            if (act && rk >= ts.q0 && rk < ts.q0 + ts.count) {
              uint32_t t = redc(mmul(d, inv_den, mp), mp.p, mp.pinv);
              terms[rk - ts.q0] = negp ? neg_mod(t, mp.p) : t;
            }
          }
        }
      }
    }
    zb.put(q, z);
    // sum of Montgomery-form values -> normal form (redc) -> Montgomery form
    S = add_mod(S, mmul(redc(csum, mp.p, mp.pinv), mp.r2, mp), mp.p);
  }
  return S;
}

template <int M, int D, bool kTerms>
__global__ void __launch_bounds__(kMaxThreadsModp) k_modp_prefix(SingleArgs a, PrefixTable tab) {
  static_assert(M > D, "the prefix needs at least one column");
  constexpr int P = M - D;
  constexpr int CS = ((M + 3) / 4) * 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n;
  ModpSmem sm(smem_raw, n, M, CS, blockDim.x);
  const ZBuf<uint32_t, D> zb(smem_raw + modp_smem_bytes(n, M, CS, blockDim.x), threadIdx.x, blockDim.x, n - M + D);
  int needed;
  const int K = stage_modp(a, sm, M, CS, &needed);
  if (K == 0) return;  // a wide pass whose primes the bound does not need

  const int lane = threadIdx.x & 31;
  const unsigned long long gwarp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * blockDim.x / 32;
  const int bs = M + 1;
  TermsSink ts{nullptr, a.q0, a.count, sm.binom[n * bs + M], 0};

  uint32_t N[kMaxPrimes], Dn[kMaxPrimes];
#pragma unroll
  for (int k = 0; k < kMaxPrimes; ++k) {
    N[k] = 0u;
    Dn[k] = sm.mont[k].one;
  }
  for (unsigned long long t = gwarp; t < tab.total_tasks; t += nwarps) {
    int v = tab.v_lo;
    while (v < tab.v_hi && t >= tab.task_start[v + 1]) ++v;
    const unsigned long long runlen = tab.run[v], cnt = tab.count[v];
    const int lp = tab.lanes[v], grp = lane / lp, sub = lane - grp * lp;
    const unsigned long long groups = 32 / lp;
    const unsigned long long r0 = (t - tab.task_start[v]) * groups * runlen + (unsigned long long)grp * runlen;
    const unsigned long long r1 = min(r0 + runlen, cnt);
    constexpr int H = P > 1 ? P - 1 : 1;
    int head[H];
    if constexpr (P > 1) unrank<P - 1>(r0 < cnt ? r0 : 0ull, v, sm.binom, bs, head);
    for (unsigned long long it = 0; it < runlen; ++it) {
      const bool act = r0 + it < r1;
      int c[P];
#pragma unroll
      for (int j = 0; j < P - 1; ++j) c[j] = head[j];
      c[P - 1] = v;
      int sp = M * (M + 1) / 2 + D;  // sign parity of Eq. (1) without the leaf columns' own parities
#pragma unroll
      for (int j = 0; j < P; ++j) sp += c[j] + 1;
      unsigned long long rank_prefix = 0;
      if constexpr (kTerms) {
#pragma unroll
        for (int j = 0; j < P; ++j) rank_prefix += rank_part(sm.binom, bs, n, c[j], M - j);
      }
#pragma unroll 1
      for (int k = 0; k < K; ++k) {
        const Mont mp = sm.mont[k];
        const uint32_t* As = sm.As + (size_t)k * n * CS;
        uint32_t fa[M][P], piv[P], den;
        int idx[M];
        bool negp;
        modp_prefix_factor<M, D, CS>(As, c, mp, fa, idx, piv, negp, den);
        negp ^= (sp & 1) != 0;
        uint32_t inv_den = 0u;
        if constexpr (kTerms) inv_den = minv(den, mp);  // 0 for a singular prefix: its terms are 0
        uint32_t* terms = kTerms ? static_cast<uint32_t*>(a.terms) + (size_t)k * a.count : nullptr;
        const uint32_t S = modp_prefix_leaves<M, D, kTerms>(As, CS, sm.binom, n, v, fa, idx, piv, mp, zb, sub, lp,
                                                           negp, inv_den, rank_prefix, ts, terms, act);
        if constexpr (!kTerms) {
          if (act && den != 0u) acc_fraction(N, Dn, k, S, den, negp, mp);
        }
      }
      if constexpr (P > 1) {
        if (r0 + it + 1 < r1) successor<P - 1>(head, v);
      }
    }
  }
  if constexpr (!kTerms) {
    uint32_t r[kMaxPrimes];
    close_fractions(N, Dn, K, sm.mont, r);
    finish_modp(a, sm, r, K, needed);
  }
}

template <int M, int D>
const void* prefix_kernel(bool terms) {
  return terms ? reinterpret_cast<const void*>(&k_modp_prefix<M, D, true>)
               : reinterpret_cast<const void*>(&k_modp_prefix<M, D, false>);
}

}  // namespace

const void* modp_prefix_kernel(int m, int depth, bool terms) {
  switch (m) {
    case 3: return depth == 2 ? prefix_kernel<3, 2>(terms) : nullptr;
    case 4: return depth == 3 ? prefix_kernel<4, 3>(terms) : prefix_kernel<4, 2>(terms);
    case 5: return depth == 3 ? prefix_kernel<5, 3>(terms) : prefix_kernel<5, 2>(terms);
    case 6: return depth == 3 ? prefix_kernel<6, 3>(terms) : prefix_kernel<6, 2>(terms);
    case 7: return depth == 3 ? prefix_kernel<7, 3>(terms) : prefix_kernel<7, 2>(terms);
    case 8: return depth == 3 ? prefix_kernel<8, 3>(terms) : prefix_kernel<8, 2>(terms);
    case 9: return depth == 3 ? prefix_kernel<9, 3>(terms) : prefix_kernel<9, 2>(terms);
    case 10: return depth == 3 ? prefix_kernel<10, 3>(terms) : prefix_kernel<10, 2>(terms);
    case 11: return depth == 3 ? prefix_kernel<11, 3>(terms) : prefix_kernel<11, 2>(terms);
    case 12: return depth == 3 ? prefix_kernel<12, 3>(terms) : prefix_kernel<12, 2>(terms);
    default: return nullptr;
  }
}

}  // namespace radic
