// Exact path for integer matrices: every minor is eliminated modulo K 31-bit
// primes (K from a Hadamard bound on |det_R(A)|), the signed terms of Eq. (1)
// are summed modulo each prime, and the last block reconstructs the signed
// 128-bit value by Chinese remaindering (Garner's mixed-radix form).
//
// Arithmetic is Montgomery multiplication with R = 2^32.  The thread mapping
// uses fraction-free elimination
//     a_ij <- a_kk a_ij - a_ik a_kj   (one Montgomery reduction per update)
// so the hot loop needs no modular inverse: det = pi_{m-1} / D with
// D = prod_{k <= m-3} (pi_0 ... pi_k); each thread keeps its running sum as
// one fraction and inverts its denominator once at the end.  To make a zero
// leading pivot as unlikely as a random residue (small integer entries are
// often 0), A is first multiplied modulo p by a fixed pseudo-random
// unimodular matrix T = L U.  Every minor of T A has the same determinant as
// the minor of A (det T = 1), and the rare zero pivot that remains takes a
// slow path with row exchanges.  The group mapping chooses a nonzero pivot
// row by ballot and needs no slow path.  The prefix mapping shares the
// elimination of each (m-D)-column prefix among the minors of its subtree,
// as the floating-point prefix kernels do, in non-dividing modular form.
#include "radic_prefix.cuh"

namespace radic {

namespace {

constexpr int kMaxThreadsModp = 128;

__host__ __device__ __forceinline__ uint32_t prime_at(int k) {
  return k == 0 ? kPrime0 : k == 1 ? kPrime1 : k == 2 ? kPrime2 : kPrime3;
}

struct Mont {
  uint32_t p, pinv, one, r2;
  uint64_t p2;
};

__device__ __forceinline__ uint32_t redc(uint64_t t, uint32_t p, uint32_t pinv) {
  const uint32_t mq = static_cast<uint32_t>(t) * pinv;
  const uint32_t u = static_cast<uint32_t>((t + static_cast<uint64_t>(mq) * p) >> 32);
  return u >= p ? u - p : u;
}
__device__ __forceinline__ uint32_t mmul(uint32_t a, uint32_t b, const Mont& mp) {
  return redc(static_cast<uint64_t>(a) * b, mp.p, mp.pinv);
}
// Montgomery form of (akk * aij - aik * akj) from Montgomery-form inputs.
__device__ __forceinline__ uint32_t ff_update(uint32_t akk, uint32_t aij, uint32_t aik, uint32_t akj,
                                              const Mont& mp) {
  const uint64_t t = static_cast<uint64_t>(akk) * aij + mp.p2 - static_cast<uint64_t>(aik) * akj;
  return redc(t, mp.p, mp.pinv);
}
__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t p) {
  const uint32_t s = a + b;
  return s >= p ? s - p : s;
}
__device__ __forceinline__ uint32_t neg_mod(uint32_t a, uint32_t p) { return a ? p - a : 0u; }

__device__ inline Mont make_mont(uint32_t p) {
  Mont mp;
  mp.p = p;
  uint32_t x = p;  // inverse of p modulo 2^32 by Newton iteration x <- x (2 - p x)
  for (int i = 0; i < 5; ++i) x *= 2u - p * x;
  mp.pinv = 0u - x;
  const uint64_t r1 = (1ull << 32) % p;
  mp.one = static_cast<uint32_t>(r1);
  mp.r2 = static_cast<uint32_t>((r1 * r1) % p);
  mp.p2 = static_cast<uint64_t>(p) * p;
  return mp;
}

// x^e in Montgomery form.
__device__ inline uint32_t mpow(uint32_t x, uint32_t e, const Mont& mp) {
  uint32_t r = mp.one;
  while (e) {
    if (e & 1u) r = mmul(r, x, mp);
    x = mmul(x, x, mp);
    e >>= 1;
  }
  return r;
}
__device__ inline uint32_t minv(uint32_t x, const Mont& mp) { return mpow(x, mp.p - 2u, mp); }

__device__ inline uint64_t mix64(uint64_t z) {  // SplitMix64 finaliser
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Shared-memory layout: binom | K x (n x cs) residues (column-major, Montgomery
// form) | m x n scratch rows | scratch words for reductions.
__host__ __device__ inline size_t modp_smem_bytes(int n, int m, int cs, int threads) {
  size_t off = ((size_t)(n + 1) * (m + 1) * 8 + 15) / 16 * 16;
  off += (size_t)kMaxPrimes * n * cs * 4;
  off += ((size_t)m * n * 4 + 15) / 16 * 16;
  off += (size_t)(threads / 32) * kMaxPrimes * 4;
  off += 64 + kMaxPrimes * sizeof(Mont);
  return off;
}

struct ModpSmem {
  uint64_t* binom;
  uint32_t* As;  // prime k at As + k * n * cs
  uint32_t* rows;
  uint32_t* scratch;
  int* misc;
  Mont* mont;
  __device__ ModpSmem(unsigned char* base, int n, int m, int cs, int threads) {
    size_t off = ((size_t)(n + 1) * (m + 1) * 8 + 15) / 16 * 16;
    binom = reinterpret_cast<uint64_t*>(base);
    As = reinterpret_cast<uint32_t*>(base + off);
    off += (size_t)kMaxPrimes * n * cs * 4;
    rows = reinterpret_cast<uint32_t*>(base + off);
    off += ((size_t)m * n * 4 + 15) / 16 * 16;
    scratch = reinterpret_cast<uint32_t*>(base + off);
    off += (size_t)(threads / 32) * kMaxPrimes * 4;
    misc = reinterpret_cast<int*>(base + off);
    off += 64;
    mont = reinterpret_cast<Mont*>(base + off);
  }
};

__device__ __forceinline__ long long load_int(const void* A, int dtype, long long idx) {
  return dtype == kI8 ? static_cast<long long>(static_cast<const int8_t*>(A)[idx])
                      : static_cast<long long>(static_cast<const int32_t*>(A)[idx]);
}

// Number of primes for |det_R(A)| <= C(n,m) prod_i ||row_i||_2 (Hadamard's
// inequality for every minor), plus a sign bit and a margin.  One warp per
// row computes the squared row norms into row_sq[]; thread 0 sums the logs.
__device__ inline int primes_needed(const void* A, int dtype, int m, int n, long long lda, double log2_count,
                                    double* row_sq) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < m; i += nw) {
    double s = 0.0;
    for (int j = lane; j < n; j += 32) {
      const double v = static_cast<double>(load_int(A, dtype, (long long)i * lda + j));
      s += v * v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
    if (lane == 0) row_sq[i] = s;
  }
  __syncthreads();
  double bits = log2_count;
  for (int i = 0; i < m; ++i) bits += 0.5 * log2(fmax(row_sq[i], 1.0));
  const int k = static_cast<int>(ceil((bits + 2.0) / 30.99));
  return k < 1 ? 1 : k;
}

// Stage binom and, for each prime, (T A mod p) in Montgomery form.  Returns K
// (primes used) in every thread; sets *needed to the primes the bound asks for.
__device__ inline int stage_modp(const SingleArgs& a, const ModpSmem& sm, int m, int cs, int* needed) {
  const int n = a.n;
  build_binom(sm.binom, n, m);
  if (threadIdx.x < kMaxPrimes) sm.mont[threadIdx.x] = make_mont(prime_at(threadIdx.x));
  {
    // the rows scratch (m x n words) is free until the residues are staged
    double* row_sq = reinterpret_cast<double*>(sm.rows);
    const double cnt = static_cast<double>(sm.binom[n * (m + 1) + m]);
    const int need = primes_needed(a.A, a.dtype, m, n, a.lda, log2(fmax(cnt, 1.0)), row_sq);
    if (threadIdx.x == 0) sm.misc[0] = need;
  }
  __syncthreads();
  *needed = sm.misc[0];
  const int K = min(sm.misc[0], kMaxPrimes);
  for (int k = 0; k < K; ++k) {
    const uint32_t p = prime_at(k);
    for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
      const int i = idx / n, j = idx - i * n;
      long long v = load_int(a.A, a.dtype, (long long)i * a.lda + j) % (long long)p;
      if (v < 0) v += p;
      sm.rows[idx] = static_cast<uint32_t>(v);
    }
    __syncthreads();
    // rows <- U rows (unit upper: row i += sum_{l > i} U_il row_l), ascending i
    for (int i = 0; i < m; ++i) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        uint64_t acc = sm.rows[i * n + j];
        for (int l = i + 1; l < m; ++l) {
          const uint64_t u = mix64(0x9e3779b97f4a7c15ull * (uint64_t)(k * 4096 + i * 64 + l) + 1ull) % p;
          acc = (acc + u * sm.rows[l * n + j]) % p;
        }
        sm.rows[i * n + j] = static_cast<uint32_t>(acc);
      }
      __syncthreads();
    }
    // rows <- L rows (unit lower: row i += sum_{l < i} L_il row_l), descending i
    for (int i = m - 1; i >= 0; --i) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        uint64_t acc = sm.rows[i * n + j];
        for (int l = 0; l < i; ++l) {
          const uint64_t u = mix64(0xd1b54a32d192ed03ull * (uint64_t)(k * 4096 + i * 64 + l) + 7ull) % p;
          acc = (acc + u * sm.rows[l * n + j]) % p;
        }
        sm.rows[i * n + j] = static_cast<uint32_t>(acc);
      }
      __syncthreads();
    }
    const Mont mp = make_mont(p);
    uint32_t* dst = sm.As + (size_t)k * n * cs;
    for (int idx = threadIdx.x; idx < n * cs; idx += blockDim.x) {
      const int j = idx / cs, i = idx - j * cs;
      dst[idx] = (i < m) ? mmul(sm.rows[i * n + j], mp.r2, mp) : 0u;
    }
    __syncthreads();
  }
  return K;
}

// Slow path: determinant (Montgomery form) with row exchanges and inverses.
template <int MC>
__device__ __noinline__ uint32_t det_pivoting(const uint32_t* As, int cs, const int* c, int m, Mont mp) {
  uint32_t x[MC * MC];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) x[i * MC + j] = As[c[j] * cs + i];
  uint32_t det = mp.one;
  for (int k = 0; k < m; ++k) {
    int p = -1;
    for (int i = k; i < m; ++i)
      if (x[i * MC + k] != 0u) {
        p = i;
        break;
      }
    if (p < 0) return 0u;
    if (p != k) {
      for (int j = 0; j < m; ++j) {
        const uint32_t t = x[k * MC + j];
        x[k * MC + j] = x[p * MC + j];
        x[p * MC + j] = t;
      }
      det = neg_mod(det, mp.p);
    }
    det = mmul(det, x[k * MC + k], mp);
    const uint32_t inv = minv(x[k * MC + k], mp);
    for (int i = k + 1; i < m; ++i) {
      const uint32_t l = mmul(x[i * MC + k], inv, mp);
      for (int j = k + 1; j < m; ++j)
        x[i * MC + j] = add_mod(x[i * MC + j], neg_mod(mmul(l, x[k * MC + j], mp), mp.p), mp.p);
    }
  }
  return det;
}

template <int M, int CS>
__device__ __forceinline__ void gather_u32(const uint32_t* __restrict__ As, const int (&c)[M],
                                           uint32_t (&x)[M][M]) {
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const uint32_t* col = As + c[j] * CS;
#pragma unroll
    for (int i = 0; i < M; i += 4) {
      const uint4 v = *reinterpret_cast<const uint4*>(col + i);
      x[i][j] = v.x;
      if (i + 1 < M) x[i + 1][j] = v.y;
      if (i + 2 < M) x[i + 2][j] = v.z;
      if (i + 3 < M) x[i + 3][j] = v.w;
    }
  }
}

// Fraction-free elimination of one minor: det = num / den (Montgomery form).
template <int M>
__device__ __forceinline__ bool ff_det(uint32_t (&x)[M][M], const Mont& mp, uint32_t& num, uint32_t& den) {
  uint32_t P = mp.one, D = mp.one;
  bool zero_pivot = false;
#pragma unroll
  for (int k = 0; k < M - 1; ++k) {
    const uint32_t piv = x[k][k];
    zero_pivot |= (piv == 0u);
    if (k <= M - 3) {
      P = mmul(P, piv, mp);
      D = mmul(D, P, mp);
    }
#pragma unroll
    for (int i = k + 1; i < M; ++i)
#pragma unroll
      for (int j = k + 1; j < M; ++j) x[i][j] = ff_update(piv, x[i][j], x[i][k], x[k][j], mp);
  }
  num = x[M - 1][M - 1];
  den = D;
  return zero_pivot;
}

// Block sum modulo each prime; result in thread 0's r[].
__device__ inline void block_reduce_modp(uint32_t (&r)[kMaxPrimes], int K, uint32_t* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < kMaxPrimes; ++k) {
    if (k < K) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) r[k] = add_mod(r[k], __shfl_xor_sync(kFull, r[k], off), prime_at(k));
    }
  }
  __syncthreads();
  if (lane == 0)
    for (int k = 0; k < K; ++k) scratch[warp * kMaxPrimes + k] = r[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < K; ++k) {
      uint32_t s = 0;
      for (int w = 0; w < nw; ++w) s = add_mod(s, scratch[w * kMaxPrimes + k], prime_at(k));
      r[k] = s;
    }
  }
}

__device__ inline uint64_t powmod64(uint64_t b, uint64_t e, uint64_t p) {
  uint64_t r = 1 % p;
  b %= p;
  while (e) {
    if (e & 1) r = (r * b) % p;
    b = (b * b) % p;
    e >>= 1;
  }
  return r;
}

// Garner reconstruction of the signed value in (-P/2, P/2].
__device__ inline void crt_write(radic_result* out, const uint32_t* res, int K, int needed, int status,
                                 unsigned long long total) {
  uint64_t v[kMaxPrimes];
  for (int i = 0; i < K; ++i) {
    const uint64_t p = prime_at(i);
    // value of the digits so far modulo p, and prod_{l<i} p_l modulo p
    uint64_t acc = 0, prod = 1;
    for (int l = 0; l < i; ++l) {
      acc = (acc + v[l] * prod) % p;
      prod = (prod * (prime_at(l) % p)) % p;
    }
    const uint64_t diff = (res[i] + p - acc) % p;
    v[i] = (diff * powmod64(prod, p - 2, p)) % p;
  }
  unsigned __int128 x = 0, big = 1;
  for (int i = 0; i < K; ++i) {
    x += static_cast<unsigned __int128>(v[i]) * big;
    big *= prime_at(i);
  }
  __int128 sx = static_cast<__int128>(x);
  if (x > big / 2) sx = static_cast<__int128>(x) - static_cast<__int128>(big);
  const unsigned __int128 ux = static_cast<unsigned __int128>(sx);
  out->exact_lo = static_cast<long long>(static_cast<uint64_t>(ux));
  out->exact_hi = static_cast<long long>(static_cast<uint64_t>(ux >> 64));
  const bool negv = sx < 0;
  const unsigned __int128 mag = negv ? static_cast<unsigned __int128>(-sx) : static_cast<unsigned __int128>(sx);
  const double val = ldexp(static_cast<double>(static_cast<uint64_t>(mag >> 64)), 64) +
                     static_cast<double>(static_cast<uint64_t>(mag));
  out->value = negv ? -val : val;
  out->abs_sum = 0.0;
  out->err_est = 0.0;
  out->minors = static_cast<long long>(total);
  out->flagged = 0;
  out->status = (needed > kMaxPrimes) ? RADIC_EOVERFLOW : status;
  out->n_primes = K;
  out->tier = kModeExact;
  for (int i = 0; i < 6; ++i) out->reserved[i] = 0;
}

// Last-block epilogue shared by both mappings.
__device__ inline void finish_modp(const SingleArgs& a, const ModpSmem& sm, uint32_t (&r)[kMaxPrimes], int K,
                                   int needed) {
  block_reduce_modp(r, K, sm.scratch);
  if (threadIdx.x == 0)
    for (int k = 0; k < kMaxPrimes; ++k) a.modp_partials[blockIdx.x * kMaxPrimes + k] = (k < K) ? r[k] : 0u;
  if (last_block(&a.hdr->ticket[0])) {
    uint32_t t[kMaxPrimes] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      for (int k = 0; k < K; ++k) t[k] = add_mod(t[k], __ldcg(&a.modp_partials[b * kMaxPrimes + k]), prime_at(k));
    block_reduce_modp(t, K, sm.scratch);
    if (threadIdx.x == 0) crt_write(a.out, t, K, needed, __ldcg(&a.hdr->status), a.total);
  }
}

// Adds the signed term num/den of one minor to the running fraction N/Dn of
// prime slot `k` (fraction form: N/Dn + s*num/den = (N*den + s*num*Dn)/(Dn*den)).
__device__ __forceinline__ void acc_fraction(uint32_t (&N)[kMaxPrimes], uint32_t (&Dn)[kMaxPrimes], int k,
                                             uint32_t num, uint32_t den, bool neg, const Mont& mp) {
#pragma unroll
  for (int kk = 0; kk < kMaxPrimes; ++kk) {
    if (kk == k) {
      uint32_t t = mmul(num, Dn[kk], mp);
      if (neg) t = neg_mod(t, mp.p);
      N[kk] = add_mod(mmul(N[kk], den, mp), t, mp.p);
      Dn[kk] = mmul(Dn[kk], den, mp);
    }
  }
}

// Residue N/Dn in normal form for every used prime.
__device__ inline void close_fractions(const uint32_t (&N)[kMaxPrimes], const uint32_t (&Dn)[kMaxPrimes], int K,
                                       const Mont* mont, uint32_t (&r)[kMaxPrimes]) {
#pragma unroll
  for (int k = 0; k < kMaxPrimes; ++k) {
    r[k] = 0u;
    if (k < K) {
      const Mont mp = mont[k];
      r[k] = redc(mmul(N[k], minv(Dn[k], mp), mp), mp.p, mp.pinv);
    }
  }
}

// ---------------------------------------------------------------------------
// Thread mapping (m = M <= 12).
// ---------------------------------------------------------------------------
template <int M, bool kTerms>
__global__ void __launch_bounds__(kMaxThreadsModp) k_modp_thread(SingleArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int CS = ((M + 3) / 4) * 4;
  const int n = a.n;
  ModpSmem sm(smem_raw, n, M, CS, blockDim.x);
  int needed;
  const int K = stage_modp(a, sm, M, CS, &needed);

  const int lane = threadIdx.x & 31;
  const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long L = a.ranks_per_task;
  const unsigned long long qbase = kTerms ? a.q0 : 0ull;
  const unsigned long long qlim = kTerms ? a.q0 + a.count : a.total;

  uint32_t N[kMaxPrimes], Dn[kMaxPrimes];
#pragma unroll
  for (int k = 0; k < kMaxPrimes; ++k) {
    N[k] = 0u;
    Dn[k] = sm.mont[k].one;
  }
  for (unsigned long long base = g - lane; base < a.tasks; base += nthreads) {
    const unsigned long long task = base + lane;
    const bool tact = task < a.tasks;
    const unsigned long long q0 = qbase + (tact ? task : 0ull) * L;
    const unsigned long long q1 = min(q0 + L, qlim);
    int c[M];
    unrank<M>(q0, n, sm.binom, M + 1, c);
    for (unsigned long long it = 0; it < L; ++it) {
      const unsigned long long q = q0 + it;
      const bool act = tact && q < q1;
      const bool neg = sign_negative<M>(c);
#pragma unroll 1
      for (int k = 0; k < K; ++k) {
        const Mont mp = sm.mont[k];
        const uint32_t* As = sm.As + (size_t)k * n * CS;
        uint32_t x[M][M];
        gather_u32<M, CS>(As, c, x);
        uint32_t num, den;
        const bool zp = ff_det<M>(x, mp, num, den);
        if constexpr (kTerms) {
          uint32_t d = zp ? det_pivoting<M>(As, CS, c, M, mp) : mmul(num, minv(den, mp), mp);
          d = redc(d, mp.p, mp.pinv);
          if (neg) d = neg_mod(d, mp.p);
          if (act) static_cast<uint32_t*>(a.terms)[(size_t)k * a.count + (q - a.q0)] = d;
        } else if (act) {
          if (zp) {
            num = det_pivoting<M>(As, CS, c, M, mp);
            den = mp.one;
          }
          acc_fraction(N, Dn, k, num, den, neg, mp);
        }
      }
      if (q + 1 < q1) successor<M>(c, n);
    }
  }
  if constexpr (!kTerms) {
    uint32_t r[kMaxPrimes];
    close_fractions(N, Dn, K, sm.mont, r);
    finish_modp(a, sm, r, K, needed);
  }
}

// ---------------------------------------------------------------------------
// Group mapping (m <= G): lane `sub` holds row `sub`; the pivot row of step k
// is the lowest active row with a nonzero entry in column k.  All lanes of the
// warp run the same number of steps (no early exit), so shuffles stay
// converged when one group meets a singular minor.
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ void group_ff(uint32_t (&x)[G], int m, int sub, int seg, const Mont& mp,
                                         uint32_t& num, uint32_t& den, bool& neg) {
  bool alive = sub < m;
  bool singular = false;
  uint32_t P = mp.one, D = mp.one;
  int par = 0;
  num = 0u;
  const unsigned segbits = (G == 32) ? kFull : ((1u << G) - 1u);
#pragma unroll
  for (int k = 0; k < G; ++k) {
    if (k >= m) break;
    const unsigned cand = (__ballot_sync(kFull, alive && x[k] != 0u) >> (seg * G)) & segbits;
    singular |= (cand == 0u);
    const int p = cand ? __ffs(cand) - 1 : 0;
    const uint32_t piv = __shfl_sync(kFull, x[k], p, G);
    const unsigned alive_bits = (__ballot_sync(kFull, alive) >> (seg * G)) & segbits;
    par ^= __popc(alive_bits & ((1u << p) - 1u)) & 1;
    if (sub == p) alive = false;
    if (k == m - 1) num = piv;
    if (k <= m - 3) {
      P = mmul(P, piv, mp);
      D = mmul(D, P, mp);
    }
    const uint32_t xk = x[k];
#pragma unroll
    for (int j = k + 1; j < G; ++j) {
      if (j < m) {
        const uint32_t u = __shfl_sync(kFull, x[j], p, G);
        if (alive) x[j] = ff_update(piv, x[j], xk, u, mp);
      }
    }
  }
  if (singular) {
    num = 0u;
    D = mp.one;
  }
  den = D;
  neg ^= (par != 0);
}

template <int G, bool kTerms>
__global__ void __launch_bounds__(kMaxThreadsModp) k_modp_group(SingleArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n, m = a.m;
  const int cs = m;
  ModpSmem sm(smem_raw, n, m, cs, blockDim.x);
  int needed;
  const int K = stage_modp(a, sm, m, cs, &needed);

  const int lane = threadIdx.x & 31, sub = lane & (G - 1), seg = lane / G;
  constexpr int kSegs = 32 / G;
  const unsigned long long gwarp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nsegs = (unsigned long long)gridDim.x * blockDim.x / G;
  const unsigned long long L = a.ranks_per_task;
  const unsigned long long qbase = kTerms ? a.q0 : 0ull;
  const unsigned long long qlim = kTerms ? a.q0 + a.count : a.total;

  uint32_t N[kMaxPrimes], Dn[kMaxPrimes];
#pragma unroll
  for (int k = 0; k < kMaxPrimes; ++k) {
    N[k] = 0u;
    Dn[k] = sm.mont[k].one;
  }
  for (unsigned long long base = gwarp * kSegs; base < a.tasks; base += nsegs) {
    const unsigned long long task = base + seg;
    const bool tact = task < a.tasks;
    const unsigned long long q0 = qbase + (tact ? task : 0ull) * L;
    const unsigned long long q1 = min(q0 + L, qlim);
    int c[G];
    unrank_dyn<G>(q0, n, m, sm.binom, m + 1, c);
    for (unsigned long long it = 0; it < L; ++it) {
      const unsigned long long q = q0 + it;
      const bool lead = tact && q < q1 && sub == 0;
      const bool sgn = sign_negative_dyn<G>(c, m);
#pragma unroll 1
      for (int k = 0; k < K; ++k) {
        const Mont mp = sm.mont[k];
        const uint32_t* As = sm.As + (size_t)k * n * cs;
        uint32_t x[G];
#pragma unroll
        for (int j = 0; j < G; ++j) x[j] = (j < m && sub < m) ? As[c[j] * cs + sub] : 0u;
        uint32_t num, den;
        bool neg = sgn;
        group_ff<G>(x, m, sub, seg, mp, num, den, neg);
        if constexpr (kTerms) {
          uint32_t d = redc(mmul(num, minv(den, mp), mp), mp.p, mp.pinv);
          if (neg) d = neg_mod(d, mp.p);
          if (lead) static_cast<uint32_t*>(a.terms)[(size_t)k * a.count + (q - a.q0)] = d;
        } else if (lead) {
          acc_fraction(N, Dn, k, num, den, neg, mp);
        }
      }
      if (q + 1 < q1) successor_dyn<G>(c, n, m);
    }
  }
  if constexpr (!kTerms) {
    uint32_t r[kMaxPrimes];
    close_fractions(N, Dn, K, sm.mont, r);
    finish_modp(a, sm, r, K, needed);
  }
}

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

template <int M>
const void* thread_kernel(bool terms) {
  return terms ? reinterpret_cast<const void*>(&k_modp_thread<M, true>)
               : reinterpret_cast<const void*>(&k_modp_thread<M, false>);
}
template <int G>
const void* group_kernel(bool terms) {
  return terms ? reinterpret_cast<const void*>(&k_modp_group<G, true>)
               : reinterpret_cast<const void*>(&k_modp_group<G, false>);
}

const void* pick(const SinglePlan& p, bool terms) {
  if (p.mapping == RADIC_MAP_PREFIX) {
    switch (p.m) {
      case 3: return p.depth == 2 ? prefix_kernel<3, 2>(terms) : nullptr;
      case 4: return p.depth == 3 ? prefix_kernel<4, 3>(terms) : prefix_kernel<4, 2>(terms);
      case 5: return p.depth == 3 ? prefix_kernel<5, 3>(terms) : prefix_kernel<5, 2>(terms);
      case 6: return p.depth == 3 ? prefix_kernel<6, 3>(terms) : prefix_kernel<6, 2>(terms);
      case 7: return p.depth == 3 ? prefix_kernel<7, 3>(terms) : prefix_kernel<7, 2>(terms);
      case 8: return p.depth == 3 ? prefix_kernel<8, 3>(terms) : prefix_kernel<8, 2>(terms);
      case 9: return p.depth == 3 ? prefix_kernel<9, 3>(terms) : prefix_kernel<9, 2>(terms);
      case 10: return p.depth == 3 ? prefix_kernel<10, 3>(terms) : prefix_kernel<10, 2>(terms);
      case 11: return p.depth == 3 ? prefix_kernel<11, 3>(terms) : prefix_kernel<11, 2>(terms);
      case 12: return p.depth == 3 ? prefix_kernel<12, 3>(terms) : prefix_kernel<12, 2>(terms);
      default: return nullptr;
    }
  }
  if (p.mapping == RADIC_MAP_THREAD) {
    switch (p.m) {
      case 1: return thread_kernel<1>(terms);
      case 2: return thread_kernel<2>(terms);
      case 3: return thread_kernel<3>(terms);
      case 4: return thread_kernel<4>(terms);
      case 5: return thread_kernel<5>(terms);
      case 6: return thread_kernel<6>(terms);
      case 7: return thread_kernel<7>(terms);
      case 8: return thread_kernel<8>(terms);
      case 9: return thread_kernel<9>(terms);
      case 10: return thread_kernel<10>(terms);
      case 11: return thread_kernel<11>(terms);
      case 12: return thread_kernel<12>(terms);
      default: return nullptr;
    }
  }
  if (p.group == 16) return group_kernel<16>(terms);
  if (p.group == 32) return group_kernel<32>(terms);
  return nullptr;
}

}  // namespace

size_t smem_modp(const SinglePlan& p) {
  const int cs = (p.mapping != RADIC_MAP_GROUP) ? ((p.m + 3) / 4) * 4 : p.m;
  size_t b = modp_smem_bytes(p.n, p.m, cs, p.threads);
  if (p.mapping == RADIC_MAP_PREFIX) b += zbuf_bytes(p.n - p.m + p.depth, p.threads, p.depth, 4);
  return b;
}

int blocks_per_sm_modp(const SinglePlan& p) {
  const void* k = pick(p, false);
  if (!k) return 0;
  if (!allow_smem(k, smem_modp(p))) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, p.threads, smem_modp(p)) != cudaSuccess) return 0;
  return nb;
}

int launch_modp(const SinglePlan& p, const SingleArgs& a, cudaStream_t s) {
  const void* k = pick(p, a.terms != nullptr);
  if (!k) return RADIC_EUNSUPPORTED;
  if (!allow_smem(k, smem_modp(p))) return RADIC_EUNSUPPORTED;
  SingleArgs args = a;
  PrefixTable tab = p.ptab;
  void* params[] = {&args, &tab};
  cudaEvent_t* ev = static_cast<cudaEvent_t*>(p.events);
  if (ev && cudaEventRecord(ev[0], s) != cudaSuccess) return RADIC_ECUDA;
  if (cudaLaunchKernel(k, dim3(p.blocks), dim3(p.threads), params, smem_modp(p), s) != cudaSuccess)
    return RADIC_ECUDA;
  if (ev && cudaEventRecord(ev[1], s) != cudaSuccess) return RADIC_ECUDA;
  return RADIC_OK;
}

}  // namespace radic
