// Shared parts of the exact (multi-modular) path: Montgomery arithmetic,
// staging of T A mod p, fraction sums, block reduction and the CRT epilogue.
// Included by the per-minor kernels (radic_modp.cu) and the prefix kernels
// (radic_modp_prefix.cu); everything here has internal linkage per file.
#pragma once

#include "radic_prefix.cuh"

namespace radic {

namespace {

constexpr int kMaxThreadsModp = 128;

__constant__ uint32_t c_prime_table[kWidePrimes] = {
    kPrimeTable[0],  kPrimeTable[1],  kPrimeTable[2],  kPrimeTable[3],  kPrimeTable[4],  kPrimeTable[5],
    kPrimeTable[6],  kPrimeTable[7],  kPrimeTable[8],  kPrimeTable[9],  kPrimeTable[10], kPrimeTable[11],
    kPrimeTable[12], kPrimeTable[13], kPrimeTable[14], kPrimeTable[15], kPrimeTable[16], kPrimeTable[17],
    kPrimeTable[18], kPrimeTable[19], kPrimeTable[20], kPrimeTable[21], kPrimeTable[22], kPrimeTable[23],
    kPrimeTable[24], kPrimeTable[25], kPrimeTable[26], kPrimeTable[27], kPrimeTable[28], kPrimeTable[29],
    kPrimeTable[30], kPrimeTable[31]};

__host__ __device__ __forceinline__ uint32_t prime_at(int k) {
#ifdef __CUDA_ARCH__
  return c_prime_table[k];
#else
  return kPrimeTable[k];
#endif
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
  off += (size_t)kMaxM * 4;  // row exponents of floating-point inputs
  return off;
}

struct ModpSmem {
  uint64_t* binom;
  uint32_t* As;  // prime k at As + k * n * cs
  uint32_t* rows;
  uint32_t* scratch;
  int* misc;  // [0] primes the bound needs, [1] total row exponent, [2] non-finite flag
  Mont* mont;
  int* row_e;  // floating-point inputs: row i times 2^-row_e[i] is integer
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
    off += kMaxPrimes * sizeof(Mont);
    row_e = reinterpret_cast<int*>(base + off);
  }
};

__device__ __forceinline__ long long load_int(const void* A, int dtype, long long idx) {
  return dtype == kI8 ? static_cast<long long>(static_cast<const int8_t*>(A)[idx])
                      : static_cast<long long>(static_cast<const int32_t*>(A)[idx]);
}

// ---------------------------------------------------------------------------
// Floating-point inputs.  A binary64 number (binary32 widens to it exactly)
// is +-mant * 2^t with an integer mant < 2^53, so every entry is a dyadic
// rational.  Row i times 2^-e_i, with e_i the exponent of the lowest set bit
// over the row's nonzero entries, is an integer row; every minor is linear
// in each row, so det_R(A) = 2^(sum_i e_i) det_R(M) with M that integer
// matrix, and det_R(M) is found exactly by the modular path.
// ---------------------------------------------------------------------------
struct FpBits {
  uint64_t mant;
  int t;
  bool neg, finite;
};
__device__ __forceinline__ FpBits fp_bits(double x) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  const int E = static_cast<int>((b >> 52) & 0x7ffu);
  const uint64_t f = b & ((1ull << 52) - 1ull);
  FpBits r;
  r.neg = (b >> 63) != 0;
  r.finite = E != 0x7ff;
  r.mant = E ? (f | (1ull << 52)) : f;
  r.t = E ? E - 1075 : -1074;
  return r;
}
__device__ __forceinline__ double load_fp(const void* A, int dtype, long long idx) {
  return dtype == kF32 ? static_cast<double>(static_cast<const float*>(A)[idx]) : static_cast<const double*>(A)[idx];
}
__device__ __forceinline__ bool is_fp_dtype(int dtype) { return dtype == kF32 || dtype == kF64; }

// 2^k mod p, k >= 0 (square and multiply).
__device__ inline uint64_t pow2_mod(int k, uint64_t p) {
  uint64_t r = 1, b = 2 % p;
  while (k) {
    if (k & 1) r = r * b % p;
    b = b * b % p;
    k >>= 1;
  }
  return r % p;
}

// Residue of the integer x * 2^-e modulo p (e at most the exponent of x's
// lowest set bit, so that the shift below drops only zeros).
__device__ inline uint32_t fp_residue(double x, int e, uint32_t p) {
  const FpBits f = fp_bits(x);
  if (f.mant == 0) return 0u;
  uint64_t r;
  if (f.t >= e) {
    r = (f.mant % p) * pow2_mod(f.t - e, p) % p;
  } else {
    r = (f.mant >> (e - f.t)) % p;
  }
  return (f.neg && r) ? static_cast<uint32_t>(p - r) : static_cast<uint32_t>(r);
}

// Row exponents e_i (into row_e) and, per row, the bits of a bound on the
// Euclidean norm of the integer row: |entry| < 2^(top_i + 1 - e_i) with top_i
// the exponent of the highest set bit, so ||M_i|| < sqrt(n) 2^(top_i + 1 - e_i).
// A zero row has e_i = 0 and no bits (all its minors are zero).  Sets
// *nonfinite (shared) when an entry is infinite or NaN.
__device__ inline void fp_row_scales(const void* A, int dtype, int m, int n, long long lda, int* row_e,
                                     double* row_bits, int* nonfinite) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < m; i += nw) {
    int lo = 0x7fffffff, hi = -0x7fffffff;
    bool bad = false;
    for (int j = lane; j < n; j += 32) {
      const FpBits f = fp_bits(load_fp(A, dtype, (long long)i * lda + j));
      if (!f.finite) {
        bad = true;
      } else if (f.mant) {
        lo = min(lo, f.t + __ffsll(static_cast<long long>(f.mant)) - 1);
        hi = max(hi, f.t + 63 - __clzll(static_cast<long long>(f.mant)));
      }
    }
    lo = __reduce_min_sync(kFull, lo);
    hi = __reduce_max_sync(kFull, hi);
    bad = __any_sync(kFull, bad);
    if (lane == 0) {
      const bool zero = hi == -0x7fffffff;
      row_e[i] = zero ? 0 : lo;
      row_bits[i] = zero ? 0.0 : static_cast<double>(hi + 1 - lo) + 0.5 * log2(static_cast<double>(n));
      if (bad) *nonfinite = 1;
    }
  }
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

// Stage binom and, for each prime of the pass, (T A mod p) in Montgomery
// form.  Slot k holds prime a.prime_base + k.  Returns K (primes this pass
// uses; 0 when the bound needs none of them) in every thread; sets *needed
// to the primes the bound asks for.
__device__ inline int stage_modp(const SingleArgs& a, const ModpSmem& sm, int m, int cs, int* needed) {
  const int n = a.n;
  const int base = a.prime_base;
  build_binom(sm.binom, n, m);
  if (threadIdx.x < kMaxPrimes && base + (int)threadIdx.x < kWidePrimes)
    sm.mont[threadIdx.x] = make_mont(prime_at(base + threadIdx.x));
  const bool fp = is_fp_dtype(a.dtype);
  {
    // the rows scratch (m x n words) is free until the residues are staged
    double* row_sq = reinterpret_cast<double*>(sm.rows);
    const double cnt = static_cast<double>(sm.binom[n * (m + 1) + m]);
    if (fp) {
      if (threadIdx.x == 0) sm.misc[2] = 0;
      __syncthreads();
      fp_row_scales(a.A, a.dtype, m, n, a.lda, sm.row_e, row_sq, &sm.misc[2]);
      __syncthreads();
      if (threadIdx.x == 0) {
        double bits = log2(fmax(cnt, 1.0));
        int esum = 0;
        for (int i = 0; i < m; ++i) {
          bits += row_sq[i];
          esum += sm.row_e[i];
        }
        const int k = static_cast<int>(ceil((bits + 2.0) / 30.99));
        sm.misc[0] = k < 1 ? 1 : k;
        sm.misc[1] = esum;
        if (sm.misc[2]) atomicExch(&a.hdr->status, RADIC_EINVAL);  // an entry is not finite
      }
    } else {
      const int need = primes_needed(a.A, a.dtype, m, n, a.lda, log2(fmax(cnt, 1.0)), row_sq);
      if (threadIdx.x == 0) {
        sm.misc[0] = need;
        sm.misc[1] = 0;
      }
    }
  }
  __syncthreads();
  *needed = sm.misc[0];
  const int K = max(0, min(min(sm.misc[0], kWidePrimes) - base, kMaxPrimes));
  for (int k = 0; k < K; ++k) {
    const uint32_t p = prime_at(base + k);
    for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
      const int i = idx / n, j = idx - i * n;
      if (fp) {
        sm.rows[idx] = fp_residue(load_fp(a.A, a.dtype, (long long)i * a.lda + j), sm.row_e[i], p);
      } else {
        long long v = load_int(a.A, a.dtype, (long long)i * a.lda + j) % (long long)p;
        if (v < 0) v += p;
        sm.rows[idx] = static_cast<uint32_t>(v);
      }
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
__device__ inline void block_reduce_modp(uint32_t (&r)[kMaxPrimes], int K, uint32_t* scratch, const Mont* mont) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < kMaxPrimes; ++k) {
    if (k < K) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) r[k] = add_mod(r[k], __shfl_xor_sync(kFull, r[k], off), mont[k].p);
    }
  }
  __syncthreads();
  if (lane == 0)
    for (int k = 0; k < K; ++k) scratch[warp * kMaxPrimes + k] = r[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < K; ++k) {
      uint32_t s = 0;
      for (int w = 0; w < nw; ++w) s = add_mod(s, scratch[w * kMaxPrimes + k], mont[k].p);
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
                                 unsigned long long total, int escale) {
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
  out->value = ldexp(negv ? -val : val, escale);
  out->abs_sum = 0.0;
  out->err_bound = 0.0;
  out->minors = static_cast<long long>(total);
  out->flagged = 0;
  out->status = (needed > kMaxPrimes) ? RADIC_EOVERFLOW : status;
  out->n_primes = K;
  out->tier = kModeExact;
  out->exact_exp = escale;
  for (int i = 0; i < 5; ++i) out->reserved[i] = 0;
}

// Last-block epilogue shared by both mappings.
// Wide passes write the pass's residues into a.wide[prime index] instead;
// the pass with the first primes also writes needed, the exponent and the
// status after the kWidePrimes residue slots.
__device__ inline void finish_modp(const SingleArgs& a, const ModpSmem& sm, uint32_t (&r)[kMaxPrimes], int K,
                                   int needed) {
  block_reduce_modp(r, K, sm.scratch, sm.mont);
  if (threadIdx.x == 0)
    for (int k = 0; k < kMaxPrimes; ++k) a.modp_partials[blockIdx.x * kMaxPrimes + k] = (k < K) ? r[k] : 0u;
  if (last_block(&a.hdr->ticket[0])) {
    uint32_t t[kMaxPrimes] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      for (int k = 0; k < K; ++k) t[k] = add_mod(t[k], __ldcg(&a.modp_partials[b * kMaxPrimes + k]), sm.mont[k].p);
    block_reduce_modp(t, K, sm.scratch, sm.mont);
    if (threadIdx.x == 0) {
      if (a.wide) {
        for (int k = 0; k < K; ++k) a.wide[a.prime_base + k] = t[k];
        if (a.prime_base == 0) {
          a.wide[kWidePrimes] = static_cast<uint32_t>(needed);
          a.wide[kWidePrimes + 1] = static_cast<uint32_t>(sm.misc[1]);
          a.wide[kWidePrimes + 2] = static_cast<uint32_t>(__ldcg(&a.hdr->status));
        }
      } else {
        crt_write(a.out, t, K, needed, __ldcg(&a.hdr->status), a.total, sm.misc[1]);
      }
    }
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

}  // namespace

}  // namespace radic
