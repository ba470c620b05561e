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
#include "radic_modp.cuh"

namespace radic {

namespace {
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
  if (K == 0) return;  // a wide pass whose primes the bound does not need

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
  if (K == 0) return;  // a wide pass whose primes the bound does not need

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
  if (p.mapping == RADIC_MAP_PREFIX) return modp_prefix_kernel(p.m, p.depth, terms);
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

// ---------------------------------------------------------------------------
// Wide exact result: mixed-radix (Garner) reconstruction of the integer from
// its residues modulo the first K primes, then base-2^32 limbs by Horner's
// rule over the mixed-radix digits, the symmetric range (-M/2, M/2) for the
// sign, M the product of the primes.  One thread; K <= 32.
// ---------------------------------------------------------------------------
__device__ void limbs_mul_add(uint32_t* x, int nl, uint32_t mul, uint32_t add) {
  uint64_t carry = add;
  for (int i = 0; i < nl; ++i) {
    const uint64_t t = static_cast<uint64_t>(x[i]) * mul + carry;
    x[i] = static_cast<uint32_t>(t);
    carry = t >> 32;
  }
}

__global__ void k_wide_crt(const uint32_t* wide, radic_wide_result* out, unsigned long long total) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  constexpr int NL = RADIC_WIDE_LIMBS + 1;  // one spare limb for M
  const int needed = static_cast<int>(wide[kWidePrimes]);
  const int escale = static_cast<int>(wide[kWidePrimes + 1]);
  const int status = static_cast<int>(wide[kWidePrimes + 2]);
  const int K = needed < kWidePrimes ? needed : kWidePrimes;
  uint64_t v[kWidePrimes];
  for (int i = 0; i < K; ++i) {
    const uint64_t p = prime_at(i);
    uint64_t acc = 0, prod = 1;  // digits so far and prod_{l<i} p_l, modulo p
    for (int l = 0; l < i; ++l) {
      acc = (acc + v[l] * prod) % p;
      prod = (prod * (prime_at(l) % p)) % p;
    }
    const uint64_t diff = (wide[i] + p - acc) % p;
    v[i] = (diff * powmod64(prod, p - 2, p)) % p;
  }
  uint32_t x[NL], mm[NL];
  for (int i = 0; i < NL; ++i) x[i] = mm[i] = 0u;
  mm[0] = 1u;
  for (int i = K - 1; i >= 0; --i) limbs_mul_add(x, NL, prime_at(i), static_cast<uint32_t>(v[i]));
  for (int i = 0; i < K; ++i) limbs_mul_add(mm, NL, prime_at(i), 0u);
  // d = M - x; the value is x when x < d (that is x < M/2), else -(M - x)
  uint32_t d[NL];
  long long borrow = 0;
  for (int i = 0; i < NL; ++i) {
    const long long t = static_cast<long long>(mm[i]) - x[i] - borrow;
    d[i] = static_cast<uint32_t>(t);
    borrow = t < 0 ? 1 : 0;
  }
  bool x_less = false;
  for (int i = NL - 1; i >= 0; --i) {
    if (x[i] != d[i]) {
      x_less = x[i] < d[i];
      break;
    }
  }
  const uint32_t* mag = x_less ? x : d;
  int nl = 0;
  for (int i = 0; i < RADIC_WIDE_LIMBS; ++i)
    if (mag[i]) nl = i + 1;
  for (int i = 0; i < RADIC_WIDE_LIMBS; ++i) out->limbs[i] = mag[i];
  double val = 0.0;
  const int lo = nl > 3 ? nl - 3 : 0;
  for (int i = nl - 1; i >= lo; --i) val = val * 4294967296.0 + static_cast<double>(mag[i]);
  const int sgn = nl == 0 ? 0 : (x_less ? 1 : -1);
  out->value = sgn < 0 ? -ldexp(val, 32 * lo + escale) : ldexp(val, 32 * lo + escale);
  out->status = (needed > kWidePrimes) ? RADIC_EOVERFLOW : status;
  out->n_primes = K;
  out->exact_exp = escale;
  out->sign = sgn;
  out->n_limbs = nl;
  out->minors = static_cast<long long>(total);
  out->reserved = 0;
}

__global__ void k_wide_zero(radic_wide_result* out) {
  out->value = 0.0;
  out->status = RADIC_OK;
  out->n_primes = 0;
  out->exact_exp = 0;
  out->sign = 0;
  out->n_limbs = 0;
  out->minors = 0;
  out->reserved = 0;
  for (int i = 0; i < RADIC_WIDE_LIMBS; ++i) out->limbs[i] = 0u;
}

int launch_wide_crt(const uint32_t* wide, radic_wide_result* out, unsigned long long total, cudaStream_t s) {
  if (total == 0) k_wide_zero<<<1, 1, 0, s>>>(out);
  else k_wide_crt<<<1, 32, 0, s>>>(wide, out, total);
  return cudaGetLastError() == cudaSuccess ? RADIC_OK : RADIC_ECUDA;
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
