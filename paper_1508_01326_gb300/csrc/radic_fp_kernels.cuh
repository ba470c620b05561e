// Floating-point kernels of the Radic determinant (binary64 and mixed
// binary32/binary64), one matrix per launch.
//
// Per thread (thread mapping) or per group of lanes (group mapping) the hot
// loop is: unrank the first dictionary rank of a task (Section 4), then for
// every rank of the task gather the minor, factor it with partial pivoting,
// apply the sign of Eq. (1) and accumulate, and step to the next rank with
// the dictionary successor (Section 5).  Tasks are contiguous runs of ranks
// dealt round-robin to threads (the chunked split of Section 5); per-block
// partial sums are combined by the last block in block order (Section 6).
#pragma once

#include <cfloat>
#include <map>
#include <mutex>
#include <utility>

#include "radic_device.cuh"

namespace radic {

constexpr int kMaxThreadsFp = 256;

// Kernels whose dynamic shared memory exceeds the default 48 KiB must opt in.
// Raises a kernel's dynamic shared-memory limit above the 48 KB default.  The
// attribute persists in the device's context, so each (device, kernel) pair
// is set once to the largest size asked for so far.
inline bool allow_smem(const void* kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return true;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = done[{dev, kernel}];
  if (have >= bytes) return true;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)) !=
      cudaSuccess)
    return false;
  have = bytes;
  return true;
}

// Shared-memory layout of the floating-point kernels: binomial table, the
// staged matrix, row exponents, column norms (error bounds), reduction
// scratch.
// The pair arithmetic also keeps a binary64 copy of the staged matrix (its
// prefixes are factored in binary64): `dbl` adds n x (m rounded up to even)
// binary64 words.
__host__ __device__ inline size_t fp_smem_bytes(int n, int m, int cs, int elem, int threads, bool dbl = false) {
  size_t off = ((size_t)(n + 1) * (m + 1) * 8 + 15) / 16 * 16;
  off += ((size_t)n * cs * elem + 15) / 16 * 16;
  off += ((size_t)m * 4 + 15) / 16 * 16;
  off += ((size_t)n * 8 + 15) / 16 * 16;
  off += (size_t)kScratchWords * (threads / 32) * 8;
  if (dbl) off += (size_t)n * ((m + 1) / 2 * 2) * 8;
  return off;
}

template <typename T>
struct FpSmem {
  uint64_t* binom;
  T* As;
  int* row_exp;
  Rad<T>* colnorm;
  double* scratch;
  double* As64;  // pairs only: binary64 copy, column stride m rounded up to even
  __device__ FpSmem(unsigned char* base, int n, int m, int cs) {
    size_t off = 0;
    binom = reinterpret_cast<uint64_t*>(base);
    off = ((size_t)(n + 1) * (m + 1) * 8 + 15) / 16 * 16;
    As = reinterpret_cast<T*>(base + off);
    off += ((size_t)n * cs * sizeof(T) + 15) / 16 * 16;
    row_exp = reinterpret_cast<int*>(base + off);
    off += ((size_t)m * 4 + 15) / 16 * 16;
    colnorm = reinterpret_cast<Rad<T>*>(base + off);
    off += ((size_t)n * 8 + 15) / 16 * 16;
    scratch = reinterpret_cast<double*>(base + off);
    off += (size_t)kScratchWords * (blockDim.x / 32) * 8;
    As64 = std::is_same<T, ff>::value ? reinterpret_cast<double*>(base + off) : nullptr;
  }
};

// Binary64 copy (column stride cs64) of a pair-staged matrix, exact.
__device__ __forceinline__ void stage_double_copy(const ff* As, int cs, int m, int n, double* As64, int cs64, int t0,
                                                  int nt) {
  for (int idx = t0; idx < n * cs64; idx += nt) {
    const int j = idx / cs64, i = idx - j * cs64;
    As64[idx] = i < m ? as_double(As[j * cs + i]) : 0.0;
  }
}

// ||A[:, j]||_2 of the staged matrix for every column j (column stride cs),
// rounded up, computed by the threads [t0, t0 + nt) of the block; the caller
// synchronises before use.
template <typename T>
__device__ __forceinline__ void column_norms(const T* As, int cs, int m, int n, Rad<T>* colnorm, int t0, int nt) {
  using R = Rad<T>;
  for (int j = t0; j < n; j += nt) {
    R s = R(0);
    for (int i = 0; i < m; ++i) {
      const R a = mag(As[j * cs + i]);
      s += a * a;
    }
    colnorm[j] = sqrt(s) * R(1.000001);
  }
}

// Flag test of the mixed mode: not finite, or pivot growth above threshold.
template <typename T>
__device__ __forceinline__ bool mixed_flag(T det, T gmax, T thr) {
  return !(fabs(det) <= static_cast<T>(FLT_MAX)) || !(gmax <= thr);
}

// Writes the final radic_result from block-ordered partial sums.  `bound`
// is the sum of the lanes' error bounds (scaled rows); the result's
// err_bound adds the margin of radic_bound.cuh and the rounding of the
// accumulation across lanes and blocks: binary64 two-sums lose at most
// 2^-70 sum|terms| over chains of up to 2^17 additions per lane plus one
// rounding of the value, float-float lane totals (binary32 elimination) at
// most 2^-30 sum|terms| over up to 2^16 prefixes per lane.
__device__ inline void write_fp_result(radic_result* out, const Dd& t, double abs_sum, double bound, int escale,
                                       int m, unsigned long long total, long long flagged, int status, int tier) {
  (void)m;
  const double acc = (tier == kModeMixed ? 0x1p-30 : 0x1p-70) * abs_sum + 0x1p-52 * fabs(t.hi + t.lo);
  out->value = scale_pow2(t.hi + t.lo, -escale);
  out->abs_sum = scale_pow2(abs_sum, -escale);
  out->err_bound = scale_pow2(kBoundMargin * bound + acc, -escale);
  out->exact_lo = 0;
  out->exact_hi = 0;
  out->minors = static_cast<long long>(total);
  out->flagged = flagged;
  out->status = status;
  out->n_primes = 0;
  out->tier = tier;
  out->exact_exp = 0;
  for (int i = 0; i < 5; ++i) out->reserved[i] = 0;
}

// Last block of the main kernel: sums the per-block partials in block order
// and writes the result.  In the mixed mode it also leaves the totals and the
// number of flagged entries in the workspace header for the fix-up kernel,
// which rewrites the result only when something was flagged.
// Tier (mode) that produced a floating-point result: binary64, binary32
// elimination (MIXED) or pairs of binary32 (PAIR).
template <typename T, bool kMixed>
__host__ __device__ constexpr int tier_of() {
  return !kMixed ? kModeFp64 : (std::is_same<T, ff>::value ? kModePair : kModeMixed);
}

constexpr int kFinishUnroll = 8;

template <bool kMixed>
__device__ inline void finish_fp_main(const SingleArgs& a, double* scratch, int escale, int m, int tier) {
  if (!last_block(&a.hdr->ticket[0])) return;
  Dd t;
  double ab = 0.0, bd_sum = 0.0;
  long long fl = 0;
  // partials b = tid, tid + blockDim, ... in that order; kFinishUnroll of
  // them are loaded before any is added, so that their L2 round trips overlap
  const int nb = gridDim.x, bd = blockDim.x;
  for (int b0 = threadIdx.x; b0 < nb; b0 += kFinishUnroll * bd) {
    double2 v[kFinishUnroll];
    double va[kFinishUnroll], vb[kFinishUnroll];
    long long vc[kFinishUnroll];
#pragma unroll
    for (int u = 0; u < kFinishUnroll; ++u) {
      const int b = b0 + u * bd;
      v[u] = b < nb ? __ldcg(reinterpret_cast<const double2*>(&a.partials[b])) : make_double2(0.0, 0.0);
      va[u] = b < nb ? __ldcg(&a.partials[b].abs_sum) : 0.0;
      vb[u] = b < nb ? __ldcg(&a.partials[b].bound) : 0.0;
      vc[u] = b < nb ? __ldcg(&a.partials[b].count) : 0ll;
    }
#pragma unroll
    for (int u = 0; u < kFinishUnroll; ++u) {
      if (b0 + u * bd < nb) {
        Dd o;
        o.hi = v[u].x;
        o.lo = v[u].y;
        t.merge(o);
        ab += va[u];
        bd_sum += vb[u];
        fl += vc[u];
      }
    }
  }
  block_reduce_dd(t, ab, fl, bd_sum, scratch);
  if (threadIdx.x == 0) {
    if constexpr (kMixed) {
      a.hdr->main_hi = t.hi;
      a.hdr->main_lo = t.lo;
      a.hdr->main_abs = ab;
      a.hdr->main_bnd = bd_sum;
      a.hdr->flag_total = fl;
      a.hdr->escale = escale;
    }
    write_fp_result(a.out, t, ab, bd_sum, escale, m, a.total, 0, a.hdr->status, tier);
  }
}

// The same for the binary32-elimination prefix kernel, whose partials are
// float-float (FfPartial): the sum over blocks stays on the binary32 pipe and
// is widened to binary64 once.  The rounding of these merges (about 2^-46 of
// the magnitudes added, per level) lies far below the binary32 rounding of
// the minors, and write_fp_result's accumulation term covers it.
__device__ inline void finish_ff_main(const SingleArgs& a, double* scratch, int escale, int m) {
  if (!last_block(&a.hdr->ticket[0])) return;
  const FfPartial* p = reinterpret_cast<const FfPartial*>(a.partials);
  Ff t, ta;
  long long fl = 0;
  double bd_sum = 0.0;
  const int nb = gridDim.x, bd = blockDim.x;
  for (int b0 = threadIdx.x; b0 < nb; b0 += kFinishUnroll * bd) {
    float4 v[kFinishUnroll];
    long long vc[kFinishUnroll];
    double vb[kFinishUnroll];
#pragma unroll
    for (int u = 0; u < kFinishUnroll; ++u) {
      const int b = b0 + u * bd;
      v[u] = b < nb ? __ldcg(reinterpret_cast<const float4*>(&p[b])) : make_float4(0.f, 0.f, 0.f, 0.f);
      vc[u] = b < nb ? __ldcg(&p[b].count) : 0ll;
      vb[u] = b < nb ? __ldcg(&p[b].bound) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kFinishUnroll; ++u) {
      if (b0 + u * bd < nb) {
        t.merge(Ff{v[u].x, v[u].y});
        ta.merge(Ff{v[u].z, v[u].w});
        fl += vc[u];
        bd_sum += vb[u];
      }
    }
  }
  block_reduce_ff(t, ta, fl, bd_sum, scratch);
  if (threadIdx.x == 0) {
    Dd d;  // exact widening of the pair
    d.hi = static_cast<double>(t.hi);
    d.lo = static_cast<double>(t.lo);
    const double ab = static_cast<double>(ta.hi) + static_cast<double>(ta.lo);
    a.hdr->main_hi = d.hi;
    a.hdr->main_lo = d.lo;
    a.hdr->main_abs = ab;
    a.hdr->main_bnd = bd_sum;
    a.hdr->flag_total = fl;
    a.hdr->escale = escale;
    write_fp_result(a.out, d, ab, bd_sum, escale, m, a.total, 0, a.hdr->status, kModeMixed);
  }
}

// ---------------------------------------------------------------------------
// Thread mapping: one thread per minor, the minor in registers.
// ---------------------------------------------------------------------------
template <typename T, int M, bool kMixed, bool kTerms>
__global__ void __launch_bounds__(kMaxThreadsFp) k_fp_thread(SingleArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int CS = ColStride<T, M>::value;
  FpSmem<T> sm(smem_raw, a.n, M, CS);
  const int n = a.n;
  build_binom(sm.binom, n, M);
  bool exact_in;
  const int escale = stage_scaled<T>(a.A, a.dtype, M, n, a.lda, sm.As, CS, sm.row_exp, &exact_in);
  const float uin = exact_in ? 0.0f : static_cast<float>(BoundTraits<T>::u_in);

  const int lane = threadIdx.x & 31;
  const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long L = a.ranks_per_task;
  const unsigned long long qbase = kTerms ? a.q0 : 0ull;
  const unsigned long long qlim = kTerms ? a.q0 + a.count : a.total;
  const T thr = static_cast<T>(a.growth);

  Dd acc;
  double abs_sum = 0.0, bnd = 0.0;
  int fcnt = 0;  // flagged ranks of this warp so far (warp-uniform)
  unsigned long long* flist = nullptr;
  if constexpr (kMixed && !kTerms) flist = a.flag_ranks + (g >> 5) * (unsigned long long)a.flag_cap;

  for (unsigned long long base = g - lane; base < a.tasks; base += nthreads) {
    const unsigned long long task = base + lane;
    const bool tact = task < a.tasks;
    const unsigned long long q0 = qbase + (tact ? task : 0ull) * L;
    const unsigned long long q1 = min(q0 + L, qlim);
    int c[M];
    unrank<M>(q0, n, sm.binom, M + 1, c);
    Ff run;
    float run_abs = 0.0f, run_bnd = 0.0f;
    for (unsigned long long it = 0; it < L; ++it) {
      const unsigned long long q = q0 + it;
      const bool act = tact && q < q1;
      T mm[M][M];
      gather<T, M, CS>(sm.As, c, mm);
      T gmax, det;
      float b = 0.0f;
      bool bad = false;
      if constexpr (kTerms) {
        det = lu_det<T, M>(mm, gmax);
      } else {
        det = lu_det_b<T, M>(mm, gmax, b, bad, uin);
      }
      if (sign_negative<M>(c)) det = -det;
      bool flag = false;
      if constexpr (kMixed) flag = mixed_flag<T>(det, gmax, thr) || bad;
      if constexpr (kTerms) {
        if (act) {
          double* terms = static_cast<double*>(a.terms);
          terms[q - a.q0] = flag ? __longlong_as_double(0x7ff8000000000000ll) : ldexp((double)det, escale);
        }
      } else if constexpr (kMixed) {
        if (act && !flag) {
          run.add(static_cast<float>(det));
          run_abs += fabsf(static_cast<float>(det));
          run_bnd += b;
        }
        const unsigned fm = __ballot_sync(kFull, act && flag);
        if (fm) {
          if (act && flag) {
            const int pos = fcnt + __popc(fm & ((1u << lane) - 1u));
            if (pos < a.flag_cap) flist[pos] = q;
          }
          fcnt += __popc(fm);
        }
      } else {
        if (act) {
          acc.add(static_cast<double>(det));
          abs_sum += fabs(static_cast<double>(det));
          run_bnd += b;
        }
      }
      if constexpr (!kTerms) {
        if ((it & 255) == 255) {  // keep the binary32 partial sums short
          if constexpr (kMixed) {
            acc.add(static_cast<double>(run.hi));
            acc.add(static_cast<double>(run.lo));
            abs_sum += static_cast<double>(run_abs);
            run = Ff();
            run_abs = 0.0f;
          }
          bnd += static_cast<double>(run_bnd);
          run_bnd = 0.0f;
        }
      }
      if (q + 1 < q1) successor<M>(c, n);
    }
    if constexpr (!kTerms) {
      if constexpr (kMixed) {
        acc.add(static_cast<double>(run.hi));
        acc.add(static_cast<double>(run.lo));
        abs_sum += static_cast<double>(run_abs);
      }
      bnd += static_cast<double>(run_bnd);
    }
  }
  if constexpr (!kTerms) {
    long long cnt = 0;
    if constexpr (kMixed) {
      if (lane == 0) {
        a.flag_count[g >> 5] = fcnt;
        if (fcnt > a.flag_cap) atomicOr(&a.hdr->overflow, 1);
        cnt = fcnt;
      }
    }
    block_reduce_dd(acc, abs_sum, cnt, bnd, sm.scratch);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = FpPartial{acc.hi, acc.lo, abs_sum, cnt, bnd, 0.0};
    finish_fp_main<kMixed>(a, sm.scratch, escale, M, tier_of<T, kMixed>());
  }
}

// ---------------------------------------------------------------------------
// Group mapping: G lanes of a warp per minor, lane `sub` holds row `sub` of
// the minor.  Pivot search is a butterfly max over the group, the pivot row
// is broadcast by shuffles, and rows are never moved: the sign of the row
// permutation is the parity of the number of still-active rows above each
// chosen pivot.
// ---------------------------------------------------------------------------
template <typename T, int G>
__device__ __forceinline__ T group_det(T (&x)[G], int m, int sub, int seg, T& gmax) {
  bool alive = sub < m;
  T det = T(1);
  int par = 0;
  gmax = T(0);
  const unsigned segbits = (G == 32) ? kFull : ((1u << G) - 1u);
#pragma unroll
  for (int k = 0; k < G; ++k) {
    if (k >= m) break;
    uint32_t key = alive ? ((mag_key(x[k]) & ~31u) | (uint32_t)(G - 1 - sub)) : 0u;
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) key = max(key, __shfl_xor_sync(kFull, key, off));
    const int p = G - 1 - (int)(key & 31u);
    const T piv = __shfl_sync(kFull, x[k], p, G);
    const unsigned alive_bits = (__ballot_sync(kFull, alive) >> (seg * G)) & segbits;
    par ^= __popc(alive_bits & ((1u << p) - 1u)) & 1;
    if (sub == p) alive = false;
    det *= piv;
    gmax = fmax(gmax, fabs(piv));
    T r;
    if constexpr (sizeof(T) == 8) r = rcp_f64(piv);
    else r = rcp_f32(piv);
    const T l = alive ? x[k] * r : T(0);
#pragma unroll
    for (int j = k + 1; j < G; ++j) {
      if (j < m) {
        const T u = __shfl_sync(kFull, x[j], p, G);
        x[j] = fma(-l, u, x[j]);
      }
    }
  }
  return par ? -det : det;
}

// group_det with running error radii (binary32, one per entry of the
// lane's row; radic_bound.cuh): the pivot row's radii travel with it by the
// same shuffles.  bnd and bad are valid in every lane of the group.
template <typename T, int G>
__device__ __forceinline__ T group_det_b(T (&x)[G], int m, int sub, int seg, T& gmax, float& bnd, bool& bad,
                                         float u_in = static_cast<float>(BoundTraits<T>::u_in)) {
  constexpr float u = static_cast<float>(BoundTraits<T>::u);
  constexpr float c_div = static_cast<float>(BoundTraits<T>::c_div);
  float rx[G];
#pragma unroll
  for (int j = 0; j < G; ++j) rx[j] = u_in * mag(x[j]);
  bool alive = sub < m;
  T det = T(1);
  int par = 0;
  float rel = 0.0f, pr = 1.0f;  // pr = prod (|p_k| + r_k)
  bool last_open = false;
  bad = false;
  gmax = T(0);
  const unsigned segbits = (G == 32) ? kFull : ((1u << G) - 1u);
#pragma unroll
  for (int k = 0; k < G; ++k) {
    if (k >= m) break;
    uint32_t key = alive ? ((mag_key(x[k]) & ~31u) | (uint32_t)(G - 1 - sub)) : 0u;
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) key = max(key, __shfl_xor_sync(kFull, key, off));
    const int p = G - 1 - (int)(key & 31u);
    const T piv = __shfl_sync(kFull, x[k], p, G);
    const float rp = __shfl_sync(kFull, rx[k], p, G);
    const unsigned alive_bits = (__ballot_sync(kFull, alive) >> (seg * G)) & segbits;
    par ^= __popc(alive_bits & ((1u << p) - 1u)) & 1;
    if (sub == p) alive = false;
    det *= piv;
    gmax = fmax(gmax, fabs(piv));
    const float ap = mag(piv);
    pr *= ap + rp;
    const float ipm = ap > 0.0f ? __frcp_ru(ap) : 0.0f;
    const float ipd = ap > rp ? __frcp_ru(__fsub_rd(ap, rp)) : 0.0f;
    if (k == m - 1) {
      // the last pivot divides nothing: a singular minor is bounded by the
      // product of the pivot enclosures instead
      last_open = pivot_unbounded(ap, rp) || ap == 0.0f;
    } else {
      bad |= pivot_unbounded(ap, rp);
    }
    if (!last_open) rel = fmaf(1.0f + rel, rp * ipm, rel);
    T r;
    if constexpr (sizeof(T) == 8) r = rcp_f64(piv);
    else r = rcp_f32(piv);
    const T l = alive ? x[k] * r : T(0);
    const float al = mag(l);
    const float rl = alive ? (rx[k] + al * rp) * ipd + c_div * u * al : 0.0f;
#pragma unroll
    for (int j = k + 1; j < G; ++j) {
      if (j < m) {
        const T uj = __shfl_sync(kFull, x[j], p, G);
        const float ru = __shfl_sync(kFull, rx[j], p, G);
        const float au = mag(uj), old = mag(x[j]);
        x[j] = fma(-l, uj, x[j]);
        rx[j] += al * ru + (au + ru) * rl + u * (al * au + old);
      }
    }
  }
  rel = fmaf(1.0f + rel, static_cast<float>(m - 1) * u * 1.01f, rel);
  bnd = last_open ? (pr * (1.0f + static_cast<float>(m) * u) + static_cast<float>(m) * u *
                                                                      mag(det)) * 1.0000002f
                  : rel * mag(det) * 1.0000001f;
  return par ? -det : det;
}

template <typename T, int G, bool kMixed, bool kTerms>
__global__ void __launch_bounds__(kMaxThreadsFp) k_fp_group(SingleArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n, m = a.m;
  FpSmem<T> sm(smem_raw, n, m, m);
  build_binom(sm.binom, n, m);
  bool exact_in;
  const int escale = stage_scaled<T>(a.A, a.dtype, m, n, a.lda, sm.As, m, sm.row_exp, &exact_in);
  const float uin = exact_in ? 0.0f : static_cast<float>(BoundTraits<T>::u_in);
  if constexpr (!kTerms) {
    column_norms<T>(sm.As, m, m, n, sm.colnorm, threadIdx.x, blockDim.x);
    __syncthreads();
  }

  const int lane = threadIdx.x & 31, sub = lane & (G - 1), seg = lane / G;
  constexpr int kSegs = 32 / G;
  const unsigned long long gwarp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nsegs = (unsigned long long)gridDim.x * blockDim.x / G;
  const unsigned long long L = a.ranks_per_task;
  const unsigned long long qbase = kTerms ? a.q0 : 0ull;
  const unsigned long long qlim = kTerms ? a.q0 + a.count : a.total;
  const T thr = static_cast<T>(a.growth);

  Dd acc;
  double abs_sum = 0.0, bnd = 0.0;
  int fcnt = 0;
  unsigned long long* flist = nullptr;
  if constexpr (kMixed && !kTerms) flist = a.flag_ranks + gwarp * (unsigned long long)a.flag_cap;

  for (unsigned long long base = gwarp * kSegs; base < a.tasks; base += nsegs) {
    const unsigned long long task = base + seg;
    const bool tact = task < a.tasks;
    const unsigned long long q0 = qbase + (tact ? task : 0ull) * L;
    const unsigned long long q1 = min(q0 + L, qlim);
    int c[G];
    unrank_dyn<G>(q0, n, m, sm.binom, m + 1, c);
    Ff run;
    float run_abs = 0.0f, run_bnd = 0.0f;
    for (unsigned long long it = 0; it < L; ++it) {
      const unsigned long long q = q0 + it;
      const bool act = tact && q < q1;
      T x[G];
#pragma unroll
      for (int j = 0; j < G; ++j) x[j] = (j < m && sub < m) ? sm.As[c[j] * m + sub] : T(0);
      T gmax, det;
      float b = 0.0f;
      bool bad = false;
      if constexpr (kTerms) {
        det = group_det<T, G>(x, m, sub, seg, gmax);
      } else {
        det = group_det_b<T, G>(x, m, sub, seg, gmax, b, bad, uin);
        if (bad && !kMixed) {  // Hadamard's inequality alone
          float h = 1.0f;
#pragma unroll
          for (int j = 0; j < G; ++j)
            if (j < m) h *= static_cast<float>(sm.colnorm[c[j]]);
          b = mag(det) * 1.0000002f + h;
        }
      }
      if (sign_negative_dyn<G>(c, m)) det = -det;
      bool flag = false;
      if constexpr (kMixed) flag = mixed_flag<T>(det, gmax, thr) || bad;
      const bool lead = act && sub == 0;
      if constexpr (kTerms) {
        if (lead) {
          double* terms = static_cast<double*>(a.terms);
          terms[q - a.q0] = flag ? __longlong_as_double(0x7ff8000000000000ll) : ldexp((double)det, escale);
        }
      } else if constexpr (kMixed) {
        if (lead && !flag) {
          run.add(static_cast<float>(det));
          run_abs += fabsf(static_cast<float>(det));
          run_bnd += b;
        }
        const unsigned fm = __ballot_sync(kFull, lead && flag);
        if (fm) {
          if (lead && flag) {
            const int pos = fcnt + __popc(fm & ((1u << lane) - 1u));
            if (pos < a.flag_cap) flist[pos] = q;
          }
          fcnt += __popc(fm);
        }
      } else {
        if (lead) {
          acc.add(static_cast<double>(det));
          abs_sum += fabs(static_cast<double>(det));
          run_bnd += b;
        }
      }
      if constexpr (!kTerms) {
        if ((it & 255) == 255) {
          if constexpr (kMixed) {
            acc.add(static_cast<double>(run.hi));
            acc.add(static_cast<double>(run.lo));
            abs_sum += static_cast<double>(run_abs);
            run = Ff();
            run_abs = 0.0f;
          }
          bnd += static_cast<double>(run_bnd);
          run_bnd = 0.0f;
        }
      }
      if (q + 1 < q1) successor_dyn<G>(c, n, m);
    }
    if constexpr (!kTerms) {
      if constexpr (kMixed) {
        acc.add(static_cast<double>(run.hi));
        acc.add(static_cast<double>(run.lo));
        abs_sum += static_cast<double>(run_abs);
      }
      bnd += static_cast<double>(run_bnd);
    }
  }
  if constexpr (!kTerms) {
    long long cnt = 0;
    if constexpr (kMixed) {
      if (lane == 0) {
        a.flag_count[gwarp] = fcnt;
        if (fcnt > a.flag_cap) atomicOr(&a.hdr->overflow, 1);
        cnt = fcnt;
      }
    }
    block_reduce_dd(acc, abs_sum, cnt, bnd, sm.scratch);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = FpPartial{acc.hi, acc.lo, abs_sum, cnt, bnd, 0.0};
    finish_fp_main<kMixed>(a, sm.scratch, escale, m, tier_of<T, kMixed>());
  }
}

}  // namespace radic
