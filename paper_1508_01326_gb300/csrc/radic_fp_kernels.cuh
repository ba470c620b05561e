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

// Shared-memory layout of the floating-point kernels.
__host__ __device__ inline size_t fp_smem_bytes(int n, int m, int cs, int elem, int threads) {
  size_t off = ((size_t)(n + 1) * (m + 1) * 8 + 15) / 16 * 16;
  off += ((size_t)n * cs * elem + 15) / 16 * 16;
  off += ((size_t)m * 4 + 15) / 16 * 16;
  off += (size_t)4 * (threads / 32) * 8;
  return off;
}

template <typename T>
struct FpSmem {
  uint64_t* binom;
  T* As;
  int* row_exp;
  double* scratch;
  __device__ FpSmem(unsigned char* base, int n, int m, int cs) {
    size_t off = 0;
    binom = reinterpret_cast<uint64_t*>(base);
    off = ((size_t)(n + 1) * (m + 1) * 8 + 15) / 16 * 16;
    As = reinterpret_cast<T*>(base + off);
    off += ((size_t)n * cs * sizeof(T) + 15) / 16 * 16;
    row_exp = reinterpret_cast<int*>(base + off);
    off += ((size_t)m * 4 + 15) / 16 * 16;
    scratch = reinterpret_cast<double*>(base + off);
  }
};

// Flag test of the mixed mode: not finite, or pivot growth above threshold.
template <typename T>
__device__ __forceinline__ bool mixed_flag(T det, T gmax, T thr) {
  return !(fabs(det) <= static_cast<T>(FLT_MAX)) || !(gmax <= thr);
}

// Writes the final radic_result from block-ordered partial sums.
__device__ inline void write_fp_result(radic_result* out, const Dd& t, double abs_sum, int escale, int m,
                                       unsigned long long total, long long flagged, int status, int tier) {
  // unit roundoff of the elimination: binary64, pairs of binary32 (about
  // 2^-46 per operation, 2^-44 allows for the renormalisations), binary32
  const double u = (tier == kModeFp64) ? 0x1p-53 : (tier == kModePair ? 0x1p-44 : 0x1p-24);
  out->value = scale_pow2(t.hi + t.lo, -escale);
  out->abs_sum = scale_pow2(abs_sum, -escale);
  out->err_est = static_cast<double>(m) * u * out->abs_sum;
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
  double ab = 0.0;
  long long fl = 0;
  // partials b = tid, tid + blockDim, ... in that order; kFinishUnroll of
  // them are loaded before any is added, so that their L2 round trips overlap
  const int nb = gridDim.x, bd = blockDim.x;
  for (int b0 = threadIdx.x; b0 < nb; b0 += kFinishUnroll * bd) {
    double2 v[kFinishUnroll];
    double va[kFinishUnroll];
    long long vc[kFinishUnroll];
#pragma unroll
    for (int u = 0; u < kFinishUnroll; ++u) {
      const int b = b0 + u * bd;
      v[u] = b < nb ? __ldcg(reinterpret_cast<const double2*>(&a.partials[b])) : make_double2(0.0, 0.0);
      va[u] = b < nb ? __ldcg(&a.partials[b].abs_sum) : 0.0;
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
        fl += vc[u];
      }
    }
  }
  block_reduce_dd(t, ab, fl, scratch);
  if (threadIdx.x == 0) {
    if constexpr (kMixed) {
      a.hdr->main_hi = t.hi;
      a.hdr->main_lo = t.lo;
      a.hdr->main_abs = ab;
      a.hdr->flag_total = fl;
      a.hdr->escale = escale;
    }
    write_fp_result(a.out, t, ab, escale, m, a.total, 0, a.hdr->status, tier);
  }
}

// The same for the binary32-elimination prefix kernel, whose partials are
// float-float (FfPartial): the sum over blocks stays on the binary32 pipe and
// is widened to binary64 once.  The rounding of these merges (about 2^-46 of
// the magnitudes added, per level) lies far below the binary32 rounding of
// the minors that the mixed mode's error estimate states.
__device__ inline void finish_ff_main(const SingleArgs& a, double* scratch, int escale, int m) {
  if (!last_block(&a.hdr->ticket[0])) return;
  const FfPartial* p = reinterpret_cast<const FfPartial*>(a.partials);
  Ff t, ta;
  long long fl = 0;
  const int nb = gridDim.x, bd = blockDim.x;
  for (int b0 = threadIdx.x; b0 < nb; b0 += kFinishUnroll * bd) {
    float4 v[kFinishUnroll];
    long long vc[kFinishUnroll];
#pragma unroll
    for (int u = 0; u < kFinishUnroll; ++u) {
      const int b = b0 + u * bd;
      v[u] = b < nb ? __ldcg(reinterpret_cast<const float4*>(&p[b])) : make_float4(0.f, 0.f, 0.f, 0.f);
      vc[u] = b < nb ? __ldcg(&p[b].count) : 0ll;
    }
#pragma unroll
    for (int u = 0; u < kFinishUnroll; ++u) {
      if (b0 + u * bd < nb) {
        t.merge(Ff{v[u].x, v[u].y});
        ta.merge(Ff{v[u].z, v[u].w});
        fl += vc[u];
      }
    }
  }
  block_reduce_ff(t, ta, fl, scratch);
  if (threadIdx.x == 0) {
    Dd d;  // exact widening of the pair
    d.hi = static_cast<double>(t.hi);
    d.lo = static_cast<double>(t.lo);
    const double ab = static_cast<double>(ta.hi) + static_cast<double>(ta.lo);
    a.hdr->main_hi = d.hi;
    a.hdr->main_lo = d.lo;
    a.hdr->main_abs = ab;
    a.hdr->flag_total = fl;
    a.hdr->escale = escale;
    write_fp_result(a.out, d, ab, escale, m, a.total, 0, a.hdr->status, kModeMixed);
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
  const int escale = stage_scaled<T>(a.A, a.dtype, M, n, a.lda, sm.As, CS, sm.row_exp);

  const int lane = threadIdx.x & 31;
  const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long L = a.ranks_per_task;
  const unsigned long long qbase = kTerms ? a.q0 : 0ull;
  const unsigned long long qlim = kTerms ? a.q0 + a.count : a.total;
  const T thr = static_cast<T>(a.growth);

  Dd acc;
  double abs_sum = 0.0;
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
    float run_abs = 0.0f;
    for (unsigned long long it = 0; it < L; ++it) {
      const unsigned long long q = q0 + it;
      const bool act = tact && q < q1;
      T mm[M][M];
      gather<T, M, CS>(sm.As, c, mm);
      T gmax;
      T det = lu_det<T, M>(mm, gmax);
      if (sign_negative<M>(c)) det = -det;
      bool flag = false;
      if constexpr (kMixed) flag = mixed_flag<T>(det, gmax, thr);
      if constexpr (kTerms) {
        if (act) {
          double* terms = static_cast<double*>(a.terms);
          terms[q - a.q0] = flag ? __longlong_as_double(0x7ff8000000000000ll) : ldexp((double)det, escale);
        }
      } else if constexpr (kMixed) {
        if (act && !flag) {
          run.add(static_cast<float>(det));
          run_abs += fabsf(static_cast<float>(det));
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
        }
      }
      if constexpr (kMixed && !kTerms) {
        if ((it & 255) == 255) {  // keep the binary32 partial sums short
          acc.add(static_cast<double>(run.hi));
          acc.add(static_cast<double>(run.lo));
          abs_sum += static_cast<double>(run_abs);
          run = Ff();
          run_abs = 0.0f;
        }
      }
      if (q + 1 < q1) successor<M>(c, n);
    }
    if constexpr (kMixed && !kTerms) {
      acc.add(static_cast<double>(run.hi));
      acc.add(static_cast<double>(run.lo));
      abs_sum += static_cast<double>(run_abs);
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
    block_reduce_dd(acc, abs_sum, cnt, sm.scratch);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = FpPartial{acc.hi, acc.lo, abs_sum, cnt};
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

template <typename T, int G, bool kMixed, bool kTerms>
__global__ void __launch_bounds__(kMaxThreadsFp) k_fp_group(SingleArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n, m = a.m;
  FpSmem<T> sm(smem_raw, n, m, m);
  build_binom(sm.binom, n, m);
  const int escale = stage_scaled<T>(a.A, a.dtype, m, n, a.lda, sm.As, m, sm.row_exp);

  const int lane = threadIdx.x & 31, sub = lane & (G - 1), seg = lane / G;
  constexpr int kSegs = 32 / G;
  const unsigned long long gwarp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nsegs = (unsigned long long)gridDim.x * blockDim.x / G;
  const unsigned long long L = a.ranks_per_task;
  const unsigned long long qbase = kTerms ? a.q0 : 0ull;
  const unsigned long long qlim = kTerms ? a.q0 + a.count : a.total;
  const T thr = static_cast<T>(a.growth);

  Dd acc;
  double abs_sum = 0.0;
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
    float run_abs = 0.0f;
    for (unsigned long long it = 0; it < L; ++it) {
      const unsigned long long q = q0 + it;
      const bool act = tact && q < q1;
      T x[G];
#pragma unroll
      for (int j = 0; j < G; ++j) x[j] = (j < m && sub < m) ? sm.As[c[j] * m + sub] : T(0);
      T gmax;
      T det = group_det<T, G>(x, m, sub, seg, gmax);
      if (sign_negative_dyn<G>(c, m)) det = -det;
      bool flag = false;
      if constexpr (kMixed) flag = mixed_flag<T>(det, gmax, thr);
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
        }
      }
      if constexpr (kMixed && !kTerms) {
        if ((it & 255) == 255) {
          acc.add(static_cast<double>(run.hi));
          acc.add(static_cast<double>(run.lo));
          abs_sum += static_cast<double>(run_abs);
          run = Ff();
          run_abs = 0.0f;
        }
      }
      if (q + 1 < q1) successor_dyn<G>(c, n, m);
    }
    if constexpr (kMixed && !kTerms) {
      acc.add(static_cast<double>(run.hi));
      acc.add(static_cast<double>(run.lo));
      abs_sum += static_cast<double>(run_abs);
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
    block_reduce_dd(acc, abs_sum, cnt, sm.scratch);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = FpPartial{acc.hi, acc.lo, abs_sum, cnt};
    finish_fp_main<kMixed>(a, sm.scratch, escale, m, tier_of<T, kMixed>());
  }
}

}  // namespace radic
