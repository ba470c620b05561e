// Mixed path: binary32 partial-pivot LU per minor with a float-float running
// sum per task flushed into binary64 two-sums.  Minors whose binary32 result
// is not finite or whose pivot growth exceeds the threshold are left out of
// the sum and their ranks are recorded in per-warp lists; a second kernel on
// the same stream recomputes exactly those minors in binary64 and performs
// the final fixed-order reduction.  If any list overflowed, the second kernel
// recomputes every minor in binary64 instead.
#include "radic_prefix.cuh"

namespace radic {

namespace {

template <int MC>
__device__ double signed_minor_f64(const FpSmem<double>& sm, int n, int m, unsigned long long q, double& absd,
                                   double& bnd) {
  int c[MC];
  unrank_dyn<MC>(q, n, m, sm.binom, m + 1, c);
  double a[MC * MC];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) a[i * MC + j] = sm.As[c[j] * m + i];
  double det = lu_det_local<MC>(a, m, &bnd);
  absd = fabs(det);
  return sign_negative_dyn<MC>(c, m) ? -det : det;
}

// Binary64 sum over every minor of the lexicographic subtree of one
// (m-2)-column prefix (given by its rank among all (m-2)-subsets of
// {0..n-1}): the minors that the prefix kernel left out after flagging.
template <int MC>
__device__ long long prefix_leaves_f64(const FpSmem<double>& sm, int n, int m, int P, unsigned long long rp, Dd& acc,
                                       double& abs_sum, double& bnd_sum) {
  long long cnt = 0;
  int cols[MC];
  // the binomial table is built for k <= m, which covers P
  unrank_dyn<MC>(rp, n, P, sm.binom, m + 1, cols);
  const int v = cols[P - 1], D = m - P;
  // every D-subset of {v+1 .. n-1}, in dictionary order
  for (int d = 0; d < D; ++d) cols[P + d] = v + 1 + d;
  if (cols[m - 1] >= n) return 0;
  for (;;) {
    double a[MC * MC], b;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) a[i * MC + j] = sm.As[cols[j] * m + i];
    double det = lu_det_local<MC>(a, m, &b);
    if (sign_negative_dyn<MC>(cols, m)) det = -det;
    acc.add(det);
    abs_sum += fabs(det);
    bnd_sum += b;
    ++cnt;
    int pos = m - 1;
    while (pos >= P && cols[pos] == n - m + pos) --pos;
    if (pos < P) break;
    ++cols[pos];
    for (int j = pos + 1; j < m; ++j) cols[j] = cols[j - 1] + 1;
  }
  return cnt;
}

// Binary64 recomputation of the flagged minors (or of every minor when a flag
// list overflowed).  The main kernel has already written the result without
// the flagged minors; when nothing was flagged every block returns at once.
// Otherwise block b owns the flag lists of a contiguous range of warps of the
// main kernel, and the last block adds the recomputed sums to the main totals
// kept in the workspace header and rewrites the result.
template <int MC>
__global__ void __launch_bounds__(128) k_mixed_fixup(SingleArgs a, int main_blocks, int tier) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int has_work;
  const bool overflow = __ldcg(&a.hdr->overflow) != 0;
  if (!overflow && __ldcg(&a.hdr->flag_total) == 0) return;
  const int n = a.n, m = a.m;
  FpSmem<double> sm(smem_raw, n, m, m);
  const int wpb = (a.n_warps + gridDim.x - 1) / gridDim.x;
  const int w0 = blockIdx.x * wpb, w1 = min(w0 + wpb, a.n_warps);
  if (threadIdx.x == 0) has_work = overflow ? 1 : 0;
  __syncthreads();
  if (!overflow) {
    int mine = 0;
    for (int w = w0 + threadIdx.x; w < w1; w += blockDim.x) mine |= (__ldcg(&a.flag_count[w]) > 0);
    if (mine) has_work = 1;
  }
  __syncthreads();

  Dd acc;
  double abs_sum = 0.0, bnd = 0.0;
  long long done = 0;
  if (has_work) {
    build_binom(sm.binom, n, m);
    stage_scaled<double>(a.A, a.dtype, m, n, a.lda, sm.As, m, sm.row_exp);
    if (overflow) {
      const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
      const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
      const unsigned long long L = a.ranks_per_task;
      for (unsigned long long task = g; task < a.tasks; task += nthreads) {
        const unsigned long long q0 = task * L, q1 = min(q0 + L, a.total);
        for (unsigned long long q = q0; q < q1; ++q) {
          double absd, b;
          acc.add(signed_minor_f64<MC>(sm, n, m, q, absd, b));
          abs_sum += absd;
          bnd += b;
          ++done;
        }
      }
    } else {
      const long long s0 = (long long)w0 * a.flag_cap, s1 = (long long)w1 * a.flag_cap;
      for (long long s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const long long w = s / a.flag_cap, i = s - w * a.flag_cap;
        if (i < __ldcg(&a.flag_count[w])) {
          const unsigned long long e = __ldcg(&a.flag_ranks[s]);
          if (a.flag_prefix == 0) {
            double absd, b;
            acc.add(signed_minor_f64<MC>(sm, n, m, e, absd, b));
            abs_sum += absd;
            bnd += b;
            ++done;
          } else {
            done += prefix_leaves_f64<MC>(sm, n, m, a.flag_prefix, e, acc, abs_sum, bnd);
          }
        }
      }
    }
  }
  block_reduce_dd(acc, abs_sum, done, bnd, sm.scratch);
  if (threadIdx.x == 0) a.partials2[blockIdx.x] = FpPartial{acc.hi, acc.lo, abs_sum, done, bnd, 0.0};
  if (last_block(&a.hdr->ticket[1])) {
    Dd t;
    double ab = 0.0, bt = 0.0;
    long long flagged = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      Dd o;
      o.hi = __ldcg(&a.partials2[b].hi);
      o.lo = __ldcg(&a.partials2[b].lo);
      t.merge(o);
      ab += __ldcg(&a.partials2[b].abs_sum);
      bt += __ldcg(&a.partials2[b].bound);
      flagged += __ldcg(&a.partials2[b].count);
    }
    block_reduce_dd(t, ab, flagged, bt, sm.scratch);
    if (threadIdx.x == 0) {
      if (!overflow) {
        Dd mainsum;
        mainsum.hi = __ldcg(&a.hdr->main_hi);
        mainsum.lo = __ldcg(&a.hdr->main_lo);
        t.merge(mainsum);
        ab += __ldcg(&a.hdr->main_abs);
        bt += __ldcg(&a.hdr->main_bnd);
      }
      // the main kernel's part of the accumulation term (binary32 lane
      // totals in the binary32-elimination prefix kernel) is kept by using
      // the tier of that kernel
      write_fp_result(a.out, t, ab, bt, __ldcg(&a.hdr->escale), m, a.total, flagged, __ldcg(&a.hdr->status), tier);
    }
  }
}

template <int M>
const void* thread_kernel(bool terms) {
  return terms ? reinterpret_cast<const void*>(&k_fp_thread<float, M, true, true>)
               : reinterpret_cast<const void*>(&k_fp_thread<float, M, true, false>);
}

template <int G>
const void* group_kernel(bool terms) {
  return terms ? reinterpret_cast<const void*>(&k_fp_group<float, G, true, true>)
               : reinterpret_cast<const void*>(&k_fp_group<float, G, true, false>);
}

template <int M, int D>
const void* prefix_kernel(bool terms) {
  return terms ? reinterpret_cast<const void*>(&k_fp_prefix<float, M, D, true, true>)
               : reinterpret_cast<const void*>(&k_fp_prefix<float, M, D, true, false>);
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

const void* mixed_fixup_kernel(int m) {
  if (m <= 8) return reinterpret_cast<const void*>(&k_mixed_fixup<8>);
  if (m <= 16) return reinterpret_cast<const void*>(&k_mixed_fixup<16>);
  return reinterpret_cast<const void*>(&k_mixed_fixup<32>);
}

size_t mixed_fixup_smem(const SinglePlan& p) { return fp_smem_bytes(p.n, p.m, p.m, 8, 128); }

size_t smem_mixed(const SinglePlan& p) {
  const int cs = (p.mapping != RADIC_MAP_GROUP) ? ((p.m + 3) / 4) * 4 : p.m;
  if (p.mapping == RADIC_MAP_PREFIX) return prefix_smem_bytes(p.n, p.m, cs, 4, p.threads, p.depth);
  return fp_smem_bytes(p.n, p.m, cs, 4, p.threads);
}

int blocks_per_sm_mixed(const SinglePlan& p) {
  const void* k = pick(p, false);
  if (!k) return 0;
  int nb = 0;
  if (!allow_smem(k, smem_mixed(p))) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, p.threads, smem_mixed(p)) != cudaSuccess) return 0;
  return nb;
}

int launch_mixed(const SinglePlan& p, const SingleArgs& a, cudaStream_t s) {
  const bool terms = a.terms != nullptr;
  const void* k = pick(p, terms);
  if (!k) return RADIC_EUNSUPPORTED;
  if (!allow_smem(k, smem_mixed(p))) return RADIC_EUNSUPPORTED;
  SingleArgs args = a;
  PrefixTable tab = p.ptab;
  void* params[] = {&args, &tab};
  cudaEvent_t* ev = static_cast<cudaEvent_t*>(p.events);
  if (ev && cudaEventRecord(ev[0], s) != cudaSuccess) return RADIC_ECUDA;
  if (cudaLaunchKernel(k, dim3(p.blocks), dim3(p.threads), params, smem_mixed(p), s) != cudaSuccess)
    return RADIC_ECUDA;
  if (ev && cudaEventRecord(ev[1], s) != cudaSuccess) return RADIC_ECUDA;
  if (terms) return RADIC_OK;
  int main_blocks = p.blocks, tier = kModeMixed;
  void* params2[] = {&args, &main_blocks, &tier};
  if (cudaLaunchKernel(mixed_fixup_kernel(p.m), dim3(p.blocks2), dim3(128), params2, mixed_fixup_smem(p), s) !=
      cudaSuccess)
    return RADIC_ECUDA;
  return RADIC_OK;
}

}  // namespace radic
