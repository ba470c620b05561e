// Mixed path: binary32 partial-pivot LU per minor with a float-float running
// sum per task flushed into binary64 two-sums.  Minors whose binary32 result
// is not finite or whose pivot growth exceeds the threshold are left out of
// the sum and their ranks are recorded in per-warp lists; a second kernel on
// the same stream recomputes exactly those minors in binary64 and performs
// the final fixed-order reduction.  If any list overflowed, the second kernel
// recomputes every minor in binary64 instead.
#include "radic_fp_kernels.cuh"

namespace radic {

namespace {

// Partial-pivot LU of an m x m row-major matrix in local memory (m <= MC).
template <int MC>
__device__ double lu_det_local(double (&a)[MC * MC], int m) {
  double det = 1.0;
  bool neg = false;
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
      }
      neg = !neg;
    }
    const double piv = a[k * MC + k];
    det *= piv;
    if (piv == 0.0) return 0.0;
    for (int i = k + 1; i < m; ++i) {
      const double l = a[i * MC + k] / piv;
      for (int j = k + 1; j < m; ++j) a[i * MC + j] = fma(-l, a[k * MC + j], a[i * MC + j]);
    }
  }
  return neg ? -det : det;
}

template <int MC>
__device__ double signed_minor_f64(const FpSmem<double>& sm, int n, int m, unsigned long long q, double& absd) {
  int c[MC];
  unrank_dyn<MC>(q, n, m, sm.binom, m + 1, c);
  double a[MC * MC];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) a[i * MC + j] = sm.As[c[j] * m + i];
  double det = lu_det_local<MC>(a, m);
  absd = fabs(det);
  return sign_negative_dyn<MC>(c, m) ? -det : det;
}

// Row exponents of the staging scale (sum_i e_i), computed without staging A.
__device__ inline int row_scale_exponent(const SingleArgs& a, int* row_exp) {
  for (int i = threadIdx.x; i < a.m; i += blockDim.x) {
    double mx = 0.0;
    for (int j = 0; j < a.n; ++j) mx = fmax(mx, fabs(load_elem(a.A, a.dtype, (long long)i * a.lda + j)));
    int e = 0;
    if (mx > 0.0 && isfinite(mx)) frexp(mx, &e);
    row_exp[i] = e;
  }
  __syncthreads();
  int tot = 0;
  for (int i = 0; i < a.m; ++i) tot += row_exp[i];
  return tot;
}

// Binary64 recomputation of the flagged minors and final reduction.  Block b
// owns the flag lists of a contiguous range of warps of the main kernel; a
// block whose lists are empty skips staging altogether.
template <int MC>
__global__ void __launch_bounds__(128) k_mixed_fixup(SingleArgs a, int main_blocks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int has_work;
  const int n = a.n, m = a.m;
  FpSmem<double> sm(smem_raw, n, m, m);
  const bool overflow = __ldcg(&a.hdr->overflow) != 0;
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
  double abs_sum = 0.0;
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
          double absd;
          acc.add(signed_minor_f64<MC>(sm, n, m, q, absd));
          abs_sum += absd;
        }
      }
    } else {
      const long long s0 = (long long)w0 * a.flag_cap, s1 = (long long)w1 * a.flag_cap;
      for (long long s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const long long w = s / a.flag_cap, i = s - w * a.flag_cap;
        if (i < __ldcg(&a.flag_count[w])) {
          double absd;
          acc.add(signed_minor_f64<MC>(sm, n, m, __ldcg(&a.flag_ranks[s]), absd));
          abs_sum += absd;
        }
      }
    }
  }
  long long cnt = 0;
  block_reduce_dd(acc, abs_sum, cnt, sm.scratch);
  if (threadIdx.x == 0) a.partials2[blockIdx.x] = FpPartial{acc.hi, acc.lo, abs_sum, 0};
  if (last_block(&a.hdr->ticket[1])) {
    const int escale = row_scale_exponent(a, sm.row_exp);
    Dd t;
    double ab = 0.0;
    long long flagged = 0;
    if (!overflow) {
      for (int b = threadIdx.x; b < main_blocks; b += blockDim.x) {
        Dd o;
        o.hi = __ldcg(&a.partials[b].hi);
        o.lo = __ldcg(&a.partials[b].lo);
        t.merge(o);
        ab += __ldcg(&a.partials[b].abs_sum);
        flagged += __ldcg(&a.partials[b].count);
      }
    }
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      Dd o;
      o.hi = __ldcg(&a.partials2[b].hi);
      o.lo = __ldcg(&a.partials2[b].lo);
      t.merge(o);
      ab += __ldcg(&a.partials2[b].abs_sum);
    }
    block_reduce_dd(t, ab, flagged, sm.scratch);
    if (threadIdx.x == 0) {
      if (overflow) flagged = static_cast<long long>(a.total);
      write_fp_result(a.out, t, ab, escale, m, a.total, flagged, __ldcg(&a.hdr->status), kModeMixed);
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

const void* pick(const SinglePlan& p, bool terms) {
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

const void* pick_fixup(int m) {
  if (m <= 8) return reinterpret_cast<const void*>(&k_mixed_fixup<8>);
  if (m <= 16) return reinterpret_cast<const void*>(&k_mixed_fixup<16>);
  return reinterpret_cast<const void*>(&k_mixed_fixup<32>);
}

}  // namespace

size_t smem_mixed(const SinglePlan& p) {
  const int cs = (p.mapping == RADIC_MAP_THREAD) ? ((p.m + 3) / 4) * 4 : p.m;
  return fp_smem_bytes(p.n, p.m, cs, 4, p.threads);
}

static size_t smem_fixup(const SinglePlan& p) { return fp_smem_bytes(p.n, p.m, p.m, 8, 128); }

int blocks_per_sm_mixed(const SinglePlan& p) {
  const void* k = pick(p, false);
  if (!k) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, p.threads, smem_mixed(p)) != cudaSuccess) return 0;
  return nb;
}

int launch_mixed(const SinglePlan& p, const SingleArgs& a, cudaStream_t s) {
  const bool terms = a.terms != nullptr;
  const void* k = pick(p, terms);
  if (!k) return RADIC_EUNSUPPORTED;
  SingleArgs args = a;
  void* params[] = {&args};
  cudaEvent_t* ev = static_cast<cudaEvent_t*>(p.events);
  if (ev && cudaEventRecord(ev[0], s) != cudaSuccess) return RADIC_ECUDA;
  if (cudaLaunchKernel(k, dim3(p.blocks), dim3(p.threads), params, smem_mixed(p), s) != cudaSuccess)
    return RADIC_ECUDA;
  if (ev && cudaEventRecord(ev[1], s) != cudaSuccess) return RADIC_ECUDA;
  if (terms) return RADIC_OK;
  int main_blocks = p.blocks;
  void* params2[] = {&args, &main_blocks};
  if (cudaLaunchKernel(pick_fixup(p.m), dim3(p.blocks2), dim3(128), params2, smem_fixup(p), s) != cudaSuccess)
    return RADIC_ECUDA;
  return RADIC_OK;
}

}  // namespace radic
