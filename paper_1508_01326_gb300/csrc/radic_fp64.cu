// Plain binary64 path: partial-pivot LU per minor in binary64 and a binary64
// compensated (two-sum) reduction.
#include "radic_prefix.cuh"

namespace radic {

namespace {

template <int M>
const void* thread_kernel(bool terms) {
  return terms ? reinterpret_cast<const void*>(&k_fp_thread<double, M, false, true>)
               : reinterpret_cast<const void*>(&k_fp_thread<double, M, false, false>);
}

template <int G>
const void* group_kernel(bool terms) {
  return terms ? reinterpret_cast<const void*>(&k_fp_group<double, G, false, true>)
               : reinterpret_cast<const void*>(&k_fp_group<double, G, false, false>);
}

template <int M, int D>
const void* prefix_kernel(bool terms) {
  return terms ? reinterpret_cast<const void*>(&k_fp_prefix<double, M, D, false, true>)
               : reinterpret_cast<const void*>(&k_fp_prefix<double, M, D, false, false>);
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
      default: return nullptr;
    }
  }
  if (p.group == 16) return group_kernel<16>(terms);
  if (p.group == 32) return group_kernel<32>(terms);
  return nullptr;
}

}  // namespace

size_t smem_fp64(const SinglePlan& p) {
  const int cs = (p.mapping != RADIC_MAP_GROUP) ? ((p.m + 1) / 2) * 2 : p.m;
  if (p.mapping == RADIC_MAP_PREFIX) return prefix_smem_bytes(p.n, p.m, cs, 8, p.threads, p.depth);
  return fp_smem_bytes(p.n, p.m, cs, 8, p.threads);
}

int blocks_per_sm_fp64(const SinglePlan& p) {
  const void* k = pick(p, false);
  if (!k) return 0;
  int nb = 0;
  if (!allow_smem(k, smem_fp64(p))) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, p.threads, smem_fp64(p)) != cudaSuccess) return 0;
  return nb;
}

int launch_fp64(const SinglePlan& p, const SingleArgs& a, cudaStream_t s) {
  const void* k = pick(p, a.terms != nullptr);
  if (!k) return RADIC_EUNSUPPORTED;
  if (!allow_smem(k, smem_fp64(p))) return RADIC_EUNSUPPORTED;
  SingleArgs args = a;
  PrefixTable tab = p.ptab;
  void* params[] = {&args, &tab};
  cudaEvent_t* ev = static_cast<cudaEvent_t*>(p.events);
  if (ev && cudaEventRecord(ev[0], s) != cudaSuccess) return RADIC_ECUDA;
  if (cudaLaunchKernel(k, dim3(p.blocks), dim3(p.threads), params, smem_fp64(p), s) != cudaSuccess)
    return RADIC_ECUDA;
  if (ev && cudaEventRecord(ev[1], s) != cudaSuccess) return RADIC_ECUDA;
  return RADIC_OK;
}

}  // namespace radic
