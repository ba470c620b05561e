// PAIR mode of the single-matrix path: the prefix mapping of the MIXED mode
// with the elimination carried out in pairs of binary32 numbers (about 48
// significant bits on the binary32 pipe).  Prefixes whose pivot growth
// exceeds the threshold, or whose scale is not finite, are left out and
// recomputed in binary64 by the fix-up kernel of the MIXED mode.
#include "radic_prefix.cuh"

namespace radic {

namespace {

template <int M, int D>
const void* pair_kernel(bool terms) {
  return terms ? reinterpret_cast<const void*>(&k_fp_prefix<ff, M, D, true, true>)
               : reinterpret_cast<const void*>(&k_fp_prefix<ff, M, D, true, false>);
}

const void* pick(const SinglePlan& p, bool terms) {
  if (p.mapping != RADIC_MAP_PREFIX) return nullptr;
  switch (p.m) {
    case 3: return p.depth == 2 ? pair_kernel<3, 2>(terms) : nullptr;
    case 4: return p.depth == 3 ? pair_kernel<4, 3>(terms) : pair_kernel<4, 2>(terms);
    case 5: return p.depth == 3 ? pair_kernel<5, 3>(terms) : pair_kernel<5, 2>(terms);
    case 6: return p.depth == 3 ? pair_kernel<6, 3>(terms) : pair_kernel<6, 2>(terms);
    case 7: return p.depth == 3 ? pair_kernel<7, 3>(terms) : pair_kernel<7, 2>(terms);
    case 8: return p.depth == 3 ? pair_kernel<8, 3>(terms) : pair_kernel<8, 2>(terms);
    case 9: return p.depth == 3 ? pair_kernel<9, 3>(terms) : pair_kernel<9, 2>(terms);
    case 10: return p.depth == 3 ? pair_kernel<10, 3>(terms) : pair_kernel<10, 2>(terms);
    default: return nullptr;
  }
}

}  // namespace

size_t smem_pair(const SinglePlan& p) {
  const int cs = ((p.m + 1) / 2) * 2;  // ColStride of 8-byte elements
  return prefix_smem_bytes(p.n, p.m, cs, 8, p.threads, p.depth, true);
}

int blocks_per_sm_pair(const SinglePlan& p) {
  const void* k = pick(p, false);
  if (!k) return 0;
  int nb = 0;
  if (!allow_smem(k, smem_pair(p))) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, p.threads, smem_pair(p)) != cudaSuccess) return 0;
  return nb;
}

int launch_pair(const SinglePlan& p, const SingleArgs& a, cudaStream_t s) {
  const bool terms = a.terms != nullptr;
  const void* k = pick(p, terms);
  if (!k) return RADIC_EUNSUPPORTED;
  if (!allow_smem(k, smem_pair(p))) return RADIC_EUNSUPPORTED;
  SingleArgs args = a;
  PrefixTable tab = p.ptab;
  void* params[] = {&args, &tab};
  cudaEvent_t* ev = static_cast<cudaEvent_t*>(p.events);
  if (ev && cudaEventRecord(ev[0], s) != cudaSuccess) return RADIC_ECUDA;
  if (cudaLaunchKernel(k, dim3(p.blocks), dim3(p.threads), params, smem_pair(p), s) != cudaSuccess)
    return RADIC_ECUDA;
  if (ev && cudaEventRecord(ev[1], s) != cudaSuccess) return RADIC_ECUDA;
  if (terms) return RADIC_OK;
  int main_blocks = p.blocks, tier = kModePair;
  void* params2[] = {&args, &main_blocks, &tier};
  if (cudaLaunchKernel(mixed_fixup_kernel(p.m), dim3(p.blocks2), dim3(128), params2, mixed_fixup_smem(p), s) !=
      cudaSuccess)
    return RADIC_ECUDA;
  return RADIC_OK;
}

}  // namespace radic
