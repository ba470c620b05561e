// Allocation-free entry point: radic_det in binary64 mode with the library's
// own static scratch array in place of a caller workspace.  It serves callers
// that cannot allocate device memory when they need a determinant (device
// memory owned by another allocator or a fixed pool, or loops that cannot
// take an allocation's synchronisation).  The array is looked up once per
// device and cached; calls on one device share it and must not overlap.  A
// cudaDeviceReset (or any teardown of the device's primary context) unloads
// the module that holds the array, so the cached address is then stale: a
// process that resets a device must not call radic_det_noalloc on it again.
#include <mutex>

#include "radic_internal.h"

namespace radic {
namespace {

constexpr int kNoallocMaxDevices = 64;

// The scratch array itself (one copy on every device that loads the library).
static __device__ __align__(256) unsigned char g_noalloc_scratch[RADIC_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (first call per
// device performs the lookup).  Returns a RADIC_* code.
int noalloc_scratch(void** ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RADIC_ECUDA;
  if (dev < 0 || dev >= kNoallocMaxDevices) return RADIC_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return RADIC_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  *ptr = g_noalloc_ptr[dev];
  return RADIC_OK;
}

}  // namespace
}  // namespace radic

extern "C" int radic_det_noalloc(const void* A, int m, int n, int64_t lda, int dtype, const radic_options* opts,
                                 radic_result* out, void* stream) {
  if (!A || !out || lda < n) return RADIC_EINVAL;
  if (m >= 1 && n >= 1 && m <= n) {
    // A plan that cannot be made (size 0) falls through to radic_det, which
    // reports the planning error (RADIC_EUNSUPPORTED, RADIC_ECUDA, ...)
    // before it touches the scratch array.
    const size_t need = radic_workspace_bytes(m, n, RADIC_MODE_FP64, opts);
    if (need > RADIC_NOALLOC_SCRATCH_BYTES) return RADIC_EWORKSPACE;
  }
  void* scratch = nullptr;
  const int rc = radic::noalloc_scratch(&scratch);
  if (rc != RADIC_OK) return rc;
  // radic_det clears the header of the scratch (tickets) before its kernel.
  return radic_det(A, m, n, lda, dtype, RADIC_MODE_FP64, opts, out, scratch, RADIC_NOALLOC_SCRATCH_BYTES, stream);
}
