// Persistent kernels of the batched path, pair tier, one per m.
#include "radic_batched.cuh"

namespace radic {

const void* batch_kernel_pair(int m) { return batch_kernel<ff, true>(m); }

}  // namespace radic
