// Persistent kernels of the batched path, pair tier, one per m and task path.
#include "radic_batched.cuh"

namespace radic {

const void* batch_kernel_pair(int m, int path) { return batch_kernel<ff, true>(m, path); }

}  // namespace radic
