// Persistent kernels of the batched path, binary64 tier (and the binary64 redo of flagged tasks), one per m and task path.
#include "radic_batched.cuh"

namespace radic {

const void* batch_kernel_f64(int m, int path) { return batch_kernel<double, false>(m, path); }

}  // namespace radic
