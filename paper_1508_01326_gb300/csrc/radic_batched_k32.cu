// Persistent kernels of the batched path, binary32 tier, one per m and task path.
#include "radic_batched.cuh"

namespace radic {

const void* batch_kernel_f32(int m, int path) { return batch_kernel<float, true>(m, path); }

}  // namespace radic
