// Persistent kernels of the batched path, binary32 tier, one per m.
#include "radic_batched.cuh"

namespace radic {

const void* batch_kernel_f32(int m) { return batch_kernel<float, true>(m); }

}  // namespace radic
