// Pipe-throughput probe: the measured peaks that the roofline fractions of
// the determinant kernels are quoted against.  It is a measuring instrument
// (built into its own library, libradic_peaks.so), not part of the method.
//
// Each thread runs kChains independent dependency chains of one operation
// for `iters` rounds, so that every SM sub-partition always has a ready
// instruction of that kind and the pipe, not latency, sets the rate:
//   kind 0  binary32 FMA   x = x * a + b         (2 flop each)
//   kind 1  binary64 FMA   x = x * a + b         (2 flop each)
//   kind 2  32-bit integer multiply-add x = x * a + b (mod 2^32)
//   kind 3  32 x 32 -> 64-bit integer multiply-add (the wide product the
//           modular arithmetic of the exact mode is built from)
// The operands are kernel arguments and the chains' final values feed one
// conditional store, so the compiler can neither fold nor drop the work.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <typename T>
__device__ __forceinline__ T step(T x, T a, T b);
// Integer chains are written as single PTX instructions: the compiler may
// reassociate integer arithmetic and fold a run of affine steps into one.
template <>
__device__ __forceinline__ uint32_t step<uint32_t>(uint32_t x, uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(a), "r"(b));
  return r;
}
template <>
__device__ __forceinline__ float step<float>(float x, float a, float b) {
  return fmaf(x, a, b);
}
template <>
__device__ __forceinline__ double step<double>(double x, double a, double b) {
  return fma(x, a, b);
}

template <typename T>
__global__ void __launch_bounds__(256) k_chain(T* out, T a, T b, int iters) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = static_cast<T>(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = step<T>(x[c], a, b);
    }
  }
  T s = x[0];
#pragma unroll
  for (int c = 1; c < kChains; ++c) s = s + x[c];
  if (s == static_cast<T>(-12345)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 32 x 32 -> 64-bit products added into 64-bit accumulators.
__global__ void __launch_bounds__(256) k_chain_wide(unsigned long long* out, uint32_t a, unsigned long long b,
                                                    int iters) {
  unsigned long long x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        unsigned long long r;
        asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(static_cast<uint32_t>(x[c])), "r"(a), "l"(b));
        x[c] = r;
      }
    }
  }
  unsigned long long s = x[0];
#pragma unroll
  for (int c = 1; c < kChains; ++c) s += x[c];
  if (s == 12345ull) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

// Runs probe `kind` once to warm up and once timed, on the current device and
// the given stream (cudaStream_t as void*), with `blocks_per_sm` blocks of
// 256 threads per SM and `iters` rounds (each round kChains * kUnroll
// operations per thread).  `scratch`: device memory of at least
// blocks_per_sm * SMs * 256 * 8 bytes (written only if a chain hits a value
// no chain reaches).  Writes the operations per second (FMA or multiply-add
// count, not flops) to *ops_per_s and the timed kernel's milliseconds to *ms.
// Returns 0, 1 for a bad argument, 3 for a CUDA error.
int radic_peak_probe(int kind, int blocks_per_sm, int iters, void* scratch, void* stream, double* ops_per_s,
                     double* ms) {
  if (kind < 0 || kind > 3 || blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || !scratch || !ops_per_s || !ms)
    return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 3;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 3;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const dim3 grid(sms * blocks_per_sm), block(256);
  auto launch = [&]() {
    switch (kind) {
      case 0: k_chain<float><<<grid, block, 0, s>>>(static_cast<float*>(scratch), 0.9999f, 1e-4f, iters); break;
      case 1: k_chain<double><<<grid, block, 0, s>>>(static_cast<double*>(scratch), 0.9999, 1e-4, iters); break;
      case 2: k_chain<uint32_t><<<grid, block, 0, s>>>(static_cast<uint32_t*>(scratch), 2654435761u, 12345u, iters);
        break;
      default:
        k_chain_wide<<<grid, block, 0, s>>>(static_cast<unsigned long long*>(scratch), 2654435761u, 12345ull, iters);
        break;
    }
    return cudaGetLastError();
  };
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 3;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return 3;
  }
  int rc = 0;
  float t = 0.0f;
  if (launch() != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess || launch() != cudaSuccess ||
      cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
    rc = 3;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  const double ops = (double)grid.x * block.x * (double)iters * kUnroll * kChains;
  *ms = t;
  *ops_per_s = ops / (t * 1e-3);
  return 0;
}

}  // extern "C"
