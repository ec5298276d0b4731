// Measurement aid: the dp4a issue rate of this GPU's CUDA cores, the
// arithmetic ceiling of the plain int32 comparison kernel (xe_cudacore.cu),
// whose inner loop is one dp4a per complex multiply-accumulate.
//
// Launched with one CTA per SM (the caller sizes the grid), so a CTA's
// clock64 span is its SM's span and dp4a per SM per clock = the CTA's dp4a /
// its span.  Every thread runs 8 independent dp4a chains on register
// operands (8 warps x 8 chains per SM keep the pipe busy); each chain feeds
// its sum back in as the multiplied operand, so no step can be folded away,
// and the loop is bound by dp4a issue alone.  Thread 0 of each CTA records
// the clock64 cycles its CTA ran; every thread stores its sums so the work
// cannot be removed.  On B300 dp4a issues to the FMA-heavy pipe only, which
// takes a warp instruction every other clock: 64 dp4a per SM per clock.
#include <cuda_runtime.h>

#include <cstdint>

#include "xengine.h"

namespace xe {
namespace probe {

constexpr int kChains = 8;
constexpr int kUnroll = 32;

__global__ void __launch_bounds__(256, 1) dp4a_rate_kernel(int iters, long long* cycles, int* sink) {
  int a[kChains], acc[kChains];
  const int b = 0x01020304 ^ static_cast<int>(threadIdx.x);
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    a[k] = static_cast<int>(threadIdx.x * 0x9E3779B1u + k);
    acc[k] = k;
  }
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) acc[k] = __dp4a(acc[k], b, a[k]);
  }
  __syncthreads();
  const long long t1 = clock64();
  int s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += acc[k];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace probe
}  // namespace xe

extern "C" XE_API xe_status xe_probe_dp4a_rate(int iters, int ctas, long long* d_cycles, int* d_sink,
                                               long long* dp4a_per_cta, void* stream) {
  if (iters < 1 || iters > (1 << 20) || ctas < 1 || ctas > (1 << 16) || !d_cycles || !d_sink ||
      !dp4a_per_cta)
    return XE_ERR_INVALID_ARG;
  *dp4a_per_cta = 256LL * iters * xe::probe::kUnroll * xe::probe::kChains;
  xe::probe::dp4a_rate_kernel<<<ctas, 256, 0, static_cast<cudaStream_t>(stream)>>>(iters, d_cycles, d_sink);
  return cudaGetLastError() == cudaSuccess ? XE_OK : XE_ERR_CUDA;
}
