// Test-only: Philox-4x32-10 words from the CUDA toolkit's own device
// function (curand_Philox4x32_10, called, not reimplemented), used to pin
// both the oracle's and the library's Philox against a third implementation.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void k_curand_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t n,
                                uint4* out) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = curand_Philox4x32_10(make_uint4(t, c1, c2, c3), make_uint2(k0, k1));
}

extern "C" int curand_philox_fill(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t n,
                                  uint32_t* out) {
  if (n == 0) return 0;
  k_curand_philox<<<(n + 255) / 256, 256>>>(k0, k1, c1, c2, c3, n, reinterpret_cast<uint4*>(out));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}
