// hsg_noalloc.cu -- E/N of a caller-held lattice without allocating memory.
//
// hsg_energy computes the energy of a context, whose device buffers (including
// the scratch array of per-block partial sums of its two-pass reduction) the
// library allocated.  Some callers cannot let a library allocate: an
// application that hands all device memory to its own arena or caching
// allocator at start-up and forbids raw cudaMalloc calls beside it, or a
// latency-critical loop that cannot afford the device-wide synchronisation an
// allocation or free may cause.  hsg_energy_noalloc serves them: the caller
// passes its own device arrays and output, and the partial sums live in a
// fixed, file-scope device array that exists from the moment the library is
// loaded on a device until the process exits.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents; each call overwrites exactly the slots it later reads, so
// nothing needs clearing.  Two calls whose kernels overlap on the GPU (for
// example on two streams) race on the array; callers must order them.  The
// array's device address is looked up once per device and cached; a
// cudaDeviceReset ends the context that address belongs to, so the cache
// does not survive it.
#include <mutex>
#include <string>

#include "hsg.h"
#include "hsg_device.cuh"
#include "hsg_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kFinalThreads = 1024;
constexpr int kScratchDoubles = HSG_NOALLOC_SCRATCH_BYTES / (int)sizeof(double);
constexpr int kMaxDevices = 64;
constexpr int kMaxL = 1624;

// Per-block partial sums of the first pass.  In host code the name is only a
// stand-in for the symbol: the device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) double g_energy_scratch[kScratchDoubles];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// First pass over site-major arrays (Eq. 1, each bond once): site i adds
// J[3i+d] s_i . s_{i+e_d} for d = x, y, z, formed in fp32; the sum over sites
// is fp64.  Block b writes partials[b].
__global__ void __launch_bounds__(kThreads) k_energy_sitemajor_partial(const float* __restrict__ s,
                                                                      const float* __restrict__ J, int L,
                                                                      double* __restrict__ partials) {
  const long long n = (long long)L * L * L;
  const long long plane = (long long)L * L;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % L);
    const long long r = i / L;
    const int y = (int)(r % L);
    const int z = (int)(r / L);
    const long long ix = x + 1 == L ? i - (L - 1) : i + 1;
    const long long iy = y + 1 == L ? i - (long long)(L - 1) * L : i + L;
    const long long iz = z + 1 == L ? i - (long long)(L - 1) * plane : i + plane;
    const float3 si = make_float3(s[3 * i], s[3 * i + 1], s[3 * i + 2]);
    const float3 sx = make_float3(s[3 * ix], s[3 * ix + 1], s[3 * ix + 2]);
    const float3 sy = make_float3(s[3 * iy], s[3 * iy + 1], s[3 * iy + 2]);
    const float3 sz = make_float3(s[3 * iz], s[3 * iz + 1], s[3 * iz + 2]);
    const float e = fmaf(J[3 * i + 2], hsg::dot3(si, sz),
                         fmaf(J[3 * i + 1], hsg::dot3(si, sy), J[3 * i] * hsg::dot3(si, sx)));
    acc += (double)e;
  }
  __shared__ double warp_part[kThreads / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kThreads / 32 ? warp_part[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
}

// Second pass: one block adds the first n partials in a fixed order and
// writes E/N = -(sum)/N.
__global__ void __launch_bounds__(kFinalThreads) k_energy_sitemajor_final(const double* __restrict__ partials, int n,
                                                                         double inv_n_sites, double* __restrict__ out) {
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += kFinalThreads) v += partials[k];
  __shared__ double warp_part[kFinalThreads / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = warp_sum(warp_part[threadIdx.x]);
    if (threadIdx.x == 0) *out = -w * inv_n_sites;
  }
}

hsg_status noalloc_fail(hsg_status st, const std::string& msg) {
  hsg::set_thread_error(msg);
  return st;
}

// HSG_OK when `p` is device memory of device `dev` or managed memory, else
// HSG_EINVAL (a host pointer would make the kernels fault).  Allocates
// nothing.
hsg_status check_device_pointer(const void* p, int dev, const char* name) {
  cudaPointerAttributes a{};
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // an unknown pointer must not stick to the next call
    return noalloc_fail(HSG_EINVAL, std::string("hsg_energy_noalloc: ") + name + " is not a device pointer (" +
                                        cudaGetErrorString(e) + ")");
  }
  if (a.type == cudaMemoryTypeManaged) return HSG_OK;
  if (a.type != cudaMemoryTypeDevice)
    return noalloc_fail(HSG_EINVAL, std::string("hsg_energy_noalloc: ") + name + " is not device memory");
  if (a.device != dev)
    return noalloc_fail(HSG_EINVAL, std::string("hsg_energy_noalloc: ") + name + " belongs to device " +
                                        std::to_string(a.device) + ", not the current device " + std::to_string(dev));
  return HSG_OK;
}

}  // namespace

extern "C" hsg_status hsg_energy_noalloc(int L, const float* spins, const float* J, double* e_out,
                                         void* cuda_stream) {
  if (L < 4 || L > kMaxL || (L & 1))
    return noalloc_fail(HSG_EINVAL, "hsg_energy_noalloc: L must be even and in [4, " + std::to_string(kMaxL) +
                                        "], got " + std::to_string(L));
  if (!spins || !J || !e_out) return noalloc_fail(HSG_EINVAL, "hsg_energy_noalloc: NULL pointer");
  if (reinterpret_cast<uintptr_t>(e_out) % alignof(double) != 0)
    return noalloc_fail(HSG_EINVAL, "hsg_energy_noalloc: e_out must be 8-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(HSG_ECUDA, std::string("hsg_energy_noalloc: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(HSG_EINVAL, "hsg_energy_noalloc: device ordinal too large");
  const struct {
    const void* p;
    const char* name;
  } args[] = {{spins, "spins"}, {J, "J"}, {e_out, "e_out"}};
  for (const auto& a : args) {
    const hsg_status st = check_device_pointer(a.p, dev, a.name);
    if (st != HSG_OK) return st;
  }
  void* scratch = nullptr;
  {
    // First call on this device: look up the device address of the scratch
    // array (this device is current).
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_energy_scratch);
      if (e != cudaSuccess || !p)
        return noalloc_fail(HSG_ECUDA, std::string("hsg_energy_noalloc: cudaGetSymbolAddress: ") +
                                           cudaGetErrorString(e));
      g_scratch_ptr[dev] = p;
    }
    scratch = g_scratch_ptr[dev];
  }
  const long long n = (long long)L * L * L;
  const long long want = (n + kThreads - 1) / kThreads;
  const int blocks = (int)(want < kScratchDoubles ? want : kScratchDoubles);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double* partials = static_cast<double*>(scratch);
  k_energy_sitemajor_partial<<<blocks, kThreads, 0, s>>>(spins, J, L, partials);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_energy_sitemajor_final<<<1, kFinalThreads, 0, s>>>(partials, blocks, 1.0 / (double)n, e_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return noalloc_fail(HSG_ECUDA, std::string("hsg_energy_noalloc: ") + cudaGetErrorString(e));
  return HSG_OK;
}
