// hsg_aux.cu -- kernels around the sweep: spin initialisation, layout
// conversion between the site-major host layout and the colour-split device
// layout, the FP64 energy (Eq. 1) and the FP64 renormalisation.
#include "hsg_device.cuh"
#include "hsg_internal.h"

namespace hsg {
namespace {

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Spin (c, q) of a lattice in either layout (hsg_device.cuh): float4
// S[c][N/2], or packed float S[c][a][N/2].
template <bool PACKED>
__device__ __forceinline__ float4 spin_get(const void* S, long long nh, int c, long long q) {
  if constexpr (PACKED) {
    const float* b = static_cast<const float*>(S) + 3 * c * nh + q;
    return make_float4(__ldg(b), __ldg(b + nh), __ldg(b + 2 * nh), 0.0f);
  } else {
    return __ldg(static_cast<const float4*>(S) + c * nh + q);
  }
}
template <bool PACKED>
__device__ __forceinline__ void spin_put(void* S, long long nh, int c, long long q, float4 v) {
  if constexpr (PACKED) {
    float* b = static_cast<float*>(S) + 3 * c * nh + q;
    b[0] = v.x;
    b[nh] = v.y;
    b[2 * nh] = v.z;
  } else {
    static_cast<float4*>(S)[c * nh + q] = v;
  }
}

constexpr int ENERGY_THREADS = 256;
// First-pass grid of the energy: fixed, so that the summation order is fixed.
// 760 = 5 CTAs of 256 threads (k_energy_partial takes 48 registers) on each
// of GB300's 152 SMs: one full, even wave.  Measured at L = 256: 92.6 us,
// against 121 us with 1024 CTAs (1.35 waves), and 174 us for a 34-register
// build on 1064 CTAs, whose registers, allocated per warp, leave room for
// only six CTAs per SM.
constexpr int ENERGY_BLOCKS = 760;
constexpr int FINAL_THREADS = 1024;

// Spin initialisation: site i gets the sphere point of Philox counter
// (i, 0, INIT<<24, 0).  Grid (Lh/32, L/8, 2L): blockIdx.z = 2 z + colour.
template <bool PACKED>
__global__ void k_init_spins(void* __restrict__ S, int L, uint32_t k0, uint32_t k1) {
  const int Lh = L / 2;
  const int xh = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const int c = blockIdx.z & 1, z = blockIdx.z >> 1;
  if (xh >= Lh || y >= L) return;
  const int p = (c + y + z) & 1;
  const uint32_t site = (uint32_t)(2 * xh + p) + (uint32_t)y * L + (uint32_t)z * L * L;
  const uint4 r = philox4x32_10(make_uint4(site, 0u, KIND_INIT << 24, 0u), k0, k1);
  const float3 v = sphere_point(u01(r.x), u01(r.y));
  const long long nh = (long long)L * L * Lh;
  spin_put<PACKED>(S, nh, c, ((long long)z * L + y) * Lh + xh, make_float4(v.x, v.y, v.z, 0.0f));
}

// Site-major -> colour-split couplings.  Thread per site (x, y, z).
template <typename T>
__global__ void k_scatter_couplings(const T* __restrict__ src, float* __restrict__ J, int L, float* __restrict__ Jp) {
  const int x = blockIdx.x * 64 + threadIdx.x;
  const int y = blockIdx.y * 4 + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L || y >= L) return;
  const int Lh = L / 2;
  const long long nh = (long long)L * L * Lh;
  const long long i = (long long)x + (long long)y * L + (long long)z * L * L;
  const int c = (x + y + z) & 1;
  const long long q = ((long long)z * L + y) * Lh + (x >> 1);
  float v[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    v[d] = (float)src[3 * i + d];
    J[(2 * d + c) * nh + q] = v[d];
  }
  if (Jp) {
    // The padded copy holds this bond at (y + 2, xh + 2) and at the
    // periodic images inside its halo: rows y + 2 +- L, columns xh + 2 +- L/2.
    const int xh = x >> 1, W = (int)padded_width(L), H = L + 2 * kPadY;
    const int rows[2] = {y + kPadY, y < kPadY ? y + kPadY + L : (y >= L - kPadY ? y + kPadY - L : -1)};
    const int cols[2] = {xh + kPadX, xh + kPadX + Lh < W ? xh + kPadX + Lh : (xh >= Lh - kPadX ? xh + kPadX - Lh : -1)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float* plane = Jp + ((size_t)(2 * d + c) * L + z) * H * W;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          if (rows[a] >= 0 && cols[b] >= 0) plane[(size_t)rows[a] * W + cols[b]] = v[d];
    }
  }
}

// Gaussian couplings from Philox kind JGEN (key of (seed, sample), shared by
// the replicas): site i draws (u0..u3) at counter (i, 0, JGEN<<24, 0) and the
// Box-Muller transform (Box & Muller 1958) in fp64 gives its +x, +y, +z bonds
// sqrt(-2 ln u0) cos(2 pi u1), sqrt(-2 ln u0) sin(2 pi u1), sqrt(-2 ln u2)
// cos(2 pi u3), each rounded once to fp32.  Thread per site (x, y, z).
__global__ void k_gen_couplings(float* __restrict__ J, int L, uint32_t k0, uint32_t k1) {
  const int x = blockIdx.x * 64 + threadIdx.x;
  const int y = blockIdx.y * 4 + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L || y >= L) return;
  const int Lh = L / 2;
  const long long nh = (long long)L * L * Lh;
  const uint32_t i = (uint32_t)x + (uint32_t)y * L + (uint32_t)z * L * L;
  const int c = (x + y + z) & 1;
  const long long q = ((long long)z * L + y) * Lh + (x >> 1);
  const uint4 r = philox4x32_10(make_uint4(i, 0u, KIND_JGEN << 24, 0u), k0, k1);
  const double u0 = u01(r.x), u1 = u01(r.y), u2 = u01(r.z), u3 = u01(r.w);
  const double a = sqrt(-2.0 * log(u0)), b = sqrt(-2.0 * log(u2));
  double s1, c1;
  sincospi(2.0 * u1, &s1, &c1);
  J[(0 + c) * nh + q] = (float)(a * c1);
  J[(2 + c) * nh + q] = (float)(a * s1);
  J[(4 + c) * nh + q] = (float)(b * cospi(2.0 * u3));
}

// Colour-split couplings -> site-major fp32.  Thread per site (x, y, z).
__global__ void k_gather_couplings(const float* __restrict__ J, float* __restrict__ dst, int L) {
  const int x = blockIdx.x * 64 + threadIdx.x;
  const int y = blockIdx.y * 4 + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L || y >= L) return;
  const int Lh = L / 2;
  const long long nh = (long long)L * L * Lh;
  const long long i = (long long)x + (long long)y * L + (long long)z * L * L;
  const int c = (x + y + z) & 1;
  const long long q = ((long long)z * L + y) * Lh + (x >> 1);
#pragma unroll
  for (int d = 0; d < 3; ++d) dst[3 * i + d] = J[(2 * d + c) * nh + q];
}

template <bool PACKED>
__global__ void k_scatter_spins(const float* __restrict__ src, void* __restrict__ S, int L) {
  const int x = blockIdx.x * 64 + threadIdx.x;
  const int y = blockIdx.y * 4 + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L || y >= L) return;
  const int Lh = L / 2;
  const long long nh = (long long)L * L * Lh;
  const long long i = (long long)x + (long long)y * L + (long long)z * L * L;
  const int c = (x + y + z) & 1;
  spin_put<PACKED>(S, nh, c, ((long long)z * L + y) * Lh + (x >> 1),
                   make_float4(src[3 * i], src[3 * i + 1], src[3 * i + 2], 0.0f));
}

template <bool PACKED>
__global__ void k_gather_spins(const void* __restrict__ S, float* __restrict__ dst, int L) {
  const int x = blockIdx.x * 64 + threadIdx.x;
  const int y = blockIdx.y * 4 + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L || y >= L) return;
  const int Lh = L / 2;
  const long long nh = (long long)L * L * Lh;
  const long long i = (long long)x + (long long)y * L + (long long)z * L * L;
  const int c = (x + y + z) & 1;
  const float4 v = spin_get<PACKED>(S, nh, c, ((long long)z * L + y) * Lh + (x >> 1));
  dst[3 * i] = v.x;
  dst[3 * i + 1] = v.y;
  dst[3 * i + 2] = v.z;
}

// Spins and +d bonds of listed sites (site-major indices i < N): out[3k + a]
// = component a of site sites[k], bonds[3k + d] = J of its bond to +e_d.
template <bool PACKED>
__global__ void k_gather_sites(const void* __restrict__ S, const float* __restrict__ J, int L,
                               const uint32_t* __restrict__ sites, int n, float* __restrict__ spins,
                               float* __restrict__ bonds) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t Lu = (uint32_t)L, Lh = Lu / 2, i = sites[k];
  const uint32_t x = i % Lu, y = (i / Lu) % Lu, z = i / (Lu * Lu);
  const uint32_t c = (x + y + z) & 1u;
  const size_t nh = (size_t)Lu * Lu * Lh;
  const size_t q = ((size_t)z * Lu + y) * Lh + (x >> 1);
  const float4 v = spin_get<PACKED>(S, (long long)nh, (int)c, (long long)q);
  spins[3 * (size_t)k] = v.x;
  spins[3 * (size_t)k + 1] = v.y;
  spins[3 * (size_t)k + 2] = v.z;
  for (int d = 0; d < 3; ++d) bonds[3 * (size_t)k + d] = J[(2 * d + c) * nh + q];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// Energy, first pass.  Every bond joins a colour-0 and a colour-1 site, so
// sum_bonds J s_i.s_j = sum over colour-0 sites of s_i . h_i with h_i the
// local field of Eq. 2.  The site term s_i . h_i is formed in FP32 (as in
// the updates, relative error a few ulp); every sum over sites is FP64.
// Block b writes partials[b].
template <bool PACKED>
__global__ void __launch_bounds__(ENERGY_THREADS) k_energy_partial(const void* __restrict__ S,
                                                                   const float* __restrict__ J, int L,
                                                                   double* __restrict__ partials) {
  const uint32_t Lh = (uint32_t)L / 2;
  const uint32_t nh = (uint32_t)L * (uint32_t)L * Lh;
  const float *jx0 = J, *jx1 = J + nh, *jy0 = J + 2ull * nh, *jy1 = J + 3ull * nh, *jz0 = J + 4ull * nh,
              *jz1 = J + 5ull * nh;
  double acc = 0.0;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nh; t += gridDim.x * blockDim.x) {
    const int xh = (int)(t % Lh);
    const uint32_t r = t / Lh;
    const int y = (int)(r % (uint32_t)L), z = (int)(r / (uint32_t)L);
    const int p = (y + z) & 1;  // colour 0
    const long long row = (long long)r * Lh;
    const long long q_xp = row + (p ? wrap_inc(xh, (int)Lh) : xh);
    const long long q_xm = row + (p ? xh : wrap_dec(xh, (int)Lh));
    const long long q_yp = ((long long)z * L + wrap_inc(y, L)) * Lh + xh;
    const long long q_ym = ((long long)z * L + wrap_dec(y, L)) * Lh + xh;
    const long long q_zp = ((long long)wrap_inc(z, L) * L + y) * Lh + xh;
    const long long q_zm = ((long long)wrap_dec(z, L) * L + y) * Lh + xh;
    const float3 h = local_field(spin_get<PACKED>(S, nh, 1, q_xp), spin_get<PACKED>(S, nh, 1, q_xm),
                                 spin_get<PACKED>(S, nh, 1, q_yp), spin_get<PACKED>(S, nh, 1, q_ym),
                                 spin_get<PACKED>(S, nh, 1, q_zp), spin_get<PACKED>(S, nh, 1, q_zm), __ldg(jx0 + t),
                                 __ldg(jx1 + q_xm), __ldg(jy0 + t), __ldg(jy1 + q_ym), __ldg(jz0 + t),
                                 __ldg(jz1 + q_zm));
    const float4 s = spin_get<PACKED>(S, nh, 0, t);
    acc += (double)dot3(make_float3(s.x, s.y, s.z), h);
  }
  __shared__ double warp_part[ENERGY_THREADS / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < ENERGY_THREADS / 32 ? warp_part[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
}

// Energy, second pass: one block adds the partials in a fixed order and
// writes E/N = -(sum)/N to *out, or, with log_idx set, to out[*log_idx]
// and then advances *log_idx.
__global__ void __launch_bounds__(FINAL_THREADS) k_energy_final(const double* __restrict__ partials, int n,
                                                                double inv_n_sites, double* __restrict__ out,
                                                                unsigned long long* __restrict__ log_idx) {
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += FINAL_THREADS) v += partials[k];
  __shared__ double warp_part[FINAL_THREADS / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = warp_part[threadIdx.x];
    w = warp_sum(w);
    if (threadIdx.x == 0) {
      if (log_idx) {
        const unsigned long long k = *log_idx;
        out[k] = -w * inv_n_sites;
        *log_idx = k + 1;
      } else {
        *out = -w * inv_n_sites;
      }
    }
  }
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long v) { *p = v; }
__global__ void k_add_u64(unsigned long long* p, unsigned long long d) { *p += d; }

// Renormalisation of every spin (renorm_spin, hsg_device.cuh); n = N sites,
// t = c * N/2 + q.
template <bool PACKED>
__global__ void k_renorm(void* __restrict__ S, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    if constexpr (PACKED) {
      const long long nh = n / 2;
      const int c = t >= nh;
      const long long q = t - c * nh;
      spin_put<true>(S, nh, c, q, renorm_spin(spin_get<true>(S, nh, c, q)));
    } else {
      float4* S4 = static_cast<float4*>(S);
      S4[t] = renorm_spin(S4[t]);
    }
  }
}

__global__ void k_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t n,
                         uint4* __restrict__ out) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = philox4x32_10(make_uint4(t, c1, c2, c3), k0, k1);
}

}  // namespace

cudaError_t launch_init_spins(void* S, bool packed, int L, uint32_t k0, uint32_t k1, cudaStream_t s) {
  const dim3 grid(cdiv(L / 2, 32), cdiv(L, 8), 2u * L), block(32, 8);
  if (packed)
    k_init_spins<true><<<grid, block, 0, s>>>(S, L, k0, k1);
  else
    k_init_spins<false><<<grid, block, 0, s>>>(S, L, k0, k1);
  return cudaGetLastError();
}

cudaError_t launch_scatter_couplings(const void* src, bool f64, float* J, int L, cudaStream_t s, float* Jp) {
  if (Jp && L < kWaveTmaMinL) return cudaErrorInvalidValue;
  const dim3 grid(cdiv(L, 64), cdiv(L, 4), (unsigned)L), block(64, 4);
  if (f64)
    k_scatter_couplings<double><<<grid, block, 0, s>>>(static_cast<const double*>(src), J, L, Jp);
  else
    k_scatter_couplings<float><<<grid, block, 0, s>>>(static_cast<const float*>(src), J, L, Jp);
  return cudaGetLastError();
}

cudaError_t launch_gen_couplings(float* J, int L, uint32_t k0, uint32_t k1, cudaStream_t s) {
  k_gen_couplings<<<dim3(cdiv(L, 64), cdiv(L, 4), (unsigned)L), dim3(64, 4), 0, s>>>(J, L, k0, k1);
  return cudaGetLastError();
}

cudaError_t launch_gather_couplings(const float* J, float* dst, int L, cudaStream_t s) {
  k_gather_couplings<<<dim3(cdiv(L, 64), cdiv(L, 4), (unsigned)L), dim3(64, 4), 0, s>>>(J, dst, L);
  return cudaGetLastError();
}

cudaError_t launch_scatter_spins(const float* src, void* S, bool packed, int L, cudaStream_t s) {
  const dim3 grid(cdiv(L, 64), cdiv(L, 4), (unsigned)L), block(64, 4);
  if (packed)
    k_scatter_spins<true><<<grid, block, 0, s>>>(src, S, L);
  else
    k_scatter_spins<false><<<grid, block, 0, s>>>(src, S, L);
  return cudaGetLastError();
}

cudaError_t launch_gather_spins(const void* S, bool packed, float* dst, int L, cudaStream_t s) {
  const dim3 grid(cdiv(L, 64), cdiv(L, 4), (unsigned)L), block(64, 4);
  if (packed)
    k_gather_spins<true><<<grid, block, 0, s>>>(S, dst, L);
  else
    k_gather_spins<false><<<grid, block, 0, s>>>(S, dst, L);
  return cudaGetLastError();
}

cudaError_t launch_gather_sites(const void* S, bool packed, const float* J, int L, const uint32_t* sites, int n,
                                float* spins, float* bonds, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (packed)
    k_gather_sites<true><<<cdiv(n, 256), 256, 0, s>>>(S, J, L, sites, n, spins, bonds);
  else
    k_gather_sites<false><<<cdiv(n, 256), 256, 0, s>>>(S, J, L, sites, n, spins, bonds);
  return cudaGetLastError();
}

size_t energy_partials(int L) {
  const long long nh = (long long)L * L * (L / 2);
  const long long b = (nh + ENERGY_THREADS - 1) / ENERGY_THREADS;
  return (size_t)(b < ENERGY_BLOCKS ? b : ENERGY_BLOCKS);
}

cudaError_t launch_energy(const void* S, bool packed, const float* J, int L, double* partials, double* out,
                          unsigned long long* log_idx, cudaStream_t s) {
  const int nb = (int)energy_partials(L);
  if (packed)
    k_energy_partial<true><<<nb, ENERGY_THREADS, 0, s>>>(S, J, L, partials);
  else
    k_energy_partial<false><<<nb, ENERGY_THREADS, 0, s>>>(S, J, L, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_energy_final<<<1, FINAL_THREADS, 0, s>>>(partials, nb, 1.0 / ((double)L * L * L), out, log_idx);
  return cudaGetLastError();
}

cudaError_t launch_set_u64(unsigned long long* p, unsigned long long v, cudaStream_t s) {
  k_set_u64<<<1, 1, 0, s>>>(p, v);
  return cudaGetLastError();
}

cudaError_t launch_add_u64(unsigned long long* p, unsigned long long d, cudaStream_t s) {
  k_add_u64<<<1, 1, 0, s>>>(p, d);
  return cudaGetLastError();
}

// Grid-stride over the spins on the CTAs that are resident at once (one
// even wave; the float4 kernel holds eight CTAs of 256 per SM, the packed one
// six).
template <bool PACKED>
cudaError_t launch_renorm_layout(void* S, long long n, int sm_count, cudaStream_t s) {
  static PerDevice resident;  // CTAs of 256 per SM, looked up once per device
  cudaError_t e = cudaSuccess;
  std::atomic<int>* slot = device_slot(resident, &e);
  if (!slot) return e;
  int per_sm = slot->load(std::memory_order_acquire);
  if (per_sm == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_renorm<PACKED>, 256, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    slot->store(per_sm, std::memory_order_release);
  }
  const long long want = (n + 255) / 256;
  const long long cap = (long long)(sm_count > 0 ? sm_count : 1) * per_sm;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  k_renorm<PACKED><<<grid, 256, 0, s>>>(S, n);
  return cudaGetLastError();
}

cudaError_t launch_renorm(void* S, bool packed, long long n, int sm_count, cudaStream_t s) {
  return packed ? launch_renorm_layout<true>(S, n, sm_count, s) : launch_renorm_layout<false>(S, n, sm_count, s);
}

cudaError_t launch_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t n, uint32_t* out,
                          cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_philox<<<cdiv(n, 256), 256, 0, s>>>(k0, k1, c1, c2, c3, n, reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

}  // namespace hsg
