// hsg_sweep.cu -- checkerboard half-sweep kernels (Sec. 4: the sites of one
// colour do not interact, so a half-sweep updates all of them in parallel
// from the other colour; one launch per colour keeps the two colours
// ordered).
//
// Two variants over the colour-split layout of hsg_device.cuh:
//   global : one thread per updated site; the six neighbours come through
//            L1/L2 (the lattice is streamed once per half-sweep from HBM).
//            Its heat-bath launches march a thread up a short column of
//            planes instead (k_half_sweep_column).
//   slab   : a CTA owns a (32 xh) x (4 y) column tile and marches up a chunk
//            of z planes.  The other colour's plane z (with a one-site halo)
//            is staged in shared memory for the x and y neighbours; planes
//            z-1 and z+1 stay in registers, so each other-colour spin is
//            read from memory about once per half-sweep.
#include "hsg_device.cuh"
#include "hsg_internal.h"

namespace hsg {
namespace {

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

__device__ __forceinline__ uint32_t site_number(int xh, int p, int y, int z, int L) {
  return (uint32_t)(2 * xh + p) + (uint32_t)y * (uint32_t)L + (uint32_t)z * (uint32_t)L * (uint32_t)L;
}

// ---------------------------------------------------------------------------
// Global variant.  Block shape (chosen at launch): 64 x 2 threads when a row
// holds at least 64 sites of a colour, else 32 x 4 (measured at L = 256:
// 64 x 2 and 128 x 2 beat 32 x 8 by ~4 %).
// ---------------------------------------------------------------------------
constexpr int G_THREADS = 128;

// Indices are 32-bit: q < N/2 <= 1624^3/2 < 2^31.  The over-relaxation
// kernel is held to 32 registers so that 16 blocks (full occupancy) fit on
// an SM (measured at L = 256: OR 92 us at 32 registers vs 99 us at 36-40);
// Metropolis, which would spill, keeps its registers.  A grid of exactly
// the resident CTAs looping over the sites (grid-stride, or an equal
// contiguous range per CTA; 10 or 12 CTAs per SM) made the 4-hit Metropolis
// half-sweep at L = 128 slower: 28.1-30.1 us against 25.9 us.
template <int U>
__global__ void __launch_bounds__(G_THREADS, U == U_OR ? 16 : 1) k_half_sweep_global(const SweepArgs a) {
  const uint32_t xh = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t y = blockIdx.y * blockDim.y + threadIdx.y;
  const uint32_t z = blockIdx.z;
  const uint32_t L = a.L, Lh = a.Lh;
  if (xh >= Lh || y >= L) return;
  uint32_t sweep_lo = a.sweep_lo, sweep_hi = a.sweep_hi;
  if constexpr (U != U_OR) {
    if (a.sweep_ptr) {
      const unsigned long long sw = *a.sweep_ptr;
      sweep_lo = (uint32_t)sw;
      sweep_hi = (uint32_t)(sw >> 32);
    }
  }
  half_sweep_site<U>(a.own, a.oth, a.jx_own, a.jy_own, a.jz_own, a.jx_oth, a.jy_oth, a.jz_oth, xh, y, z, L, Lh,
                     (uint32_t)a.colour, sweep_lo, sweep_hi, a.k0, a.k1, a.beta, a.step, a.hits);
}

// Heat-bath half-sweeps of the global variant: one thread per (xh, y)
// column of the updated colour over ZM_PLANES consecutive planes.  The
// other colour's spins in the thread's own column on planes z-1 and z (the
// site's -z neighbour and one of its x neighbours) are carried from the
// plane before, so a site loads four neighbour spins instead of six; the
// inputs and the site code are those of k_half_sweep_global, so the results
// are the same bit for bit.  Measured on the L = 256 heat-bath half-sweep:
// 6 planes and 40 registers (12 blocks per SM) 94.0 us, against 100.9 us
// for one site per thread at 32 registers; 8 planes 95.1, 4 planes 96.0,
// 16 planes 97.3, 32 planes 107; at 32 registers (spilling) 104-106 us.
// A persistent grid that deals out equal contiguous (column block, plane)
// ranges, one CTA per resident slot (no partial last wave), took 105.7 us:
// neighbouring column blocks then work on different planes, so the rows
// they share are probably no longer found in L2.  Blocks of 16 x 8 threads
// (a warp spans two rows, so a block's y-neighbour rows are mostly its own
// and come from L1): 89.4 us against 90.7 us for 64 x 2 (fp32 subnormals
// flushed); 32 x 4, 128 x 1, 8 x 16 and 256-thread blocks 89.9-91.1 us;
// streaming (evict-first) stores of the new spins gained 0.2 us more.
constexpr int ZM_PLANES = 6;
constexpr int ZM_BX = 16, ZM_BY = 8;

template <int U>
__global__ void __launch_bounds__(G_THREADS, 12) k_half_sweep_column(const SweepArgs a) {
  const uint32_t xh = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t y = blockIdx.y * blockDim.y + threadIdx.y;
  const uint32_t L = a.L, Lh = a.Lh;
  if (xh >= Lh || y >= L) return;
  uint32_t sweep_lo = a.sweep_lo, sweep_hi = a.sweep_hi;
  if (a.sweep_ptr) {
    const unsigned long long sw = *a.sweep_ptr;
    sweep_lo = (uint32_t)sw;
    sweep_hi = (uint32_t)(sw >> 32);
  }
  const uint32_t plane = L * Lh;
  const uint32_t z0 = blockIdx.z * ZM_PLANES, z1 = min(z0 + ZM_PLANES, L);
  // rows y, y+1, y-1 and columns xh+1, xh-1, wrapped (the layout comment of
  // hsg_device.cuh; the same indices as site_index)
  const uint32_t row = y * Lh, row_p = (y + 1 == L ? 0u : y + 1) * Lh, row_m = (y == 0 ? L - 1 : y - 1) * Lh;
  const uint32_t xm1 = xh == 0 ? Lh - 1 : xh - 1, xp1 = xh + 1 == Lh ? 0u : xh + 1;
  const float4* __restrict__ oth = a.oth;
  uint32_t zmo = (z0 == 0 ? L - 1 : z0 - 1) * plane, zo = z0 * plane;
  float4 s_m = __ldg(oth + zmo + row + xh), s_0 = __ldg(oth + zo + row + xh);
  for (uint32_t z = z0; z < z1; ++z) {
    const uint32_t zpo = z + 1 == L ? 0u : zo + plane;
    const uint32_t p = ((uint32_t)a.colour + y + z) & 1u;  // x = 2 xh + p
    const uint32_t q = zo + row + xh;
    const float4 s_p = __ldg(oth + zpo + row + xh);
    const float4 side = __ldg(oth + zo + row + (p ? xp1 : xm1));
    SiteInputs in;
    in.sxp = p ? side : s_0;
    in.sxm = p ? s_0 : side;
    in.syp = __ldg(oth + zo + row_p + xh);
    in.sym = __ldg(oth + zo + row_m + xh);
    in.szp = s_p;
    in.szm = s_m;
    in.jxp = __ldg(a.jx_own + q);
    in.jxm = __ldg(a.jx_oth + (p ? q : zo + row + xm1));
    in.jyp = __ldg(a.jy_own + q);
    in.jym = __ldg(a.jy_oth + zo + row_m + xh);
    in.jzp = __ldg(a.jz_own + q);
    in.jzm = __ldg(a.jz_oth + zmo + row + xh);
    in.s = make_float3(0.0f, 0.0f, 0.0f);
    if constexpr (U != U_HB) {
      const float4 o = a.own[q];
      in.s = make_float3(o.x, o.y, o.z);
    }
    in.q = q;
    in.site = (2 * xh + p) + y * L + z * L * L;
    a.own[q] = site_result<U>(in, (uint32_t)a.colour, sweep_lo, sweep_hi, a.k0, a.k1, a.beta, a.step, a.hits);
    s_m = s_0;
    s_0 = s_p;
    zmo = zo;
    zo = zpo;
  }
}

// The global variant over the packed layout (three fp32 arrays per colour,
// 12 bytes a spin: 60 bytes per over-relaxation update instead of 72).  Same
// site code on the same values, so bit-identical to the float4 kernel.
template <int U>
__global__ void __launch_bounds__(G_THREADS, (U == U_OR || U == U_HB) ? 16 : 1)
    k_half_sweep_global_packed(const SweepArgs a) {
  const uint32_t xh = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t y = blockIdx.y * blockDim.y + threadIdx.y;
  const uint32_t z = blockIdx.z;
  const uint32_t L = a.L, Lh = a.Lh;
  if (xh >= Lh || y >= L) return;
  uint32_t sweep_lo = a.sweep_lo, sweep_hi = a.sweep_hi;
  if constexpr (U != U_OR) {
    if (a.sweep_ptr) {
      const unsigned long long sw = *a.sweep_ptr;
      sweep_lo = (uint32_t)sw;
      sweep_hi = (uint32_t)(sw >> 32);
    }
  }
  const SpinsSoA own{reinterpret_cast<float*>(a.own), a.stride};
  const SpinsSoA oth{const_cast<float*>(reinterpret_cast<const float*>(a.oth)), a.stride};
  half_sweep_site_packed<U>(own, oth, a.jx_own, a.jy_own, a.jz_own, a.jx_oth, a.jy_oth, a.jz_oth, xh, y, z, L, Lh,
                            (uint32_t)a.colour, sweep_lo, sweep_hi, a.k0, a.k1, a.beta, a.step, a.hits);
}

// ---------------------------------------------------------------------------
// Slab variant.  A CTA of TX x SLAB_TY threads owns a column tile of the
// updated colour and marches up zc planes; zc is chosen at launch so that
// the grid holds SLAB_CTAS_PER_SM CTAs per SM (at L = 128: 7 planes, 1216
// CTAs; from L = 256 the cap of 16 planes).  Indices are 32-bit: every
// offset is below N/2 < 2^31.  Registers are held to what 10 (over-
// relaxation) or 8 (the others) resident CTAs allow.  Measured on GB300
// (bit-identical throughout): the L = 128 4-hit Metropolis + OR workload
// 15.0 us (OR) and 34.0 us (Metropolis) per half-sweep against 26.0 and
// 45.3 us with 32 x 8 tiles of 16 planes, 64-bit indices and no register
// bound; the L = 256 OR half-sweep 144 us against 162 us.
// ---------------------------------------------------------------------------
constexpr int TX = 32, SLAB_TY = 4, SLAB_ZC_MAX = 16, SLAB_CTAS_PER_SM = 8;
template <int U>
constexpr int slab_min_blocks() {
  return U == U_OR ? 10 : 8;
}

template <int U>
__global__ void __launch_bounds__(TX* SLAB_TY, slab_min_blocks<U>()) k_half_sweep_slab(const SweepArgs a, int zc) {
  constexpr int TY = SLAB_TY;
  // Two buffers of the other colour's plane tile: slot (r, c) holds the site
  // ((x0 + c - 1) mod Lh, (y0 + r - 1) mod L); the corners are unused.
  __shared__ float4 plane[2][TY + 2][TX + 2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int L = a.L, Lh = a.Lh;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, L);
  const int xh = x0 + tx, y = y0 + ty;
  const bool valid = xh < Lh && y < L;
  // Threads past the lattice edge fill their slot with the periodic image.
  const uint32_t xw = (uint32_t)(xh % Lh), yw = (uint32_t)(y % L);
  const uint32_t x_left = (uint32_t)((x0 + Lh - 1) % Lh), x_right = (uint32_t)((x0 + TX) % Lh);
  const uint32_t y_top = (uint32_t)((y0 + L - 1) % L), y_bot = (uint32_t)((y0 + TY) % L);
  const uint32_t Lhu = (uint32_t)Lh;
  const uint32_t plane_sz = (uint32_t)L * Lhu;
  const uint32_t col = yw * Lhu + xw;  // this slot's offset in a plane
  uint32_t sweep_lo = a.sweep_lo, sweep_hi = a.sweep_hi;
  if constexpr (U != U_OR) {
    if (a.sweep_ptr) {
      const unsigned long long sw = *a.sweep_ptr;
      sweep_lo = (uint32_t)sw;
      sweep_hi = (uint32_t)(sw >> 32);
    }
  }

  const uint32_t zprev = (uint32_t)wrap_dec(z0, L);
  float4 s_zm = __ldg(a.oth + zprev * plane_sz + col);
  float4 s_z = __ldg(a.oth + (uint32_t)z0 * plane_sz + col);
  float jzm = valid ? __ldg(a.jz_oth + zprev * plane_sz + col) : 0.0f;

  for (int z = z0; z < z1; ++z) {
    const uint32_t zn = (uint32_t)wrap_inc(z, L);
    const float4 s_zp = __ldg(a.oth + zn * plane_sz + col);
    const uint32_t pz = (uint32_t)z * plane_sz;
    float4(*buf)[TX + 2] = plane[(z - z0) & 1];
    buf[ty + 1][tx + 1] = s_z;
    if (ty == 0) buf[0][tx + 1] = __ldg(a.oth + pz + y_top * Lhu + xw);
    if (ty == 1) buf[TY + 1][tx + 1] = __ldg(a.oth + pz + y_bot * Lhu + xw);
    if (tx == 0) buf[ty + 1][0] = __ldg(a.oth + pz + yw * Lhu + x_left);
    if (tx == 1) buf[ty + 1][TX + 1] = __ldg(a.oth + pz + yw * Lhu + x_right);
    __syncthreads();
    if (valid) {
      const int p = (a.colour + y + z) & 1;
      const uint32_t row = pz + (uint32_t)y * Lhu;
      const uint32_t q = row + (uint32_t)xh;
      const float jxp = __ldg(a.jx_own + q), jyp = __ldg(a.jy_own + q), jzp = __ldg(a.jz_own + q);
      const float jxm = __ldg(a.jx_oth + row + (uint32_t)(p ? xh : wrap_dec(xh, Lh)));
      const float jym = __ldg(a.jy_oth + pz + (uint32_t)wrap_dec(y, L) * Lhu + (uint32_t)xh);
      const float jz_here = __ldg(a.jz_oth + q);  // -z bond of the site above
      float3 s = make_float3(0.0f, 0.0f, 0.0f);
      if constexpr (U != U_HB) {
        const float4 o = a.own[q];
        s = make_float3(o.x, o.y, o.z);
      }
      const float3 h = local_field(buf[ty + 1][tx + 1 + p], buf[ty + 1][tx + p], buf[ty + 2][tx + 1],
                                   buf[ty][tx + 1], s_zp, s_zm, jxp, jxm, jyp, jym, jzp, jzm);
      const float3 t = update_site<U>(s, h, site_number(xh, p, y, z, L), (uint32_t)a.colour, sweep_lo, sweep_hi,
                                      a.k0, a.k1, a.beta, a.step, a.hits);
      a.own[q] = make_float4(t.x, t.y, t.z, 0.0f);
      jzm = jz_here;
    }
    s_zm = s_z;
    s_z = s_zp;
  }
}

// Planes per slab CTA: the grid holds SLAB_CTAS_PER_SM CTAs per SM where
// the lattice allows, at most SLAB_ZC_MAX planes each.
int slab_zc(int L, unsigned tiles, int sm_count) {
  const long long want = (long long)SLAB_CTAS_PER_SM * (sm_count > 0 ? sm_count : 1);
  long long chunks = (want + tiles - 1) / tiles;
  if (chunks < 1) chunks = 1;
  int zc = (int)((L + chunks - 1) / chunks);
  return zc < 1 ? 1 : (zc > SLAB_ZC_MAX ? SLAB_ZC_MAX : zc);
}

template <int U>
cudaError_t launch_kind(int variant, const SweepArgs& a, int sm_count, cudaStream_t s) {
  if (a.packed) {
    const dim3 block = a.Lh >= 64 ? dim3(64, 2) : dim3(32, 4);
    const dim3 grid(cdiv(a.Lh, block.x), cdiv(a.L, block.y), (unsigned)a.L);
    k_half_sweep_global_packed<U><<<grid, block, 0, s>>>(a);
  } else if (variant == V_SLAB) {
    const unsigned tx = cdiv(a.Lh, TX), ty = cdiv(a.L, SLAB_TY);
    const int zc = slab_zc(a.L, tx * ty, sm_count);
    const dim3 grid(tx, ty, cdiv(a.L, zc));
    k_half_sweep_slab<U><<<grid, dim3(TX, SLAB_TY), 0, s>>>(a, zc);
  } else {
    const dim3 block = a.Lh >= 64 ? dim3(64, 2) : dim3(32, 4);
    const dim3 grid(cdiv(a.Lh, block.x), cdiv(a.L, block.y), (unsigned)a.L);
    if constexpr (U == U_HB) {
      const dim3 gcol(cdiv(a.Lh, ZM_BX), cdiv(a.L, ZM_BY), cdiv(a.L, ZM_PLANES));
      k_half_sweep_column<U><<<gcol, dim3(ZM_BX, ZM_BY), 0, s>>>(a);
    } else {
      k_half_sweep_global<U><<<grid, block, 0, s>>>(a);
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_half_sweep(int upd, int variant, const SweepArgs& a, int sm_count, cudaStream_t s) {
  switch (upd) {
    case U_OR: return launch_kind<U_OR>(variant, a, sm_count, s);
    case U_MET_SPHERE: return launch_kind<U_MET_SPHERE>(variant, a, sm_count, s);
    case U_MET_BALL: return launch_kind<U_MET_BALL>(variant, a, sm_count, s);
    case U_HB: return launch_kind<U_HB>(variant, a, sm_count, s);
    case U_MET_OR_SPHERE: return launch_kind<U_MET_OR_SPHERE>(variant, a, sm_count, s);
    case U_MET_OR_BALL: return launch_kind<U_MET_OR_BALL>(variant, a, sm_count, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hsg
