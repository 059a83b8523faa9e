// hsg_wave.cu -- temporally blocked over-relaxation sweep: colour 0 then
// colour 1 in a single pass over the lattice.
//
// Sec. 4 updates all white spins, then all black spins, one pass over memory
// per colour; the paper's shared-memory kernels (Sec. 5, SM and SM4P) keep
// z planes on chip to reuse each spin within one colour's pass.  This kernel
// also reuses them across the two colours.  A CTA owns a tile of WX x WY
// sites of each colour in the colour-split (xh, y) plane and marches up a
// chunk of z planes.  At step k it
//   stage 0: reflects colour 0 on plane k+1 over the tile grown by one site
//            on every side (region R0, one thread per site), from the old
//            colour-1 planes k, k+1, k+2 (region R1, the tile grown by two
//            sites: a ring of four plane tiles in shared memory, filled by
//            cp.async one plane ahead);
//   stage 1: reflects colour 1 on plane k over the tile, from the new colour-0
//            planes k-1, k, k+1 (a ring of three in shared memory).
// The bonds and old spins of stage 0 are loaded into registers one step
// ahead; stage 0 leaves its bonds in shared memory, where stage 1 finds its
// own (each bond joins a colour-0 and a colour-1 site).  Each spin and bond
// thus leaves HBM about once per full sweep instead of once per half-sweep:
// 44 B per site update instead of 72 B.  A thread marches up one column, so
// the neighbours in its own column on three consecutive planes (its -z, one
// x and its +z neighbour) are read from shared memory once and carried in
// registers: four shared-memory reads per site instead of six.  The RENORM
// instantiation also renormalises every spin it stores, for a
// renormalisation due right after the sweep.
//
// Neighbouring tiles both compute the colour-0 sites of their shared halo;
// they read the same old values and run the same code (site_result), so the
// copies agree bit for bit, and only the owner stores them.  Tiles read the
// old state while others write the new one, so the sweep goes from one spin
// buffer to another.  The result equals colour 0 then colour 1 of
// launch_half_sweep exactly.
//
// Shape (measured on GB300 at L = 256): 16 x 14 tiles make R0 exactly nine
// warps; 51 KB of shared memory per CTA, three CTAs per SM, and the rest of
// the SM's unified L1/shared array left to L1 (launch_wave).  Bringing the
// colour-1 planes in by TMA instead of per-thread cp.async was slower: one
// 3-D tensor box per plane 165 us, bulk row copies 231 us, against 155 us.
// The heat-bath is not blocked this way: recomputing the halo's Philox draws
// and transcendentals made it compute-bound and slower than two half-sweeps.
#include "hsg_device.cuh"
#include "hsg_internal.h"

namespace hsg {
namespace {

constexpr int WX = 16, WY = 14;            // tile: WX columns (xh) x WY rows (y)
constexpr int R1X = WX + 4, R1Y = WY + 4;  // old colour-1 region: halo 2
constexpr int R1N = R1X * R1Y;             // 360
constexpr int R0X = WX + 2, R0Y = WY + 2;  // colour-0 region: halo 1
constexpr int R0N = R0X * R0Y;             // 288
constexpr int W_THREADS = R0N;             // nine warps
constexpr int W_MIN_BLOCKS = 3;            // resident CTAs per SM (at most 72 registers)
constexpr int NS1 = 4, NS0 = 3;            // ring slots
constexpr int MIN_ZC = 8;                  // shortest z chunk
static_assert(W_THREADS % 32 == 0 && WX * WY <= W_THREADS && R1N <= 2 * W_THREADS, "thread roles");

// Bond slots of an R0 site: its +x, +y, +z bonds and its -x, -y, -z bonds.
enum { B_XP = 0, B_YP = 1, B_ZP = 2, B_XM = 3, B_YM = 4, B_ZM = 5, NB = 6 };

struct WaveSmem {
  float4 c1[NS1][R1N];  // old colour 1 over R1
  float4 c0[NS0][R0N];  // new colour 0 over R0
  float jb[2][NB][R0N];  // bonds of the R0 sites of two planes
};  // 51,264 bytes
constexpr size_t W_SMEM = sizeof(WaveSmem);

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// v mod n for v >= -2n (region coordinates never go further below 0).
__device__ __forceinline__ int wrap_mod(int v, int n) { return (v + 2 * n) % n; }

// The six bonds of a site.
struct SiteBonds {
  float xp, xm, yp, ym, zp, zm;
};

// In-plane offsets of a site (x = 2 xh + p, y): its own, the -x bond's
// when p = 0 (the row's previous xh, wrapped) and the -y bond's.
struct SiteOffsets {
  uint32_t off, off_xm, off_ym;
};

__device__ __forceinline__ SiteOffsets site_offsets(uint32_t xh, uint32_t y, uint32_t L, uint32_t Lh) {
  SiteOffsets o;
  o.off = y * Lh + xh;
  o.off_xm = y * Lh + (xh == 0 ? Lh - 1 : xh - 1);
  o.off_ym = (y == 0 ? L - 1 : y - 1) * Lh + xh;
  return o;
}

// Read-only loads issued where they stand: the register prefetch of the
// next step must leave before this step's compute, not be moved to its use.
__device__ __forceinline__ float ld_early(const float* g) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];\n" : "=f"(v) : "l"(g));
  return v;
}
__device__ __forceinline__ float4 ld_early4(const float4* g) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];\n" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(g));
  return v;
}

// Bonds of a site of colour c on plane z (offsets zo = z*plane, zmo =
// (z-1)*plane): its +d bonds in J[d][c], its -d bonds in J[d][1-c] at the
// -d neighbour (the layout comment of hsg_device.cuh).
__device__ __forceinline__ SiteBonds load_bonds(const float* __restrict__ jc, const float* __restrict__ jo,
                                                size_t Nh2, const SiteOffsets& o, uint32_t p, uint32_t zo,
                                                uint32_t zmo) {
  const uint32_t q = zo + o.off;
  SiteBonds b;
  b.xp = ld_early(jc + q);
  b.xm = ld_early(jo + (p ? q : zo + o.off_xm));
  b.yp = ld_early(jc + Nh2 + q);
  b.ym = ld_early(jo + Nh2 + zo + o.off_ym);
  b.zp = ld_early(jc + 2 * Nh2 + q);
  b.zm = ld_early(jo + 2 * Nh2 + zmo + o.off);
  return b;
}

// RENORM: the stored spins are renormalised (renorm_spin), as by a
// renormalisation pass right after the sweep; the colour-0 values that
// stage 1 reads from shared memory are the unrenormalised ones, as in the
// unfused order.
template <bool RENORM>
__global__ void __launch_bounds__(W_THREADS, W_MIN_BLOCKS) k_or_sweep_wave(const WaveArgs a, int zc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WaveSmem& sm = *reinterpret_cast<WaveSmem*>(smem_raw);
  float4(*c1s)[R1N] = sm.c1;
  float4(*c0s)[R0N] = sm.c0;

  const int t = threadIdx.x;
  const int L = a.L, Lh = a.Lh;
  const uint32_t Lu = (uint32_t)L, Lhu = (uint32_t)Lh;
  const uint32_t plane = Lu * Lhu;
  const uint32_t Nh = plane * Lu;
  const int xh0 = blockIdx.x * WX, y0 = blockIdx.y * WY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, L);
  const int nsteps = z1 - z0 + 2;

  const float4* __restrict__ src0 = a.src;
  const float4* __restrict__ src1 = a.src + Nh;
  float4* __restrict__ dst0 = a.dst;
  float4* __restrict__ dst1 = a.dst + Nh;
  // J[d][c]: colour c's +d bonds at a.J + (2d + c) Nh; the stride between
  // directions of one colour is 2 Nh.
  const float* __restrict__ j0 = a.J;
  const float* __restrict__ j1 = a.J + Nh;
  const size_t Nh2 = 2 * (size_t)Nh;

  // R1 sites this thread copies in (in-plane offsets).
  uint32_t l1_off[2];
  const bool l1_second = t + W_THREADS < R1N;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int i = t + j * W_THREADS;
    l1_off[j] = (uint32_t)wrap_mod(y0 - 2 + i / R1X, L) * Lhu + (uint32_t)wrap_mod(xh0 - 2 + i % R1X, Lh);
  }

  // This thread's stage-0 site: R0 position t.
  const int r0 = t / R0X, cc0 = t % R0X;
  const uint32_t y_0 = (uint32_t)wrap_mod(y0 - 1 + r0, L), xh_0 = (uint32_t)wrap_mod(xh0 - 1 + cc0, Lh);
  const bool owned0 = r0 >= 1 && r0 <= WY && cc0 >= 1 && cc0 <= WX && y0 + r0 - 1 < L && xh0 + cc0 - 1 < Lh;
  const SiteOffsets o0 = site_offsets(xh_0, y_0, Lu, Lhu);
  const int b1 = (r0 + 1) * R1X + (cc0 + 1);  // in R1 coordinates

  // This thread's stage-1 site: tile position (t / WX, t % WX).
  const int r1 = t / WX, cc1 = t % WX;
  const bool valid1 = t < WX * WY && y0 + r1 < L && xh0 + cc1 < Lh;
  const uint32_t y_1 = (uint32_t)min(y0 + r1, L - 1), xh_1 = (uint32_t)min(xh0 + cc1, Lh - 1);
  const uint32_t off1 = y_1 * Lhu + xh_1;
  const int b0 = (r1 + 1) * R0X + (cc1 + 1);    // in R0 coordinates (valid1 only)
  const int own1 = (r1 + 2) * R1X + (cc1 + 2);  // in R1 coordinates (valid1 only)

  // Planes are numbered j = 0, 1, ... from z0 - 2; the colour-1 tile of
  // plane j sits in c1 slot j % NS1, the new colour-0 tile in c0 slot j % NS0.
  // z_of(zs, k): the plane k after plane zs, wrapped (k <= 3 < L).
  auto z_of = [&](uint32_t zs, uint32_t k) { return zs + k >= Lu ? zs + k - Lu : zs + k; };
  auto z_below = [&](uint32_t z) { return z == 0 ? Lu - 1 : z - 1; };
  auto load_c1 = [&](int slot_i, uint32_t z) {
    const uint32_t zo = z * plane;
    float4* slot = c1s[slot_i];
    cp_async16(&slot[t], src1 + zo + l1_off[0]);
    if (l1_second) cp_async16(&slot[t + W_THREADS], src1 + zo + l1_off[1]);
  };
  // Register inputs of stage 0 on plane z: its bonds and old spin.
  auto load0 = [&](uint32_t z, SiteBonds& b, float3& s) {
    const uint32_t zo = z * plane;
    b = load_bonds(j0, j1, Nh2, o0, (y_0 + z) & 1u, zo, z_below(z) * plane);
    const float4 v = ld_early4(src0 + zo + o0.off);
    s = make_float3(v.x, v.y, v.z);
  };

  SiteBonds cb0{}, nb0{};
  float jzm1 = 0.0f;  // stage 1: the -z bond of this column, from the plane before
  float3 cs0 = make_float3(0.0f, 0.0f, 0.0f), ns0 = cs0;
  // Column carries: stage 0's old colour 1 on planes s, s + 1 (a0, a1),
  // stage 1's new colour 0 on planes s - 1, s (bm, bc).
  float4 a0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), a1 = a0, bm = a0, bc = a0;
  uint32_t zs = (uint32_t)wrap_mod(z0 - 2, L);  // plane of j = s
  load_c1(0, zs);
  load_c1(1, z_of(zs, 1));
  load_c1(2, z_of(zs, 2));
  cp_async_commit();
  load0(z_of(zs, 1), cb0, cs0);

  for (int s = 0; s < nsteps; ++s) {
    // Ring slots of planes s .. s + 3 (colour 1) and s - 1 .. s + 1 (colour 0).
    const int k0 = s % NS1, k1 = (s + 1) % NS1, k2 = (s + 2) % NS1, k3 = (s + 3) % NS1;
    const int c00 = s % NS0, c0p = (s + 1) % NS0;
    const uint32_t z1p = z_of(zs, 1), z2p = z_of(zs, 2), z3p = z_of(zs, 3);
    asm volatile("cp.async.wait_all;\n" ::: "memory");  // colour-1 planes up to s + 2
    __syncthreads();  // ... visible to all; step s-1 is done with the slot refilled next
    if (s + 3 <= nsteps + 1) load_c1(k3, z3p);
    cp_async_commit();
    // Next step's register inputs of stage 0 (plane s + 2).
    if (s + 1 < nsteps) load0(z2p, nb0, ns0);

    // Stage 0: colour 0 on plane j = s + 1 (stored when s in [1, z1 - z0]).
    // Its -z, +z and one of its x neighbours sit in its own column on
    // planes s, s + 2 and s + 1; only plane s + 2 is new, the other two
    // are carried from the steps before.
    {
      const uint32_t z = z1p;
      const uint32_t p = (y_0 + z) & 1u;
      if (s == 0) {
        a0 = c1s[k0][b1];
        a1 = c1s[k1][b1];
      }
      const float4 a2 = c1s[k2][b1];
      const float4* p1 = c1s[k1] + b1;
      const float4 side = p1[p ? 1 : -1];
      SiteInputs in;
      in.sxp = p ? side : a1;
      in.sxm = p ? a1 : side;
      in.syp = p1[R1X];
      in.sym = p1[-R1X];
      in.szp = a2;
      in.szm = a0;
      a0 = a1;
      a1 = a2;
      in.jxp = cb0.xp;
      in.jxm = cb0.xm;
      in.jyp = cb0.yp;
      in.jym = cb0.ym;
      in.jzp = cb0.zp;
      in.jzm = cb0.zm;
      in.s = cs0;
      in.q = 0;
      in.site = 0;  // over-relaxation draws no random numbers
      const float4 v = site_result<U_OR>(in, 0u, 0u, 0u, 0u, 0u, 0.0f, 0.0f, 1);
      c0s[c0p][t] = v;
      if (owned0 && s >= 1 && s <= z1 - z0) dst0[z * plane + o0.off] = RENORM ? renorm_spin(v) : v;
      float(*jb)[R0N] = sm.jb[(s + 1) & 1];
      jb[B_XP][t] = cb0.xp;
      jb[B_YP][t] = cb0.yp;
      jb[B_ZP][t] = cb0.zp;
      jb[B_XM][t] = cb0.xm;
      jb[B_YM][t] = cb0.ym;
      jb[B_ZM][t] = cb0.zm;
    }
    __syncthreads();

    // Stage 1: colour 1 on plane j = s, for s >= 2.  Each of its bonds
    // joins it to a colour-0 site, whose bond list (plane j, or j + 1 for
    // +z) holds it: +x = the -x bond of its +x neighbour, -x = the +x bond of
    // its -x neighbour, +y / -y likewise, +z = the -z bond of the site above,
    // -z = the +z bond of the site below (kept from the step before).
    // Its own column of new colour 0 on planes s - 1, s, s + 1 likewise:
    // plane s + 1 (just written by stage 0) is loaded, the others carried.
    const float(*jb)[R0N] = sm.jb[s & 1];
    const float4 b2 = valid1 ? c0s[c0p][b0] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (s >= 2 && valid1) {
      const uint32_t z = zs;
      const uint32_t p = (1u + y_1 + z) & 1u;
      const float4* n0 = c0s[c00] + b0;
      const float4 side = n0[p ? 1 : -1];
      SiteInputs in;
      in.sxp = p ? side : bc;
      in.sxm = p ? bc : side;
      in.syp = n0[R0X];
      in.sym = n0[-R0X];
      in.szp = b2;
      in.szm = bm;
      in.jxp = jb[B_XM][b0 + (int)p];
      in.jxm = jb[B_XP][b0 - 1 + (int)p];
      in.jyp = jb[B_YM][b0 + R0X];
      in.jym = jb[B_YP][b0 - R0X];
      in.jzp = sm.jb[(s + 1) & 1][B_ZM][b0];
      in.jzm = jzm1;
      const float4 o = c1s[k0][own1];
      in.s = make_float3(o.x, o.y, o.z);
      in.q = 0;
      in.site = 0;
      const float4 r = site_result<U_OR>(in, 1u, 0u, 0u, 0u, 0u, 0.0f, 0.0f, 1);
      dst1[z * plane + off1] = RENORM ? renorm_spin(r) : r;
    }
    if (s >= 1 && valid1) jzm1 = jb[B_ZP][b0];
    bm = bc;
    bc = b2;
    cb0 = nb0;
    cs0 = ns0;
    zs = z1p;
  }
}

// Launch shape, measured at L = 256 (OR sweep time; bit-identical results
// in every case):
//  * carveout hint 58 %: the CUDA driver takes the next supported configuration,
//    164 KB of shared memory -- the smallest that holds three 51 KB CTAs --
//    and leaves 92 KB of the SM's unified array as L1 for the in-flight bond
//    loads of stage 0: 166 us.  With 60 KB of L1 left (196 KB shared) 178 us,
//    with 28 KB 267 us;
//  * grid: three CTAs per SM over the tiles (z chunks of L / 3 at L = 256),
//    one full wave: 166 us; six per SM (two waves) 167 us; two per SM 196 us;
//    four per SM (a partial second wave) 234 us.
constexpr int W_CARVEOUT_PCT = 58;
constexpr int W_GRID_PER_SM = 3;

// The kernel attributes are per device: applied once on each device used.
template <bool RENORM>
cudaError_t configure_wave() {
  static PerDevice configured;
  cudaError_t e = cudaSuccess;
  std::atomic<int>* slot = device_slot(configured, &e);
  if (!slot) return e;
  if (slot->load(std::memory_order_acquire) == 0) {
    e = cudaFuncSetAttribute(k_or_sweep_wave<RENORM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W_SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_or_sweep_wave<RENORM>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               W_CARVEOUT_PCT);
    if (e != cudaSuccess) return e;
    slot->store(1, std::memory_order_release);
  }
  return cudaSuccess;
}

cudaError_t launch_wave(const WaveArgs& a, int sm_count, cudaStream_t s) {
  const cudaError_t e = a.renorm ? configure_wave<true>() : configure_wave<false>();
  if (e != cudaSuccess) return e;
  const unsigned tx = cdiv(a.Lh, WX), ty = cdiv(a.L, WY);
  long long chunks = (long long)W_GRID_PER_SM * sm_count / ((long long)tx * ty);
  if (chunks < 1) chunks = 1;
  int zc = (int)cdiv(a.L, chunks);
  if (zc < MIN_ZC) zc = MIN_ZC;
  if (zc > a.L) zc = a.L;
  const dim3 grid(tx, ty, cdiv(a.L, zc));
  if (a.renorm)
    k_or_sweep_wave<true><<<grid, W_THREADS, W_SMEM, s>>>(a, zc);
  else
    k_or_sweep_wave<false><<<grid, W_THREADS, W_SMEM, s>>>(a, zc);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_or_sweep_wave(const WaveArgs& a, int sm_count, cudaStream_t s) {
  if (a.L < 4 || (a.L & 1) || a.src == a.dst) return cudaErrorInvalidValue;
  return launch_wave(a, sm_count, s);
}

}  // namespace hsg
