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
//            sites: a ring of plane tiles in shared memory, filled by
//            cp.async ahead of their use);
//   stage 1: reflects colour 1 on plane k over the tile, from the new colour-0
//            planes k-1, k, k+1 (a ring in shared memory).
// Each bond joins a colour-0 and a colour-1 site, so both stages read their
// bonds from one shared-memory copy of the plane's bonds.  Each spin and
// bond thus leaves HBM about once per full sweep instead of once per
// half-sweep: 44 B per site update instead of 72 B.  A thread marches up one
// column, so the neighbours in its own column on three consecutive planes
// (its -z, one x and its +z neighbour) are read from shared memory once and
// carried in registers: four shared-memory reads per site instead of six.
// The RENORM instantiations also renormalise every spin they store, for a
// renormalisation due right after the sweep.
//
// Neighbouring tiles both compute the colour-0 sites of their shared halo;
// they read the same old values and run the same code (site_result), so the
// copies agree bit for bit, and only the owner stores them.  Tiles read the
// old state while others write the new one, so the sweep goes from one spin
// buffer to another.  The result equals colour 0 then colour 1 of
// launch_half_sweep exactly.
//
// Two kernels, bit-identical to each other:
//   k_or_sweep_wave (from L = 32, when the device has room for a halo-padded
//     copy of the couplings): each plane's bonds come as ONE tensor box per
//     CTA (TMA, cp.async.bulk.tensor) from the padded copy, whose rows and
//     columns carry the periodic images of the lattice's edges so that no
//     box wraps; the colour-1 planes come by cp.async completing on
//     mbarriers; stage 0's old spins by cp.async into the slot where its new
//     value goes.  One CTA barrier per plane (the pipeline is described at
//     the kernel).  131.5 us per sweep at L = 256.
//   k_or_sweep_wave_regs (smaller lattices, or no room for the copy): stage
//     0 loads each site's bonds and old spin into registers a step ahead and
//     leaves the bonds in shared memory for stage 1; two barriers per plane.
//     155 us at L = 256.
//
// Shape (measured on GB300 at L = 256): 16 x 14 tiles make R0 exactly nine
// warps; three CTAs per SM (74 KB of shared memory each for the tensor-box
// kernel; 51 KB for the register kernel, the rest of the SM's unified array
// left to L1 for its loads).  Measured and dropped (bit-identical, slower):
// the colour-1 planes by one 3-D tensor box per plane (165 us against 155
// us, register bonds) or by bulk row copies (231 us); with tensor-box bonds
// and two barriers per plane (142 us), spin boxes for the tiles whose
// regions do not wrap (145.8 us; the wrapping tiles, still on cp.async,
// set the time), tiles of 32 x 14 or 16 x 30 at two CTAs per SM (149, 159
// us), deeper or shallower rings (144.6-185 us).
// The heat-bath is not blocked this way: recomputing the halo's Philox draws
// and transcendentals made it compute-bound and slower than two half-sweeps.
#include <cstddef>
#include <mutex>

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
constexpr int MIN_ZC = 8;                  // shortest z chunk
static_assert(W_THREADS % 32 == 0 && WX * WY <= W_THREADS && R1N <= 2 * W_THREADS, "thread roles");

// Register kernel.  Bond slots of an R0 site: its +x, +y, +z bonds and its
// -x, -y, -z bonds.
enum { B_XP = 0, B_YP = 1, B_ZP = 2, B_XM = 3, B_YM = 4, B_ZM = 5, NB = 6 };
constexpr int NS1_REGS = 4, NS0_REGS = 3;  // colour-1 ring (one plane in flight), colour-0 ring
struct WaveSmem {
  float4 c1[NS1_REGS][R1N];  // old colour 1 over R1
  float4 c0[NS0_REGS][R0N];  // new colour 0 over R0
  float jb[2][NB][R0N];      // bonds of the R0 sites of two planes
};  // 51,264 bytes

// Tensor-box kernel.  One box per plane holds all six bond arrays (a = 2d +
// c) of the rows y0 - 2 .. y0 + 14 and the columns xh0 - 2 .. xh0 + 17 of
// the halo-padded copy -- every bond any site of the CTA's two stages needs
// on that plane.  Box element (a, row k, col m) is the bond of (y0 - 2 + k,
// xh0 - 2 + m).  Each slot is rounded up to 128 bytes.
constexpr int TB_X = WX + 4, TB_Y = WY + 3, TB_A = 6;  // 20 x 17 x 6 floats
static_assert(TB_X % 4 == 0, "a box row is a multiple of 16 bytes");
constexpr int TB_ARRAY = TB_X * TB_Y;                      // 340 floats
constexpr uint32_t TB_BYTES = TB_A * TB_ARRAY * 4;         // 8160
constexpr int TB_SLOT = (TB_BYTES + 127) / 128 * 128 / 4;  // 2048 floats
constexpr int PAD_X = kPadX, PAD_Y = kPadY;
// Ring depth of every buffer of the tensor-box kernel.  Rings of three
// (refills half a step ahead, 55.7 KB) fit four CTAs per SM, 36 warps:
// 145.2 us against 131.3 us with rings of four at three CTAs per SM.
constexpr int NR = 4;
// Warps 7 and 8 have no stage-1 site (WX * WY = 224 = 7 warps): the first
// thread of warp 7 issues the tensor-box kernel's bond boxes (131.5 us
// against 131.8 us from thread 0).  Handing them the colour-1 copies as well
// (six per thread) was slower: 133.8 us.
constexpr int BOX_ISSUER = WX * WY;
static_assert(BOX_ISSUER % 32 == 0 && BOX_ISSUER < W_THREADS, "an idle warp issues the boxes");
struct WaveBoxSmem {
  float4 c1[NR][R1N];  // old colour 1, plane j in slot j % NR
  float4 c0[NR][R0N];  // colour 0 of plane j: its old spins, then its new ones
  float tb[NR][TB_SLOT];
  unsigned long long bar[NR];   // bond boxes
  unsigned long long full[NR];  // colour-1 planes
};  // 74,304 bytes
static_assert(R0X == 18 && R0Y == 16 && WX == 16 && WY == 14 && TB_X == 20 && R1X == 20 && W_THREADS == 9 * 32,
              "the tensor-box kernel's thread-to-site maps assume this tile");
static_assert(offsetof(WaveBoxSmem, c0) % 128 == 0 && offsetof(WaveBoxSmem, tb) % 128 == 0 &&
                  offsetof(WaveBoxSmem, bar) % 8 == 0,
              "slot alignment");

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Wait until at most N of this thread's cp.async groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Wait until phase `parity` of the mbarrier has completed, for at most
// about `limit_ns` (and 2^22 polls): false if it gave up.
__device__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t i = 1; i < (1u << 22); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0 && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}
// One tensor box of `map` at coordinates (x, y, z, a) into shared memory,
// completing on `bar` (its transaction count must expect the box's bytes).
__device__ __forceinline__ void tma_box_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int a,
                                           unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(a), "r"(smem_addr(bar))
      : "memory");
}
constexpr unsigned long long kBoxWaitNs = 200000000ull;  // 0.2 s

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

// Arrive on `bar` once this thread's cp.async copies issued so far have
// landed (the barrier's count includes the arrival).
__device__ __forceinline__ void cp_async_arrive(unsigned long long* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}

// The register kernel: stage 0 loads its bonds and old spin into registers
// a step ahead and leaves the bonds in shared memory for stage 1; the
// colour-1 planes come by cp.async one plane ahead.
template <bool RENORM>
__global__ void __launch_bounds__(W_THREADS, W_MIN_BLOCKS) k_or_sweep_wave_regs(const WaveArgs a, int zc) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  WaveSmem& sm = *reinterpret_cast<WaveSmem*>(smem_raw);
  constexpr int NS0 = NS0_REGS, NS1 = NS1_REGS;
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
  float3 cs0 = make_float3(0.0f, 0.0f, 0.0f), ns0 = cs0;  // stage 0's old spins, planes s + 1, s + 2
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
    // Ring slots of planes s .. s + 2 (colour 1) and s, s + 1 (colour 0).
    const int k0 = s % NS1, k1 = (s + 1) % NS1, k2 = (s + 2) % NS1;
    const int c00 = s % NS0, c0p = (s + 1) % NS0;
    const uint32_t z1p = z_of(zs, 1), z2p = z_of(zs, 2);
    cp_async_wait<0>();  // colour-1 planes up to s + 2
    __syncthreads();     // ... visible to all; step s-1 is done with the slot refilled next
    if (s + 3 <= nsteps + 1) load_c1((s + 3) % NS1, z_of(zs, 3));
    cp_async_commit();
    if (s + 1 < nsteps) load0(z2p, nb0, ns0);  // stage 0's inputs, a step ahead

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
      const float(*jb)[R0N] = sm.jb[s & 1];
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
    if (s >= 1 && valid1) jzm1 = sm.jb[s & 1][B_ZP][b0];
    bm = bc;
    bc = b2;
    cb0 = nb0;
    cs0 = ns0;
    zs = z1p;
  }
}

// The tensor-box kernel, with one CTA barrier per plane.  Per step s (plane
// s + 1 for stage 0, plane s for stage 1) a warp
//   waits (mbarriers) for the colour-1 plane s + 2 and the bond box of plane
//       s + 1, and (cp.async.wait_group) for its own old spin of plane s + 1;
//   runs stage 0;
//   meets the others at the one barrier (stage 0's new colour 0 then visible);
//   refills the slots that no warp reads any more: colour-1 plane s + 4 (into
//       plane s's slot), its old colour-0 spin of plane s + 3 (into plane
//       s - 1's colour-0 slot) and (one thread) the bond box of plane s + 3 (into
//       box s - 1's slot) -- each a step and a half ahead of its use;
//   runs stage 1, reading its own old colour-1 spin of plane s from a
//       register loaded a step earlier, so that plane s's slot is free once
//       stage 0 of step s is done everywhere.
// Colour-1 planes complete on an mbarrier per slot that each thread's
// cp.async copies arrive on (cp.async.mbarrier.arrive.noinc: all 288
// threads per plane).  The old colour-0 spin of plane j goes into the slot
// where stage 0 later writes the site's new value, by the thread that reads
// it: a thread-private value, so it needs no barrier.  Measured at L = 256:
// 135.6 us against 142.2 us with the same rings and loads behind two
// barriers per plane (the second at the top of each step); 131.8 us once
// each warp's sites lie in two rows four apart (no bank conflicts on the
// box and colour-1 reads; the maps are at the kernel's top), 131.5 us with
// the boxes issued by a warp that has no stage-1 site.  Bounded waits:
// one that gives up sets a.err, the CTA runs to its end, and the issuing thread waits
// (bounded) for its boxes still in flight before it exits.
template <bool RENORM>
__global__ void __launch_bounds__(W_THREADS, W_MIN_BLOCKS)
    k_or_sweep_wave(const WaveArgs a, int zc, const __grid_constant__ CUtensorMap bond_map) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  WaveBoxSmem& sm = *reinterpret_cast<WaveBoxSmem*>(smem_raw);

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

  // R1 sites this thread copies in (in-plane offsets).
  uint32_t l1_off[2];
  const bool l1_second = t + W_THREADS < R1N;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int i = t + j * W_THREADS;
    l1_off[j] = (uint32_t)wrap_mod(y0 - 2 + i / R1X, L) * Lhu + (uint32_t)wrap_mod(xh0 - 2 + i % R1X, Lh);
  }
  // Stage-0 site: R0 position (r0, cc0) at pos0.  The slots are 20 floats
  // (bonds) or 20 float4 (colour 1) wide, so a warp that reads two adjacent
  // rows meets itself in a bank; rows four apart sit 80 floats = 16 banks
  // apart.  Warps 0-7 therefore take columns 0-15 of two rows four apart
  // ((0, 4), (1, 5), (2, 6), (3, 7), (8, 12) .. (11, 15)), and warp 8 columns
  // 16-17 of every row, two columns per quarter-warp row pair.
  int r0, cc0;
  if (t < 8 * 32) {
    const int w = t >> 5, l = t & 31;
    r0 = (w < 4 ? w : w + 4) + ((l >> 4) << 2);
    cc0 = l & 15;
  } else {
    r0 = (t - 8 * 32) >> 1;
    cc0 = 16 + (t & 1);
  }
  const int pos0 = r0 * R0X + cc0;
  const uint32_t y_0 = (uint32_t)wrap_mod(y0 - 1 + r0, L), xh_0 = (uint32_t)wrap_mod(xh0 - 1 + cc0, Lh);
  const bool owned0 = r0 >= 1 && r0 <= WY && cc0 >= 1 && cc0 <= WX && y0 + r0 - 1 < L && xh0 + cc0 - 1 < Lh;
  const uint32_t off0 = y_0 * Lhu + xh_0;
  const int b1 = (r0 + 1) * R1X + (cc0 + 1);
  // Stage-1 site: tile position (r1, cc1), for t < WX * WY: columns 0-15 of
  // two rows four apart likewise ((0, 4) .. (3, 7), (8, 12), (9, 13); the
  // last warp (10, 11)).
  const int w1 = t >> 5, hi1 = (t >> 4) & 1;
  const int ra = w1 < 4 ? w1 : (w1 < 6 ? w1 + 4 : 10);
  const int r1 = t < WX * WY ? (hi1 ? (w1 < 6 ? ra + 4 : 11) : ra) : 0, cc1 = t & 15;
  const bool valid1 = t < WX * WY && y0 + r1 < L && xh0 + cc1 < Lh;
  const uint32_t y_1 = (uint32_t)min(y0 + r1, L - 1), xh_1 = (uint32_t)min(xh0 + cc1, Lh - 1);
  const uint32_t off1 = y_1 * Lhu + xh_1;
  const int b0 = (r1 + 1) * R0X + (cc1 + 1);
  const int own1 = (r1 + 2) * R1X + (cc1 + 2);
  const int tb0 = (r0 + 1) * TB_X + (cc0 + 1);
  const int tb1 = (r1 + 2) * TB_X + (cc1 + 2);

  auto z_of = [&](uint32_t zs, uint32_t k) { return zs + k >= Lu ? zs + k - Lu : zs + k; };  // k < L
  auto load_c1 = [&](int j, uint32_t z) {
    float4* slot = sm.c1[j % NR];
    const uint32_t zo = z * plane;
    cp_async16(&slot[t], src1 + zo + l1_off[0]);
    if (l1_second) cp_async16(&slot[t + W_THREADS], src1 + zo + l1_off[1]);
    cp_async_arrive(&sm.full[j % NR]);
  };
  auto load_old = [&](int j, uint32_t z) { cp_async16(&sm.c0[j % NR][pos0], src0 + z * plane + off0); };

  // Bounded waits: one that gives up marks the sweep as failed (a.err) and
  // stops this thread's further waits (and, for BOX_ISSUER, its boxes); the
  // CTA runs to its end, and BOX_ISSUER then waits, again bounded, for the
  // boxes still in flight.
  bool ok = true;
  int boxes_issued = 0, boxes_seen = 0;
  auto give_up = [&] {
    ok = false;
    atomicOr(a.err, 1ull);
  };
  auto issue_box = [&](int j, uint32_t z) {
    const int k = j % NR;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // earlier reads of the slot, then the box
    mbar_expect_tx(&sm.bar[k], TB_BYTES + a.box_extra_tx);
    tma_box_4d(sm.tb[k], &bond_map, xh0, y0, (int)z, 0, &sm.bar[k]);
    boxes_issued = j + 1;
  };
  auto wait_box = [&](int j) {
    if (!ok) return;
    if (mbar_wait_bounded(&sm.bar[j % NR], (uint32_t)(j / NR) & 1u, kBoxWaitNs))
      boxes_seen = j + 1;
    else
      give_up();
  };
  auto wait_c1 = [&](int j) {
    if (ok && !mbar_wait_bounded(&sm.full[j % NR], (uint32_t)(j / NR) & 1u, kBoxWaitNs)) give_up();
  };

  uint32_t zs = (uint32_t)wrap_mod(z0 - 2, L);  // plane of j = s
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      mbar_init(&sm.bar[k], 1);
      mbar_init(&sm.full[k], W_THREADS + a.c1_extra_arrivals);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (t == BOX_ISSUER)
#pragma unroll
    for (int j = 0; j < 3; ++j) issue_box(j, z_of(zs, j));
#pragma unroll
  for (int j = 0; j < NR; ++j) load_c1(j, z_of(zs, j));  // nsteps + 1 >= 4 > 3
  load_old(1, z_of(zs, 1));
  cp_async_commit();
  load_old(2, z_of(zs, 2));
  cp_async_commit();
  wait_c1(0);
  wait_c1(1);
  wait_box(0);

  float jzm1 = 0.0f;  // stage 1: the -z bond of this column, from the plane before
  // Column carries: stage 0's old colour 1 on planes s, s + 1 (a0, a1),
  // stage 1's new colour 0 on planes s - 1, s (bm, bc), its own old colour 1
  // on plane s (own).
  float4 a0 = sm.c1[0][b1], a1 = sm.c1[1][b1], bm = make_float4(0.0f, 0.0f, 0.0f, 0.0f), bc = bm;
  float4 own = bm;
  for (int s = 0; s < nsteps; ++s) {
    const uint32_t z1p = z_of(zs, 1);
    wait_c1(s + 2);
    wait_box(s + 1);
    cp_async_wait<1>();  // this thread's old spin of plane s + 1

    // Stage 0: colour 0 on plane j = s + 1 (stored when s in [1, z1 - z0]).
    {
      const uint32_t z = z1p;
      const uint32_t p = (y_0 + z) & 1u;
      const float4 a2 = sm.c1[(s + 2) % NR][b1];
      const float4* p1 = sm.c1[(s + 1) % NR] + b1;
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
      const float* B = sm.tb[(s + 1) % NR];
      in.jxp = B[0 * TB_ARRAY + tb0];
      in.jxm = B[1 * TB_ARRAY + tb0 - (p ? 0 : 1)];
      in.jyp = B[2 * TB_ARRAY + tb0];
      in.jym = B[3 * TB_ARRAY + tb0 - TB_X];
      in.jzp = B[4 * TB_ARRAY + tb0];
      in.jzm = sm.tb[s % NR][5 * TB_ARRAY + tb0];
      float4* slot = &sm.c0[(s + 1) % NR][pos0];
      const float4 o = *slot;
      in.s = make_float3(o.x, o.y, o.z);
      in.q = 0;
      in.site = 0;  // over-relaxation draws no random numbers
      const float4 v = site_result<U_OR>(in, 0u, 0u, 0u, 0u, 0u, 0.0f, 0.0f, 1);
      *slot = v;
      if (owned0 && s >= 1 && s <= z1 - z0) dst0[z * plane + off0] = RENORM ? renorm_spin(v) : v;
    }
    __syncthreads();

    // Refills, each into a slot that no warp reads from here on.
    if (s + 4 <= nsteps + 1) load_c1(s + 4, z_of(zs, 4));
    if (s + 3 <= nsteps) load_old(s + 3, z_of(zs, 3));
    cp_async_commit();
    if (t == BOX_ISSUER && ok && s + 3 <= nsteps) issue_box(s + 3, z_of(zs, 3));

    // Stage 1: colour 1 on plane j = s, for s >= 2 (bonds as in the
    // two-barrier kernel's tensor-box path).
    const float4 b2 = valid1 ? sm.c0[(s + 1) % NR][b0] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (s >= 2 && valid1) {
      const uint32_t z = zs;
      const uint32_t p = (1u + y_1 + z) & 1u;
      const float4* n0 = sm.c0[s % NR] + b0;
      const float4 side = n0[p ? 1 : -1];
      SiteInputs in;
      in.sxp = p ? side : bc;
      in.sxm = p ? bc : side;
      in.syp = n0[R0X];
      in.sym = n0[-R0X];
      in.szp = b2;
      in.szm = bm;
      const float* B = sm.tb[s % NR];
      in.jxp = B[1 * TB_ARRAY + tb1];
      in.jxm = B[0 * TB_ARRAY + tb1 - 1 + (int)p];
      in.jyp = B[3 * TB_ARRAY + tb1];
      in.jym = B[2 * TB_ARRAY + tb1 - TB_X];
      in.jzp = B[5 * TB_ARRAY + tb1];
      in.jzm = jzm1;
      in.s = make_float3(own.x, own.y, own.z);
      in.q = 0;
      in.site = 0;
      const float4 r = site_result<U_OR>(in, 1u, 0u, 0u, 0u, 0u, 0.0f, 0.0f, 1);
      dst1[z * plane + off1] = RENORM ? renorm_spin(r) : r;
    }
    if (valid1) {
      own = sm.c1[(s + 1) % NR][own1];  // plane s + 1 (waited for at step s - 1)
      if (s >= 1) jzm1 = sm.tb[s % NR][4 * TB_ARRAY + tb1];
    }
    bm = bc;
    bc = b2;
    zs = z1p;
  }
  cp_async_wait<0>();
  if (t == BOX_ISSUER)
    for (int j = boxes_seen; j < boxes_issued; ++j)
      if (!mbar_wait_bounded(&sm.bar[j % NR], (uint32_t)(j / NR) & 1u, kBoxWaitNs)) break;
}

// Launch shape, measured at L = 256 (OR sweep time; bit-identical results
// in every case):
//  * register kernel: carveout hint 58 %: the CUDA driver takes the next
//    supported configuration, 164 KB of shared memory -- the smallest that
//    holds three 51 KB CTAs -- and leaves 92 KB of the SM's unified array as
//    L1 for the in-flight bond loads of stage 0: 166 us.  With 60 KB of L1
//    left (196 KB shared) 178 us, with 28 KB 267 us;
//  * tensor-box kernel: its loads do not pass through L1, so the carveout is
//    the smallest that holds three CTAs (each with the 1 KB the system
//    reserves), as a percentage of the 228 KB maximum, which the driver
//    rounds up to a supported configuration (74.3 KB per CTA: 97 % -> 228 KB);
//  * grid: three CTAs per SM over the tiles (z chunks of L / 3 at L = 256),
//    one full wave: 166 us; six per SM (two waves) 167 us; two per SM 196 us;
//    four per SM (a partial second wave) 234 us (register kernel).
constexpr int W_CARVEOUT_PCT = 58;
constexpr int W_BOX_CARVEOUT_PCT =
    (int)((100 * W_MIN_BLOCKS * (sizeof(WaveBoxSmem) + 1024) + 233471) / 233472) > 100
        ? 100
        : (int)((100 * W_MIN_BLOCKS * (sizeof(WaveBoxSmem) + 1024) + 233471) / 233472);
static_assert(W_MIN_BLOCKS * (sizeof(WaveBoxSmem) + 1024) <= 233472, "three tensor-box CTAs per SM");
constexpr int W_GRID_PER_SM = 3;

// The kernel attributes are per device: set once on each device used.
template <typename Kernel>
cudaError_t configure_once(PerDevice& configured, Kernel kernel, size_t smem, int carveout) {
  cudaError_t e = cudaSuccess;
  std::atomic<int>* slot = device_slot(configured, &e);
  if (!slot) return e;
  if (slot->load(std::memory_order_acquire) == 0) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
    if (e != cudaSuccess) return e;
    slot->store(1, std::memory_order_release);
  }
  return cudaSuccess;
}

template <bool RENORM>
cudaError_t launch_regs(const WaveArgs& a, dim3 grid, int zc, cudaStream_t s) {
  static PerDevice configured;
  const cudaError_t e = configure_once(configured, k_or_sweep_wave_regs<RENORM>, sizeof(WaveSmem), W_CARVEOUT_PCT);
  if (e != cudaSuccess) return e;
  k_or_sweep_wave_regs<RENORM><<<grid, W_THREADS, sizeof(WaveSmem), s>>>(a, zc);
  return cudaGetLastError();
}

template <bool RENORM>
cudaError_t launch_boxes(const WaveArgs& a, dim3 grid, int zc, cudaStream_t s) {
  static PerDevice configured;
  const cudaError_t e =
      configure_once(configured, k_or_sweep_wave<RENORM>, sizeof(WaveBoxSmem), W_BOX_CARVEOUT_PCT);
  if (e != cudaSuccess) return e;
  k_or_sweep_wave<RENORM><<<grid, W_THREADS, sizeof(WaveBoxSmem), s>>>(a, zc, *a.bond_map);
  return cudaGetLastError();
}

cudaError_t launch_wave(const WaveArgs& a, int sm_count, cudaStream_t s) {
  const unsigned tx = cdiv(a.Lh, WX), ty = cdiv(a.L, WY);
  long long chunks = (long long)W_GRID_PER_SM * sm_count / ((long long)tx * ty);
  if (chunks < 1) chunks = 1;
  int zc = (int)cdiv(a.L, chunks);
  if (zc < MIN_ZC) zc = MIN_ZC;
  if (zc > a.L) zc = a.L;
  const dim3 grid(tx, ty, cdiv(a.L, zc));
  if (a.bond_map) return a.renorm ? launch_boxes<true>(a, grid, zc, s) : launch_boxes<false>(a, grid, zc, s);
  return a.renorm ? launch_regs<true>(a, grid, zc, s) : launch_regs<false>(a, grid, zc, s);
}

// The padded copy, one warp per padded row (a, z, yp) at a time: the row of
// bond array a at (z, y = yp - 2 mod L), its columns shifted by PAD_X and
// wrapped.
__global__ void __launch_bounds__(256) k_pad_bonds(const float* __restrict__ J, float* __restrict__ Jp, int L,
                                                   int Lh, uint32_t W, uint32_t rows) {
  const uint32_t H = (uint32_t)L + 2 * PAD_Y;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps) {
    const uint32_t yp = row % H, za = row / H;
    const uint32_t z = za % (uint32_t)L, arr = za / (uint32_t)L;
    int y = (int)yp - PAD_Y;
    y = y < 0 ? y + L : (y >= L ? y - L : y);
    const float* __restrict__ src = J + (size_t)arr * ((size_t)L * L * Lh) + ((size_t)z * L + (size_t)y) * Lh;
    float* __restrict__ dst = Jp + (size_t)row * W;
    for (uint32_t xp = lane; xp < W; xp += 32) {
      int xh = (int)xp - PAD_X;
      while (xh < 0) xh += Lh;
      while (xh >= Lh) xh -= Lh;
      dst[xp] = __ldg(src + xh);
    }
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once (the library links the
// CUDA runtime only).
EncodeTiledFn tensor_map_encoder() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

}  // namespace

cudaError_t launch_or_sweep_wave(const WaveArgs& a, int sm_count, cudaStream_t s) {
  if (a.L < 4 || (a.L & 1) || a.src == a.dst) return cudaErrorInvalidValue;
  if (a.bond_map && (a.L < kWaveTmaMinL || !a.err)) return cudaErrorInvalidValue;
  return launch_wave(a, sm_count, s);
}

size_t padded_bonds_elems(int L) { return (size_t)6 * L * (L + 2 * PAD_Y) * padded_width(L); }

cudaError_t launch_pad_bonds(const float* J, float* Jp, int L, cudaStream_t s) {
  if (L < kWaveTmaMinL || (L & 1)) return cudaErrorInvalidValue;
  const uint32_t rows = (uint32_t)(TB_A * L * (L + 2 * PAD_Y));  // < 2^24 for L <= 1624
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const uint32_t blocks = (uint32_t)sms * 8u < (rows + 7u) / 8u ? (uint32_t)sms * 8u : (rows + 7u) / 8u;
  k_pad_bonds<<<blocks, 256, 0, s>>>(J, Jp, L, L / 2, padded_width(L), rows);
  return cudaGetLastError();
}

cudaError_t encode_padded_bond_map(CUtensorMap* map, const float* Jp, int L) {
  if (L < kWaveTmaMinL || (L & 1) || (reinterpret_cast<uintptr_t>(Jp) & 15)) return cudaErrorInvalidValue;
  const EncodeTiledFn encode = tensor_map_encoder();
  if (!encode) return cudaErrorNotSupported;
  const cuuint64_t W = padded_width(L), H = (cuuint64_t)L + 2 * PAD_Y;
  const cuuint64_t dims[4] = {W, H, (cuuint64_t)L, (cuuint64_t)TB_A};
  const cuuint64_t strides[3] = {W * 4, W * H * 4, W * H * (cuuint64_t)L * 4};
  const cuuint32_t box[4] = {TB_X, TB_Y, 1, TB_A};
  const cuuint32_t elem_strides[4] = {1, 1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(Jp), dims, strides, box,
                            elem_strides, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace hsg
