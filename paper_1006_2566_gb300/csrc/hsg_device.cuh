// hsg_device.cuh -- device-side building blocks of the checkerboard sweep:
// Philox-4x32-10, the uniform map, the three site updates and the local field.
//
// Device layout ("colour-split"): colour c of site (x,y,z) is (x+y+z) & 1.
// With Lh = L/2, the sites of colour c in row (y,z) have x = 2*xh + p,
// p = (c + y + z) & 1, and are stored at q = (z*L + y)*Lh + xh of
//   spins  float4 S[c][N/2]            (x, y, z, unused), or, packed
//          float  S[c][a][N/2]         component a = 0,1,2 (12 bytes a spin)
//   bonds  float  J[d][c][N/2]         d = 0,1,2: bond from the site to +x,+y,+z.
// A site of colour c finds its six neighbours in colour 1-c at
//   x+1: xh + p (wrapped)   x-1: xh - 1 + p (wrapped)   in the same row,
//   y+-1, z+-1: the same xh in rows (y+-1, z) and (y, z+-1).
// Its +d bonds are J[d][c][q]; its -d bonds are the +d bonds of the -d
// neighbours, J[d][1-c][q_-d], read at the same index as that neighbour's spin.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hsg {

// Update kinds of the half-sweep kernels.  U_MET_OR_* is the fused colour
// pass: the Metropolis hits, then one over-relaxation reflection about the
// same field.
enum UpdKind : int { U_OR = 0, U_MET_SPHERE = 1, U_MET_BALL = 2, U_HB = 3, U_MET_OR_SPHERE = 4, U_MET_OR_BALL = 5 };

// Philox stream kinds (third counter word, bits 24..31).
constexpr uint32_t KIND_INIT = 1u, KIND_JGEN = 2u, KIND_MET = 3u, KIND_HB = 4u;

// Philox-4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of the
// 4x32 multiply/xor bijection; the key is bumped by the Weyl increments
// between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// (2m+1) * 2^-24 with m the top 23 bits: exact in fp32, strictly inside (0,1).
// Formed as (1 + m 2^-23) - (1 - 2^-24): m placed in the mantissa of 1.0,
// minus a constant; the difference is representable, so the subtraction is
// exact and the value is the same as converting 2m+1 and scaling it.
__device__ __forceinline__ float u01(uint32_t r) {
  return __int_as_float((int)((r >> 9) | 0x3F800000u)) - 0x1.fffffep-1f;
}

// Uniform point on S^2 (z = 2 u0 - 1 uniform by Archimedes' theorem).
// 1 - z^2 = 4 u0 (1 - u0) with both factors exact in fp32.
__device__ __forceinline__ float3 sphere_point(float u0, float u1) {
  const float z = fmaf(2.0f, u0, -1.0f);
  const float rho = 2.0f * sqrtf(u0 * (1.0f - u0));
  float s, c;
  sincospif(2.0f * u1, &s, &c);
  return make_float3(rho * c, rho * s, z);
}

__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }

// Over-relaxation: reflection of s about h, s' = 2 (s.h)/(h.h) h - s;
// unchanged when h = 0.  The quotient takes the fast divide (2 ulp; h.h is
// at most (sum |J|)^2, far below the 2^126 where it would flush to 0).
__device__ __forceinline__ float3 update_or(float3 s, float3 h) {
  const float hh = dot3(h, h);
  if (hh == 0.0f) return s;
  const float f = __fdividef(2.0f * dot3(s, h), hh);
  return make_float3(fmaf(f, h.x, -s.x), fmaf(f, h.y, -s.y), fmaf(f, h.z, -s.z));
}

// The same sphere point with the fast sine/cosine (absolute error ~4e-7) on
// the angle 2 pi u1 - pi and a reciprocal-square-root radius (2 ulp).
__device__ __forceinline__ float3 sphere_point_fast(float u0, float u1) {
  const float z = fmaf(2.0f, u0, -1.0f);
  const float t = u0 * (1.0f - u0);  // > 0: u0 is strictly inside (0,1)
  const float rho = 2.0f * t * rsqrtf(t);
  float s, c;
  __sincosf(6.283185307179586f * (u1 - 0.5f), &s, &c);
  return make_float3(-rho * c, -rho * s, z);
}

// Multi-hit Metropolis at fixed field h: hits hit0 .. hit0 + hits - 1 (a
// colour's hits may be split over several passes: the field is fixed for
// the whole half-sweep, so the result does not depend on the split).  Hit
// j uses the Philox draw at counter (site, sweep_lo, MET<<24 | colour<<16 | j,
// sweep_hi).  The site
// energy in the field is -s.h, dE = -(s' - s).h, accept iff u3 < exp(-beta dE).
// The proposal uses the fast sphere point, the ball radius cbrt(u2) is
// __powf(u2, 1/3) (relative error ~1e-6 for u2 in (0,1)), the normalisation
// rsqrtf; the acceptance uses __expf, whose ~1e-6 relative error can only
// flip decisions lying within ~1e-6 of their threshold.
template <bool BALL>
__device__ __forceinline__ float3 update_metropolis(float3 s, float3 h, uint32_t site, uint32_t colour,
                                                    uint32_t sweep_lo, uint32_t sweep_hi, uint32_t k0,
                                                    uint32_t k1, float beta, float step, int hits, int hit0 = 0) {
  for (int j = hit0; j < hit0 + hits; ++j) {
    const uint4 r = philox4x32_10(make_uint4(site, sweep_lo, (KIND_MET << 24) | (colour << 16) | (uint32_t)j,
                                             sweep_hi),
                                  k0, k1);
    const float3 d = sphere_point_fast(u01(r.x), u01(r.y));
    float3 p;
    if (BALL) {
      const float a = step * __powf(u01(r.z), 0.333333343f);
      const float3 v = make_float3(fmaf(a, d.x, s.x), fmaf(a, d.y, s.y), fmaf(a, d.z, s.z));
      const float n2 = dot3(v, v);
      if (n2 == 0.0f) continue;  // no direction: rejected
      const float inv = rsqrtf(n2);
      p = make_float3(v.x * inv, v.y * inv, v.z * inv);
    } else {
      p = d;
    }
    const float de = -dot3(make_float3(p.x - s.x, p.y - s.y, p.z - s.z), h);
    if (u01(r.w) < __expf(-beta * de)) s = p;
  }
  return s;
}

// Heat-bath: s' from the density prop. to exp(beta s'.h) on S^2.  With
// x = beta|h|, 1 - cos(theta) = -log(1 + v)/x, v = u0 expm1(-2x), inverts
// the CDF of cos(theta); the azimuth 2 pi u1 is taken in the orthonormal
// frame of h/|h| built as in Duff et al., "Building an Orthonormal Basis,
// Revisited" (JCGT 2017).  Uniform on S^2 when x < 1e-6.
//
// Where s = 1 - cos(theta) > 1 (the lower hemisphere about h), the branch
// below takes 2 - s from its own exact form instead of subtracting, so that
// sin(theta) keeps relative precision up to cos(theta) = -1.
//
// fp32 evaluation of log(1 + v): where 1 + v >= 1/2, w = 1 + v rounded and
// log1p(v) = v log(w)/(w - 1) (Goldberg, "What every computer scientist
// should know about floating-point arithmetic", 1991, Theorem 4: relative
// error a few ulp); below 1/2, w = (1 - u0) + u0 e^{-2x} is summed from two
// positive terms (1 - u0 is exact), since forming 1 + v directly cancels
// when u0 (1 - e^{-2x}) is close to 1.  One logf serves both.  q = 1 - e^{-2x}
// comes from expm1 for small x and from 1 - e^{-2x} once e^{-2x} <= 1/2.
// 1/|h| is rsqrtf (2 ulp); the azimuth uses the fast sine/cosine on
// (-pi, pi) (absolute error ~4e-7); divisions by numbers in [1e-6, 2] use
// the fast divide (2 ulp).  Every one of these errors is below 1e-6.
// (Gathering ct n + c1 e1 + c2 e2 into fewer operations -- ct n + (c1, s c2,
// 0) + a D (nx, ny, 0) - (0, 0, D), D = s c1 nx + c2 ny -- executed 3.4 %
// fewer instructions in the L = 256 column kernel but took 98.9 us against
// 93.7 us: its loads were scheduled worse, long-scoreboard stalls 8.1
// against 4.8 per issue.)
__device__ __forceinline__ float3 update_heatbath(float3 h, uint32_t site, uint32_t colour, uint32_t sweep_lo,
                                                  uint32_t sweep_hi, uint32_t k0, uint32_t k1, float beta) {
  const uint4 r = philox4x32_10(make_uint4(site, sweep_lo, (KIND_HB << 24) | (colour << 16), sweep_hi), k0, k1);
  const float u0 = u01(r.x), u1 = u01(r.y);
  const float hh = dot3(h, h);
  const float inv = rsqrtf(hh);  // +inf for h = 0, and then x is NaN
  const float x = beta * (hh * inv);
  if (!(x >= 1e-6f)) return sphere_point(u0, u1);
  const float3 n = make_float3(h.x * inv, h.y * inv, h.z * inv);
  const float e2x = expf(-2.0f * x);
  const float q = e2x > 0.5f ? -expm1f(-2.0f * x) : 1.0f - e2x;
  const float v = -u0 * q;
  const bool near_one = v > -0.5f;
  const float w = near_one ? 1.0f + v : fmaf(u0, e2x, 1.0f - u0);
  float lg = logf(w);
  if (near_one) lg = (w == 1.0f) ? v : lg * __fdividef(v, w - 1.0f);
  float sv = __fdividef(-lg, x);
  sv = fminf(fmaxf(sv, 0.0f), 2.0f);
  float ct = 1.0f - sv, t = sv * (2.0f - sv);
  if (sv > 1.0f && x < 16.0f) {
    // Near cos(theta) = -1, 2 - s formed as 2 - sv cancels and sin(theta) =
    // sqrt(s (2 - s)) inherits the cancellation.  There 2 - s comes from the
    // exact identity 2 - s = log(1 + (1 - u0) (e^{2x} - 1)) / x to relative
    // precision (s > 1 needs -log(1 - u0) > x, so x < 16.7: e^{2x} is finite).
    const float d = fminf(fmaxf(__fdividef(log1pf((1.0f - u0) * expm1f(2.0f * x)), x), 0.0f), 2.0f);
    ct = d - 1.0f;
    t = (2.0f - d) * d;
  }
  const float st = t > 0.0f ? t * rsqrtf(t) : 0.0f;
  float sp, cp;
  __sincosf(6.283185307179586f * (u1 - 0.5f), &sp, &cp);  // angle 2 pi u1 - pi
  sp = -sp;
  cp = -cp;
  const float sign = copysignf(1.0f, n.z);
  const float a = __fdividef(-1.0f, sign + n.z);
  const float b = n.x * n.y * a;
  const float3 e1 = make_float3(fmaf(sign * n.x * n.x, a, 1.0f), sign * b, -sign * n.x);
  const float3 e2 = make_float3(b, fmaf(n.y * n.y, a, sign), -n.y);
  const float c1 = st * cp, c2 = st * sp;
  return make_float3(fmaf(ct, n.x, fmaf(c1, e1.x, c2 * e2.x)), fmaf(ct, n.y, fmaf(c1, e1.y, c2 * e2.y)),
                     fmaf(ct, n.z, fmaf(c1, e1.z, c2 * e2.z)));
}

// Local field from the six neighbour spins and bonds (Eq. 2):
// h = sum_k J_k s_k in the order +x, -x, +y, -y, +z, -z.
__device__ __forceinline__ float3 local_field(float4 sxp, float4 sxm, float4 syp, float4 sym, float4 szp, float4 szm,
                                              float jxp, float jxm, float jyp, float jym, float jzp, float jzm) {
  float3 h;
  h.x = fmaf(jzm, szm.x, fmaf(jzp, szp.x, fmaf(jym, sym.x, fmaf(jyp, syp.x, fmaf(jxm, sxm.x, jxp * sxp.x)))));
  h.y = fmaf(jzm, szm.y, fmaf(jzp, szp.y, fmaf(jym, sym.y, fmaf(jyp, syp.y, fmaf(jxm, sxm.y, jxp * sxp.y)))));
  h.z = fmaf(jzm, szm.z, fmaf(jzp, szp.z, fmaf(jym, sym.z, fmaf(jyp, syp.z, fmaf(jxm, sxm.z, jxp * sxp.z)))));
  return h;
}

// Site update of kind U given the old spin s (unused by the heat-bath).
template <int U>
__device__ __forceinline__ float3 update_site(float3 s, float3 h, uint32_t site, uint32_t colour, uint32_t sweep_lo,
                                              uint32_t sweep_hi, uint32_t k0, uint32_t k1, float beta, float step,
                                              int hits, int hit0 = 0) {
  if constexpr (U == U_OR) {
    return update_or(s, h);
  } else if constexpr (U == U_MET_SPHERE) {
    return update_metropolis<false>(s, h, site, colour, sweep_lo, sweep_hi, k0, k1, beta, step, hits, hit0);
  } else if constexpr (U == U_MET_BALL) {
    return update_metropolis<true>(s, h, site, colour, sweep_lo, sweep_hi, k0, k1, beta, step, hits, hit0);
  } else if constexpr (U == U_MET_OR_SPHERE) {
    return update_or(
        update_metropolis<false>(s, h, site, colour, sweep_lo, sweep_hi, k0, k1, beta, step, hits, hit0), h);
  } else if constexpr (U == U_MET_OR_BALL) {
    return update_or(
        update_metropolis<true>(s, h, site, colour, sweep_lo, sweep_hi, k0, k1, beta, step, hits, hit0), h);
  } else {
    return update_heatbath(h, site, colour, sweep_lo, sweep_hi, k0, k1, beta);
  }
}

// Knuth's two-sum: s + t = a + b exactly (round-to-nearest fp32, no
// reassociation; the build keeps additions as written).
__device__ __forceinline__ float two_sum(float a, float b, float& t) {
  const float s = a + b;
  const float bv = s - a;
  t = (a - (s - bv)) + (b - bv);
  return s;
}

// Renormalisation s <- s/|s|.  d = |s|^2 - 1 is formed from error-free fp32
// transformations: each square as p + e exactly (p = x*x rounded, e =
// fma(x, x, -p)), the three p summed by two-sums into hi + t1 + t2 exactly,
// and hi - 1 exact by Sterbenz's lemma while hi is within [1/2, 2].  The
// leftover terms (each below 2^-23) add up with an error below 2^-43, so d
// carries what an fp64 evaluation of the squares would give, far below the
// fp32 rounding of the result -- with no fp64 instruction on GB300's thin
// FP64 pipe.  Spins drift from unit length only by fp32 round-off, so |d| is
// tiny and 1/sqrt(1+d) - 1 = -d/2 + 3d^2/8 - 5d^3/16 + O(d^4) (binomial
// series; for |d| < 2^-8 the remainder is below 2^-33) is evaluated in fp32
// and applied as s + s*c with one rounding: the result is within a hair of
// the correctly rounded s/|s|.  Larger |d| (a spin set far from unit length,
// never reached by sweeps) takes the fp64 reciprocal square root of the fp64
// |s|^2; a zero spin is left as is.
__device__ __forceinline__ float4 renorm_spin(float4 v) {
  const float px = v.x * v.x, py = v.y * v.y, pz = v.z * v.z;
  const float ex = fmaf(v.x, v.x, -px), ey = fmaf(v.y, v.y, -py), ez = fmaf(v.z, v.z, -pz);
  float t1, t2;
  const float hi = two_sum(two_sum(px, py, t1), pz, t2);
  const float df = (hi - 1.0f) + (((ex + ey) + ez) + (t1 + t2));
  if (fabsf(df) < 0x1p-8f) {
    const float c = df * fmaf(df, fmaf(df, -0.3125f, 0.375f), -0.5f);
    v.x = fmaf(v.x, c, v.x);
    v.y = fmaf(v.y, c, v.y);
    v.z = fmaf(v.z, c, v.z);
  } else {
    const double dx = v.x, dy = v.y, dz = v.z;
    const double n2 = fma(dx, dx, fma(dy, dy, dz * dz));
    if (n2 > 0.0) {
      const double r = rsqrt(n2);
      v.x = (float)(dx * r);
      v.y = (float)(dy * r);
      v.z = (float)(dz * r);
    }
  }
  return v;
}

// The spins of one colour: float4 per site, or three component arrays
// (packed layout).  Both hand the site code the same float4 values, so the
// arithmetic -- and the result -- is the same in either layout.
struct SpinsF4 {
  float4* p;
  __device__ __forceinline__ float4 ldg(uint32_t q) const { return __ldg(p + q); }
  __device__ __forceinline__ float4 ld(uint32_t q) const { return p[q]; }
  __device__ __forceinline__ void st(uint32_t q, float4 v) const { p[q] = v; }
};
struct SpinsSoA {
  float* p;       // component 0; components 1 and 2 at + stride, + 2 stride
  size_t stride;  // N/2
  __device__ __forceinline__ float4 ldg(uint32_t q) const {
    return make_float4(__ldg(p + q), __ldg(p + stride + q), __ldg(p + 2 * stride + q), 0.0f);
  }
  __device__ __forceinline__ float4 ld(uint32_t q) const {
    return make_float4(p[q], p[stride + q], p[2 * stride + q], 0.0f);
  }
  __device__ __forceinline__ void st(uint32_t q, float4 v) const {
    p[q] = v.x;
    p[stride + q] = v.y;
    p[2 * stride + q] = v.z;
  }
};

// What one site of a half-sweep reads: its six other-colour neighbours and
// bonds, its own spin, its index q and its Philox site number.
struct SiteInputs {
  float4 sxp, sxm, syp, sym, szp, szm;
  float jxp, jxm, jyp, jym, jzp, jzm;
  float3 s;
  uint32_t q, site;
};

// Gather the inputs of site (x = 2 xh + p, y, z) of colour `colour` (layout
// at the top of this file).  Indices are 32-bit: q < N/2 <= 1624^3/2 < 2^31.
// Indices a site of colour `colour` at (x = 2 xh + p, y, z) reads: its own
// q, its six other-colour neighbours (periodic wrap by compare-and-select,
// no power-of-2 assumption) and its Philox site number x + y L + z L^2.
// Host and device: the CPU tests check it against coordinate arithmetic.
struct SiteIndex {
  uint32_t q, q_xp, q_xm, q_yp, q_ym, q_zp, q_zm, site;
};

__host__ __device__ __forceinline__ SiteIndex site_index(uint32_t xh, uint32_t y, uint32_t z, uint32_t L, uint32_t Lh,
                                                         uint32_t colour) {
  const uint32_t p = (colour + y + z) & 1u;  // x = 2*xh + p
  const uint32_t plane = L * Lh;
  const uint32_t row = (z * L + y) * Lh;
  SiteIndex i;
  i.q = row + xh;
  i.q_xp = p ? (xh + 1 == Lh ? row : i.q + 1) : i.q;
  i.q_xm = p ? i.q : (xh == 0 ? row + Lh - 1 : i.q - 1);
  i.q_yp = y + 1 == L ? i.q - (L - 1) * Lh : i.q + Lh;
  i.q_ym = y == 0 ? i.q + (L - 1) * Lh : i.q - Lh;
  i.q_zp = z + 1 == L ? i.q - (L - 1) * plane : i.q + plane;
  i.q_zm = z == 0 ? i.q + (L - 1) * plane : i.q - plane;
  i.site = (2 * xh + p) + y * L + z * L * L;
  return i;
}

template <int U, class Spins>
__device__ __forceinline__ void gather_site_in(SiteInputs& in, Spins own, Spins oth, const float* __restrict__ jx_own,
                                               const float* __restrict__ jy_own, const float* __restrict__ jz_own,
                                               const float* __restrict__ jx_oth, const float* __restrict__ jy_oth,
                                               const float* __restrict__ jz_oth, uint32_t xh, uint32_t y, uint32_t z,
                                               uint32_t L, uint32_t Lh, uint32_t colour) {
  const SiteIndex ix = site_index(xh, y, z, L, Lh, colour);
  const uint32_t q = ix.q, q_xp = ix.q_xp, q_xm = ix.q_xm, q_yp = ix.q_yp, q_ym = ix.q_ym, q_zp = ix.q_zp,
                 q_zm = ix.q_zm;
  in.sxp = oth.ldg(q_xp);
  in.sxm = oth.ldg(q_xm);
  in.syp = oth.ldg(q_yp);
  in.sym = oth.ldg(q_ym);
  in.szp = oth.ldg(q_zp);
  in.szm = oth.ldg(q_zm);
  in.jxp = __ldg(jx_own + q);
  in.jxm = __ldg(jx_oth + q_xm);
  in.jyp = __ldg(jy_own + q);
  in.jym = __ldg(jy_oth + q_ym);
  in.jzp = __ldg(jz_own + q);
  in.jzm = __ldg(jz_oth + q_zm);
  in.s = make_float3(0.0f, 0.0f, 0.0f);
  if constexpr (U != U_HB) {
    const float4 o = own.ld(q);
    in.s = make_float3(o.x, o.y, o.z);
  }
  in.q = q;
  in.site = ix.site;
}

template <int U>
__device__ __forceinline__ void gather_site(SiteInputs& in, const float4* __restrict__ own,
                                            const float4* __restrict__ oth, const float* __restrict__ jx_own,
                                            const float* __restrict__ jy_own, const float* __restrict__ jz_own,
                                            const float* __restrict__ jx_oth, const float* __restrict__ jy_oth,
                                            const float* __restrict__ jz_oth, uint32_t xh, uint32_t y, uint32_t z,
                                            uint32_t L, uint32_t Lh, uint32_t colour) {
  gather_site_in<U>(in, SpinsF4{const_cast<float4*>(own)}, SpinsF4{const_cast<float4*>(oth)}, jx_own, jy_own, jz_own,
                    jx_oth, jy_oth, jz_oth, xh, y, z, L, Lh, colour);
}

// Form h (Eq. 2) and apply update U: the site's new spin.
template <int U>
__device__ __forceinline__ float4 site_result(const SiteInputs& in, uint32_t colour, uint32_t sweep_lo,
                                              uint32_t sweep_hi, uint32_t k0, uint32_t k1, float beta, float step,
                                              int hits, int hit0 = 0) {
  const float3 h = local_field(in.sxp, in.sxm, in.syp, in.sym, in.szp, in.szm, in.jxp, in.jxm, in.jyp, in.jym,
                               in.jzp, in.jzm);
  const float3 t = update_site<U>(in.s, h, in.site, colour, sweep_lo, sweep_hi, k0, k1, beta, step, hits, hit0);
  return make_float4(t.x, t.y, t.z, 0.0f);
}

// Form h, apply update U and store the site's new spin.
template <int U>
__device__ __forceinline__ void finish_site(const SiteInputs& in, float4* __restrict__ own, uint32_t colour,
                                            uint32_t sweep_lo, uint32_t sweep_hi, uint32_t k0, uint32_t k1,
                                            float beta, float step, int hits, int hit0 = 0) {
  own[in.q] = site_result<U>(in, colour, sweep_lo, sweep_hi, k0, k1, beta, step, hits, hit0);
}

// One site of a half-sweep: gather, then finish.  Every half-sweep kernel
// that updates sites one by one goes through gather_site / finish_site, so
// they give bit-identical results.
template <int U>
__device__ __forceinline__ void half_sweep_site(float4* __restrict__ own, const float4* __restrict__ oth,
                                                const float* __restrict__ jx_own, const float* __restrict__ jy_own,
                                                const float* __restrict__ jz_own, const float* __restrict__ jx_oth,
                                                const float* __restrict__ jy_oth, const float* __restrict__ jz_oth,
                                                uint32_t xh, uint32_t y, uint32_t z, uint32_t L, uint32_t Lh,
                                                uint32_t colour, uint32_t sweep_lo, uint32_t sweep_hi, uint32_t k0,
                                                uint32_t k1, float beta, float step, int hits, int hit0 = 0) {
  SiteInputs in;
  gather_site<U>(in, own, oth, jx_own, jy_own, jz_own, jx_oth, jy_oth, jz_oth, xh, y, z, L, Lh, colour);
  finish_site<U>(in, own, colour, sweep_lo, sweep_hi, k0, k1, beta, step, hits, hit0);
}

// One site of a half-sweep in the packed layout (same arithmetic).
template <int U>
__device__ __forceinline__ void half_sweep_site_packed(SpinsSoA own, SpinsSoA oth, const float* __restrict__ jx_own,
                                                       const float* __restrict__ jy_own,
                                                       const float* __restrict__ jz_own,
                                                       const float* __restrict__ jx_oth,
                                                       const float* __restrict__ jy_oth,
                                                       const float* __restrict__ jz_oth, uint32_t xh, uint32_t y,
                                                       uint32_t z, uint32_t L, uint32_t Lh, uint32_t colour,
                                                       uint32_t sweep_lo, uint32_t sweep_hi, uint32_t k0, uint32_t k1,
                                                       float beta, float step, int hits) {
  SiteInputs in;
  gather_site_in<U>(in, own, oth, jx_own, jy_own, jz_own, jx_oth, jy_oth, jz_oth, xh, y, z, L, Lh, colour);
  own.st(in.q, site_result<U>(in, colour, sweep_lo, sweep_hi, k0, k1, beta, step, hits));
}

// Unsigned division by an invariant d (Granlund & Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994): with l = ceil(log2 d)
// and m = floor(2^32 (2^l - d) / d) + 1, n / d = (t + ((n - t) >> s1)) >> s2
// for every 32-bit n, where t = mulhi(m, n), s1 = min(l, 1), s2 = max(l - 1, 0).
struct FastDiv {
  uint32_t m, s1, s2;
};

// The constants for divisor d >= 1 (host).
inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;  // ceil(log2 d)
  const unsigned long long m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
  return FastDiv{(uint32_t)m, l < 1 ? l : 1u, l > 1 ? l - 1 : 0u};
}

__host__ __device__ __forceinline__ uint32_t fast_div(uint32_t n, FastDiv f) {
#ifdef __CUDA_ARCH__
  const uint32_t t = __umulhi(n, f.m);
#else
  const uint32_t t = (uint32_t)(((unsigned long long)n * f.m) >> 32);
#endif
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

__device__ __forceinline__ int wrap_inc(int v, int n) { return v + 1 == n ? 0 : v + 1; }
__device__ __forceinline__ int wrap_dec(int v, int n) { return v == 0 ? n - 1 : v - 1; }

}  // namespace hsg
