/*
 * hsg_oracle.c -- plain, slow, FP64 CPU oracle for the checkerboard Monte Carlo
 * sweep of the 3D Heisenberg spin glass (Bernaschi, Parisi & Parisi, "The
 * Heisenberg spin glass model on GPU: myths and actual facts").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference legs may load this library.  The CUDA
 * library never includes, links or calls anything here, and nothing here
 * includes a header of the CUDA library: the two share no code.
 *
 * Everything is written for a reader checking it against the paper:
 * site-major arrays, one loop over sites, no blocking, no fusion.
 *
 * Layout (the paper's own indexing, Sec. 2 text after Eq. 1):
 *   site i = x + y*L + z*L*L,  0 <= x,y,z < L, periodic in all three axes
 *   (Sec. 4, "periodic boundary conditions along X, Y and Z").
 *   s[3*i + a]  spin component a of site i (a unit 3-vector).
 *   J[3*i + d]  coupling of the bond joining i and i + e_d, d = 0:x 1:y 2:z.
 *
 * Readings of the paper used here (the paper is silent or garbled on these):
 *   R1 Eq. 1 sums over ordered pairs; each bond is counted once here:
 *      E = - sum_i sum_d J[3i+d] s_i . s_{i+e_d}.
 *   R2 Eq. 2 is the site's bond sum; "J_{x+1,y,z}" is read as the bond
 *      between (x,y,z) and (x+1,y,z); the local field is
 *      h_i = sum over the 6 neighbours of J_bond * s_nb, and the energy of
 *      site i in the field of its neighbours is -s_i . h_i.
 *   R3 Over-relaxation (Sec. 4, the "maximal move that leaves the energy
 *      invariant"): reflection of s about h, s' = 2 (s.h)/(h.h) h - s;
 *      unchanged when h = 0.
 *   R4 Checkerboard (Sec. 4): colour c(i) = (x+y+z) mod 2; a half-sweep
 *      updates every site of one colour from the other colour's values;
 *      colour 0 ("white") goes first.
 *   R5 Metropolis and heat-bath are only named (Sec. 2); their formulas,
 *      the random-number map (Philox-4x32-10 counters) and the proposals
 *      are the project's reading, written out at each function below.
 *
 * Parity status: every function is pinned by the CPU tests against values
 * fixed by the mathematics (closed forms, brute force, an independent
 * Philox implementation); none is "parity unpinned".
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* Update kinds and random-number stream kinds.  ORACLE_MET_OR is the fused
 * colour pass: the Metropolis hits, then one over-relaxation reflection
 * about the same local field (an opt-in schedule, not the paper's). */
enum { ORACLE_OR = 0, ORACLE_MET = 1, ORACLE_HB = 2, ORACLE_MET_OR = 3 };
enum { ORACLE_PROP_SPHERE = 0, ORACLE_PROP_BALL = 1 };
enum { ORACLE_KIND_INIT = 1, ORACLE_KIND_JGEN = 2, ORACLE_KIND_MET = 3, ORACLE_KIND_HB = 4 };

/* Parameters of one half-sweep. */
typedef struct {
  uint32_t key[2];   /* Philox key of this (seed, sample, replica) */
  uint64_t sweep;    /* sweep counter, part of the Philox counter */
  double beta;       /* inverse temperature, 0 for T = infinity */
  double step;       /* ball-proposal scale */
  int hits;          /* Metropolis hits per site */
  int proposal;      /* ORACLE_PROP_SPHERE or ORACLE_PROP_BALL */
} oracle_params;

/* A sweep schedule. */
typedef struct {
  int kind;          /* main update: -1 none, ORACLE_MET, ORACLE_HB or ORACLE_MET_OR */
  int hits;
  int proposal;
  double step;
  int n_or;          /* over-relaxation sweeps after the main update */
  double beta;
  int renorm_every;  /* 0 = never */
  int energy_every;  /* 0 = never */
} oracle_schedule;

/* ------------------------------------------------------------------------
 * Philox-4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11).  Ten rounds of a multiply-based bijection of
 * a 128-bit counter; the 64-bit key is bumped by the Weyl constants between
 * rounds.  The paper leaves the generator out of its scope (Sec. 2), so this
 * is a project choice.
 * ---------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += weyl0;
      k1 += weyl1;
    }
    uint64_t p0 = (uint64_t)mult0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)mult1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Key of one (seed, sample, replica): k0 = low word of the seed, k1 = high
 * word XOR (2*sample + replica) * 0x9E3779B9 (mod 2^32).  The stream number
 * 2*sample + replica names each (sample, replica) once only while
 * replica < 2 and sample < 2^31 (beyond, two pairs would share a key and
 * every random number): returns -1 and writes nothing outside that range,
 * else 0. */
int oracle_key(uint64_t seed, uint32_t sample, uint32_t replica, uint32_t key[2]) {
  if (replica > 1u || sample >= 0x80000000u) return -1;
  uint32_t stream = (uint32_t)(2u * sample + replica) * 0x9E3779B9u;
  key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
  key[1] = (uint32_t)(seed >> 32) ^ stream;
  return 0;
}

/* Counter of one draw: (site, sweep low word, kind<<24 | colour<<16 | hit,
 * sweep high word). */
void oracle_counter(uint32_t site, uint64_t sweep, int kind, int colour, int hit, uint32_t ctr[4]) {
  ctr[0] = site;
  ctr[1] = (uint32_t)(sweep & 0xFFFFFFFFu);
  ctr[2] = ((uint32_t)kind << 24) | ((uint32_t)colour << 16) | (uint32_t)hit;
  ctr[3] = (uint32_t)(sweep >> 32);
}

/* Uniform in the open interval (0,1): the top 23 bits m of r give
 * (2m+1) * 2^-24, which fp32 and fp64 both hold exactly. */
double oracle_u01(uint32_t r) {
  uint32_t m = r >> 9;
  return (2.0 * (double)m + 1.0) * (1.0 / 16777216.0);
}

/* Point uniform on the unit sphere from two uniforms (Archimedes' theorem:
 * the z coordinate of a uniform point on S^2 is uniform on [-1,1]). */
static void sphere_point(double u0, double u1, double v[3]) {
  double z = 2.0 * u0 - 1.0;
  double rho = sqrt(1.0 - z * z);
  double phi = 2.0 * ORACLE_PI * u1;
  v[0] = rho * cos(phi);
  v[1] = rho * sin(phi);
  v[2] = z;
}

static int64_t site_index(int L, int x, int y, int z) {
  return (int64_t)x + (int64_t)y * L + (int64_t)z * L * L;
}

static void site_coords(int L, int64_t i, int* x, int* y, int* z) {
  *x = (int)(i % L);
  *y = (int)((i / L) % L);
  *z = (int)(i / ((int64_t)L * L));
}

/* Neighbour of i one step along axis d in direction dir (+1 or -1), with
 * periodic wrap. */
static int64_t neighbour(int L, int64_t i, int d, int dir) {
  int c[3];
  site_coords(L, i, &c[0], &c[1], &c[2]);
  c[d] = (c[d] + dir + L) % L;
  return site_index(L, c[0], c[1], c[2]);
}

int oracle_colour(int L, int64_t i) {
  int x, y, z;
  site_coords(L, i, &x, &y, &z);
  return (x + y + z) % 2;
}

/* Spin initialisation: site i takes the sphere point of the draw
 * (site = i, sweep 0, kind INIT, colour 0, hit 0). */
/* Initial spin of site i under key `key`: the sphere map of the Philox draw
 * at counter (i, 0, INIT<<24, 0). */
static void init_spin_at(const uint32_t key[2], uint32_t i, double out[3]) {
  uint32_t ctr[4], r[4];
  oracle_counter(i, 0, ORACLE_KIND_INIT, 0, 0, ctr);
  oracle_philox4x32_10(ctr, key, r);
  sphere_point(oracle_u01(r[0]), oracle_u01(r[1]), out);
}

int oracle_init_spins(int L, uint64_t seed, uint32_t sample, uint32_t replica, double* s) {
  uint32_t key[2];
  int64_t n = (int64_t)L * L * L;
  if (oracle_key(seed, sample, replica, key) != 0) return -1;
  for (int64_t i = 0; i < n; ++i) init_spin_at(key, (uint32_t)i, &s[3 * i]);
  return 0;
}

/* The same for n listed sites (any lattice size): out[3k..3k+2] = spin of sites[k]. */
int oracle_init_spin_sites(uint64_t seed, uint32_t sample, uint32_t replica, const uint32_t* sites, int n,
                           double* out) {
  uint32_t key[2];
  if (oracle_key(seed, sample, replica, key) != 0) return -1;
  for (int k = 0; k < n; ++k) init_spin_at(key, sites[k], &out[3 * k]);
  return 0;
}

/* Gaussian couplings J ~ N(0,1) (Sec. 2: Gaussian, mean 0, variance 1),
 * drawn from Philox so that a sample's disorder needs no host-side arrays:
 * site i draws (u0,u1,u2,u3) at counter (i, 0, JGEN<<24, 0) under the key of
 * (seed, sample, replica 0) -- replicas of a sample share J -- and the
 * Box-Muller transform (Box & Muller, Ann. Math. Stat. 29, 1958) gives
 *   J[3i]   = sqrt(-2 ln u0) cos(2 pi u1),
 *   J[3i+1] = sqrt(-2 ln u0) sin(2 pi u1),
 *   J[3i+2] = sqrt(-2 ln u2) cos(2 pi u3). */
static void couplings_at(const uint32_t key[2], uint32_t i, double out[3]) {
  uint32_t ctr[4], r[4];
  oracle_counter(i, 0, ORACLE_KIND_JGEN, 0, 0, ctr);
  oracle_philox4x32_10(ctr, key, r);
  double u0 = oracle_u01(r[0]), u1 = oracle_u01(r[1]);
  double u2 = oracle_u01(r[2]), u3 = oracle_u01(r[3]);
  double a = sqrt(-2.0 * log(u0)), b = sqrt(-2.0 * log(u2));
  out[0] = a * cos(2.0 * ORACLE_PI * u1);
  out[1] = a * sin(2.0 * ORACLE_PI * u1);
  out[2] = b * cos(2.0 * ORACLE_PI * u3);
}

int oracle_gaussian_couplings(int L, uint64_t seed, uint32_t sample, double* J) {
  uint32_t key[2];
  int64_t n = (int64_t)L * L * L;
  if (oracle_key(seed, sample, 0, key) != 0) return -1;
  for (int64_t i = 0; i < n; ++i) couplings_at(key, (uint32_t)i, &J[3 * i]);
  return 0;
}

/* The same for n listed sites: out[3k + d] = J of the bond from sites[k] to +e_d. */
int oracle_gaussian_coupling_sites(uint64_t seed, uint32_t sample, const uint32_t* sites, int n, double* out) {
  uint32_t key[2];
  if (oracle_key(seed, sample, 0, key) != 0) return -1;
  for (int k = 0; k < n; ++k) couplings_at(key, sites[k], &out[3 * k]);
  return 0;
}

/* Local field of site i (Eq. 2 with reading R2):
 * h_i = sum_d ( J[3i+d] s_{i+e_d} + J[3(i-e_d)+d] s_{i-e_d} ). */
void oracle_local_field(int L, const double* J, const double* s, int64_t i, double h[3]) {
  h[0] = h[1] = h[2] = 0.0;
  for (int d = 0; d < 3; ++d) {
    int64_t up = neighbour(L, i, d, +1);
    int64_t dn = neighbour(L, i, d, -1);
    double j_up = J[3 * i + d];
    double j_dn = J[3 * dn + d];
    for (int a = 0; a < 3; ++a) h[a] += j_up * s[3 * up + a] + j_dn * s[3 * dn + a];
  }
}

/* The same sum for one site from its six neighbours given explicitly (for
   samples of lattices too large to hold): for d = x, y, z in turn, nb[2d] is
   the spin at i + e_d with bond Jb[2d] = J[3i + d], nb[2d + 1] the spin at
   i - e_d with bond Jb[2d + 1] = J[3(i - e_d) + d]; same order of terms as
   oracle_local_field, so the two agree bit for bit. */
void oracle_local_field_nb(const double nb[18], const double Jb[6], double h[3]) {
  h[0] = h[1] = h[2] = 0.0;
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < 3; ++a) h[a] += Jb[2 * d] * nb[3 * (2 * d) + a] + Jb[2 * d + 1] * nb[3 * (2 * d + 1) + a];
}

/* Total energy, Eq. 1 with each bond counted once (reading R1). */
double oracle_energy(int L, const double* J, const double* s) {
  int64_t n = (int64_t)L * L * L;
  double e = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    for (int d = 0; d < 3; ++d) {
      int64_t up = neighbour(L, i, d, +1);
      double dot = s[3 * i] * s[3 * up] + s[3 * i + 1] * s[3 * up + 1] + s[3 * i + 2] * s[3 * up + 2];
      e -= J[3 * i + d] * dot;
    }
  }
  return e;
}

static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Over-relaxation (Sec. 4, reading R3): s' = 2 (s.h)/(h.h) h - s. */
static void update_or(const double s[3], const double h[3], double out[3]) {
  double hh = dot3(h, h);
  if (hh == 0.0) {
    out[0] = s[0]; out[1] = s[1]; out[2] = s[2];
    return;
  }
  double f = 2.0 * dot3(s, h) / hh;
  for (int a = 0; a < 3; ++a) out[a] = f * h[a] - s[a];
}

/* Metropolis, multi-hit at fixed h (the paper names Metropolis and the
 * multi-hit technique, Sec. 2 and Table 3; the formulas are the project's).
 * Hit j draws (u0,u1,u2,u3) from counter (site, sweep, MET, colour, j).
 *   sphere proposal: s' = sphere_point(u0,u1)
 *   ball proposal:   d = sphere_point(u0,u1), rho = cbrt(u2) (so rho*d is
 *                    uniform in the unit ball), s' = (s + step*rho*d)/|..|;
 *                    a zero-length vector is rejected.
 * The site energy in the field is -s.h, so dE = -(s' - s).h; the hit is
 * accepted iff u3 < exp(-beta dE).  *margin receives the smallest
 * |u3 - exp(-beta dE)| over the hits. */
static void update_metropolis(const double s[3], const double h[3], const oracle_params* p,
                              uint32_t site, int colour, double out[3], double* margin) {
  double cur[3] = {s[0], s[1], s[2]};
  double m = INFINITY;
  uint32_t ctr[4], r[4];
  for (int hit = 0; hit < p->hits; ++hit) {
    oracle_counter(site, p->sweep, ORACLE_KIND_MET, colour, hit, ctr);
    oracle_philox4x32_10(ctr, p->key, r);
    double u0 = oracle_u01(r[0]), u1 = oracle_u01(r[1]);
    double u2 = oracle_u01(r[2]), u3 = oracle_u01(r[3]);
    double prop[3];
    double d[3];
    sphere_point(u0, u1, d);
    if (p->proposal == ORACLE_PROP_SPHERE) {
      prop[0] = d[0]; prop[1] = d[1]; prop[2] = d[2];
    } else {
      double rho = cbrt(u2);
      double v[3];
      for (int a = 0; a < 3; ++a) v[a] = cur[a] + p->step * rho * d[a];
      double nv = sqrt(dot3(v, v));
      if (nv == 0.0) continue; /* rejected: no direction */
      for (int a = 0; a < 3; ++a) prop[a] = v[a] / nv;
    }
    double de = 0.0;
    for (int a = 0; a < 3; ++a) de -= (prop[a] - cur[a]) * h[a];
    double pacc = exp(-p->beta * de);
    double gap = fabs(u3 - pacc);
    if (gap < m) m = gap;
    if (u3 < pacc) {
      cur[0] = prop[0]; cur[1] = prop[1]; cur[2] = prop[2];
    }
  }
  out[0] = cur[0]; out[1] = cur[1]; out[2] = cur[2];
  if (margin) *margin = m;
}

/* Orthonormal pair (e1, e2) perpendicular to the unit vector n, by the
 * branch-free construction of Duff, Burgess, Christensen, Hery, Kensler,
 * Liani & Villemin, "Building an Orthonormal Basis, Revisited", JCGT 6(1),
 * 2017.  sign is +1 for n_z >= 0 (including +0) and -1 for n_z < 0. */
static void orthonormal_frame(const double n[3], double e1[3], double e2[3]) {
  double sign = copysign(1.0, n[2]);
  double a = -1.0 / (sign + n[2]);
  double b = n[0] * n[1] * a;
  e1[0] = 1.0 + sign * n[0] * n[0] * a;
  e1[1] = sign * b;
  e1[2] = -sign * n[0];
  e2[0] = b;
  e2[1] = sign + n[1] * n[1] * a;
  e2[2] = -n[1];
}

/* Heat-bath (named in Sec. 2 and 4; the formula is the project's): the new
 * spin is drawn from the density proportional to exp(beta s'.h) on S^2,
 * independently of the old spin.  With x = beta|h| and t = cos of the angle
 * to h, t has density prop. to exp(x t) on [-1,1]; inverting its CDF in the
 * variable s = 1 - t gives  s = -log1p(u0 * expm1(-2x)) / x.  The azimuth
 * is 2 pi u1 in the frame (e1, e2) of h/|h|.  For x < 1e-6 (or h = 0) the
 * spin is uniform on S^2 from (u0, u1). */
static void update_heatbath(const double h[3], const oracle_params* p, uint32_t site, int colour,
                            double out[3]) {
  uint32_t ctr[4], r[4];
  oracle_counter(site, p->sweep, ORACLE_KIND_HB, colour, 0, ctr);
  oracle_philox4x32_10(ctr, p->key, r);
  double u0 = oracle_u01(r[0]), u1 = oracle_u01(r[1]);
  double hn = sqrt(dot3(h, h));
  double x = p->beta * hn;
  if (!(x >= 1e-6)) {
    sphere_point(u0, u1, out);
    return;
  }
  double n[3] = {h[0] / hn, h[1] / hn, h[2] / hn};
  double sv = -log1p(u0 * expm1(-2.0 * x)) / x;
  if (sv < 0.0) sv = 0.0;
  if (sv > 2.0) sv = 2.0;
  double ct = 1.0 - sv;
  double st = sqrt(fmax(sv * (2.0 - sv), 0.0));
  double phi = 2.0 * ORACLE_PI * u1;
  double e1[3], e2[3];
  orthonormal_frame(n, e1, e2);
  double cp = cos(phi), sp = sin(phi);
  for (int a = 0; a < 3; ++a) out[a] = ct * n[a] + st * (cp * e1[a] + sp * e2[a]);
}

/* One site update of kind upd given the spin s and its local field h.
 * site is the linear site index, colour its checkerboard colour. */
void oracle_update_site(int upd, const double s[3], const double h[3], const oracle_params* p,
                        uint32_t site, int colour, double out[3], double* margin) {
  if (margin) *margin = INFINITY;
  if (upd == ORACLE_OR) {
    update_or(s, h, out);
  } else if (upd == ORACLE_MET) {
    update_metropolis(s, h, p, site, colour, out, margin);
  } else if (upd == ORACLE_MET_OR) {
    /* The neighbours do not move during a colour's pass, so h is the same
     * for the Metropolis hits and the reflection that follows them. */
    double mid[3];
    update_metropolis(s, h, p, site, colour, mid, margin);
    update_or(mid, h, out);
  } else {
    update_heatbath(h, p, site, colour, out);
  }
}

/* One half-sweep (reading R4) restricted to the sites i0 <= i < i1: every
 * site of colour `colour` in the range is updated from the current values
 * of the other colour.  Sites of one colour do not interact, so the loop
 * order does not change the result.  margins, if not NULL, receives per
 * site of the range the Metropolis margin (INFINITY elsewhere). */
/* Threads of the half-sweep loop below (OpenMP, when the library is built
   with it): the sites of one colour read only the other colour and each is
   written once, so any number of threads gives the same result.  Default 1;
   only the timed CPU baseline raises it. */
static int g_threads = 1;
void oracle_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_num_procs();
#else
  return 1;
#endif
}

void oracle_half_sweep_range(int L, const double* J, double* s, int upd, int colour,
                             const oracle_params* p, int64_t i0, int64_t i1, double* margins) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
#endif
  for (int64_t i = i0; i < i1; ++i) {
    if (margins) margins[i] = INFINITY;
    if (oracle_colour(L, i) != colour) continue;
    double h[3], out[3], m;
    oracle_local_field(L, J, s, i, h);
    oracle_update_site(upd, &s[3 * i], h, p, (uint32_t)i, colour, out, &m);
    s[3 * i] = out[0]; s[3 * i + 1] = out[1]; s[3 * i + 2] = out[2];
    if (margins) margins[i] = m;
  }
}

/* The same half-sweep over all sites. */
void oracle_half_sweep(int L, const double* J, double* s, int upd, int colour,
                       const oracle_params* p, double* margins) {
  oracle_half_sweep_range(L, J, s, upd, colour, p, 0, (int64_t)L * L * L, margins);
}

/* Renormalisation: s <- s/|s| for every site. */
void oracle_renorm(int L, double* s) {
  int64_t n = (int64_t)L * L * L;
  for (int64_t i = 0; i < n; ++i) {
    double nrm = sqrt(dot3(&s[3 * i], &s[3 * i]));
    if (nrm > 0.0)
      for (int a = 0; a < 3; ++a) s[3 * i + a] /= nrm;
  }
}

/* n_sweeps sweeps of a schedule.  One sweep: the main update on colour 0
 * then colour 1 (if any), then n_or over-relaxation sweeps, each colour 0
 * then colour 1; the sweep counter then advances by one; every
 * renorm_every sweeps the spins are renormalised, and every energy_every
 * sweeps E/N is appended to elog (renormalisation first when both fall on
 * the same sweep).  *n_elog counts the appended values. */
void oracle_sweeps(int L, const double* J, double* s, const oracle_schedule* sch, const uint32_t key[2],
                   int n_sweeps, uint64_t* sweep, double* elog, int* n_elog) {
  oracle_params p;
  p.key[0] = key[0];
  p.key[1] = key[1];
  p.beta = sch->beta;
  p.step = sch->step;
  p.hits = sch->hits;
  p.proposal = sch->proposal;
  double n = (double)L * L * L;
  for (int k = 0; k < n_sweeps; ++k) {
    p.sweep = *sweep;
    if (sch->kind == ORACLE_MET || sch->kind == ORACLE_HB || sch->kind == ORACLE_MET_OR) {
      oracle_half_sweep(L, J, s, sch->kind, 0, &p, NULL);
      oracle_half_sweep(L, J, s, sch->kind, 1, &p, NULL);
    }
    for (int o = 0; o < sch->n_or; ++o) {
      oracle_half_sweep(L, J, s, ORACLE_OR, 0, &p, NULL);
      oracle_half_sweep(L, J, s, ORACLE_OR, 1, &p, NULL);
    }
    *sweep += 1;
    if (sch->renorm_every > 0 && (*sweep % (uint64_t)sch->renorm_every) == 0) oracle_renorm(L, s);
    if (sch->energy_every > 0 && (*sweep % (uint64_t)sch->energy_every) == 0) {
      if (elog) elog[*n_elog] = oracle_energy(L, J, s) / n;
      *n_elog += 1;
    }
  }
}
