/*
 * hsg.h -- C ABI of libhsg: checkerboard Monte Carlo sweeps of the 3D
 * Heisenberg spin glass on one GB300 GPU (sm_103a).
 *
 * Model (Bernaschi, Parisi & Parisi, "The Heisenberg spin glass model on
 * GPU: myths and actual facts", Sec. 2, Eq. 1 and Eq. 2): unit 3-vector
 * spins s_i on an L^3 periodic cubic lattice, Gaussian couplings J on the
 * nearest-neighbour bonds, H = - sum over bonds J s_i . s_j (each bond
 * counted once), local field h_i = sum over the six neighbours J_bond s_nb.
 *
 * Host-visible layout ("site-major", the paper's indexing, Sec. 2):
 *   site i = x + y*L + z*L*L;
 *   spins  float s[3*N],  s[3*i + a] = component a of site i;
 *   J      J[3*N],        J[3*i + d] = coupling of the bond from i to
 *                         i + e_d (d = 0, 1, 2 for +x, +y, +z), periodic.
 * The library keeps its own colour-split copy on the device and converts
 * on the way in and out.
 *
 * Conventions for every function:
 *   - Returns HSG_OK (0) or an error code; never throws, never aborts.
 *   - Arguments are checked on the host before anything is launched; a bad
 *     argument returns HSG_EINVAL and leaves the context unchanged.
 *   - Work is queued on the stream given to hsg_create, in call order.
 *     Functions that return host data synchronise that stream; the others
 *     are asynchronous.
 *   - A context or pool belongs to the device that was current when it was
 *     created.  Each call makes that device current for its duration and
 *     then restores the caller's, so objects of several devices can be used
 *     from one thread in any order.
 *   - Device memory is owned by the context (stream-ordered allocations),
 *     released by hsg_destroy.  Caller arrays are copied, never retained.
 *   - hsg_last_error() gives a message for the last failure.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef HSG_H
#define HSG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int hsg_status;
enum {
  HSG_OK = 0,
  HSG_EINVAL = 1,   /* bad argument or call order */
  HSG_ENOMEM = 2,   /* device or pinned-host allocation failed */
  HSG_ECUDA = 3,    /* a CUDA runtime call failed (message in hsg_last_error) */
  HSG_ETIMEOUT = 4, /* a bounded device wait gave up (see hsg_energy) */
  HSG_EBUSY = 5     /* resource in use */
};

/* Main update of a sweep, and the update of a single half-sweep. */
enum {
  HSG_NONE = 0,
  HSG_METROPOLIS = 1, /* multi-hit Metropolis (named in Sec. 2; Table 3) */
  HSG_HEATBATH = 2,   /* heat-bath (named in Sec. 2 and Sec. 4) */
  HSG_OVERRELAX = 3,  /* over-relaxation (Sec. 4); only for hsg_half_sweep */
  /* Fused colour pass (opt-in; not in the paper): at every site the
   * Metropolis hits, then one over-relaxation reflection about the same
   * local field -- within a colour's pass the neighbours do not move.  A
   * different chain from Metropolis followed by OR sweeps, with the same
   * equilibrium; it moves each spin twice per half-sweep of memory traffic. */
  HSG_METROPOLIS_OR = 4
};

/* Metropolis proposals. */
enum {
  HSG_PROP_SPHERE = 0, /* s' uniform on the unit sphere */
  HSG_PROP_BALL = 1    /* s' = (s + step*u)/|s + step*u|, u uniform in the unit ball */
};

/* Element types and memory spaces of caller arrays. */
enum { HSG_F32 = 0, HSG_F64 = 1 };
enum { HSG_HOST = 0, HSG_DEVICE = 1 };

/* Half-sweep kernel variant. */
enum {
  HSG_KERNEL_AUTO = 0,   /* library's choice: HSG_KERNEL_WAVE when the lattice's
                          * spins and bonds (28 N bytes) exceed three quarters of
                          * the device's L2, so that the sweep streams much of it
                          * from HBM; else GLOBAL */
  HSG_KERNEL_GLOBAL = 1, /* one thread per site, neighbours through L1/L2 (heat-bath:
                          * one thread per six-plane column, carrying its column's
                          * neighbours; the same results) */
  HSG_KERNEL_SLAB = 2,   /* z-marching tiles: other colour staged in shared memory */
  /* Temporally blocked over-relaxation: each over-relaxation sweep
   * runs colour 0 and colour 1 in ONE pass over the lattice (z-marching
   * tiles; the new colour-0 planes stay in shared memory for the colour-1
   * update), so each spin and bond leaves HBM about once per sweep instead of
   * once per half-sweep (44 instead of 72 bytes per site update).  Results
   * are bit-identical to HSG_KERNEL_GLOBAL.  The pass writes a second spin
   * buffer of 16 N bytes, allocated by the first hsg_sweep that needs it and
   * kept until hsg_destroy; the two buffers alternate.  The main update of a
   * sweep and hsg_half_sweep use the global kernel.  A renormalisation due
   * right after a sweep is done by that sweep's last wave pass, as it
   * stores (bit-identical to a renormalisation of its own).  From L = 32
   * the pass also keeps a halo-padded copy of the couplings for its tensor
   * loads (about 12 N (1 + 4/L)(1 + 8/L) bytes), made by the first hsg_sweep
   * that needs it when the device has that much free beside 1 GiB, written
   * by hsg_set_couplings from then on, and rebuilt (one launch) by the first
   * sweep after hsg_generate_couplings; without it
   * the pass loads the couplings through registers, with the same results. */
  HSG_KERNEL_WAVE = 3
};

/* Device layout of the spins (hsg_create_layout). */
enum {
  HSG_LAYOUT_FLOAT4 = 0, /* one float4 per spin (16 bytes: x, y, z, unused) */
  HSG_LAYOUT_PACKED = 1  /* three fp32 arrays per colour (12 bytes a spin): 60 instead of 72
                          * bytes per over-relaxation update; global kernel only */
};

/* Kernel classes reported by the profiler. */
enum {
  HSG_PROF_INIT = 0,
  HSG_PROF_LAYOUT = 1,   /* coupling / spin layout conversion */
  HSG_PROF_OVERRELAX = 2,
  HSG_PROF_METROPOLIS = 3,
  HSG_PROF_HEATBATH = 4,
  HSG_PROF_ENERGY = 5,   /* both energy kernels */
  HSG_PROF_RENORM = 6,
  HSG_PROF_OVERRELAX_RENORM = 7, /* an over-relaxation wave sweep that also renormalises what it stores
                                  * (a renormalisation due right after it, fused into it) */
  HSG_PROF_COUNT = 8
};

/*
 * One sweep = the main update (`kind`) on colour 0 then colour 1, then
 * `n_or` over-relaxation sweeps (colour 0 then colour 1 each); then the
 * sweep counter advances by one.  After the counter advances, every
 * `renorm_every` sweeps the spins are renormalised in FP64, and every
 * `energy_every` sweeps E/N (FP64) is appended to the energy log, the
 * renormalisation first.  Colour of site (x,y,z) = (x+y+z) mod 2; colour 0
 * goes first (Sec. 4: all white spins, then all black spins).
 *
 * Random numbers: Philox-4x32-10 (Salmon et al., SC'11), key (k0, k1) =
 * (seed low word, seed high word XOR (2*sample + replica)*0x9E3779B9),
 * counter (site, sweep low word, kind<<24 | colour<<16 | hit, sweep high
 * word) with kind 1 = init, 3 = Metropolis, 4 = heat-bath; uniform
 * u = ((r >> 9)*2 + 1) * 2^-24.  One draw per Metropolis hit (u0, u1:
 * direction; u2: ball radius cbrt(u2); u3: accept iff u3 < exp(-beta dE))
 * and one per heat-bath update (u0: polar angle via
 * 1 - cos = -log1p(u0*expm1(-2x))/x with x = beta|h|; u1: azimuth 2 pi u1
 * in the Duff et al. (JCGT 2017) frame of h; uniform on S^2 if x < 1e-6).
 */
typedef struct hsg_schedule {
  int kind;         /* HSG_NONE | HSG_METROPOLIS | HSG_HEATBATH | HSG_METROPOLIS_OR */
  int hits;         /* Metropolis hits per site per half-sweep, 1..65535 */
  int proposal;     /* HSG_PROP_SPHERE | HSG_PROP_BALL */
  float step;       /* ball-proposal scale, > 0 */
  int n_or;         /* over-relaxation sweeps after the main update, >= 0 */
  double T;         /* temperature, > 0; +inf allowed (beta = 0) */
  int renorm_every; /* 0 = never, else > 0 */
  int energy_every; /* 0 = never, else > 0 */
  int kernel;       /* HSG_KERNEL_* */
} hsg_schedule;

typedef struct hsg_ctx hsg_ctx; /* opaque, library-owned */

/*
 * Create a lattice of side L on the current CUDA device, queued on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * Spins start uniform on S^2, drawn from Philox kind 1 at counter site i,
 * sweep 0 (Sec. 2: unit 3-vector spins).  The sweep counter starts at 0.
 * L must be even (the checkerboard needs it under periodic wrap) and in
 * [4, 1624] (site indices fit 32 bits).  replica must be 0 or 1 and
 * sample < 2^31: the key's stream number 2*sample + replica (see
 * hsg_schedule) names each pair once only in that range, and two pairs
 * sharing a key would share every random number.  Couplings must be set
 * with hsg_set_couplings before any sweep.
 * Errors: HSG_EINVAL (out == NULL, bad L, replica > 1, sample >= 2^31),
 * HSG_ENOMEM, HSG_ECUDA (no device); *out is NULL on error and nothing
 * leaks.
 */
hsg_status hsg_create(hsg_ctx** out, int L, uint64_t seed, uint32_t sample, uint32_t replica,
                      void* cuda_stream);

/*
 * hsg_create with a choice of device spin layout.  HSG_LAYOUT_PACKED keeps
 * each colour as three fp32 component arrays instead of float4: the paper's
 * own footprint of six single-precision words per lattice point, three spin
 * components and three bonds (Sec. 4), 25 % fewer spin bytes per update than
 * float4, the same results bit for bit.  A packed
 * lattice sweeps with the global kernel (HSG_KERNEL_AUTO or _GLOBAL;
 * _SLAB / _WAVE return HSG_EINVAL).  Library-specific (the paper has one
 * layout).  Errors as hsg_create, and HSG_EINVAL for an unknown layout.
 */
hsg_status hsg_create_layout(hsg_ctx** out, int L, uint64_t seed, uint32_t sample, uint32_t replica,
                             void* cuda_stream, int layout);

/* Release everything the context owns; waits for its stream.  NULL is a
 * no-op returning HSG_OK. */
hsg_status hsg_destroy(hsg_ctx* ctx);

/*
 * Set the couplings (Eq. 1: Gaussian J_ij on nearest-neighbour bonds).
 * J: 3*N values, site-major J[3*i + d] (see top), of type `dtype`
 * (HSG_F32 | HSG_F64) in memory space `where` (HSG_HOST | HSG_DEVICE).
 * FP64 values are rounded to FP32 (round to nearest) on upload; all spin
 * arithmetic is FP32.  A host array is copied before the call returns; a
 * device array must stay valid until the stream reaches this call.
 * Errors: HSG_EINVAL (NULL, bad dtype/where), HSG_ENOMEM, HSG_ECUDA.
 */
hsg_status hsg_set_couplings(hsg_ctx* ctx, const void* J, int dtype, int where);

/*
 * Draw the couplings on the device (Sec. 2: Gaussian J, mean 0, variance
 * 1) from the context's (seed, sample): bond d of site i comes from the
 * Philox draw of kind 2 at counter (i, 0, 2<<24, 0) under the key of
 * (seed, sample, replica 0) -- the replicas of a sample share their J --
 * through the Box-Muller transform in FP64 (J_x, J_y from (u0, u1), J_z
 * from (u2, u3)), rounded once to FP32.  Queued on the stream.
 * hsg_get_couplings returns the FP32 couplings site-major, J[3*i + d], in
 * memory space `where` (HOST synchronises).
 */
hsg_status hsg_generate_couplings(hsg_ctx* ctx);
hsg_status hsg_get_couplings(hsg_ctx* ctx, float* out, int where);

/*
 * Run n_sweeps sweeps of `schedule` (see hsg_schedule), asynchronously on
 * the context's stream.  n_sweeps = 0 is a no-op.
 * Checkerboard half-sweeps follow Sec. 4 (non-interacting spins in
 * parallel, one launch per colour); the local field is Eq. 2;
 * over-relaxation is the reflection s' = 2 (s.h)/(h.h) h - s (Sec. 4, the
 * energy-conserving maximal move; s unchanged when h = 0).
 * Errors: HSG_EINVAL (bad schedule, n_sweeps < 0, couplings not set),
 * HSG_ENOMEM (energy log growth), HSG_ECUDA.
 */
hsg_status hsg_sweep(hsg_ctx* ctx, const hsg_schedule* schedule, int n_sweeps);

/*
 * E/N of the current state (Eq. 1, each bond once, divided by N = L^3):
 * per-site local fields in FP32, dot products and the deterministic
 * two-pass sum in FP64.  Synchronises the stream.
 * Errors: HSG_EINVAL (NULL, couplings not set), HSG_ECUDA, HSG_ETIMEOUT (a
 * temporally blocked sweep queued before gave up a bounded wait -- 0.2 s --
 * for its couplings' tensor loads; the spins since then are not valid).
 */
hsg_status hsg_energy(hsg_ctx* ctx, double* e_per_spin);

/* Energy log written by hsg_sweep: copies min(max_n, logged) values of
 * E/N, oldest first, into host `out` and the number logged into *n (either
 * pointer may be NULL when max_n = 0).  Synchronises the stream. */
hsg_status hsg_get_energy_log(hsg_ctx* ctx, double* out, int max_n, int* n);
hsg_status hsg_clear_energy_log(hsg_ctx* ctx);

/*
 * Spins and bonds of n listed sites (site-major indices i = x + y*L +
 * z*L*L < N, host array `sites`): spins[3k + a] = component a of site
 * sites[k], and, if `bonds` is not NULL, bonds[3k + d] = J of its bond to
 * +e_d (d = 0, 1, 2).  Host output arrays of 3n floats; synchronises the
 * stream.  For checking samples of lattices too large to copy whole
 * (library-specific; the paper has no counterpart).
 * Errors: HSG_EINVAL (NULL arrays with n > 0, n < 0, an index >= N, bonds
 * requested before couplings are set).
 */
hsg_status hsg_get_sites(hsg_ctx* ctx, const uint32_t* sites, int n, float* spins, float* bonds);

/*
 * Spins as site-major FP32 s[3*N] (see top), in memory space `where`.
 * hsg_get_spins with HSG_HOST synchronises; with HSG_DEVICE it is queued
 * on the stream.  hsg_set_spins stores the values as given (no
 * normalisation).  Together with hsg_get_sweep / hsg_set_sweep this is a
 * full checkpoint: the random numbers depend only on (key, counter), so a
 * resumed run repeats the continuous one bit for bit.
 */
hsg_status hsg_get_spins(hsg_ctx* ctx, float* out, int where);
hsg_status hsg_set_spins(hsg_ctx* ctx, const float* in, int where);
hsg_status hsg_get_sweep(hsg_ctx* ctx, uint64_t* sweep);
hsg_status hsg_set_sweep(hsg_ctx* ctx, uint64_t sweep);

/*
 * One half-sweep: update `update` (HSG_OVERRELAX, HSG_METROPOLIS or
 * HSG_HEATBATH, with the temperature / hits / proposal / kernel fields of
 * `schedule`) on every site of `colour` (0 or 1) at the current sweep
 * counter, which is not advanced.  Used to check single half-sweeps
 * against the oracle and to build custom schedules.
 */
hsg_status hsg_half_sweep(hsg_ctx* ctx, const hsg_schedule* schedule, int update, int colour);

/* Renormalise every spin, s <- s/|s|, computed in FP64, stored FP32. */
hsg_status hsg_renorm(hsg_ctx* ctx);

/*
 * The kernel variant hsg_sweep runs for the over-relaxation sweeps of
 * `schedule` on this lattice (HSG_KERNEL_GLOBAL, _SLAB or _WAVE: what
 * HSG_KERNEL_AUTO resolves to).  Library-specific; the paper has no
 * counterpart.  Errors: HSG_EINVAL (NULL argument, bad schedule).
 */
hsg_status hsg_kernel_for(hsg_ctx* ctx, const hsg_schedule* schedule, int* kernel);

/*
 * Profiler: with on != 0 every kernel the context launches is bracketed
 * by CUDA events on its stream.  hsg_profile_read synchronises, adds the
 * elapsed time (ms) and the number of launches of class `kclass`
 * (HSG_PROF_*) recorded since the last reset, and hsg_profile_reset
 * clears the records.  hsg_launch_count counts every kernel launch of the
 * context since creation, profiled or not.
 */
hsg_status hsg_profile(hsg_ctx* ctx, int on);
hsg_status hsg_profile_read(hsg_ctx* ctx, int kclass, double* total_ms, uint64_t* launches);
hsg_status hsg_profile_reset(hsg_ctx* ctx);
hsg_status hsg_launch_count(hsg_ctx* ctx, uint64_t* launches);

/* Message of the context's last failure ("" if none).  With ctx == NULL:
 * the calling thread's last failure of a call without a context
 * (hsg_create, hsg_philox). */
const char* hsg_last_error(const hsg_ctx* ctx);
const char* hsg_status_string(hsg_status s);

/* Library version as major*10000 + minor*100 + patch. */
int hsg_version(void);

/*
 * Philox-4x32-10 stream of one key, on the device: for t < n,
 * out[4*t + w] = word w of Philox((t, c1, c2, c3), key(seed, sample,
 * replica)).  out: device array of 4*n uint32, queued on `cuda_stream`.
 * The same device function feeds every update kernel; this entry point
 * exposes it so that its words can be compared with other Philox
 * implementations.  Errors: HSG_EINVAL (out NULL or not 16-byte aligned,
 * replica > 1, sample >= 2^31, as for hsg_create), HSG_ECUDA.
 */
hsg_status hsg_philox(uint64_t seed, uint32_t sample, uint32_t replica, uint32_t c1, uint32_t c2, uint32_t c3,
                      uint32_t n, uint32_t* out, void* cuda_stream);

/*
 * Pools: many independent lattices (disorder samples, replicas, requests) of
 * uneven L in one device arena, swept together.  Every half-sweep of a pool
 * is ONE persistent kernel over a work list of (lattice, site-range) tiles
 * covering all admitted lattices, and a sweep's launches are captured once
 * in a CUDA graph and replayed (on a non-default stream) while lattices come
 * and go.  Each lattice keeps its own side, Philox key, temperature and
 * sweep counter, and is updated by the same device code with the same
 * random numbers as a single-lattice context: its spins are bit-identical
 * to those of the same lattice swept alone with hsg_sweep.
 */
typedef struct hsg_pool hsg_pool;

/* A pool with an arena of `budget_bytes` of device memory (allocated once,
 * here) and room for `max_slots` lattices, queued on `cuda_stream`.  A
 * lattice of side L takes 28 L^3 bytes (float4 spins + 3 fp32 bonds per
 * site), rounded up to 256.  Errors: HSG_EINVAL, HSG_ENOMEM, HSG_ECUDA. */
hsg_status hsg_pool_create(hsg_pool** out, uint64_t budget_bytes, int max_slots, void* cuda_stream);
hsg_status hsg_pool_destroy(hsg_pool* pool); /* NULL ok; waits for the stream */

/* Admit one lattice: side L (even, 4..1624), Philox key from (seed,
 * sample, replica) with replica 0 or 1 and sample < 2^31 (HSG_EINVAL
 * otherwise, as for hsg_create), temperature T (> 0, inf allowed); spins
 * start as in hsg_create; couplings from J (site-major, dtype / where as in
 * hsg_set_couplings) or, with J == NULL, generated on the device as by
 * hsg_generate_couplings.  *slot receives the lattice's slot index, its
 * sweep counter starts at 0.  HSG_EBUSY (nothing changed) when no slot is
 * free or the arena has no free block large enough. */
hsg_status hsg_pool_admit(hsg_pool* pool, int L, uint64_t seed, uint32_t sample, uint32_t replica, double T,
                          const void* J, int dtype, int where, int* slot);

/* Release a lattice's slot and arena block.  Does not wait: work already
 * queued for the slot runs first, and the block is reused only by work
 * queued on the pool's stream after this call (stream order). */
hsg_status hsg_pool_retire(hsg_pool* pool, int slot);

/* n_sweeps sweeps of every admitted lattice, each at its own temperature
 * (schedule.T and schedule.kernel are ignored; energy_every must be 0;
 * renorm_every applies to each lattice's own counter).  Asynchronous. */
hsg_status hsg_pool_sweep(hsg_pool* pool, const hsg_schedule* schedule, int n_sweeps);

/* E/N of every slot into out[0..n) (NaN for free slots); FP32 site terms,
 * FP64 sums, fixed order (Eq. 1, as hsg_energy).  Synchronises. */
hsg_status hsg_pool_energies(hsg_pool* pool, double* out, int n);

/* The same energies without waiting: hsg_pool_energies_async queues the
 * energy kernels and the copy of every slot's E/N into the pool's pinned
 * buffer `buffer` (0 or 1) after the work already queued, and returns;
 * hsg_pool_energies_read waits for that copy and writes the values into
 * out[0..n) (NaN for slots free at queueing time and for i >= max_slots).
 * A slot retired after hsg_pool_energies_async still gets its final E/N.
 * Reading a buffer with nothing queued is HSG_EINVAL; queueing into a
 * buffer that was not read waits for and drops its previous values. */
hsg_status hsg_pool_energies_async(hsg_pool* pool, int buffer);
hsg_status hsg_pool_energies_read(hsg_pool* pool, int buffer, double* out, int n);

/* As hsg_pool_energies_async for the n active slots listed in slots[]
 * only (read back with hsg_pool_energies_read; every other slot reads
 * NaN): the energy kernels skip the other lattices' sites.  A slot that is
 * not active is HSG_EINVAL (nothing queued). */
hsg_status hsg_pool_energies_slots_async(hsg_pool* pool, int buffer, const int* slots, int n);

/* One lattice's spins, site-major fp32 (as hsg_get_spins), and counter. */
hsg_status hsg_pool_get_spins(hsg_pool* pool, int slot, float* out, int where);
hsg_status hsg_pool_get_sweep(hsg_pool* pool, int slot, uint64_t* sweep);

/* Arena bytes in use, the budget, and the number of admitted lattices. */
hsg_status hsg_pool_usage(hsg_pool* pool, uint64_t* bytes_used, uint64_t* bytes_budget, int* active);

/* Launch configuration of the pool kernels: threads per CTA (64, 128 or
 * 256), sites per tile (a multiple of threads, <= 8192), CTAs per SM of the
 * persistent grid (1..32), and Metropolis hits per pass (0: all of a
 * colour's hits in one pass; h > 0: the hits in passes of at most h, each a
 * launch that reads and writes the colour again -- the neighbours are fixed
 * for the whole half-sweep and hit j draws the Philox numbers keyed by j,
 * so the result is the same; Table 3 of the paper runs the hits in one
 * pass).  hsg_pool_autotune times every launch shape with all hits in one
 * pass, then the best shape with 1, 2, 4, ... hits per pass (Metropolis
 * schedules with more than one hit), on the admitted lattices (one warm-up
 * and two timed sweeps each), restores the lattices and counters
 * afterwards, keeps the fastest configuration and reports it.  Results do
 * not depend on the configuration.  Errors: HSG_EINVAL (NULL pool, values
 * out of range; autotune with no lattice admitted or on the legacy default
 * stream). */
hsg_status hsg_pool_config(hsg_pool* pool, int threads, int tile_sites, int blocks_per_sm, int hits_per_pass);
hsg_status hsg_pool_autotune(hsg_pool* pool, const hsg_schedule* schedule, int* threads, int* tile_sites,
                             int* blocks_per_sm, int* hits_per_pass);

/* Kernel launches issued for this pool (graph replays count their kernels). */
hsg_status hsg_pool_launch_count(hsg_pool* pool, uint64_t* launches);
const char* hsg_pool_last_error(const hsg_pool* pool);

/*
 * Fault injection for tests: the k-th device allocation from now (k >= 1)
 * fails as if the device were out of memory; k = 0 disables.  Process-wide.
 */
hsg_status hsg_test_fail_alloc(int k);

/*
 * Fault injection for tests of the bounded waits of the temporally blocked
 * sweep's tensor-box kernel (L >= 32).  Bit 0 of `on`: every sweep launched
 * from now waits for more bytes than each of its couplings' tensor loads
 * delivers; bit 1: for one arrival more than the copies of each of its
 * colour-1 planes make.  Every such wait runs out (after 0.2 s; nothing
 * hangs, nothing faults), the sweep's spins are not valid, and the next
 * hsg_energy on the context returns HSG_ETIMEOUT (once).  on = 0 restores;
 * HSG_EINVAL outside 0 .. 3.  Process-wide; a sweep captured in a CUDA
 * graph keeps the setting it was captured with.  Library-specific.
 */
hsg_status hsg_test_stall_tensor_loads(int on);

/*
 * E/N of a lattice held in the caller's own device memory, without any
 * allocation.  The paper has no counterpart: this entry point exists for
 * callers that cannot let a library allocate device memory -- applications
 * that give all device memory to their own arena or caching allocator at
 * start-up and forbid raw cudaMalloc beside it, and latency-critical loops
 * that cannot afford the device-wide synchronisation an allocation or free
 * may cause.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * spins: device, site-major fp32 s[3*N]; J: device, site-major fp32 J[3*N]
 * (layouts at the top of this file); e_out: device, one double, receives
 * E/N, where E = - sum over the 3N nearest-neighbour bonds of J times the
 * dot product of the two spins it joins, each bond counted once (per-site
 * terms fp32, sums fp64).  Queued on `cuda_stream` (NULL = legacy default
 * stream); nothing is synchronised.  L must be even and in [4, 1624];
 * larger or odd L is rejected with HSG_EINVAL and a message in
 * hsg_last_error(NULL).  Each of spins, J and e_out must be device memory
 * of the current device (or managed memory), else HSG_EINVAL before any
 * launch; the arrays' lengths cannot be checked here and are the caller's
 * to get right.
 *
 * Scratch: the per-block partial sums live in a fixed device array of
 * HSG_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  The first call on a device (with that device current)
 * looks up the array's device address and caches it; make that first call
 * before any stream capture.  The cached address does not survive
 * cudaDeviceReset: do not call this entry point on a device after resetting
 * it.  All calls share the array: calls whose kernels overlap on the GPU
 * (e.g. on two streams) race and must be ordered by the caller.
 * Errors: HSG_EINVAL, HSG_ECUDA.
 */
#define HSG_NOALLOC_SCRATCH_BYTES 8192
hsg_status hsg_energy_noalloc(int L, const float* spins, const float* J, double* e_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* HSG_H */
