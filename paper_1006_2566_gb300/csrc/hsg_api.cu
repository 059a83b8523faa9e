// hsg_api.cu -- the C ABI declared in include/hsg.h.
//
// Host code only: argument checks, stream-ordered device memory, the sweep
// schedule (which kernels run in which order), the energy log and the
// event-based profiler.  Every step of the Monte Carlo itself runs in the
// kernels of hsg_sweep.cu and hsg_aux.cu.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

#include "hsg.h"
#include "hsg_device.cuh"
#include "hsg_internal.h"

namespace {

constexpr int kVersion = 100;  // 0.1.0
constexpr int kMaxL = 1624;    // L^3 < 2^32: site indices are 32-bit Philox counters
constexpr int kElogInit = 64;
constexpr long long kMaxGraphPeriod = 64;  // longest sweep period captured as one graph

thread_local std::string g_thread_error;
int g_fail_alloc_countdown = 0;  // test hook: k-th allocation from now fails
std::atomic<int> g_test_stall_boxes{0};  // test hook: hsg_test_stall_tensor_loads

// A run of consecutive launches of one kernel class, bracketed by one pair
// of events (count = launches in the run).
struct ProfRec {
  int kclass;
  cudaEvent_t start, stop;
  uint32_t count;
};

}  // namespace

struct hsg_ctx {
  int L = 0, Lh = 0;
  long long N = 0, Nh = 0;
  uint64_t seed = 0;
  uint32_t sample = 0, replica = 0, k0 = 0, k1 = 0;
  cudaStream_t stream = nullptr;
  int device = 0, sm_count = 0;
  long long l2_bytes = 0;  // the device's L2 size
  bool packed = false;          // spin layout: three fp32 arrays per colour instead of float4
  float4* spins = nullptr;      // [2][Nh] float4 (or [2][3][Nh] floats, packed), the current state
  float4* spins_alt = nullptr;  // [2][Nh], target of the temporally blocked sweeps (allocated on first use)
  float* J = nullptr;       // [3][2][Nh]
  bool have_J = false;
  // Halo-padded copy of J for the temporally blocked sweep's tensor boxes
  // (allocated with its tensor map by the first such sweep at L >= 32 when
  // the device has room for it; rebuilt after every change of J).
  float* Jpad = nullptr;
  bool Jpad_ok = false;  // Jpad holds the current J
  bool use_tma = false;  // bond_map describes Jpad
  CUtensorMap bond_map{};
  uint64_t sweep = 0;
  void* stage = nullptr;  // site-major staging for host copies
  size_t stage_bytes = 0;
  double* partials = nullptr;  // energy first-pass sums
  double* e_out = nullptr;     // hsg_energy result
  double* elog = nullptr;      // energy log
  int elog_cap = 0, elog_n = 0;
  double* host_e = nullptr;  // pinned, 2 doubles: E/N and the bond-box wait flag
  bool prof = false;
  bool group = false;     // inside hsg_sweep: one event pair per run of same-class launches
  bool run_open = false;  // recs.back() still lacks its stop event
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> free_events;
  uint64_t launches = 0;
  // Device counters: [0] the sweep counter the kernels read, [1] the energy
  // log position; the host mirrors both (sweep, elog_n).  [2] is set by a
  // temporally blocked sweep whose bounded wait for a bond box gave up.
  unsigned long long* d_ctr = nullptr;
  // One captured period of sweeps (see hsg_sweep), replayed while the
  // schedule, the kernel variant and the energy log buffer stay the same.
  cudaGraphExec_t gexec = nullptr;
  hsg_schedule gsched{};
  int gvariant = 0, gperiod = 0, glaunches = 0;
  double* gelog = nullptr;
  float4* gspins = nullptr;  // current spin buffer when the period was captured
  std::string err;
};

namespace {

hsg_status fail(hsg_ctx* c, hsg_status st, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_thread_error = msg;
  return st;
}

hsg_status cuda_fail(hsg_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) return fail(c, HSG_ENOMEM, m);
  return fail(c, HSG_ECUDA, m);
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (g_fail_alloc_countdown > 0 && --g_fail_alloc_countdown == 0) return cudaErrorMemoryAllocation;
  return cudaMallocAsync(p, bytes, s);
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

cudaEvent_t take_event(hsg_ctx* c) {
  if (!c->free_events.empty()) {
    cudaEvent_t e = c->free_events.back();
    c->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Record the stop event of the open profiler run, if any.
void close_run(hsg_ctx* c) {
  if (!c->run_open) return;
  cudaEvent_t b = take_event(c);
  if (b) cudaEventRecord(b, c->stream);
  c->recs.back().stop = b;
  c->run_open = false;
}

// Run `fn` (which launches `n_kernels` kernels on the context stream).  With
// the profiler on, each launch is bracketed by CUDA events on the stream;
// inside hsg_sweep consecutive launches of one class share one bracket, so
// that the events perturb the sweep as little as possible.
template <typename F>
hsg_status launch(hsg_ctx* c, int kclass, int n_kernels, const char* what, F&& fn) {
  if (c->prof && !(c->group && c->run_open && c->recs.back().kclass == kclass)) {
    close_run(c);
    cudaEvent_t a = take_event(c);
    if (!a) return fail(c, HSG_ECUDA, "cudaEventCreate failed");
    cudaEventRecord(a, c->stream);
    c->recs.push_back(ProfRec{kclass, a, nullptr, 0});
    c->run_open = true;
  }
  cudaError_t e = fn();
  if (e != cudaSuccess) {
    close_run(c);
    return cuda_fail(c, e, what);
  }
  c->launches += (uint64_t)n_kernels;
  if (c->prof) {
    c->recs.back().count += 1;
    if (!c->group) close_run(c);
  }
  return HSG_OK;
}

// Inside hsg_sweep: group same-class launches; the run closes on exit.
struct SweepGroup {
  hsg_ctx* c;
  explicit SweepGroup(hsg_ctx* ctx) : c(ctx) { c->group = true; }
  ~SweepGroup() {
    close_run(c);
    c->group = false;
  }
};

hsg_status ensure_stage(hsg_ctx* c, size_t bytes) {
  if (c->stage_bytes >= bytes) return HSG_OK;
  dev_free(c->stage, c->stream);
  c->stage = nullptr;
  c->stage_bytes = 0;
  cudaError_t e = dev_alloc(&c->stage, bytes, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "staging buffer");
  c->stage_bytes = bytes;
  return HSG_OK;
}

void release(hsg_ctx* c) {
  if (!c) return;
  const hsg::DeviceGuard device_guard(c->device);
  cudaStream_t s = c->stream;
  dev_free(c->spins, s);
  dev_free(c->spins_alt, s);
  dev_free(c->J, s);
  dev_free(c->Jpad, s);
  dev_free(c->stage, s);
  dev_free(c->partials, s);
  dev_free(c->e_out, s);
  dev_free(c->elog, s);
  dev_free(c->d_ctr, s);
  cudaStreamSynchronize(s);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->host_e) cudaFreeHost(c->host_e);
  for (auto& r : c->recs) {
    cudaEventDestroy(r.start);
    if (r.stop) cudaEventDestroy(r.stop);
  }
  for (auto e : c->free_events) cudaEventDestroy(e);
  delete c;
}

hsg::SweepArgs sweep_args(hsg_ctx* c, int colour, float beta, float step, int hits) {
  hsg::SweepArgs a{};
  const int o = 1 - colour;
  a.own = c->spins + colour * c->Nh;
  a.oth = c->spins + o * c->Nh;
  a.jx_own = c->J + (0 + colour) * c->Nh;
  a.jy_own = c->J + (2 + colour) * c->Nh;
  a.jz_own = c->J + (4 + colour) * c->Nh;
  a.jx_oth = c->J + (0 + o) * c->Nh;
  a.jy_oth = c->J + (2 + o) * c->Nh;
  a.jz_oth = c->J + (4 + o) * c->Nh;
  a.L = c->L;
  a.Lh = c->Lh;
  a.colour = colour;
  a.hits = hits;
  a.k0 = c->k0;
  a.k1 = c->k1;
  a.sweep_lo = (uint32_t)(c->sweep & 0xFFFFFFFFu);
  a.sweep_hi = (uint32_t)(c->sweep >> 32);
  a.beta = beta;
  a.step = step;
  a.sweep_ptr = c->d_ctr;  // the device counter equals c->sweep in stream order
  if (c->packed) {
    float* base = reinterpret_cast<float*>(c->spins);
    a.own = reinterpret_cast<float4*>(base + 3 * colour * c->Nh);
    a.oth = reinterpret_cast<const float4*>(base + 3 * o * c->Nh);
    a.packed = true;
    a.stride = (size_t)c->Nh;
  }
  return a;
}

hsg_status check_schedule(hsg_ctx* c, const hsg_schedule* s, bool need_kind) {
  if (!s) return fail(c, HSG_EINVAL, "schedule is NULL");
  if (need_kind && s->kind != HSG_NONE && s->kind != HSG_METROPOLIS && s->kind != HSG_HEATBATH &&
      s->kind != HSG_METROPOLIS_OR)
    return fail(c, HSG_EINVAL, "schedule.kind must be HSG_NONE, HSG_METROPOLIS, HSG_HEATBATH or HSG_METROPOLIS_OR");
  if (s->hits < 1 || s->hits > 65535) return fail(c, HSG_EINVAL, "schedule.hits must be in [1, 65535]");
  if (s->proposal != HSG_PROP_SPHERE && s->proposal != HSG_PROP_BALL)
    return fail(c, HSG_EINVAL, "schedule.proposal must be HSG_PROP_SPHERE or HSG_PROP_BALL");
  if (!(s->step > 0.0f) || !std::isfinite(s->step)) return fail(c, HSG_EINVAL, "schedule.step must be finite and > 0");
  if (s->n_or < 0) return fail(c, HSG_EINVAL, "schedule.n_or must be >= 0");
  if (!(s->T > 0.0)) return fail(c, HSG_EINVAL, "schedule.T must be > 0 (inf allowed)");
  if (s->renorm_every < 0 || s->energy_every < 0) return fail(c, HSG_EINVAL, "cadences must be >= 0");
  if (s->kernel != HSG_KERNEL_AUTO && s->kernel != HSG_KERNEL_GLOBAL && s->kernel != HSG_KERNEL_SLAB &&
      s->kernel != HSG_KERNEL_WAVE)
    return fail(c, HSG_EINVAL, "schedule.kernel must be HSG_KERNEL_AUTO, _GLOBAL, _SLAB or _WAVE");
  if (c->packed && (s->kernel == HSG_KERNEL_SLAB || s->kernel == HSG_KERNEL_WAVE))
    return fail(c, HSG_EINVAL, "the packed spin layout runs the global kernel only (HSG_KERNEL_AUTO or _GLOBAL)");
  return HSG_OK;
}

float beta_of(double T) { return std::isinf(T) ? 0.0f : (float)(1.0 / T); }

// HSG_KERNEL_AUTO: the temporally blocked over-relaxation once the spins
// and bonds (16 + 12 bytes per site) exceed three quarters of L2 -- it
// saves HBM traffic, and pays where the sweeps stream much of their state
// from HBM.  Measured on GB300 (126 MB L2), whole sweeps of 4-hit
// Metropolis + 1 OR sweep: L = 128 (59 MB) 73.6 against 66.4 us with the
// global kernel, L = 144 (84 MB) 123-127 against 121-125 us, L = 152 (98
// MB) 135-139 against 144-147 us, L = 160 157 against 167 us; at L = 256
// one OR sweep 131.7 us against 2 x 87.9 us.
int pick_variant(const hsg_ctx* c, int requested) {
  if (requested == HSG_KERNEL_GLOBAL || requested == HSG_KERNEL_SLAB || requested == HSG_KERNEL_WAVE) return requested;
  if (c->packed) return hsg::V_GLOBAL;
  return 4 * 28LL * c->N > 3 * c->l2_bytes ? hsg::V_WAVE : hsg::V_GLOBAL;
}

// Temporally blocked launches of one sweep under schedule s with the wave
// variant: one per over-relaxation sweep (the main update stays two
// half-sweeps).  Each one swaps the spin buffers.
int wave_sweeps_per_sweep(const hsg_schedule* s) { return s->n_or; }

hsg_status run_half_sweep(hsg_ctx* c, const hsg_schedule* s, int update, int colour) {
  int upd, kclass;
  if (update == HSG_OVERRELAX) {
    upd = hsg::U_OR;
    kclass = HSG_PROF_OVERRELAX;
  } else if (update == HSG_METROPOLIS) {
    upd = s->proposal == HSG_PROP_BALL ? hsg::U_MET_BALL : hsg::U_MET_SPHERE;
    kclass = HSG_PROF_METROPOLIS;
  } else if (update == HSG_METROPOLIS_OR) {
    upd = s->proposal == HSG_PROP_BALL ? hsg::U_MET_OR_BALL : hsg::U_MET_OR_SPHERE;
    kclass = HSG_PROF_METROPOLIS;
  } else {
    upd = hsg::U_HB;
    kclass = HSG_PROF_HEATBATH;
  }
  const hsg::SweepArgs a = sweep_args(c, colour, beta_of(s->T), s->step, s->hits);
  int variant = pick_variant(c, s->kernel);
  if (variant == hsg::V_WAVE) variant = hsg::V_GLOBAL;  // a single colour: the plain kernel
  return launch(c, kclass, 1, "half-sweep kernel", [&] { return hsg::launch_half_sweep(upd, variant, a, c->sm_count, c->stream); });
}

// Both colours of one over-relaxation sweep in one temporally blocked launch
// from c->spins into c->spins_alt (renormalising what it stores when
// `renorm`); then the two buffers swap.
hsg_status run_or_sweep_wave(hsg_ctx* c, bool renorm) {
  hsg::WaveArgs a{};
  a.src = c->spins;
  a.dst = c->spins_alt;
  a.J = c->J;
  a.L = c->L;
  a.Lh = c->Lh;
  a.renorm = renorm;
  a.bond_map = c->use_tma ? &c->bond_map : nullptr;
  a.err = c->d_ctr + 2;
  const int stall = g_test_stall_boxes.load();
  a.box_extra_tx = (stall & 1) ? 16u : 0u;
  a.c1_extra_arrivals = (stall & 2) ? 1u : 0u;
  hsg_status st = launch(c, renorm ? HSG_PROF_OVERRELAX_RENORM : HSG_PROF_OVERRELAX, 1, "over-relaxation sweep kernel",
                         [&] { return hsg::launch_or_sweep_wave(a, c->sm_count, c->stream); });
  if (st == HSG_OK) std::swap(c->spins, c->spins_alt);
  return st;
}

// The temporally blocked sweep's tensor-box bonds: at L >= 32, the first
// sweep allocates the halo-padded copy of J (when the device has room for
// it beside a margin of 1 GiB; else the sweep keeps its register loads) and
// encodes its tensor map; a copy older than J is rebuilt (one launch).
hsg_status prepare_bond_boxes(hsg_ctx* c) {
  if (c->L < hsg::kWaveTmaMinL || c->packed) return HSG_OK;
  if (!c->Jpad) {
    const size_t bytes = sizeof(float) * hsg::padded_bonds_elems(c->L);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || free_b < bytes + ((size_t)1 << 30)) {
      cudaGetLastError();
      return HSG_OK;  // no room: register loads
    }
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(&c->Jpad), bytes, c->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->Jpad = nullptr;
      return e == cudaErrorMemoryAllocation ? HSG_OK : cuda_fail(c, e, "padded couplings");
    }
    c->Jpad_ok = false;
    c->use_tma = hsg::encode_padded_bond_map(&c->bond_map, c->Jpad, c->L) == cudaSuccess;
  }
  if (c->use_tma && !c->Jpad_ok) {
    hsg_status st = launch(c, HSG_PROF_LAYOUT, 1, "coupling padding kernel",
                           [&] { return hsg::launch_pad_bonds(c->J, c->Jpad, c->L, c->stream); });
    if (st != HSG_OK) return st;
    c->Jpad_ok = true;
  }
  return HSG_OK;
}

// The bond-box wait flag of the temporally blocked sweeps: queue its copy
// into the second pinned word (after the work queued so far), and, once the
// stream has been synchronised, HSG_ETIMEOUT if one of them gave up.
cudaError_t queue_box_flag(hsg_ctx* c) {
  if (!c->use_tma) return cudaSuccess;
  return cudaMemcpyAsync(c->host_e + 1, c->d_ctr + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
}
hsg_status check_box_waits(hsg_ctx* c) {
  if (!c->use_tma) return HSG_OK;
  unsigned long long flag = 0;
  std::memcpy(&flag, c->host_e + 1, sizeof(flag));
  if (!flag) return HSG_OK;
  // Reported once: the flag is cleared for the sweeps that follow.
  cudaError_t e = cudaMemsetAsync(c->d_ctr + 2, 0, sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "wait flag reset");
  c->host_e[1] = 0.0;
  return fail(c, HSG_ETIMEOUT,
              "an over-relaxation sweep gave up waiting for its couplings (bounded wait): the spins since are not "
              "valid");
}

// E/N into *out_dev, or (logged) into the energy log at the device position.
hsg_status run_energy(hsg_ctx* c, double* out_dev, bool logged) {
  unsigned long long* idx = logged ? c->d_ctr + 1 : nullptr;
  return launch(c, HSG_PROF_ENERGY, 2, "energy kernels",
                [&] { return hsg::launch_energy(c->spins, c->packed, c->J, c->L, c->partials, out_dev, idx, c->stream); });
}

hsg_status run_advance(hsg_ctx* c) {
  return launch(c, HSG_PROF_LAYOUT, 1, "counter kernel", [&] { return hsg::launch_add_u64(c->d_ctr, 1, c->stream); });
}

hsg_status run_renorm(hsg_ctx* c) {
  return launch(c, HSG_PROF_RENORM, 1, "renorm kernel",
                [&] { return hsg::launch_renorm(c->spins, c->packed, c->N, c->sm_count, c->stream); });
}

// One sweep's launches in schedule order; the host mirrors of the sweep
// counter and the energy-log position advance as the device ones will.
hsg_status enqueue_one_sweep(hsg_ctx* c, const hsg_schedule* s) {
  hsg_status st;
  const bool wave = pick_variant(c, s->kernel) == hsg::V_WAVE;
  if (s->kind != HSG_NONE)
    for (int colour = 0; colour < 2; ++colour)
      if ((st = run_half_sweep(c, s, s->kind, colour)) != HSG_OK) return st;
  // A renormalisation due after this sweep is fused into its last wave
  // launch (the same renorm_spin on the same values; the counter kernel in
  // between touches no spin).
  const bool renorm_due = s->renorm_every > 0 && (c->sweep + 1) % (uint64_t)s->renorm_every == 0;
  const bool fuse_renorm = renorm_due && wave && s->n_or > 0;
  for (int o = 0; o < s->n_or; ++o) {
    if (wave) {
      if ((st = run_or_sweep_wave(c, fuse_renorm && o == s->n_or - 1)) != HSG_OK) return st;
      continue;
    }
    for (int colour = 0; colour < 2; ++colour)
      if ((st = run_half_sweep(c, s, HSG_OVERRELAX, colour)) != HSG_OK) return st;
  }
  if ((st = run_advance(c)) != HSG_OK) return st;
  c->sweep += 1;
  if (renorm_due && !fuse_renorm)
    if ((st = run_renorm(c)) != HSG_OK) return st;
  if (s->energy_every > 0 && c->sweep % (uint64_t)s->energy_every == 0) {
    if ((st = run_energy(c, c->elog, true)) != HSG_OK) return st;
    c->elog_n += 1;
  }
  return HSG_OK;
}

bool same_schedule(const hsg_schedule& a, const hsg_schedule& b) {
  return a.kind == b.kind && a.hits == b.hits && a.proposal == b.proposal && a.step == b.step && a.n_or == b.n_or &&
         a.T == b.T && a.renorm_every == b.renorm_every && a.energy_every == b.energy_every && a.kernel == b.kernel;
}

bool graph_matches(const hsg_ctx* c, const hsg_schedule* s, int variant, int period) {
  return c->gexec && same_schedule(c->gsched, *s) && c->gvariant == variant && c->gperiod == period &&
         c->gelog == c->elog && c->gspins == c->spins;
}

// Capture `period` sweeps starting at the current counter (a multiple of
// the period) into c->gexec.  Capturing runs nothing, so the host mirrors
// are restored afterwards.
hsg_status capture_period(hsg_ctx* c, const hsg_schedule* s, int variant, int period) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  const uint64_t sweep0 = c->sweep, launches0 = c->launches;
  const int elog0 = c->elog_n;
  float4* const spins0 = c->spins;
  float4* const alt0 = c->spins_alt;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(c, e, "sweep capture");
  hsg_status st = HSG_OK;
  for (int j = 0; j < period && st == HSG_OK; ++j) st = enqueue_one_sweep(c, s);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->stream, &g);
  c->glaunches = (int)(c->launches - launches0);
  c->launches = launches0;
  c->sweep = sweep0;
  c->elog_n = elog0;
  c->spins = spins0;
  c->spins_alt = alt0;
  if (st == HSG_OK && e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (st != HSG_OK) return st;
  if (e != cudaSuccess) {
    c->gexec = nullptr;
    return cuda_fail(c, e, "sweep graph");
  }
  c->gsched = *s;
  c->gvariant = variant;
  c->gperiod = period;
  c->gelog = c->elog;
  c->gspins = spins0;
  return HSG_OK;
}

hsg_status grow_elog(hsg_ctx* c, int need) {
  if (need <= c->elog_cap) return HSG_OK;
  int cap = c->elog_cap > 0 ? c->elog_cap : kElogInit;
  while (cap < need) cap *= 2;
  void* p = nullptr;
  cudaError_t e = dev_alloc(&p, sizeof(double) * (size_t)cap, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "energy log");
  if (c->elog_n > 0) {
    e = cudaMemcpyAsync(p, c->elog, sizeof(double) * (size_t)c->elog_n, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) {
      dev_free(p, c->stream);
      return cuda_fail(c, e, "energy log copy");
    }
  }
  dev_free(c->elog, c->stream);
  c->elog = static_cast<double*>(p);
  c->elog_cap = cap;
  return HSG_OK;
}

}  // namespace

void hsg::set_thread_error(const std::string& msg) { g_thread_error = msg; }

extern "C" {

hsg_status hsg_create(hsg_ctx** out, int L, uint64_t seed, uint32_t sample, uint32_t replica, void* cuda_stream) {
  return hsg_create_layout(out, L, seed, sample, replica, cuda_stream, HSG_LAYOUT_FLOAT4);
}

hsg_status hsg_create_layout(hsg_ctx** out, int L, uint64_t seed, uint32_t sample, uint32_t replica,
                             void* cuda_stream, int layout) {
  if (!out) return fail(nullptr, HSG_EINVAL, "out is NULL");
  *out = nullptr;
  if (L < 4 || L > kMaxL || (L & 1))
    return fail(nullptr, HSG_EINVAL, "L must be even and in [4, " + std::to_string(kMaxL) + "]");
  if (layout != HSG_LAYOUT_FLOAT4 && layout != HSG_LAYOUT_PACKED)
    return fail(nullptr, HSG_EINVAL, "layout must be HSG_LAYOUT_FLOAT4 or HSG_LAYOUT_PACKED");
  if (!hsg::key_stream_ok(sample, replica)) return fail(nullptr, HSG_EINVAL, hsg::kKeyStreamMsg);
  hsg_ctx* c = new (std::nothrow) hsg_ctx();
  if (!c) return fail(nullptr, HSG_ENOMEM, "host allocation failed");
  c->packed = layout == HSG_LAYOUT_PACKED;
  c->L = L;
  c->Lh = L / 2;
  c->N = (long long)L * L * L;
  c->Nh = c->N / 2;
  c->seed = seed;
  c->sample = sample;
  c->replica = replica;
  // Key of (seed, sample, replica): low seed word, high seed word XOR the
  // Weyl-scrambled stream number 2*sample + replica.
  c->k0 = (uint32_t)(seed & 0xFFFFFFFFu);
  c->k1 = (uint32_t)(seed >> 32) ^ ((2u * sample + replica) * 0x9E3779B9u);
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  int l2 = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device);
  c->l2_bytes = l2;
  if (e != cudaSuccess) {
    hsg_status st = cuda_fail(nullptr, e, "no usable CUDA device");
    delete c;
    return st;
  }
  struct {
    void** p;
    size_t bytes;
    const char* what;
  } allocs[] = {
      {reinterpret_cast<void**>(&c->spins), (c->packed ? 3 * sizeof(float) : sizeof(float4)) * (size_t)c->N, "spins"},
      {reinterpret_cast<void**>(&c->J), sizeof(float) * 3 * (size_t)c->N, "couplings"},
      {reinterpret_cast<void**>(&c->partials), sizeof(double) * hsg::energy_partials(L), "energy partials"},
      {reinterpret_cast<void**>(&c->e_out), sizeof(double), "energy result"},
      {reinterpret_cast<void**>(&c->d_ctr), 3 * sizeof(unsigned long long), "device counters"},
  };
  for (auto& a : allocs) {
    e = dev_alloc(a.p, a.bytes, c->stream);
    if (e != cudaSuccess) {
      hsg_status st = cuda_fail(nullptr, e, a.what);
      release(c);
      return st;
    }
  }
  hsg_status st = grow_elog(c, kElogInit);
  if (st != HSG_OK) {
    g_thread_error = c->err;
    release(c);
    return st;
  }
  e = cudaMallocHost(&c->host_e, 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_ctr, 0, 3 * sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) {
    if (!c->host_e) c->host_e = nullptr;
    st = cuda_fail(nullptr, e, "pinned host slot / counters");
    release(c);
    return st;
  }
  st = launch(c, HSG_PROF_INIT, 1, "init kernel",
              [&] { return hsg::launch_init_spins(c->spins, c->packed, L, c->k0, c->k1, c->stream); });
  if (st != HSG_OK) {
    g_thread_error = c->err;
    release(c);
    return st;
  }
  *out = c;
  return HSG_OK;
}

hsg_status hsg_destroy(hsg_ctx* ctx) {
  release(ctx);
  return HSG_OK;
}

hsg_status hsg_set_couplings(hsg_ctx* c, const void* J, int dtype, int where) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  if (!J) return fail(c, HSG_EINVAL, "J is NULL");
  if (dtype != HSG_F32 && dtype != HSG_F64) return fail(c, HSG_EINVAL, "dtype must be HSG_F32 or HSG_F64");
  if (where != HSG_HOST && where != HSG_DEVICE) return fail(c, HSG_EINVAL, "where must be HSG_HOST or HSG_DEVICE");
  const bool f64 = dtype == HSG_F64;
  const void* src = J;
  if (where == HSG_HOST) {
    const size_t bytes = (f64 ? sizeof(double) : sizeof(float)) * 3 * (size_t)c->N;
    hsg_status st = ensure_stage(c, bytes);
    if (st != HSG_OK) return st;
    cudaError_t e = cudaMemcpyAsync(c->stage, J, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "coupling upload");
    src = c->stage;
  }
  // With a padded copy in use (temporally blocked sweeps at L >= 32) the
  // same launch writes it too.
  float* const Jp = c->use_tma ? c->Jpad : nullptr;
  hsg_status st = launch(c, HSG_PROF_LAYOUT, 1, "coupling layout kernel",
                         [&] { return hsg::launch_scatter_couplings(src, f64, c->J, c->L, c->stream, Jp); });
  if (st != HSG_OK) return st;
  if (where == HSG_HOST) {
    // The caller may reuse its array as soon as we return.
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "coupling upload sync");
  }
  c->have_J = true;
  c->Jpad_ok = Jp != nullptr;
  return HSG_OK;
}

hsg_status hsg_generate_couplings(hsg_ctx* c) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  // Key of (seed, sample, replica 0): replicas of one sample share J.
  const uint32_t k1 = (uint32_t)(c->seed >> 32) ^ ((2u * c->sample) * 0x9E3779B9u);
  hsg_status st = launch(c, HSG_PROF_LAYOUT, 1, "coupling generator kernel",
                         [&] { return hsg::launch_gen_couplings(c->J, c->L, c->k0, k1, c->stream); });
  if (st == HSG_OK) {
    c->have_J = true;
    c->Jpad_ok = false;
  }
  return st;
}

hsg_status hsg_get_couplings(hsg_ctx* c, float* out, int where) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  if (!out) return fail(c, HSG_EINVAL, "out is NULL");
  if (where != HSG_HOST && where != HSG_DEVICE) return fail(c, HSG_EINVAL, "where must be HSG_HOST or HSG_DEVICE");
  if (!c->have_J) return fail(c, HSG_EINVAL, "couplings not set");
  const size_t bytes = sizeof(float) * 3 * (size_t)c->N;
  float* dst = out;
  if (where == HSG_HOST) {
    hsg_status st = ensure_stage(c, bytes);
    if (st != HSG_OK) return st;
    dst = static_cast<float*>(c->stage);
  }
  hsg_status st = launch(c, HSG_PROF_LAYOUT, 1, "coupling gather kernel",
                         [&] { return hsg::launch_gather_couplings(c->J, dst, c->L, c->stream); });
  if (st != HSG_OK) return st;
  if (where == HSG_HOST) {
    cudaError_t e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "coupling readback");
  }
  return HSG_OK;
}

hsg_status hsg_sweep(hsg_ctx* c, const hsg_schedule* s, int n_sweeps) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  hsg_status st = check_schedule(c, s, true);
  if (st != HSG_OK) return st;
  if (n_sweeps < 0) return fail(c, HSG_EINVAL, "n_sweeps must be >= 0");
  if (!c->have_J) return fail(c, HSG_EINVAL, "couplings not set: call hsg_set_couplings first");
  if (s->energy_every > 0) {
    const uint64_t end = c->sweep + (uint64_t)n_sweeps;
    const uint64_t logged = end / (uint64_t)s->energy_every - c->sweep / (uint64_t)s->energy_every;
    st = grow_elog(c, c->elog_n + (int)logged);
    if (st != HSG_OK) return st;
  }
  const int variant = pick_variant(c, s->kernel);
  const int swaps = variant == hsg::V_WAVE ? wave_sweeps_per_sweep(s) : 0;
  if (swaps > 0 && !c->spins_alt) {
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(&c->spins_alt), sizeof(float4) * (size_t)c->N, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "second spin buffer");
  }
  if (swaps > 0 && (st = prepare_bond_boxes(c)) != HSG_OK) return st;
  SweepGroup group_guard(c);
  // Sweeps run in periods of P = lcm(renorm_every, energy_every) sweeps
  // (1 without cadences).  On a non-default stream and without the
  // profiler, a period that starts at a multiple of P is captured once as a
  // CUDA graph (the kernels read the sweep counter and the energy-log
  // position from device memory) and replayed; other sweeps are launched
  // directly.  Both paths issue the same kernels in the same order.  A
  // captured period leaves the spins in the buffer it found them in (an even
  // number of buffer swaps), so that the graph can be replayed.
  long long period = 1;
  if (s->renorm_every > 0) period = std::lcm(period, (long long)s->renorm_every);
  if (s->energy_every > 0) period = std::lcm(period, (long long)s->energy_every);
  if ((period * swaps) % 2 == 1) period *= 2;
  const bool graphs = c->stream != nullptr && !c->prof && period <= kMaxGraphPeriod;
  int k = 0;
  while (k < n_sweeps) {
    if (graphs && c->sweep % (uint64_t)period == 0 && n_sweeps - k >= period) {
      if (!graph_matches(c, s, variant, (int)period) && (st = capture_period(c, s, variant, (int)period)) != HSG_OK)
        return st;
      cudaError_t e = cudaGraphLaunch(c->gexec, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "sweep graph launch");
      c->launches += (uint64_t)c->glaunches;
      c->sweep += (uint64_t)period;
      if (s->energy_every > 0) c->elog_n += (int)(period / s->energy_every);
      k += (int)period;
    } else {
      if ((st = enqueue_one_sweep(c, s)) != HSG_OK) return st;
      k += 1;
    }
  }
  return HSG_OK;
}

hsg_status hsg_energy(hsg_ctx* c, double* e_per_spin) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  if (!e_per_spin) return fail(c, HSG_EINVAL, "e_per_spin is NULL");
  if (!c->have_J) return fail(c, HSG_EINVAL, "couplings not set");
  hsg_status st = run_energy(c, c->e_out, false);
  if (st != HSG_OK) return st;
  cudaError_t e = cudaMemcpyAsync(c->host_e, c->e_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = queue_box_flag(c);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "energy readback");
  *e_per_spin = *c->host_e;
  return check_box_waits(c);
}

hsg_status hsg_get_energy_log(hsg_ctx* c, double* out, int max_n, int* n) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  if (max_n < 0 || (max_n > 0 && !out)) return fail(c, HSG_EINVAL, "bad output buffer");
  const int k = max_n < c->elog_n ? max_n : c->elog_n;
  cudaError_t e = cudaSuccess;
  if (k > 0) e = cudaMemcpyAsync(out, c->elog, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "energy log readback");
  if (n) *n = c->elog_n;
  return HSG_OK;
}

hsg_status hsg_clear_energy_log(hsg_ctx* c) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  hsg_status st = launch(c, HSG_PROF_LAYOUT, 1, "counter kernel",
                         [&] { return hsg::launch_set_u64(c->d_ctr + 1, 0, c->stream); });
  if (st != HSG_OK) return st;
  c->elog_n = 0;
  return HSG_OK;
}

hsg_status hsg_get_spins(hsg_ctx* c, float* out, int where) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  if (!out) return fail(c, HSG_EINVAL, "out is NULL");
  if (where != HSG_HOST && where != HSG_DEVICE) return fail(c, HSG_EINVAL, "where must be HSG_HOST or HSG_DEVICE");
  const size_t bytes = sizeof(float) * 3 * (size_t)c->N;
  float* dst = out;
  if (where == HSG_HOST) {
    hsg_status st = ensure_stage(c, bytes);
    if (st != HSG_OK) return st;
    dst = static_cast<float*>(c->stage);
  }
  hsg_status st = launch(c, HSG_PROF_LAYOUT, 1, "spin gather kernel",
                         [&] { return hsg::launch_gather_spins(c->spins, c->packed, dst, c->L, c->stream); });
  if (st != HSG_OK) return st;
  if (where == HSG_HOST) {
    cudaError_t e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "spin readback");
  }
  return HSG_OK;
}

hsg_status hsg_set_spins(hsg_ctx* c, const float* in, int where) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  if (!in) return fail(c, HSG_EINVAL, "in is NULL");
  if (where != HSG_HOST && where != HSG_DEVICE) return fail(c, HSG_EINVAL, "where must be HSG_HOST or HSG_DEVICE");
  const float* src = in;
  if (where == HSG_HOST) {
    const size_t bytes = sizeof(float) * 3 * (size_t)c->N;
    hsg_status st = ensure_stage(c, bytes);
    if (st != HSG_OK) return st;
    cudaError_t e = cudaMemcpyAsync(c->stage, in, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "spin upload");
    src = static_cast<const float*>(c->stage);
  }
  hsg_status st = launch(c, HSG_PROF_LAYOUT, 1, "spin scatter kernel",
                         [&] { return hsg::launch_scatter_spins(src, c->spins, c->packed, c->L, c->stream); });
  if (st != HSG_OK) return st;
  if (where == HSG_HOST) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "spin upload sync");
  }
  return HSG_OK;
}

hsg_status hsg_get_sites(hsg_ctx* c, const uint32_t* sites, int n, float* spins, float* bonds) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  if (n < 0) return fail(c, HSG_EINVAL, "n must be >= 0");
  if (n == 0) return HSG_OK;
  if (!sites || !spins) return fail(c, HSG_EINVAL, "sites and spins must not be NULL");
  if (bonds && !c->have_J) return fail(c, HSG_EINVAL, "couplings not set");
  for (int k = 0; k < n; ++k)
    if ((long long)sites[k] >= c->N) return fail(c, HSG_EINVAL, "site index out of range");
  const size_t nb = (size_t)n;
  hsg_status st = ensure_stage(c, nb * (4 + 12 + 12));
  if (st != HSG_OK) return st;
  uint32_t* d_sites = static_cast<uint32_t*>(c->stage);
  float* d_spins = reinterpret_cast<float*>(d_sites + nb);
  float* d_bonds = d_spins + 3 * nb;
  cudaError_t e = cudaMemcpyAsync(d_sites, sites, 4 * nb, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "site list upload");
  st = launch(c, HSG_PROF_LAYOUT, 1, "site gather kernel",
              [&] {
                return hsg::launch_gather_sites(c->spins, c->packed, c->J, c->L, d_sites, n, d_spins, d_bonds,
                                                c->stream);
              });
  if (st != HSG_OK) return st;
  e = cudaMemcpyAsync(spins, d_spins, 12 * nb, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && bonds) e = cudaMemcpyAsync(bonds, d_bonds, 12 * nb, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "site readback");
  return HSG_OK;
}

hsg_status hsg_get_sweep(hsg_ctx* c, uint64_t* sweep) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  if (!sweep) return fail(c, HSG_EINVAL, "sweep is NULL");
  *sweep = c->sweep;
  return HSG_OK;
}

hsg_status hsg_set_sweep(hsg_ctx* c, uint64_t sweep) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  hsg_status st = launch(c, HSG_PROF_LAYOUT, 1, "counter kernel",
                         [&] { return hsg::launch_set_u64(c->d_ctr, sweep, c->stream); });
  if (st != HSG_OK) return st;
  c->sweep = sweep;
  return HSG_OK;
}

hsg_status hsg_half_sweep(hsg_ctx* c, const hsg_schedule* s, int update, int colour) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  hsg_status st = check_schedule(c, s, false);
  if (st != HSG_OK) return st;
  if (update != HSG_OVERRELAX && update != HSG_METROPOLIS && update != HSG_HEATBATH && update != HSG_METROPOLIS_OR)
    return fail(c, HSG_EINVAL, "update must be HSG_OVERRELAX, HSG_METROPOLIS, HSG_HEATBATH or HSG_METROPOLIS_OR");
  if (colour != 0 && colour != 1) return fail(c, HSG_EINVAL, "colour must be 0 or 1");
  if (!c->have_J) return fail(c, HSG_EINVAL, "couplings not set");
  return run_half_sweep(c, s, update, colour);
}

hsg_status hsg_renorm(hsg_ctx* c) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  return run_renorm(c);
}

hsg_status hsg_kernel_for(hsg_ctx* c, const hsg_schedule* s, int* kernel) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  if (!kernel) return fail(c, HSG_EINVAL, "kernel is NULL");
  hsg_status st = check_schedule(c, s, true);
  if (st != HSG_OK) return st;
  *kernel = pick_variant(c, s->kernel);
  return HSG_OK;
}

hsg_status hsg_profile(hsg_ctx* c, int on) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  if (!on) close_run(c);
  c->prof = on != 0;
  return HSG_OK;
}

hsg_status hsg_profile_read(hsg_ctx* c, int kclass, double* total_ms, uint64_t* launches) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  if (kclass < 0 || kclass >= HSG_PROF_COUNT) return fail(c, HSG_EINVAL, "bad kernel class");
  close_run(c);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "profile sync");
  double ms = 0.0;
  uint64_t n = 0;
  for (const auto& r : c->recs) {
    if (r.kclass != kclass || !r.stop) continue;
    float t = 0.0f;
    e = cudaEventElapsedTime(&t, r.start, r.stop);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventElapsedTime");
    ms += t;
    n += r.count;
  }
  if (total_ms) *total_ms = ms;
  if (launches) *launches = n;
  return HSG_OK;
}

hsg_status hsg_profile_reset(hsg_ctx* c) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "profile sync");
  close_run(c);
  for (auto& r : c->recs) {
    c->free_events.push_back(r.start);
    if (r.stop) c->free_events.push_back(r.stop);
  }
  c->recs.clear();
  return HSG_OK;
}

hsg_status hsg_launch_count(hsg_ctx* c, uint64_t* launches) {
  if (!c) return fail(nullptr, HSG_EINVAL, "ctx is NULL");
  const hsg::DeviceGuard device_guard(c->device);
  if (device_guard.status() != cudaSuccess) return cuda_fail(c, device_guard.status(), "cudaSetDevice");
  if (!launches) return fail(c, HSG_EINVAL, "launches is NULL");
  *launches = c->launches;
  return HSG_OK;
}

const char* hsg_last_error(const hsg_ctx* c) { return c ? c->err.c_str() : g_thread_error.c_str(); }

const char* hsg_status_string(hsg_status s) {
  switch (s) {
    case HSG_OK: return "HSG_OK";
    case HSG_EINVAL: return "HSG_EINVAL";
    case HSG_ENOMEM: return "HSG_ENOMEM";
    case HSG_ECUDA: return "HSG_ECUDA";
    case HSG_ETIMEOUT: return "HSG_ETIMEOUT";
    case HSG_EBUSY: return "HSG_EBUSY";
    default: return "HSG_UNKNOWN";
  }
}

int hsg_version(void) { return kVersion; }

hsg_status hsg_philox(uint64_t seed, uint32_t sample, uint32_t replica, uint32_t c1, uint32_t c2, uint32_t c3,
                      uint32_t n, uint32_t* out, void* cuda_stream) {
  if (!out) return fail(nullptr, HSG_EINVAL, "out is NULL");
  if (reinterpret_cast<uintptr_t>(out) % 16 != 0) return fail(nullptr, HSG_EINVAL, "out must be 16-byte aligned");
  if (!hsg::key_stream_ok(sample, replica)) return fail(nullptr, HSG_EINVAL, hsg::kKeyStreamMsg);
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu);
  const uint32_t k1 = (uint32_t)(seed >> 32) ^ ((2u * sample + replica) * 0x9E3779B9u);
  cudaError_t e = hsg::launch_philox(k0, k1, c1, c2, c3, n, out, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "philox kernel");
  return HSG_OK;
}

hsg_status hsg_test_stall_tensor_loads(int on) {
  if (on < 0 || on > 3) return fail(nullptr, HSG_EINVAL, "on must be 0 .. 3");
  g_test_stall_boxes.store(on);
  return HSG_OK;
}

hsg_status hsg_test_fail_alloc(int k) {
  if (k < 0) return fail(nullptr, HSG_EINVAL, "k must be >= 0");
  g_fail_alloc_countdown = k;
  return HSG_OK;
}

}  // extern "C"
