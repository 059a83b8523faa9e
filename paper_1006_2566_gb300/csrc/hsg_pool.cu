// hsg_pool.cu -- many independent lattices in one device arena, swept
// together: the batched engine behind hsg_pool_* (include/hsg.h).
//
// Each admitted lattice ("slot") has its own side L, Philox key, temperature
// and sweep counter, and its spins and couplings in the colour-split layout
// of hsg_device.cuh, placed at offsets of one arena allocation.  A work list
// of tiles (slot, first site index q0) covers the sites of one colour of
// every active slot; every half-sweep kernel is persistent (a fixed grid of
// a few CTAs per SM strides over the tiles) and reads the tile count from
// device memory.  So a sweep's launches can be captured once in a CUDA graph
// and replayed while lattices are admitted and retired: only the work list
// and the slot table change, in device memory, between replays.
//
// Every site is updated by half_sweep_site, the same device function as the
// single-lattice kernel, with the same key and counters: a lattice swept in
// a pool is bit-identical to the same lattice swept alone.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "hsg.h"
#include "hsg_device.cuh"
#include "hsg_internal.h"

namespace {

// One slot as the kernels see it (96 bytes).
struct PoolDesc {
  uint32_t L, Lh, nh, plane;          // side, side/2, sites per colour, per colour-plane
  uint32_t k0, k1;                    // Philox key of (seed, sample, replica)
  uint32_t sweep_lo, sweep_hi;        // the lattice's own sweep counter
  float beta;                         // 1/T (0 for T = inf)
  uint32_t active;                    // 1 while admitted
  uint32_t tile_begin, tile_count;    // the slot's tiles in the work list
  unsigned long long spin_off;        // float4 offset of colour 0 (colour 1 at + nh)
  unsigned long long j_off;           // float offset of J[0][0] (J[d][c] at + (2d + c) nh)
  hsg::FastDiv by_plane, by_lh;       // division of a site index by plane and by Lh
  uint32_t pad[2];
};
static_assert(sizeof(PoolDesc) == 96, "PoolDesc layout");


// Site index q -> (xh, y, z) of a slot.
__device__ __forceinline__ void decode_site(const PoolDesc* d, uint32_t q, uint32_t& xh, uint32_t& y, uint32_t& z) {
  z = hsg::fast_div(q, d->by_plane);
  const uint32_t r = q - z * d->plane;
  y = hsg::fast_div(r, d->by_lh);
  xh = r - y * d->Lh;
}

constexpr size_t kAlign = 256;

inline unsigned cdiv_u(unsigned long long a, unsigned long long b) { return (unsigned)((a + b - 1) / b); }

// At most 64 registers (four CTAs of 256 threads per SM): the over-relaxation
// pass is memory-bound and needs the resident warps for loads in flight
// (measured on GB300, 39 M sites: 350 us per half-sweep at 120 registers and
// two sites per thread, 243 us at 56 registers and one), and the Metropolis
// pass runs fastest at the 64 registers its code wants.
template <int U>
__global__ void __launch_bounds__(256, 4) k_pool_half_sweep(const PoolDesc* __restrict__ desc,
                                                         const uint2* __restrict__ tiles,
                                                         const uint32_t* __restrict__ n_tiles, float4* __restrict__ S,
                                                         const float* __restrict__ J, uint32_t colour, float step,
                                                         int hits, int hit0, uint32_t tile_sites) {
  const uint32_t nt = *n_tiles;
  for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const uint2 tl = tiles[t];
    const PoolDesc* d = desc + tl.x;
    const uint32_t L = d->L, Lh = d->Lh, nh = d->nh;
    float4* base = S + d->spin_off;
    float4* own = base + (colour ? nh : 0);
    const float4* oth = base + (colour ? 0 : nh);
    const float* j = J + d->j_off;
    const uint32_t o = 1u - colour;
    const float *jxo = j + (0 + colour) * (size_t)nh, *jyo = j + (2 + colour) * (size_t)nh,
                *jzo = j + (4 + colour) * (size_t)nh, *jxt = j + (0 + o) * (size_t)nh,
                *jyt = j + (2 + o) * (size_t)nh, *jzt = j + (4 + o) * (size_t)nh;
    for (uint32_t k = threadIdx.x; k < tile_sites; k += blockDim.x) {
      const uint32_t q = tl.y + k;
      if (q >= nh) break;
      uint32_t xh, y, z;
      decode_site(d, q, xh, y, z);
      hsg::half_sweep_site<U>(own, oth, jxo, jyo, jzo, jxt, jyt, jzt, xh, y, z, L, Lh, colour, d->sweep_lo,
                              d->sweep_hi, d->k0, d->k1, d->beta, step, hits, hit0);
    }
  }
}

// Counter advance of every active slot, after the last half-sweep of a sweep.
__global__ void k_pool_advance(PoolDesc* __restrict__ desc, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (!desc[i].active) continue;
    const uint32_t lo = desc[i].sweep_lo + 1u;
    desc[i].sweep_lo = lo;
    if (lo == 0u) desc[i].sweep_hi += 1u;
  }
}

// Renormalisation of the slots whose counter is a multiple of `every`
// (the single-lattice rule: after the advance, when sweep % every == 0).
__global__ void __launch_bounds__(256) k_pool_renorm(const PoolDesc* __restrict__ desc, const uint2* __restrict__ tiles,
                                                     const uint32_t* __restrict__ n_tiles, float4* __restrict__ S,
                                                     uint32_t every, uint32_t tile_sites) {
  const uint32_t nt = *n_tiles;
  for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const uint2 tl = tiles[t];
    const PoolDesc* d = desc + tl.x;
    const unsigned long long sweep = ((unsigned long long)d->sweep_hi << 32) | d->sweep_lo;
    if (sweep % every != 0) continue;
    const uint32_t nh = d->nh;
    float4* s0 = S + d->spin_off;
    for (uint32_t k = threadIdx.x; k < tile_sites; k += blockDim.x) {
      const uint32_t q = tl.y + k;
      if (q >= nh) break;
      s0[q] = hsg::renorm_spin(s0[q]);
      s0[nh + q] = hsg::renorm_spin(s0[nh + q]);
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double part[NT / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  double w = 0.0;
  if (threadIdx.x < 32) {
    w = threadIdx.x < NT / 32 ? part[threadIdx.x] : 0.0;
    w = warp_sum(w);
  }
  __syncthreads();
  return w;  // valid in thread 0
}

// Energy, first pass: per tile of colour-0 sites, sum of s . h (fp32 per
// site, fp64 sums), written to partials[tile].
__global__ void __launch_bounds__(256) k_pool_energy_partial(const PoolDesc* __restrict__ desc,
                                                             const uint2* __restrict__ tiles,
                                                             const uint32_t* __restrict__ n_tiles,
                                                             const float4* __restrict__ S, const float* __restrict__ J,
                                                             uint32_t tile_sites, const uint8_t* __restrict__ sel,
                                                             double* __restrict__ partials) {
  const uint32_t nt = *n_tiles;
  for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const uint2 tl = tiles[t];
    if (sel && !sel[tl.x]) continue;  // slot not asked for
    const PoolDesc* d = desc + tl.x;
    const uint32_t L = d->L, Lh = d->Lh, nh = d->nh, plane = d->plane;
    const float4* s0 = S + d->spin_off;
    const float4* s1 = s0 + nh;
    const float* j = J + d->j_off;
    double acc = 0.0;
    for (uint32_t k = threadIdx.x; k < tile_sites; k += blockDim.x) {
      const uint32_t q = tl.y + k;
      if (q >= nh) break;
      uint32_t xh, y, z;
      decode_site(d, q, xh, y, z);
      const uint32_t p = (y + z) & 1u;
      const uint32_t row = (z * L + y) * Lh;
      const uint32_t q_xp = p ? (xh + 1 == Lh ? row : q + 1) : q;
      const uint32_t q_xm = p ? q : (xh == 0 ? row + Lh - 1 : q - 1);
      const uint32_t q_yp = y + 1 == L ? q - (L - 1) * Lh : q + Lh;
      const uint32_t q_ym = y == 0 ? q + (L - 1) * Lh : q - Lh;
      const uint32_t q_zp = z + 1 == L ? q - (L - 1) * plane : q + plane;
      const uint32_t q_zm = z == 0 ? q + (L - 1) * plane : q - plane;
      const float3 h = hsg::local_field(s1[q_xp], s1[q_xm], s1[q_yp], s1[q_ym], s1[q_zp], s1[q_zm], j[q],
                                        j[(size_t)nh + q_xm], j[2 * (size_t)nh + q], j[3 * (size_t)nh + q_ym],
                                        j[4 * (size_t)nh + q], j[5 * (size_t)nh + q_zm]);
      const float4 s = s0[q];
      acc += (double)hsg::dot3(make_float3(s.x, s.y, s.z), h);
    }
    const double v = block_sum<256>(acc);
    if (threadIdx.x == 0) partials[t] = v;
  }
}

// Energy, second pass: block per slot adds its tiles' partials in order;
// E/N = -(sum)/N, NaN for inactive slots.
__global__ void __launch_bounds__(256) k_pool_energy_final(const PoolDesc* __restrict__ desc, int n_slots,
                                                           const uint8_t* __restrict__ sel,
                                                           const double* __restrict__ partials,
                                                           double* __restrict__ out) {
  for (int s = blockIdx.x; s < n_slots; s += gridDim.x) {
    const PoolDesc* d = desc + s;
    if (!d->active || (sel && !sel[s])) {
      if (threadIdx.x == 0) out[s] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    double v = 0.0;
    for (uint32_t k = threadIdx.x; k < d->tile_count; k += blockDim.x) v += partials[d->tile_begin + k];
    v = block_sum<256>(v);
    if (threadIdx.x == 0) out[s] = -v / (2.0 * (double)d->nh);
  }
}

struct Slot {
  bool active = false;
  int L = 0;
  uint64_t seed = 0;
  uint32_t sample = 0, replica = 0;
  double T = 0.0;
  uint64_t off = 0, bytes = 0;  // arena block
  uint64_t sweep = 0;
};

}  // namespace

struct hsg_pool {
  cudaStream_t stream = nullptr;
  int device = 0, sm_count = 0;
  char* arena = nullptr;
  uint64_t budget = 0, used = 0;
  std::map<uint64_t, uint64_t> free_blocks;  // offset -> size
  int max_slots = 0, n_active = 0;
  std::vector<Slot> slots;
  // Device tables and two pinned host mirrors of each: a rebuild writes
  // the mirror whose last upload has completed (its event), so the host
  // never waits for the sweeps in flight.
  PoolDesc* d_desc = nullptr;
  PoolDesc* h_desc = nullptr;  // pinned, 2 x max_slots
  uint2* d_tiles = nullptr;
  uint2* h_tiles = nullptr;  // pinned, 2 x tiles_cap
  size_t tiles_cap = 0;
  uint32_t* d_ntiles = nullptr;
  uint32_t* h_ntiles = nullptr;  // pinned, 2
  cudaEvent_t up_ev[2] = {nullptr, nullptr};
  bool up_rec[2] = {false, false};
  int up_buf = 0;
  double* d_partials = nullptr;
  double* d_energy = nullptr;
  // Energies read back into pinned buffer b (b = 0, 1 for
  // hsg_pool_energies_async, 2 for hsg_pool_energies), each followed by
  // an event that its reader waits for.
  static constexpr int kEnergyBufs = 3;
  double* h_energy = nullptr;  // pinned, kEnergyBufs x max_slots
  // Slots asked for by hsg_pool_energies_slots_async: a mask per buffer
  // (pinned, kEnergyBufs x max_slots, free again once the buffer's event
  // has passed) and the device copy the kernels read.
  uint8_t* h_sel = nullptr;
  uint8_t* d_sel = nullptr;
  cudaEvent_t en_ev[kEnergyBufs] = {nullptr, nullptr, nullptr};
  bool en_pending[kEnergyBufs] = {false, false, false};
  void* stage = nullptr;
  size_t stage_bytes = 0;
  bool dirty = true;
  int threads = 256, tile_sites = 512, blocks_per_sm = 8;
  // Metropolis hits per pass over a colour (0: all of them in one pass).
  int hits_per_pass = 0;
  struct GraphKey {
    int kind, hits, proposal, n_or, renorm_every, threads, tile_sites, bps, hits_per_pass;
    float step;
    bool operator==(const GraphKey& o) const { return memcmp(this, &o, sizeof(GraphKey)) == 0; }
  };
  bool have_graph = false;
  GraphKey gkey{};
  cudaGraphExec_t gexec = nullptr;
  uint64_t launches = 0;
  std::string err;
};

namespace {

hsg_status pfail(hsg_pool* p, hsg_status st, const std::string& m) {
  if (p)
    p->err = m;
  else
    hsg::set_thread_error(m);
  return st;
}

hsg_status pcuda(hsg_pool* p, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return pfail(p, e == cudaErrorMemoryAllocation ? HSG_ENOMEM : HSG_ECUDA, m);
}

void drop_graph(hsg_pool* p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  p->gexec = nullptr;
  p->have_graph = false;
}

// First-fit allocation of `bytes` (multiple of kAlign) in the arena.
bool arena_alloc(hsg_pool* p, uint64_t bytes, uint64_t* off) {
  for (auto it = p->free_blocks.begin(); it != p->free_blocks.end(); ++it) {
    if (it->second < bytes) continue;
    *off = it->first;
    const uint64_t rest = it->second - bytes;
    const uint64_t rest_off = it->first + bytes;
    p->free_blocks.erase(it);
    if (rest) p->free_blocks[rest_off] = rest;
    p->used += bytes;
    return true;
  }
  return false;
}

void arena_free(hsg_pool* p, uint64_t off, uint64_t bytes) {
  p->used -= bytes;
  auto it = p->free_blocks.emplace(off, bytes).first;
  auto next = std::next(it);
  if (next != p->free_blocks.end() && it->first + it->second == next->first) {
    it->second += next->second;
    p->free_blocks.erase(next);
  }
  if (it != p->free_blocks.begin()) {
    auto prev = std::prev(it);
    if (prev->first + prev->second == it->first) {
      prev->second += it->second;
      p->free_blocks.erase(it);
    }
  }
}

hsg_status ensure_pool_stage(hsg_pool* p, size_t bytes) {
  if (p->stage_bytes >= bytes) return HSG_OK;
  if (p->stage) cudaFreeAsync(p->stage, p->stream);
  p->stage = nullptr;
  p->stage_bytes = 0;
  cudaError_t e = cudaMallocAsync(&p->stage, bytes, p->stream);
  if (e != cudaSuccess) return pcuda(p, e, "pool staging buffer");
  p->stage_bytes = bytes;
  return HSG_OK;
}

// Host: rebuild the slot table and the work list; device: upload both.
hsg_status sync_tables(hsg_pool* p) {
  if (!p->dirty) return HSG_OK;
  const int b = p->up_buf;
  cudaError_t e = cudaSuccess;
  // this mirror may still be the source of the upload before last
  if (p->up_rec[b] && (e = cudaEventSynchronize(p->up_ev[b])) != cudaSuccess) return pcuda(p, e, "pool sync");
  size_t need = 0;
  for (const Slot& s : p->slots)
    if (s.active) need += cdiv_u((unsigned long long)s.L * s.L * s.L / 2, (unsigned long long)p->tile_sites);
  if (need > p->tiles_cap) {
    size_t cap = std::max<size_t>(1024, p->tiles_cap);
    while (cap < need) cap *= 2;
    drop_graph(p);  // the graph holds the old buffer addresses
    if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return pcuda(p, e, "pool sync");
    if (p->d_tiles) cudaFree(p->d_tiles);
    if (p->h_tiles) cudaFreeHost(p->h_tiles);
    if (p->d_partials) cudaFree(p->d_partials);
    p->d_tiles = nullptr;
    p->h_tiles = nullptr;
    p->d_partials = nullptr;
    p->tiles_cap = 0;
    if ((e = cudaMalloc(&p->d_tiles, cap * sizeof(uint2))) != cudaSuccess ||
        (e = cudaMallocHost(&p->h_tiles, 2 * cap * sizeof(uint2))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_partials, cap * sizeof(double))) != cudaSuccess)
      return pcuda(p, e, "pool work list");
    p->tiles_cap = cap;
  }
  PoolDesc* h_desc = p->h_desc + (size_t)b * p->max_slots;
  uint2* h_tiles = p->h_tiles + (size_t)b * p->tiles_cap;
  uint32_t* h_ntiles = p->h_ntiles + b;
  uint32_t nt = 0;
  for (int i = 0; i < p->max_slots; ++i) {
    const Slot& s = p->slots[i];
    PoolDesc& d = h_desc[i];
    memset(&d, 0, sizeof(d));
    if (!s.active) continue;
    const uint64_t n = (uint64_t)s.L * s.L * s.L;
    d.L = (uint32_t)s.L;
    d.Lh = (uint32_t)s.L / 2;
    d.nh = (uint32_t)(n / 2);
    d.plane = d.L * d.Lh;
    d.k0 = (uint32_t)(s.seed & 0xFFFFFFFFu);
    d.k1 = (uint32_t)(s.seed >> 32) ^ ((2u * s.sample + s.replica) * 0x9E3779B9u);
    d.sweep_lo = (uint32_t)(s.sweep & 0xFFFFFFFFu);
    d.sweep_hi = (uint32_t)(s.sweep >> 32);
    d.beta = std::isinf(s.T) ? 0.0f : (float)(1.0 / s.T);
    d.active = 1;
    d.spin_off = s.off / sizeof(float4);
    d.j_off = (s.off + sizeof(float4) * n) / sizeof(float);
    d.by_plane = hsg::make_fastdiv(d.plane);
    d.by_lh = hsg::make_fastdiv(d.Lh);
    d.tile_begin = nt;
    for (uint32_t q0 = 0; q0 < d.nh; q0 += (uint32_t)p->tile_sites) h_tiles[nt++] = make_uint2((uint32_t)i, q0);
    d.tile_count = nt - d.tile_begin;
  }
  *h_ntiles = nt;
  if ((e = cudaMemcpyAsync(p->d_desc, h_desc, sizeof(PoolDesc) * p->max_slots, cudaMemcpyHostToDevice,
                           p->stream)) != cudaSuccess ||
      (nt && (e = cudaMemcpyAsync(p->d_tiles, h_tiles, sizeof(uint2) * nt, cudaMemcpyHostToDevice, p->stream)) !=
                 cudaSuccess) ||
      (e = cudaMemcpyAsync(p->d_ntiles, h_ntiles, sizeof(uint32_t), cudaMemcpyHostToDevice, p->stream)) !=
          cudaSuccess ||
      (e = cudaEventRecord(p->up_ev[b], p->stream)) != cudaSuccess)
    return pcuda(p, e, "pool table upload");
  p->up_rec[b] = true;
  p->up_buf = 1 - b;
  p->dirty = false;
  return HSG_OK;
}

unsigned pool_grid(const hsg_pool* p) { return (unsigned)(p->sm_count * p->blocks_per_sm); }

cudaError_t launch_pool_half(hsg_pool* p, int upd, uint32_t colour, float step, int hits, int hit0) {
  const dim3 g(pool_grid(p)), b(p->threads);
  const float4* S4 = reinterpret_cast<const float4*>(p->arena);
  float4* S = const_cast<float4*>(S4);
  const float* J = reinterpret_cast<const float*>(p->arena);
  const uint32_t ts = (uint32_t)p->tile_sites;
  const PoolDesc* D = p->d_desc;
  const uint2* T = p->d_tiles;
  const uint32_t* NT = p->d_ntiles;
  cudaStream_t st = p->stream;
  switch (upd) {
    case hsg::U_OR: k_pool_half_sweep<hsg::U_OR><<<g, b, 0, st>>>(D, T, NT, S, J, colour, step, hits, hit0, ts); break;
    case hsg::U_MET_SPHERE:
      k_pool_half_sweep<hsg::U_MET_SPHERE><<<g, b, 0, st>>>(D, T, NT, S, J, colour, step, hits, hit0, ts);
      break;
    case hsg::U_MET_BALL:
      k_pool_half_sweep<hsg::U_MET_BALL><<<g, b, 0, st>>>(D, T, NT, S, J, colour, step, hits, hit0, ts);
      break;
    case hsg::U_MET_OR_SPHERE:
      k_pool_half_sweep<hsg::U_MET_OR_SPHERE><<<g, b, 0, st>>>(D, T, NT, S, J, colour, step, hits, hit0, ts);
      break;
    case hsg::U_MET_OR_BALL:
      k_pool_half_sweep<hsg::U_MET_OR_BALL><<<g, b, 0, st>>>(D, T, NT, S, J, colour, step, hits, hit0, ts);
      break;
    default: k_pool_half_sweep<hsg::U_HB><<<g, b, 0, st>>>(D, T, NT, S, J, colour, step, hits, hit0, ts); break;
  }
  p->launches += 1;
  return cudaGetLastError();
}

// Passes over each colour for the schedule's main update: the Metropolis
// hits split into groups of hits_per_pass (the field is fixed for the
// whole half-sweep and hit j is keyed by j, so any split gives the same
// result); one pass otherwise.
int main_passes(const hsg_pool* p, const hsg_schedule* s) {
  if (s->kind == HSG_NONE) return 0;
  if (s->kind == HSG_HEATBATH || p->hits_per_pass <= 0 || p->hits_per_pass >= s->hits) return 1;
  return (s->hits + p->hits_per_pass - 1) / p->hits_per_pass;
}

// The launches of one sweep, in the single-lattice order: main update on
// colour 0 then 1, n_or OR sweeps, counter advance, renormalisation.
cudaError_t enqueue_sweep(hsg_pool* p, const hsg_schedule* s) {
  cudaError_t e = cudaSuccess;
  if (s->kind != HSG_NONE) {
    const bool ball = s->proposal == HSG_PROP_BALL;
    const bool fused = s->kind == HSG_METROPOLIS_OR;
    const int met = ball ? hsg::U_MET_BALL : hsg::U_MET_SPHERE;
    const int upd = s->kind == HSG_HEATBATH ? hsg::U_HB : fused ? (ball ? hsg::U_MET_OR_BALL : hsg::U_MET_OR_SPHERE) : met;
    const int passes = main_passes(p, s);
    const int per = (s->hits + passes - 1) / passes;
    for (uint32_t c = 0; c < 2 && e == cudaSuccess; ++c)
      for (int k = 0, j0 = 0; k < passes && e == cudaSuccess; ++k, j0 += per) {
        const int n = std::min(per, s->hits - j0);
        // the fused reflection follows the colour's last hit only
        e = launch_pool_half(p, (fused && k + 1 < passes) ? met : upd, c, s->step, n, j0);
      }
  }
  for (int o = 0; o < s->n_or && e == cudaSuccess; ++o)
    for (uint32_t c = 0; c < 2 && e == cudaSuccess; ++c) e = launch_pool_half(p, hsg::U_OR, c, s->step, s->hits, 0);
  if (e != cudaSuccess) return e;
  k_pool_advance<<<cdiv_u((unsigned)p->max_slots, 256), 256, 0, p->stream>>>(p->d_desc, p->max_slots);
  p->launches += 1;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (s->renorm_every > 0) {
    k_pool_renorm<<<pool_grid(p), p->threads, 0, p->stream>>>(p->d_desc, p->d_tiles, p->d_ntiles,
                                                              reinterpret_cast<float4*>(p->arena),
                                                              (uint32_t)s->renorm_every, (uint32_t)p->tile_sites);
    p->launches += 1;
    e = cudaGetLastError();
  }
  return e;
}

hsg_status check_pool_schedule(hsg_pool* p, const hsg_schedule* s) {
  if (!s) return pfail(p, HSG_EINVAL, "schedule is NULL");
  if (s->kind != HSG_NONE && s->kind != HSG_METROPOLIS && s->kind != HSG_HEATBATH && s->kind != HSG_METROPOLIS_OR)
    return pfail(p, HSG_EINVAL, "schedule.kind must be HSG_NONE, HSG_METROPOLIS, HSG_HEATBATH or HSG_METROPOLIS_OR");
  if (s->hits < 1 || s->hits > 65535) return pfail(p, HSG_EINVAL, "schedule.hits must be in [1, 65535]");
  if (s->proposal != HSG_PROP_SPHERE && s->proposal != HSG_PROP_BALL)
    return pfail(p, HSG_EINVAL, "schedule.proposal must be HSG_PROP_SPHERE or HSG_PROP_BALL");
  if (!(s->step > 0.0f) || !std::isfinite(s->step)) return pfail(p, HSG_EINVAL, "schedule.step must be finite and > 0");
  if (s->n_or < 0 || s->renorm_every < 0) return pfail(p, HSG_EINVAL, "n_or and renorm_every must be >= 0");
  if (s->energy_every != 0) return pfail(p, HSG_EINVAL, "pools log no energies: energy_every must be 0");
  return HSG_OK;
}

bool valid_slot(const hsg_pool* p, int slot) {
  return slot >= 0 && slot < p->max_slots && p->slots[slot].active;
}

}  // namespace

extern "C" {

hsg_status hsg_pool_create(hsg_pool** out, uint64_t budget_bytes, int max_slots, void* cuda_stream) {
  if (!out) return pfail(nullptr, HSG_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_slots < 1 || max_slots > (1 << 20)) return pfail(nullptr, HSG_EINVAL, "max_slots must be in [1, 2^20]");
  if (budget_bytes < kAlign) return pfail(nullptr, HSG_EINVAL, "budget too small");
  hsg_pool* p = new (std::nothrow) hsg_pool();
  if (!p) return pfail(nullptr, HSG_ENOMEM, "host allocation failed");
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  p->max_slots = max_slots;
  p->slots.resize(max_slots);
  p->budget = budget_bytes / kAlign * kAlign;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
  if (e == cudaSuccess) e = cudaMalloc(&p->arena, p->budget);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_desc, sizeof(PoolDesc) * max_slots);
  if (e == cudaSuccess) e = cudaMallocHost(&p->h_desc, 2 * sizeof(PoolDesc) * max_slots);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_ntiles, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMallocHost(&p->h_ntiles, 2 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_energy, sizeof(double) * max_slots);
  if (e == cudaSuccess) e = cudaMallocHost(&p->h_energy, hsg_pool::kEnergyBufs * sizeof(double) * max_slots);
  if (e == cudaSuccess) e = cudaMallocHost(&p->h_sel, (size_t)hsg_pool::kEnergyBufs * max_slots);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_sel, (size_t)max_slots);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&p->up_ev[i], cudaEventDisableTiming);
  for (int i = 0; i < hsg_pool::kEnergyBufs && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&p->en_ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    hsg_status st = pcuda(nullptr, e, "pool creation");
    hsg_pool_destroy(p);
    return st;
  }
  p->free_blocks[0] = p->budget;
  p->h_ntiles[0] = p->h_ntiles[1] = 0;
  *out = p;
  return HSG_OK;
}

hsg_status hsg_pool_destroy(hsg_pool* p) {
  if (!p) return HSG_OK;
  const hsg::DeviceGuard device_guard(p->device);
  if (p->stream || p->arena) cudaStreamSynchronize(p->stream);
  drop_graph(p);
  if (p->stage) cudaFreeAsync(p->stage, p->stream);
  cudaStreamSynchronize(p->stream);
  cudaFree(p->arena);
  cudaFree(p->d_desc);
  cudaFreeHost(p->h_desc);
  cudaFree(p->d_tiles);
  cudaFreeHost(p->h_tiles);
  cudaFree(p->d_ntiles);
  cudaFreeHost(p->h_ntiles);
  cudaFree(p->d_partials);
  cudaFree(p->d_energy);
  cudaFreeHost(p->h_energy);
  cudaFreeHost(p->h_sel);
  cudaFree(p->d_sel);
  for (cudaEvent_t ev : p->up_ev)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : p->en_ev)
    if (ev) cudaEventDestroy(ev);
  delete p;
  return HSG_OK;
}

hsg_status hsg_pool_admit(hsg_pool* p, int L, uint64_t seed, uint32_t sample, uint32_t replica, double T,
                          const void* J, int dtype, int where, int* slot) {
  if (!p) return pfail(nullptr, HSG_EINVAL, "pool is NULL");
  const hsg::DeviceGuard device_guard(p->device);
  if (device_guard.status() != cudaSuccess) return pcuda(p, device_guard.status(), "cudaSetDevice");
  if (!slot) return pfail(p, HSG_EINVAL, "slot is NULL");
  *slot = -1;
  if (L < 4 || L > 1624 || (L & 1)) return pfail(p, HSG_EINVAL, "L must be even and in [4, 1624]");
  if (!(T > 0.0)) return pfail(p, HSG_EINVAL, "T must be > 0 (inf allowed)");
  if (!hsg::key_stream_ok(sample, replica)) return pfail(p, HSG_EINVAL, hsg::kKeyStreamMsg);
  if (J && dtype != HSG_F32 && dtype != HSG_F64) return pfail(p, HSG_EINVAL, "dtype must be HSG_F32 or HSG_F64");
  if (J && where != HSG_HOST && where != HSG_DEVICE) return pfail(p, HSG_EINVAL, "where must be HSG_HOST or HSG_DEVICE");
  int idx = -1;
  for (int i = 0; i < p->max_slots; ++i)
    if (!p->slots[i].active) {
      idx = i;
      break;
    }
  if (idx < 0) return pfail(p, HSG_EBUSY, "no free slot");
  const uint64_t n = (uint64_t)L * L * L;
  const uint64_t bytes = (n * (sizeof(float4) + 3 * sizeof(float)) + kAlign - 1) / kAlign * kAlign;
  uint64_t off = 0;
  if (!arena_alloc(p, bytes, &off)) return pfail(p, HSG_EBUSY, "not enough free pool memory for this lattice");
  Slot& s = p->slots[idx];
  s.active = true;
  s.L = L;
  s.seed = seed;
  s.sample = sample;
  s.replica = replica;
  s.T = T;
  s.off = off;
  s.bytes = bytes;
  s.sweep = 0;
  float4* S = reinterpret_cast<float4*>(p->arena + off);
  float* Jd = reinterpret_cast<float*>(p->arena + off + sizeof(float4) * n);
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu);
  const uint32_t k1 = (uint32_t)(seed >> 32) ^ ((2u * sample + replica) * 0x9E3779B9u);
  cudaError_t e = hsg::launch_init_spins(S, false, L, k0, k1, p->stream);
  p->launches += 1;
  if (e == cudaSuccess) {
    if (!J) {
      const uint32_t kj = (uint32_t)(seed >> 32) ^ ((2u * sample) * 0x9E3779B9u);
      e = hsg::launch_gen_couplings(Jd, L, k0, kj, p->stream);
    } else {
      const void* src = J;
      const size_t jb = (dtype == HSG_F64 ? sizeof(double) : sizeof(float)) * 3 * n;
      if (where == HSG_HOST) {
        hsg_status st = ensure_pool_stage(p, jb);
        if (st != HSG_OK) {
          arena_free(p, off, bytes);
          s.active = false;
          return st;
        }
        e = cudaMemcpyAsync(p->stage, J, jb, cudaMemcpyHostToDevice, p->stream);
        src = p->stage;
      }
      if (e == cudaSuccess) e = hsg::launch_scatter_couplings(src, dtype == HSG_F64, Jd, L, p->stream);
      if (e == cudaSuccess && where == HSG_HOST) e = cudaStreamSynchronize(p->stream);
    }
    p->launches += 1;
  }
  if (e != cudaSuccess) {
    arena_free(p, off, bytes);
    s.active = false;
    return pcuda(p, e, "pool admit");
  }
  p->n_active += 1;
  p->dirty = true;
  *slot = idx;
  return HSG_OK;
}

hsg_status hsg_pool_retire(hsg_pool* p, int slot) {
  if (!p) return pfail(nullptr, HSG_EINVAL, "pool is NULL");
  const hsg::DeviceGuard device_guard(p->device);
  if (device_guard.status() != cudaSuccess) return pcuda(p, device_guard.status(), "cudaSetDevice");
  if (!valid_slot(p, slot)) return pfail(p, HSG_EINVAL, "no such active slot");
  // No wait: the kernels already queued for this slot run first, and its
  // block is reused only by work queued on the same stream after this call.
  Slot& s = p->slots[slot];
  arena_free(p, s.off, s.bytes);
  s.active = false;
  p->n_active -= 1;
  p->dirty = true;
  return HSG_OK;
}

hsg_status hsg_pool_sweep(hsg_pool* p, const hsg_schedule* sched, int n_sweeps) {
  if (!p) return pfail(nullptr, HSG_EINVAL, "pool is NULL");
  const hsg::DeviceGuard device_guard(p->device);
  if (device_guard.status() != cudaSuccess) return pcuda(p, device_guard.status(), "cudaSetDevice");
  hsg_status st = check_pool_schedule(p, sched);
  if (st != HSG_OK) return st;
  if (n_sweeps < 0) return pfail(p, HSG_EINVAL, "n_sweeps must be >= 0");
  if (n_sweeps == 0 || p->n_active == 0) return HSG_OK;
  if ((st = sync_tables(p)) != HSG_OK) return st;
  const hsg_pool::GraphKey key{sched->kind,    sched->hits,       sched->proposal,      sched->n_or,
                               sched->renorm_every, p->threads,   p->tile_sites,        p->blocks_per_sm,
                               p->hits_per_pass, sched->step};
  cudaError_t e = cudaSuccess;
  // One sweep is captured once per (schedule, launch configuration) and
  // replayed; the legacy default stream cannot be captured, so there the
  // launches are issued directly.
  if (p->stream != nullptr) {
    if (!p->have_graph || !(p->gkey == key)) {
      drop_graph(p);
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const uint64_t before = p->launches;
        cudaError_t e2 = enqueue_sweep(p, sched);
        p->launches = before;
        e = cudaStreamEndCapture(p->stream, &g);
        if (e == cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&p->gexec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return pcuda(p, e, "pool sweep capture");
      p->have_graph = true;
      p->gkey = key;
    }
    const int per_sweep = 2 * main_passes(p, sched) + 2 * sched->n_or + 1 + (sched->renorm_every > 0);
    for (int k = 0; k < n_sweeps && e == cudaSuccess; ++k) {
      e = cudaGraphLaunch(p->gexec, p->stream);
      p->launches += (uint64_t)per_sweep;
    }
  } else {
    for (int k = 0; k < n_sweeps && e == cudaSuccess; ++k) e = enqueue_sweep(p, sched);
  }
  if (e != cudaSuccess) return pcuda(p, e, "pool sweep");
  for (Slot& s : p->slots)
    if (s.active) s.sweep += (uint64_t)n_sweeps;
  return HSG_OK;
}

namespace {

// Queue the energy kernels and the copy of the result into pinned buffer
// b, followed by b's event: every slot, or (slots != nullptr) the n listed
// active slots only, the others reading NaN.
hsg_status enqueue_energies(hsg_pool* p, int b, const int* slots = nullptr, int n = 0) {
  if (slots)
    for (int i = 0; i < n; ++i)
      if (!valid_slot(p, slots[i])) return pfail(p, HSG_EINVAL, "no such active slot");
  hsg_status st = sync_tables(p);
  if (st != HSG_OK) return st;
  cudaError_t e = cudaSuccess;
  if (p->en_pending[b] && (e = cudaEventSynchronize(p->en_ev[b])) != cudaSuccess) return pcuda(p, e, "pool sync");
  p->en_pending[b] = false;
  const uint8_t* sel = nullptr;
  if (slots) {  // the mask of buffer b is free: its last copy has passed
    uint8_t* h = p->h_sel + (size_t)b * p->max_slots;
    memset(h, 0, (size_t)p->max_slots);
    for (int i = 0; i < n; ++i) h[slots[i]] = 1;
    if ((e = cudaMemcpyAsync(p->d_sel, h, (size_t)p->max_slots, cudaMemcpyHostToDevice, p->stream)) != cudaSuccess)
      return pcuda(p, e, "pool energies");
    sel = p->d_sel;
  }
  if (p->n_active > 0 && (!slots || n > 0)) {
    k_pool_energy_partial<<<pool_grid(p), 256, 0, p->stream>>>(p->d_desc, p->d_tiles, p->d_ntiles,
                                                                reinterpret_cast<const float4*>(p->arena),
                                                                reinterpret_cast<const float*>(p->arena),
                                                                (uint32_t)p->tile_sites, sel, p->d_partials);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_pool_energy_final<<<(unsigned)std::min(p->max_slots, 4096), 256, 0, p->stream>>>(p->d_desc, p->max_slots, sel,
                                                                                        p->d_partials, p->d_energy);
    e = cudaGetLastError();
  }
  p->launches += 2;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->h_energy + (size_t)b * p->max_slots, p->d_energy, sizeof(double) * p->max_slots,
                        cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaEventRecord(p->en_ev[b], p->stream);
  if (e != cudaSuccess) return pcuda(p, e, "pool energies");
  p->en_pending[b] = true;
  return HSG_OK;
}

// Wait for buffer b's copy and hand out its first n values.
hsg_status read_energies(hsg_pool* p, int b, double* out, int n) {
  if (!p->en_pending[b]) return pfail(p, HSG_EINVAL, "no energies queued in this buffer");
  const cudaError_t e = cudaEventSynchronize(p->en_ev[b]);
  if (e != cudaSuccess) return pcuda(p, e, "pool energies");
  p->en_pending[b] = false;
  const double* h = p->h_energy + (size_t)b * p->max_slots;
  for (int i = 0; i < n; ++i) out[i] = i < p->max_slots ? h[i] : std::nan("");
  return HSG_OK;
}

}  // namespace

hsg_status hsg_pool_energies(hsg_pool* p, double* out, int n) {
  if (!p) return pfail(nullptr, HSG_EINVAL, "pool is NULL");
  const hsg::DeviceGuard device_guard(p->device);
  if (device_guard.status() != cudaSuccess) return pcuda(p, device_guard.status(), "cudaSetDevice");
  if (!out || n < 0) return pfail(p, HSG_EINVAL, "bad output buffer");
  const hsg_status st = enqueue_energies(p, 2);
  return st != HSG_OK ? st : read_energies(p, 2, out, n);
}

hsg_status hsg_pool_energies_async(hsg_pool* p, int buffer) {
  if (!p) return pfail(nullptr, HSG_EINVAL, "pool is NULL");
  const hsg::DeviceGuard device_guard(p->device);
  if (device_guard.status() != cudaSuccess) return pcuda(p, device_guard.status(), "cudaSetDevice");
  if (buffer != 0 && buffer != 1) return pfail(p, HSG_EINVAL, "buffer must be 0 or 1");
  return enqueue_energies(p, buffer);
}

hsg_status hsg_pool_energies_slots_async(hsg_pool* p, int buffer, const int* slots, int n) {
  if (!p) return pfail(nullptr, HSG_EINVAL, "pool is NULL");
  const hsg::DeviceGuard device_guard(p->device);
  if (device_guard.status() != cudaSuccess) return pcuda(p, device_guard.status(), "cudaSetDevice");
  if (buffer != 0 && buffer != 1) return pfail(p, HSG_EINVAL, "buffer must be 0 or 1");
  if (n < 0 || (n > 0 && !slots)) return pfail(p, HSG_EINVAL, "bad slot list");
  static const int none = 0;
  return enqueue_energies(p, buffer, n > 0 ? slots : &none, n);
}

hsg_status hsg_pool_energies_read(hsg_pool* p, int buffer, double* out, int n) {
  if (!p) return pfail(nullptr, HSG_EINVAL, "pool is NULL");
  const hsg::DeviceGuard device_guard(p->device);
  if (device_guard.status() != cudaSuccess) return pcuda(p, device_guard.status(), "cudaSetDevice");
  if (buffer != 0 && buffer != 1) return pfail(p, HSG_EINVAL, "buffer must be 0 or 1");
  if (!out || n < 0) return pfail(p, HSG_EINVAL, "bad output buffer");
  return read_energies(p, buffer, out, n);
}

hsg_status hsg_pool_get_spins(hsg_pool* p, int slot, float* out, int where) {
  if (!p) return pfail(nullptr, HSG_EINVAL, "pool is NULL");
  const hsg::DeviceGuard device_guard(p->device);
  if (device_guard.status() != cudaSuccess) return pcuda(p, device_guard.status(), "cudaSetDevice");
  if (!valid_slot(p, slot)) return pfail(p, HSG_EINVAL, "no such active slot");
  if (!out) return pfail(p, HSG_EINVAL, "out is NULL");
  if (where != HSG_HOST && where != HSG_DEVICE) return pfail(p, HSG_EINVAL, "where must be HSG_HOST or HSG_DEVICE");
  const Slot& s = p->slots[slot];
  const uint64_t n = (uint64_t)s.L * s.L * s.L;
  float* dst = out;
  if (where == HSG_HOST) {
    hsg_status st = ensure_pool_stage(p, sizeof(float) * 3 * n);
    if (st != HSG_OK) return st;
    dst = static_cast<float*>(p->stage);
  }
  cudaError_t e = hsg::launch_gather_spins(p->arena + s.off, false, dst, s.L, p->stream);
  p->launches += 1;
  if (e == cudaSuccess && where == HSG_HOST) {
    e = cudaMemcpyAsync(out, dst, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  }
  if (e != cudaSuccess) return pcuda(p, e, "pool spin readback");
  return HSG_OK;
}

hsg_status hsg_pool_get_sweep(hsg_pool* p, int slot, uint64_t* sweep) {
  if (!p) return pfail(nullptr, HSG_EINVAL, "pool is NULL");
  const hsg::DeviceGuard device_guard(p->device);
  if (device_guard.status() != cudaSuccess) return pcuda(p, device_guard.status(), "cudaSetDevice");
  if (!valid_slot(p, slot) || !sweep) return pfail(p, HSG_EINVAL, "no such active slot / NULL");
  *sweep = p->slots[slot].sweep;
  return HSG_OK;
}

hsg_status hsg_pool_usage(hsg_pool* p, uint64_t* bytes_used, uint64_t* bytes_budget, int* active) {
  if (!p) return pfail(nullptr, HSG_EINVAL, "pool is NULL");
  const hsg::DeviceGuard device_guard(p->device);
  if (device_guard.status() != cudaSuccess) return pcuda(p, device_guard.status(), "cudaSetDevice");
  if (bytes_used) *bytes_used = p->used;
  if (bytes_budget) *bytes_budget = p->budget;
  if (active) *active = p->n_active;
  return HSG_OK;
}

hsg_status hsg_pool_config(hsg_pool* p, int threads, int tile_sites, int blocks_per_sm, int hits_per_pass) {
  if (!p) return pfail(nullptr, HSG_EINVAL, "pool is NULL");
  const hsg::DeviceGuard device_guard(p->device);
  if (device_guard.status() != cudaSuccess) return pcuda(p, device_guard.status(), "cudaSetDevice");
  if ((threads != 64 && threads != 128 && threads != 256) || tile_sites < threads || tile_sites % threads != 0 ||
      tile_sites > 8192 || blocks_per_sm < 1 || blocks_per_sm > 32 || hits_per_pass < 0 || hits_per_pass > 65535)
    return pfail(p, HSG_EINVAL,
                 "threads in {64,128,256}, tile_sites a multiple of threads <= 8192, blocks_per_sm 1..32, "
                 "hits_per_pass 0..65535");
  if (tile_sites != p->tile_sites) p->dirty = true;
  p->threads = threads;
  p->tile_sites = tile_sites;
  p->blocks_per_sm = blocks_per_sm;
  p->hits_per_pass = hits_per_pass;
  return HSG_OK;
}

hsg_status hsg_pool_autotune(hsg_pool* p, const hsg_schedule* sched, int* threads, int* tile_sites,
                             int* blocks_per_sm, int* hits_per_pass) {
  if (!p) return pfail(nullptr, HSG_EINVAL, "pool is NULL");
  const hsg::DeviceGuard device_guard(p->device);
  if (device_guard.status() != cudaSuccess) return pcuda(p, device_guard.status(), "cudaSetDevice");
  hsg_status st = check_pool_schedule(p, sched);
  if (st != HSG_OK) return st;
  if (p->n_active == 0) return pfail(p, HSG_EINVAL, "autotune needs admitted lattices");
  if (p->stream == nullptr) return pfail(p, HSG_EINVAL, "autotune needs a non-default stream");
  // Snapshot the lattices (every trial sweep changes them) and the counters.
  uint64_t hi = 0;
  for (const Slot& s : p->slots)
    if (s.active) hi = std::max(hi, s.off + s.bytes);
  void* snap = nullptr;
  cudaError_t e = cudaMallocAsync(&snap, hi, p->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(snap, p->arena, hi, cudaMemcpyDeviceToDevice, p->stream);
  if (e != cudaSuccess) return pcuda(p, e, "autotune snapshot");
  std::vector<uint64_t> sweeps;
  for (const Slot& s : p->slots) sweeps.push_back(s.sweep);
  const int old_t = p->threads, old_ts = p->tile_sites, old_b = p->blocks_per_sm, old_h = p->hits_per_pass;
  int best_t = old_t, best_ts = old_ts, best_b = old_b, best_h = old_h;
  float best_ms = 1e30f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // One warm-up sweep (it also captures the graph), then two timed ones.
  auto trial = [&](int t, int ts, int b, int h) {
    if (hsg_pool_config(p, t, ts, b, h) != HSG_OK) return true;
    if ((st = hsg_pool_sweep(p, sched, 1)) != HSG_OK) return false;
    cudaEventRecord(e0, p->stream);
    if ((st = hsg_pool_sweep(p, sched, 2)) != HSG_OK) return false;
    cudaEventRecord(e1, p->stream);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best_t = t;
      best_ts = ts;
      best_b = b;
      best_h = h;
    }
    return true;
  };
  // Launch shape with every Metropolis hit in one pass, then, on that
  // shape, the hits split over passes of 1, 2, 4, ... hits.
  const int cand_t[] = {128, 256};
  const int cand_ts[] = {256, 512, 1024, 2048};
  const int cand_b[] = {4, 8, 16};
  bool ok = true;
  for (int t : cand_t)
    for (int ts : cand_ts)
      for (int b : cand_b)
        if (ok) ok = trial(t, ts, b, 0);
  const bool multi_hit = sched->kind == HSG_METROPOLIS || sched->kind == HSG_METROPOLIS_OR;
  const int shape_t = best_t, shape_ts = best_ts, shape_b = best_b;
  for (int h = 1; ok && multi_hit && h < sched->hits; h *= 2) ok = trial(shape_t, shape_ts, shape_b, h);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // Restore the lattices and counters; keep the fastest configuration.
  e = cudaMemcpyAsync(p->arena, snap, hi, cudaMemcpyDeviceToDevice, p->stream);
  cudaFreeAsync(snap, p->stream);
  for (size_t i = 0; i < p->slots.size(); ++i) p->slots[i].sweep = sweeps[i];
  hsg_pool_config(p, best_t, best_ts, best_b, best_h);
  p->dirty = true;
  if (st != HSG_OK) {
    hsg_pool_config(p, old_t, old_ts, old_b, old_h);
    return st;
  }
  if (e != cudaSuccess) return pcuda(p, e, "autotune restore");
  if ((st = sync_tables(p)) != HSG_OK) return st;
  if (threads) *threads = best_t;
  if (tile_sites) *tile_sites = best_ts;
  if (blocks_per_sm) *blocks_per_sm = best_b;
  if (hits_per_pass) *hits_per_pass = best_h;
  return HSG_OK;
}

hsg_status hsg_pool_launch_count(hsg_pool* p, uint64_t* launches) {
  if (!p || !launches) return pfail(p, HSG_EINVAL, "NULL argument");
  *launches = p->launches;
  return HSG_OK;
}

const char* hsg_pool_last_error(const hsg_pool* p) { return p ? p->err.c_str() : ""; }

}  // extern "C"
