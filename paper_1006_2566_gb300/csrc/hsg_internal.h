// hsg_internal.h -- host-side interface between the C-ABI layer and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda.h>  // CUtensorMap (the type only; the encoder is fetched from the driver at run time)
#include <cuda_runtime.h>

namespace hsg {

// A value kept per device and set once, by whichever host thread gets there
// first: a kernel attribute applied, an occupancy looked up (0 = not yet).
// Objects of this type live in static storage, so every slot starts at 0.
constexpr int kMaxDevices = 64;
struct PerDevice {
  std::atomic<int> v[kMaxDevices];
};

// Makes `dev` the current device for the guard's lifetime and then restores
// the caller's; no device call beyond cudaGetDevice when it is current
// already.  Every ABI entry point holds one for its context's or pool's
// device, so calls on objects of several devices may be mixed freely.
class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    err_ = cudaGetDevice(&prev_);
    if (err_ == cudaSuccess && prev_ != dev) {
      err_ = cudaSetDevice(dev);
      switched_ = err_ == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (switched_) cudaSetDevice(prev_);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
  cudaError_t status() const { return err_; }

 private:
  int prev_ = 0;
  bool switched_ = false;
  cudaError_t err_ = cudaSuccess;
};

// The current device's slot of `pd`; nullptr with *err set when the device
// cannot be read or its ordinal is beyond kMaxDevices.
inline std::atomic<int>* device_slot(PerDevice& pd, cudaError_t* err) {
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= kMaxDevices) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  return &pd.v[dev];
}

// The Philox key's stream number 2*sample + replica names each (sample,
// replica) pair once only for replica < 2 and sample < 2^31; beyond, two
// pairs would share a key and every random number.
inline bool key_stream_ok(uint32_t sample, uint32_t replica) { return replica <= 1u && sample < 0x80000000u; }
constexpr const char* kKeyStreamMsg = "replica must be 0 or 1 and sample < 2^31 (the Philox key's stream number "
                                      "2*sample + replica must name each pair once)";

// Arguments of one half-sweep (see hsg_device.cuh for the layout).
struct SweepArgs {
  float4* own;          // spins of the colour being updated
  const float4* oth;    // spins of the other colour (read only)
  const float* jx_own;  // +x / +y / +z bonds of the updated colour
  const float* jy_own;
  const float* jz_own;
  const float* jx_oth;  // +x / +y / +z bonds of the other colour
  const float* jy_oth;
  const float* jz_oth;
  int L, Lh, colour, hits;
  uint32_t k0, k1, sweep_lo, sweep_hi;
  float beta, step;
  // When set, the sweep counter is read from this device word instead of
  // sweep_lo/sweep_hi (so that a captured graph can be replayed).
  const unsigned long long* sweep_ptr;
  // Packed layout: own / oth are then component-0 arrays of three fp32
  // arrays `stride` floats apart (global kernel only).
  bool packed;
  size_t stride;
};

// Kernel variants (values match HSG_KERNEL_*).
enum Variant : int { V_AUTO = 0, V_GLOBAL = 1, V_SLAB = 2, V_WAVE = 3 };

// Half-sweep of update kind `upd` (UpdKind) with kernel `variant`
// (V_GLOBAL or V_SLAB).  One kernel launch; `sm_count` (the device's SMs)
// shapes the slab kernel's grid.
cudaError_t launch_half_sweep(int upd, int variant, const SweepArgs& a, int sm_count, cudaStream_t s);

// Arguments of one temporally blocked over-relaxation sweep (hsg_wave.cu):
// colour 0 then colour 1, read from `src` and written to `dst`.
struct WaveArgs {
  const float4* src;  // S[2][N/2] before the sweep
  float4* dst;        // S[2][N/2] after the sweep; must not overlap src
  const float* J;     // J[3][2][N/2]
  int L, Lh;
  bool renorm;  // store every new spin renormalised (renorm_spin)
  // TMA descriptor of the halo-padded bonds (launch_pad_bonds), or nullptr:
  // with it the sweep takes each plane's bonds as one tensor box per CTA.
  const CUtensorMap* bond_map;
  // Device word that a CTA sets (to 1) when a bounded wait for a tensor
  // box gave up; the sweep's results are then not to be trusted.
  unsigned long long* err;
  // Bytes each box's wait expects beyond the box (0; > 0 only to test the
  // bounded waits: the waits then cannot complete and run out).
  uint32_t box_extra_tx;
  // Arrivals each colour-1 plane's barrier expects beyond its copies (0;
  // 1 only to test the bounded waits, likewise).
  uint32_t c1_extra_arrivals;
};

// Over-relaxation sweep (both colours) in one launch, bit-identical to the
// colour-0 and colour-1 half-sweeps of launch_half_sweep(U_OR, ...), and
// with `renorm` set to those half-sweeps followed by launch_renorm.
cudaError_t launch_or_sweep_wave(const WaveArgs& a, int sm_count, cudaStream_t s);

// Halo-padded copy of the colour-split bonds, read by the sweep's tensor
// boxes: Jp[a][z][yp][xp] with a = 2d + c, yp = y + 2 in [0, L + 4) and
// xp = xh + 2 in [0, W), W = roundup(L/2 + 4, 4), holding the bond of
// (y mod L, xh mod L/2) -- the periodic images of the lattice's edges --
// so that no box ever wraps.  Used for L >= kWaveTmaMinL.
constexpr int kWaveTmaMinL = 32;
constexpr int kPadX = 2, kPadY = 2;  // halo columns / rows of the padded copy on the low side
// Width W of the padded copy's rows: room for xh in [-2, L/2 + 2), rounded
// up to a multiple of four floats (16-byte rows, as tensor maps want).
__host__ __device__ inline uint32_t padded_width(int L) { return (uint32_t)((L / 2 + kPadX + 2 + 3) / 4 * 4); }
size_t padded_bonds_elems(int L);
cudaError_t launch_pad_bonds(const float* J, float* Jp, int L, cudaStream_t s);
// The tensor map of Jp (4-D: xp, yp, z, a; box 20 x 17 x 1 x 6 floats).
cudaError_t encode_padded_bond_map(CUtensorMap* map, const float* Jp, int L);

// Spin layouts (hsg_device.cuh): `packed` = three fp32 component arrays per
// colour (12 bytes a spin), else float4 per spin.
// Spin initialisation: S from Philox kind INIT.  One launch.
cudaError_t launch_init_spins(void* S, bool packed, int L, uint32_t k0, uint32_t k1, cudaStream_t s);

// Site-major -> colour-split couplings (src: 3N fp32 or fp64); with Jp not
// NULL also its halo-padded copy (launch_pad_bonds' layout), from the same
// values.  One launch.
cudaError_t launch_scatter_couplings(const void* src, bool f64, float* J, int L, cudaStream_t s, float* Jp = nullptr);

// Gaussian couplings from Philox kind JGEN under key (k0, k1), written
// colour-split; and colour-split -> site-major fp32 couplings.  One launch each.
cudaError_t launch_gen_couplings(float* J, int L, uint32_t k0, uint32_t k1, cudaStream_t s);
cudaError_t launch_gather_couplings(const float* J, float* dst, int L, cudaStream_t s);

// Site-major fp32 spins <-> colour-split float4 spins.  One launch each.
cudaError_t launch_scatter_spins(const float* src, void* S, bool packed, int L, cudaStream_t s);
cudaError_t launch_gather_spins(const void* S, bool packed, float* dst, int L, cudaStream_t s);

// Spins (3 per site) and +x/+y/+z bonds of n listed site-major indices
// (device arrays).  One launch (none for n = 0).
cudaError_t launch_gather_sites(const void* S, bool packed, const float* J, int L, const uint32_t* sites, int n,
                                float* spins, float* bonds, cudaStream_t s);

// Energy: number of FP64 partial sums the first pass writes, and the
// two-pass E/N into *out (device).  Two launches.
// With log_idx set, E/N goes to out[*log_idx] and *log_idx is incremented
// (an energy log whose position lives in device memory).
size_t energy_partials(int L);
cudaError_t launch_energy(const void* S, bool packed, const float* J, int L, double* partials, double* out,
                          unsigned long long* log_idx, cudaStream_t s);

// Device counters: *p = v, *p += d.  One single-thread launch each.
cudaError_t launch_set_u64(unsigned long long* p, unsigned long long v, cudaStream_t s);
cudaError_t launch_add_u64(unsigned long long* p, unsigned long long d, cudaStream_t s);

// FP64 renormalisation of the n = N spins.  One launch.
cudaError_t launch_renorm(void* S, bool packed, long long n, int sm_count, cudaStream_t s);

// Record the calling thread's last error message (read by hsg_last_error(NULL)).
void set_thread_error(const std::string& msg);

// Philox words for counters (t, c1, c2, c3), t < n.  One launch.
cudaError_t launch_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t n, uint32_t* out,
                          cudaStream_t s);

}  // namespace hsg
