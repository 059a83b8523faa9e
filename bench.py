#!/usr/bin/env python
"""Benchmark: checkerboard Monte Carlo sweeps of the 3D Heisenberg spin glass.

Workload (default): L = 256 periodic lattice (16.7M spins, 470 MB of fp32
state), one disorder sample, Gaussian J; per sweep one heat-bath sweep at
T = 0.3 and four over-relaxation sweeps; FP64 renormalisation and FP64
energy every 10 sweeps.  One benchmark step = 10 sweeps (ending with the
renormalisation and the energy), so 20 steps are the 200-sweep run.

Prints one JSON line.  `value` is site updates per ns (one update = one site
visited by one heat-bath or over-relaxation pass), timed with CUDA events on
the library's stream with the inputs resident in HBM; `e2e` is the same
metric through the C ABI from pinned host buffers (couplings and spins in,
energy and spins out, every step); `roofline` is the dominant kernel (the
over-relaxation half-sweep) against the measured HBM copy bandwidth.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank runs its own disorder sample (weak scaling,
no collective on the data path); the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# Bytes per site update of each kernel (fp32, float4 spins, each
# other-colour spin and each bond read once per half-sweep):
#   over-relaxation / Metropolis: own spin read 16 + write 16, neighbours 16, bonds 24
#   heat-bath: own spin write 16, neighbours 16, bonds 24 (old spin not read)
#   energy: 28 per site (all spins 16, all bonds 12); renormalisation: 32 per site
BYTES_OR, BYTES_HB, BYTES_ENERGY, BYTES_RENORM = 72, 56, 28, 32
# Temporally blocked over-relaxation sweep (both colours in one pass), per
# site update: all spins read 16 + written 16, all bonds 12.
BYTES_OR_WAVE = 44
# Packed layout (12-byte spins): OR 12 r + 12 w + 12 + 24, heat-bath 12 w + 12
# + 24, energy 12 + 12, renormalisation 12 r + 12 w.
BYTES_OR_PACKED, BYTES_HB_PACKED, BYTES_ENERGY_PACKED, BYTES_RENORM_PACKED = 60, 48, 24, 24

WORKLOADS = {
    "l256_hb_or": dict(
        L=256, seed=3, kind="HB", T=0.3, n_or=4, hits=1, proposal="SPHERE", step=0.5, renorm_every=10,
        energy_every=10, sweeps_per_step=10,
        desc=("L=256 periodic 3D Heisenberg spin glass (16.7M spins, 470 MB fp32 state), 1 sample, fp32 float4 "
              "spins + fp32 Gaussian J; per sweep 1 heat-bath (T=0.3) + 4 over-relaxation; FP64 renorm and "
              "FP64 energy every 10 sweeps; 1 step = 10 sweeps")),
    "l16_met": dict(
        L=16, seed=1, kind="MET", T=1.0, n_or=0, hits=1, proposal="SPHERE", step=0.5, renorm_every=0,
        energy_every=10, sweeps_per_step=10, j_fp64=True,
        desc=("L=16 periodic 3D Heisenberg spin glass, 1 sample, Gaussian J in fp64 (rounded to fp32 on upload); "
              "checkerboard Metropolis 1 hit, uniform-sphere proposal, T=1.0; E/N every 10 sweeps; "
              "1 step = 10 sweeps")),
    "l128_metor_fused": dict(
        L=128, seed=2, kind="METOR", T=0.5, n_or=0, hits=4, proposal="BALL", step=0.5, renorm_every=10,
        energy_every=10, sweeps_per_step=10,
        desc=("L=128, 1 sample, fp32; per sweep the fused colour pass (4-hit Metropolis, ball 0.5, T=0.5, then one "
              "over-relaxation reflection about the same field; opt-in chain); 1 step = 10 sweeps")),
    "l128_met_or": dict(
        L=128, seed=2, kind="MET", T=0.5, n_or=1, hits=4, proposal="BALL", step=0.5, renorm_every=10,
        energy_every=10, sweeps_per_step=10,
        desc=("L=128 periodic 3D Heisenberg spin glass, 1 sample, fp32; per sweep 4-hit Metropolis (ball "
              "proposal, step 0.5, T=0.5) + 1 over-relaxation; 1 step = 10 sweeps")),
}

# The paper's own timings (context only; other hardware, other workload):
# over-relaxation on an L=128 lattice, fp32 (Table 2, Table 3).
PAPER_CONTEXT = {
    "workload": "L=128 over-relaxation sweeps, fp32 (paper Table 2)",
    "GTX480_TEXT_upd_per_ns": round(1 / 0.63, 3),
    "GTX480_GM_upd_per_ns": round(1 / 0.66, 3),
    "TeslaC1060_TEXT_upd_per_ns": round(1 / 1.8, 3),
    "i7_SSE_OpenMP_8threads_upd_per_ns": round(1 / 5.0, 3),
}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched", "l16_pooled", "serving"],
                    default="l256_hb_or")
    ap.add_argument("--kernel", choices=["auto", "global", "slab", "wave"], default="auto")
    ap.add_argument("--layout", choices=["float4", "packed"], default="float4", help="device spin layout")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the timed oracle sample")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--no-clocks", action="store_true", help="do not sample nvidia-smi")
    ap.add_argument("--no-autotune", action="store_true", help="batched workload: default pool launch shape")
    ap.add_argument("--no-batched", action="store_true",
                    help="default line: skip the batched-pool summaries (512 samples x 2 replicas; 2048 L=16 samples)")
    ap.add_argument("--no-serving", action="store_true", help="default line: skip the serving summary")
    return ap.parse_args()


def dist_env():
    from paper_1006_2566_gb300 import dist as hdist

    return hdist.env()


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, enabled: bool = True):
        self.device_index = device_index
        self.proc = None
        self.lines: list[str] = []
        self.enabled = enabled

    def start(self):
        """Start sampling every 100 ms and wait (at most 3 s) for the first
        sample, so that the timed region that follows is sampled from its
        start."""
        if not self.enabled:
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device_index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        deadline = time.time() + 3.0
        while not self.lines and time.time() < deadline:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, window=None):
        """Stop sampling; summarise the samples that arrived within `window`
        (wall-clock start, end of the timed region; one sampling interval of
        grace at the end), or all of them when none did."""
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        lines = self.lines
        in_window = window is not None and any(window[0] <= t <= window[1] + 0.1 for t, _ in lines)
        if in_window:
            lines = [(t, ln) for t, ln in lines if window[0] <= t <= window[1] + 0.1]
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
                power.append(float(parts[3].split()[0]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "power_w_max": max(power),
                "samples": len(sm), "reasons": sorted(reasons),
                "window": "timed region" if in_window else "whole run (no sample fell in the timed region)"}


# ---------------------------------------------------------------------------
# Helpers
# ---------------------------------------------------------------------------

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _code_only(text: str) -> str:
    """C/CUDA source without its comments and with runs of white space
    folded to one blank: what the compiler sees of it."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":  # a string or character literal, kept whole
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return re.sub(r"\s+", " ", "".join(out)).strip()


def kernel_source_hash() -> str:
    """First 16 hex digits of the SHA-256 of the single-lattice kernels' code
    (comments and spacing removed) and of the nvcc flags they are built with
    (paths left out), which an ncu summary records to say which kernels its
    counters belong to."""
    from paper_1006_2566_gb300 import build as _build

    h = hashlib.sha256()
    for f in ("hsg_sweep.cu", "hsg_wave.cu", "hsg_device.cuh"):
        with open(os.path.join(ROOT, "paper_1006_2566_gb300", "csrc", f)) as fh:
            h.update(_code_only(fh.read()).encode())
    h.update(" ".join(f for f in _build.NVCC_FLAGS if not os.path.isabs(f)).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_variant: str, L: int):
    """DRAM bytes per over-relaxation launch from the committed ncu summary,
    if it was taken on the current kernel source; else None."""
    name = {"wave": f"or_full_sweep_wave_L{L}.md", "packed": f"or_half_sweep_packed_L{L}.md"}.get(
        kernel_variant, f"or_half_sweep_{kernel_variant}_L{L}.md")
    return profiled_value(name, "dram_bytes_per_launch")


def profiled_value(name: str, key: str):
    """A per-launch figure `key` from the committed ncu summary `name`, if it
    was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_src = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]{16})", text)
    m_v = re.search(key + r":\s*([0-9.eE+]+)", text)
    if not m_src or not m_v or m_src.group(1) != kernel_source_hash():
        return None
    return float(m_v.group(1))


# Warp instructions one SM issues per clock: four schedulers, one each.
ISSUE_PER_SM_CLK = 4
# Maximum SM clock of a GB300 (MHz), used when no clock was sampled.
SM_MAX_MHZ_NOMINAL = 2070


def alu_roofline(L, hits_per_launch, met_ms, met_n, clk, sm_count, steps, profiled_ms):
    """The multi-hit Metropolis half-sweep is bound by instruction issue, not
    by memory: `achieved` = warp instructions it issues per second (the ncu
    count per launch over the live CUDA-event duration), `peak` = the SMs'
    issue slots per second at the maximum SM clock."""
    avg_s = met_ms / met_n / 1e3
    max_mhz = (clk or {}).get("sm_max_mhz") or SM_MAX_MHZ_NOMINAL
    peak = sm_count * ISSUE_PER_SM_CLK * max_mhz * 1e6 / 1e9
    name = f"metropolis_half_sweep_global_L{L}.md"
    insts = profiled_value(name, "warp_inst_per_launch")
    ach = insts / avg_s / 1e9 if insts else None
    return {"bound": "alu", "kernel": "multi-hit Metropolis half-sweep", "unit": "G warp-inst/s",
            "achieved": round(ach, 1) if ach else None, "peak": round(peak, 1),
            "frac": round(ach / peak, 4) if ach else None,
            "peak_source": f"{sm_count} SMs x {ISSUE_PER_SM_CLK} warp instructions/clock x {max_mhz:.0f} MHz",
            "warp_inst_per_launch": insts, "hits_per_launch": hits_per_launch,
            "hits_per_ns": round(hits_per_launch / avg_s / 1e9, 2),
            "traffic": profiled_value(name, "dram_bytes_per_launch"),
            "avg_launch_ms": round(met_ms / met_n, 5), "launches": met_n,
            "measured_over": f"{steps} steps with per-launch CUDA events ({profiled_ms / steps:.3f} "
                             f"ms/step, directly launched)"}


def step_units(wl) -> int:
    """Site updates in one step (one per site per main-update or OR pass)."""
    passes = {"HB": 1, "MET": 1, "METOR": 2}.get(wl["kind"], 0) + wl["n_or"]
    return (wl["L"] ** 3) * passes * wl["sweeps_per_step"]


def step_bytes(wl, wave: bool = False, packed: bool = False) -> int:
    n = wl["L"] ** 3
    b_or, b_hb = (BYTES_OR_PACKED, BYTES_HB_PACKED) if packed else (BYTES_OR, BYTES_HB)
    b_en, b_rn = (BYTES_ENERGY_PACKED, BYTES_RENORM_PACKED) if packed else (BYTES_ENERGY, BYTES_RENORM)
    main = {"HB": b_hb, "MET": b_or, "METOR": b_or}.get(wl["kind"], 0)
    per_sweep = n * (main + wl["n_or"] * (BYTES_OR_WAVE if wave else b_or))
    s = wl["sweeps_per_step"]
    extra = 0
    if wl["energy_every"]:
        extra += n * b_en * (s // wl["energy_every"])
    if wl["renorm_every"] and not (wave and wl["n_or"] > 0):  # else fused into the last wave sweep
        extra += n * b_rn * (s // wl["renorm_every"])
    return per_sweep * s + extra


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def run_ours(args, wl):
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_1006_2566_gb300 import build

    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1006_2566_gb300 import dist as hdist
    from paper_1006_2566_gb300 import hsg, inputs

    L = wl["L"]
    N = L ** 3
    kind = {"HB": hsg.HSG_HEATBATH, "MET": hsg.HSG_METROPOLIS, "METOR": hsg.HSG_METROPOLIS_OR,
            "NONE": hsg.HSG_NONE}[wl["kind"]]
    proposal = {"SPHERE": hsg.HSG_PROP_SPHERE, "BALL": hsg.HSG_PROP_BALL}[wl["proposal"]]
    kernel = {"auto": hsg.HSG_KERNEL_AUTO, "global": hsg.HSG_KERNEL_GLOBAL, "slab": hsg.HSG_KERNEL_SLAB,
              "wave": hsg.HSG_KERNEL_WAVE}[args.kernel]
    sched = hsg.schedule(kind=kind, hits=wl["hits"], proposal=proposal, step=wl["step"], n_or=wl["n_or"], T=wl["T"],
                         renorm_every=wl["renorm_every"], energy_every=wl["energy_every"], kernel=kernel)
    sps = wl["sweeps_per_step"]
    stream = torch.cuda.Stream()
    sample = hdist.rank_sample(rank)  # weak scaling: one disorder sample per rank
    # fp64 couplings where the workload specifies them (the library rounds
    # them to fp32 on upload), fp32 otherwise
    J = inputs.gaussian_couplings(L, seed=wl["seed"], sample=sample,
                                  dtype=np.float64 if wl.get("j_fp64") else np.float32)
    packed = args.layout == "packed"
    lat = hsg.Lattice(L, wl["seed"], sample, 0, stream,
                      layout=hsg.HSG_LAYOUT_PACKED if packed else hsg.HSG_LAYOUT_FLOAT4)
    lat.set_couplings(J)
    kernel_used = hsg.hsg_kernel_for(lat.ctx, sched)  # what HSG_KERNEL_AUTO resolves to
    # inputs resident in HBM from here on
    for _ in range(args.warmup):
        lat.sweep(sched, sps)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device(), enabled=not args.no_clocks and rank == 0)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    # Timed region: K steps as a user runs them (sweep periods replayed as
    # CUDA graphs), CUDA events on the library's stream.
    n_launch0 = hsg.hsg_launch_count(lat.ctx)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    wall0 = time.time()
    t0.record(stream)
    for _ in range(args.steps):
        lat.sweep(sched, sps)
    t1.record(stream)
    torch.cuda.synchronize()
    wall1 = time.time()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop((wall0, wall1))
    elapsed_ms = t0.elapsed_time(t1)
    launches = hsg.hsg_launch_count(lat.ctx) - n_launch0
    # The same K steps again with the library's profiler on: every kernel is
    # bracketed by CUDA events on its stream (launched directly, not from a
    # graph) -- the per-kernel durations of the roofline.
    hsg.hsg_profile_reset(lat.ctx)
    hsg.hsg_profile(lat.ctx, True)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        lat.sweep(sched, sps)
    p1.record(stream)
    torch.cuda.synchronize()
    profiled_ms = p0.elapsed_time(p1)
    per_class = {k: hsg.hsg_profile_read(lat.ctx, k) for k in range(hsg.HSG_PROF_COUNT)}
    hsg.hsg_profile(lat.ctx, False)
    e_last = float(lat.energy_log()[-1]) if wl["energy_every"] else float("nan")
    elapsed_ms = hdist.max_over_ranks(elapsed_ms, device="cuda")
    # The oracle leg, part 1 (outside every timed region): the error of the
    # reported quantities against the FP64 oracle, on this lattice as the
    # timed steps left it.
    errors = None
    if world == 1 and not args.no_cpu_baseline:
        errors = errors_vs_oracle(hsg, lat, J, wl, e_last)

    # ---- end to end through the C ABI, from pinned host memory -------------
    # Every step uploads its inputs (couplings and spins, site-major fp32)
    # from pinned host memory, runs its sweeps and reads its result back (E/N
    # and the spins).  Two lattices on two streams take alternate steps, so
    # one step's copies overlap the other's sweeps (copy engines and SMs
    # work at once); each step still waits for its own uploads before its
    # sweeps and for its sweeps before its read-back.  The sweeps of the two
    # lattices are chained by an event (a step's sweeps start once the
    # previous step's have ended): run side by side, the two lattices'
    # kernels share the SMs and break the temporally blocked sweep's single
    # wave of CTAs (7.98 against 7.81 ms per step).
    e2e = None
    if not args.no_e2e:
        Jh = torch.from_numpy(J).pin_memory()
        s_in = torch.empty(3 * N, dtype=torch.float32).pin_memory()
        outs = [torch.empty(3 * N, dtype=torch.float32).pin_memory() for _ in range(2)]
        hsg.hsg_get_spins(lat.ctx, s_in)
        stream2 = torch.cuda.Stream()
        lat2 = hsg.Lattice(L, wl["seed"], sample, 0, stream2,
                           layout=hsg.HSG_LAYOUT_PACKED if packed else hsg.HSG_LAYOUT_FLOAT4)
        pair = [lat, lat2]
        streams = {id(lat): stream, id(lat2): stream2}
        swept = [None]  # event after the last step's sweeps

        def begin(lt):
            lt.set_couplings(Jh)  # H2D 12N bytes, returns when copied
            lt.set_spins(s_in)  # H2D 12N bytes, returns when copied
            st = streams[id(lt)]
            if swept[0] is not None:
                st.wait_event(swept[0])
            lt.sweep(sched, sps)  # queued on the lattice's stream
            swept[0] = torch.cuda.Event()
            swept[0].record(st)

        def finish(lt, out):
            lt.energy()  # waits for the sweeps; D2H 8 bytes
            hsg.hsg_get_spins(lt.ctx, out)  # D2H 12N bytes

        for k in range(2):  # untimed warm-up of the host path, both lattices
            begin(pair[k])
            finish(pair[k], outs[k])
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        pending = None
        for k in range(args.steps):
            lt = pair[k % 2]
            begin(lt)
            if pending is not None:
                finish(*pending)
            pending = (lt, outs[k % 2])
        finish(*pending)
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - w0) * 1e3
        e2e_ms = hdist.max_over_ranks(e2e_ms, device="cuda")
        lat2.close()
        e2e = {"value": round(world * step_units(wl) * args.steps / (e2e_ms * 1e6), 4), "unit": "spin updates/ns",
               "h2d_bytes_per_step": int(Jh.numel() * Jh.element_size() + s_in.numel() * 4),
               "d2h_bytes_per_step": int(8 + outs[0].numel() * 4), "ms_per_step": round(e2e_ms / args.steps, 4),
               "pipelined": "two lattices on two streams take alternate steps; one step's host copies overlap "
                            "the other's sweeps, and each step's sweeps start after the previous step's"}
    lat.close()
    if world > 1:
        torch.distributed.barrier()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    value = hdist.job_throughput(step_units(wl) * args.steps, world, elapsed_ms * 1e6)
    peak, peak_kind = measured_peaks()
    or_ms, or_n = per_class[hsg.HSG_PROF_OVERRELAX]
    hb_ms, hb_n = per_class[hsg.HSG_PROF_HEATBATH]
    met_ms, met_n = per_class[hsg.HSG_PROF_METROPOLIS]
    nh = N // 2
    variant = {hsg.HSG_KERNEL_GLOBAL: "global", hsg.HSG_KERNEL_SLAB: "slab",
               hsg.HSG_KERNEL_WAVE: "wave"}[kernel_used]
    wave = variant == "wave"
    if packed:
        variant = "packed"  # the global kernel over the packed layout
    # Units one over-relaxation launch processes: N/2 sites per half-sweep,
    # N per wave sweep.
    units = N if wave else nh
    b_or = BYTES_OR_WAVE if wave else (BYTES_OR_PACKED if packed else BYTES_OR)
    b_hb = BYTES_HB_PACKED if packed else BYTES_HB
    roof = None
    if or_n:
        # `achieved` prices each site update at the per-update byte model of
        # the update kind (72 B for over-relaxation with float4 spins, 60 B
        # packed), whatever the kernel actually moves: a temporally blocked
        # sweep that moves fewer bytes shows as a fraction above 1.  The
        # kernel's own 44 B model and the DRAM bytes ncu counted for it are
        # given beside it, each against the measured copy peak and the
        # nominal 8 TB/s.
        avg_s = or_ms / or_n / 1e3
        b_model = BYTES_OR_PACKED if packed else BYTES_OR
        alg = units * b_model
        ach = alg / avg_s / 1e9
        kname = ("over-relaxation full sweep, temporally blocked" if wave else
                 "over-relaxation half-sweep, packed spins" if packed else "over-relaxation half-sweep")
        traffic = profiled_traffic(variant, L)

        def rate(nbytes):
            g = nbytes / avg_s / 1e9
            return {"GBps": round(g, 1), "frac": round(g / peak, 4), "frac_of_nominal_8TBps": round(g / 8000.0, 4)}

        roof = {"bound": "hbm", "kernel": kname, "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "peak_source": f"{peak_kind} hbm_gbs",
                "byte_model": f"{b_model} B per site update", "traffic": traffic,
                "algorithmic_bytes_per_launch": alg, "units_per_launch": units,
                "avg_launch_ms": round(or_ms / or_n, 5), "launches": or_n,
                "frac_of_nominal_8TBps": round(ach / 8000.0, 4),
                "blocked_44B_model": dict(rate(units * BYTES_OR_WAVE), bytes_per_update=BYTES_OR_WAVE) if wave else None,
                "dram_measured": dict(rate(traffic), bytes_per_launch=traffic) if traffic else None,
                "measured_over": f"{args.steps} steps with per-launch CUDA events ({profiled_ms / args.steps:.3f} "
                                 f"ms/step, directly launched)"}
    if met_n and met_ms > or_ms + hb_ms:
        # Metropolis dominates the step: its roofline is instruction issue.
        sm_count = torch.cuda.get_device_properties(local).multi_processor_count
        roof = alu_roofline(L, nh * wl["hits"], met_ms, met_n, clk, sm_count, args.steps, profiled_ms)
    kernels = {}
    for name, (ms, n), bpu, u in (("heatbath", (hb_ms, hb_n), b_hb, nh), ("overrelax", (or_ms, or_n), b_or, units),
                                  ("metropolis", (met_ms, met_n), BYTES_OR_PACKED if packed else BYTES_OR, nh)):
        if n:
            kernels[name] = {"avg_ms": round(ms / n, 5), "launches": n,
                             "GBps": round(u * bpu / (ms / n / 1e3) / 1e9, 1)}
    for name, k in (("energy", hsg.HSG_PROF_ENERGY), ("renorm", hsg.HSG_PROF_RENORM)):
        ms, n = per_class[k]
        if n:
            bpu = ((BYTES_ENERGY_PACKED if packed else BYTES_ENERGY) if name == "energy" else
                   (BYTES_RENORM_PACKED if packed else BYTES_RENORM))
            kernels[name] = {"avg_ms": round(ms / n, 5), "launches": n,
                             "GBps": round(N * bpu / (ms / n / 1e3) / 1e9, 1)}
    ms, n = per_class[hsg.HSG_PROF_OVERRELAX_RENORM]
    if n:  # the last wave sweep before a renormalisation, renormalising as it stores (same bytes, FP64 work)
        kernels["overrelax_renorm"] = {"avg_ms": round(ms / n, 5), "launches": n,
                                       "GBps": round(N * BYTES_OR_WAVE / (ms / n / 1e3) / 1e9, 1)}
    step_gbps = step_bytes(wl, wave, packed) / (elapsed_ms / args.steps / 1e3) / 1e9
    out = {
        "metric": "spin updates/ns", "value": round(value, 4), "unit": "spin updates/ns", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded Gaussian J (numpy), spins uniform on S^2 from Philox",
        "config": {"workload": wl["desc"], "L": L, "sweeps_per_step": sps, "kernel": variant,
                   "spin_layout": "packed (3 fp32 arrays per colour)" if packed else "float4",
                   "parallelism": f"samples{world}" if world > 1 else "single sample",
                   "l2": "inputs larger than L2 (state 470 MB vs 126 MB L2), no flush" if L >= 256 else
                         "state fits in L2"},
        "roofline": roof,
        "step_roofline": {"bound": "hbm", "algorithmic_bytes_per_step": step_bytes(wl, wave, packed),
                          "achieved_GBps": round(step_gbps, 1), "frac": round(step_gbps / peak, 4)},
        "kernels": kernels,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "clocks": clk,
        "energy_per_spin_last": e_last,
        "paper_context": PAPER_CONTEXT,
    }
    if world == 1 and args.workload == "l256_hb_or":
        # the batched and served forms of the path, measured in the same run
        # (after the lattice above is released): compact summaries
        if not args.no_batched:
            b = measure_batched(steps=20, warmup=3)
            out["batched"] = {k: b[k] for k in ("value", "unit", "speedup_vs_plain", "plain_one_lattice_per_launch",
                                                "hit_updates_per_ns", "lattices", "sites", "autotuned",
                                                "gpu_launches")}
            out["batched"]["workload"] = BATCH["desc"]
            p = measure_batched(steps=20, warmup=3, cfg=BATCH_L16)
            out["l16_pooled"] = {k: p[k] for k in ("value", "unit", "speedup_vs_plain", "plain_one_lattice_per_launch",
                                                   "lattices", "sites", "autotuned", "gpu_launches")}
            out["l16_pooled"]["workload"] = BATCH_L16["desc"]
        if not args.no_serving:
            m = measure_serving()
            o, sub, fifo, same = (m["overload"], m["sub_saturating"], m["plain_fifo_one_per_launch"],
                                  m["served_same_trace"])
            out["serving"] = {
                "workload": SERVE["desc"],
                "overload": {k: o[k] for k in ("requests", "rate_req_per_s", "updates_per_ns",
                                               "offered_updates_per_ns", "p50_ms", "p99_ms", "completed",
                                               "wall_s", "max_batch")},
                "sub_saturating": {k: sub[k] for k in ("requests", "rate_req_per_s", "updates_per_ns", "p50_ms",
                                                       "p99_ms", "max_batch")},
                "same_trace_served_vs_plain_fifo": {
                    "requests": same["requests"], "rate_req_per_s": fifo["rate_req_per_s"],
                    "served": {k: same[k] for k in ("p50_ms", "p99_ms", "updates_per_ns", "tick_sweeps",
                                                    "host_ms_per_tick")},
                    "plain_fifo_one_per_launch": {k: fifo[k] for k in ("p50_ms", "p99_ms", "updates_per_ns")},
                    "served_p99_over_fifo_p99": round(same["p99_ms"] / fifo["p99_ms"], 3),
                    "served_by_tick_sweeps": m["served_same_trace_by_tick_sweeps"]},
                "pool_config": m["pool_config"],
            }
    if world == 1 and not args.no_cpu_baseline:
        out["errors_vs_oracle"] = errors
        out["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# The oracle, timed on the host cores
# ---------------------------------------------------------------------------

def _oracle_setup(wl):
    import oracle
    from paper_1006_2566_gb300 import inputs

    oracle.build()
    L = wl["L"]
    J = inputs.round_to_f32(inputs.gaussian_couplings(L, seed=wl["seed"], dtype=np.float32))
    s = oracle.init_spins(L, wl["seed"])
    kind = {"HB": oracle.HB, "MET": oracle.MET, "METOR": oracle.MET_OR}.get(wl["kind"], -1)
    p = oracle.Params(key=oracle.key(wl["seed"]), sweep=0, beta=1.0 / wl["T"], step=wl["step"], hits=wl["hits"],
                      proposal=oracle.PROP_BALL if wl["proposal"] == "BALL" else oracle.PROP_SPHERE)
    return oracle, L, J, s, kind, p


def _sample_sites(L, rng, colour, n):
    """n random sites of one colour plus the lattice's corners."""
    cand = rng.integers(0, L ** 3, size=4 * n)
    x, y, z = cand % L, (cand // L) % L, cand // (L * L)
    pick = [int(i) for i in cand[(x + y + z) % 2 == colour][:n]]
    corners = [0, L - 1, L * L - 1, L ** 3 - 1, (L - 1) * L * L, L * (L - 1)]
    return pick + [i for i in corners if (i % L + (i // L) % L + i // (L * L)) % 2 == colour]


def _site_errors(oracle, L, J, before, after, sites, upd, colour, p):
    """Per-site error of one GPU half-sweep layer against the oracle's update
    of each listed site from the same state `before` (fp32 values in fp64).
    The parity rules of the tests: heat-bath sites within 1e-5 (relative)
    of the h_z = 0 plane and Metropolis sites within 1e-5 of a threshold are
    excluded (fp32 and fp64 may take different branches there); a site is
    counted as ill-conditioned when 4 kappa > 1e-5, kappa = 2^-24 sum|J| /
    |h| (its fp32 field's round-off relative to the field)."""
    u = 2.0 ** -24
    err_all, err_well, over_kappa = [], [], []
    excluded = ill = 0
    for i in sites:
        x, y, zc = i % L, (i // L) % L, i // (L * L)
        h = oracle.local_field(L, J, before, i)
        hn = float(np.linalg.norm(h))
        want, margin = oracle.update_site(upd, before[3 * i: 3 * i + 3], h, p, i, colour)
        if (upd == oracle.HB and abs(h[2]) < 1e-5 * hn) or (upd == oracle.MET and margin < 1e-5):
            excluded += 1
            continue
        bonds = [J[3 * i], J[3 * i + 1], J[3 * i + 2], J[3 * ((x - 1) % L + y * L + zc * L * L)],
                 J[3 * (x + ((y - 1) % L) * L + zc * L * L) + 1], J[3 * (x + y * L + ((zc - 1) % L) * L * L) + 2]]
        kappa = u * float(np.sum(np.abs(bonds))) / max(hn, 1e-300)
        e = float(np.max(np.abs(after[3 * i: 3 * i + 3] - want)))
        err_all.append(e)
        over_kappa.append(e / kappa)
        if 4 * kappa <= 1e-5:
            err_well.append(e)
        else:
            ill += 1
    return {"sites": len(sites), "excluded": excluded, "ill_conditioned": ill,
            "max_abs_err": max(err_all), "max_abs_err_well_conditioned": max(err_well),
            "max_err_over_kappa": round(max(over_kappa), 3)}


def errors_vs_oracle(hsg, lat, J_in, wl, e_last):
    """The error of each reported quantity against the FP64 oracle, measured
    after the timed region on the benchmark's own lattice (the oracle leg):
    the logged E/N against the oracle's energy of the same spins; one
    main-update half-sweep (colour 0) and one over-relaxation sweep of the
    kernel the benchmark times (colour 0 from the state before it, colour 1
    from the GPU's own new colour 0) at >= 3000 sampled sites per layer; and
    the FP64 renormalisation of the whole lattice against the oracle's.
    The oracle is fed the couplings the lattice holds (the input rounded to
    fp32); with fp64 input, what that rounding alone changes in E/N is
    reported apart."""
    import oracle

    oracle.build()
    L, N = wl["L"], wl["L"] ** 3
    J = np.asarray(J_in, dtype=np.float32).astype(np.float64)
    rng = np.random.default_rng(7)
    out = {"rules": "max |diff| per spin component at each sampled site; heat-bath frame-branch band and "
                    "Metropolis near-threshold sites excluded; ill-conditioned = 4 kappa > 1e-5, kappa = "
                    "2^-24 sum|J| / |h|"}
    s_end = lat.spins().astype(np.float64)
    if wl["energy_every"]:
        e_ref = oracle.energy(L, J, s_end) / N
        out["energy_per_spin"] = {"gpu": e_last, "oracle": e_ref, "abs_err": abs(e_last - e_ref)}
    if np.asarray(J_in).dtype == np.float64:
        e_raw = oracle.energy(L, np.asarray(J_in), s_end) / N
        out["fp64_coupling_rounding"] = {"energy_per_spin_raw_fp64_J": e_raw,
                                         "abs_diff_vs_rounded_J": abs(e_raw - oracle.energy(L, J, s_end) / N)}
    # FP64 renormalisation of the current state against the oracle's
    lat.renorm()
    got = lat.spins().astype(np.float64)
    ref = s_end.copy()
    oracle.renorm(L, ref)
    norms = np.linalg.norm(got.reshape(-1, 3), axis=1)
    out["renorm"] = {"sites": N, "max_abs_err": float(np.max(np.abs(got - ref))),
                     "max_norm_deviation": float(np.max(np.abs(norms - 1.0)))}
    # one main-update half-sweep on colour 0
    upd = {"HB": oracle.HB, "MET": oracle.MET}.get(wl["kind"])
    if upd is not None:
        sched = hsg.schedule(kind=hsg.HSG_HEATBATH if upd == oracle.HB else hsg.HSG_METROPOLIS, hits=wl["hits"],
                             proposal=hsg.HSG_PROP_BALL if wl["proposal"] == "BALL" else hsg.HSG_PROP_SPHERE,
                             step=wl["step"], T=wl["T"])
        before = got
        sweep = lat.sweep_count
        lat.half_sweep(sched, sched.kind, 0)
        got = lat.spins().astype(np.float64)
        p = oracle.Params(key=oracle.key(wl["seed"]), sweep=sweep, beta=1.0 / wl["T"], step=wl["step"],
                          hits=wl["hits"], proposal=oracle.PROP_BALL if wl["proposal"] == "BALL" else
                          oracle.PROP_SPHERE)
        name = "heatbath_half_sweep" if upd == oracle.HB else "metropolis_half_sweep"
        out[name] = _site_errors(oracle, L, J, before, got, _sample_sites(L, rng, 0, 3000), upd, 0, p)
    # one over-relaxation sweep with the kernel the benchmark's OR sweeps use
    if wl["n_or"]:
        before = got
        lat.sweep(hsg.schedule(kind=hsg.HSG_NONE, n_or=1, kernel=hsg.HSG_KERNEL_AUTO), 1)
        got = lat.spins().astype(np.float64)
        mid = np.where(np.repeat(np.indices((L, L, L)).sum(axis=0).reshape(-1) % 2 == 0, 3), got, before)
        p = oracle.Params()
        out["overrelax_sweep"] = {
            "colour0": _site_errors(oracle, L, J, before, got, _sample_sites(L, rng, 0, 3000), oracle.OR, 0, p),
            "colour1_from_gpu_colour0": _site_errors(oracle, L, J, mid, got, _sample_sites(L, rng, 1, 3000),
                                                     oracle.OR, 1, p)}
    return out


def _oracle_sample_sweep(oracle, L, J, s, kind, p, i0, i1):
    """One sweep of the schedule restricted to sites [i0, i1): main update on
    both colours, then the OR sweeps.  Returns the site updates done."""
    n = 0
    if kind >= 0:
        for c in (0, 1):
            oracle.half_sweep_range(L, J, s, kind, c, p, i0, i1)
        n += (i1 - i0) * (2 if kind == oracle.MET_OR else 1)
    return n


def cpu_baseline(wl, target_s: float = 10.0):
    """Full sweeps of the workload's lattice by the FP64 oracle on one
    thread -- as many as it takes to pass target_s seconds (two at L = 256
    on a Grace core, about 12 s) -- and one on every host core (the oracle's
    OpenMP half-sweep loop; the same arithmetic)."""
    oracle, L, J, s, kind, p = _oracle_setup(wl)
    N = L ** 3

    def sweep():
        t = time.perf_counter()
        updates = _oracle_sample_sweep(oracle, L, J, s, kind, p, 0, N)
        for _ in range(wl["n_or"]):
            for c in (0, 1):
                oracle.half_sweep(L, J, s, oracle.OR, c, p)
            updates += N
        return updates, time.perf_counter() - t

    updates = n_sweeps = 0
    dt = 0.0
    while dt < target_s:
        u, t = sweep()
        updates, dt, n_sweeps = updates + u, dt + t, n_sweeps + 1
    out = {"value": round(updates / (dt * 1e9), 6), "unit": "spin updates/ns", "cores": 1, "kind": "oracle",
           "sample": f"{n_sweeps} full sweep(s) (main update + {wl['n_or']} OR) of the L={L} lattice, fp64, "
                     f"1 thread, until {target_s:.0f} s had passed",
           "seconds": round(dt, 2)}
    cores = oracle.max_threads()
    if cores > 1:
        oracle.set_threads(cores)
        try:
            updates, dt = sweep()
        finally:
            oracle.set_threads(1)
        out["all_cores"] = {"value": round(updates / (dt * 1e9), 6), "cores": cores, "seconds": round(dt, 2),
                            "sample": "the same sweep, OpenMP over the sites of each half-sweep"}
    return out


def run_reference(args, wl):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    oracle, L, J, s, kind, p = _oracle_setup(wl)
    cores = oracle.max_threads()
    oracle.set_threads(cores)  # every host core (OpenMP over each half-sweep's sites)
    planes = max(1, L // 16) * (4 if cores >= 8 else 1)
    i1 = planes * L * L  # z-planes [0, planes)
    per_step = 0

    def step():
        n = _oracle_sample_sweep(oracle, L, J, s, kind, p, 0, i1)
        for _ in range(wl["n_or"]):
            for c in (0, 1):
                oracle.half_sweep_range(L, J, s, oracle.OR, c, p, 0, i1)
            n += i1
        return n

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        per_step = step()
    dt = time.perf_counter() - t
    value = per_step * args.steps / (dt * 1e9)
    sample = (f"per step: 1 sweep (main update + {wl['n_or']} OR) of z-planes [0,{planes}) of the L={L} lattice "
              f"({i1} sites), fp64 oracle, {cores} threads (OpenMP over each half-sweep's sites)")
    out = {"impl": "reference", "metric": "spin updates/ns", "value": round(value, 6), "unit": "spin updates/ns",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic: seeded Gaussian J, spins from Philox",
           "config": {"workload": wl["desc"], "L": L, "kernel": "oracle"},
           "cpu_baseline": {"value": round(value, 6), "unit": "spin updates/ns", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 6), "unit": "spin updates/ns", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# Batched workload: many small lattices in one pool
# ---------------------------------------------------------------------------

BATCH = dict(samples=512, replicas=2, sides=(16, 24, 32, 48), seed=4, hits=4, proposal="BALL", step=0.5, n_or=2,
             renorm_every=10, sweeps_per_step=10, T=None,
             desc=("batched: 512 samples x 2 replicas, L uniform in {16,24,32,48} (seeded), T_s = 0.2 + 0.8 s/511, "
                   "Gaussian J per sample (device Philox + Box-Muller), 4-hit Metropolis (ball, 0.5) + 2 OR per "
                   "sweep, renorm every 10; one pool, one graph replay per sweep; 1 step = 10 sweeps"))
# The L = 16 single-lattice workload (l16_met: 1-hit Metropolis, uniform-
# sphere proposal, T = 1) as it is meant to run: many independent samples
# in one pool.
BATCH_L16 = dict(samples=2048, replicas=1, sides=(16,), seed=1, hits=1, proposal="SPHERE", step=0.5, n_or=0,
                 renorm_every=0, sweeps_per_step=10, T=1.0,
                 desc=("pooled L=16: 2048 independent samples of the L=16 workload (Gaussian J per sample from device "
                       "Philox + Box-Muller; checkerboard Metropolis 1 hit, uniform-sphere proposal, T=1.0), one pool, "
                       "one graph replay per sweep; 1 step = 10 sweeps"))


def batch_specs(cfg=BATCH):
    """(L, seed, sample, replica, T) of every lattice of a batched workload:
    sides drawn from cfg["sides"] (seeded), T fixed or ramped over the
    samples from 0.2 to 1.0."""
    rng = np.random.default_rng([cfg["seed"], 0x4C])
    sides = rng.choice(cfg["sides"], size=cfg["samples"])
    out = []
    for s in range(cfg["samples"]):
        T = cfg["T"] if cfg["T"] is not None else 0.2 + 0.8 * s / (cfg["samples"] - 1)
        for r in range(cfg["replicas"]):
            out.append((int(sides[s]), cfg["seed"], s, r, T))
    return out


def measure_batched(steps: int, warmup: int, autotune: bool = True, cfg=BATCH) -> dict:
    """A batched workload in one pool (graph-replayed sweeps, autotuned
    launch shape) against one lattice per launch, on the current device."""
    import torch

    from paper_1006_2566_gb300 import hsg

    specs = batch_specs(cfg)
    sites = sum(L ** 3 for L, *_ in specs)
    prop = hsg.HSG_PROP_BALL if cfg["proposal"] == "BALL" else hsg.HSG_PROP_SPHERE
    sched = hsg.schedule(kind=hsg.HSG_METROPOLIS, hits=cfg["hits"], proposal=prop, step=cfg["step"],
                         n_or=cfg["n_or"], renorm_every=cfg["renorm_every"])
    sps = cfg["sweeps_per_step"]
    passes = 1 + cfg["n_or"]
    stream = torch.cuda.Stream()
    budget = int(sum(28 * L ** 3 for L, *_ in specs) * 1.05) + (1 << 24)
    with hsg.Pool(budget, len(specs), stream) as pool:
        for spec in specs:
            pool.admit(*spec)
        t0 = time.perf_counter()
        if not autotune:
            tcfg = (256, 512, 8, 0)  # the pool's default launch configuration
            hsg.hsg_pool_config(pool.pool, *tcfg)
        else:
            tcfg = hsg.hsg_pool_autotune(pool.pool, sched)
        tune_s = time.perf_counter() - t0
        for _ in range(warmup):
            pool.sweep(sched, sps)
        torch.cuda.synchronize()
        n0 = hsg.hsg_pool_launch_count(pool.pool)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            pool.sweep(sched, sps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = hsg.hsg_pool_launch_count(pool.pool) - n0
        energies = pool.energies()
    value = sites * passes * sps * steps / (ms * 1e6)
    # one lattice per launch: every lattice of a representative subset swept
    # on its own context, one after another
    sub = specs[:: max(1, len(specs) // 64)]
    sub_sites = sum(L ** 3 for L, *_ in sub)
    ctxs = []
    for (L, seed, sample, replica, T) in sub:
        lat = hsg.Lattice(L, seed, sample, replica, stream)
        lat.generate_couplings()
        ctxs.append((lat, hsg.schedule(kind=hsg.HSG_METROPOLIS, hits=cfg["hits"], proposal=prop, step=cfg["step"],
                                       n_or=cfg["n_or"], T=T, renorm_every=cfg["renorm_every"])))
    for lat, s in ctxs:
        lat.sweep(s, 1)
    torch.cuda.synchronize()
    e0.record(stream)
    for lat, s in ctxs:
        lat.sweep(s, sps)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    for lat, _ in ctxs:
        lat.close()
    plain = sub_sites * passes * sps / (plain_ms * 1e6)
    return {"value": round(value, 4), "unit": "spin updates/ns", "steps": steps, "ms_per_step": round(ms / steps, 4),
            "lattices": len(specs), "sites": sites,
            "autotuned": {"threads": tcfg[0], "tile_sites": tcfg[1], "blocks_per_sm": tcfg[2],
                          "hits_per_pass": tcfg[3] or cfg["hits"], "seconds": round(tune_s, 3)} if autotune else None,
            "hit_updates_per_ns": round(sites * (cfg["hits"] + cfg["n_or"]) * sps * steps / (ms * 1e6), 4),
            "plain_one_lattice_per_launch": {"value": round(plain, 4), "unit": "spin updates/ns",
                                             "lattices": len(sub), "sites": sub_sites,
                                             "ms_for_10_sweeps": round(plain_ms, 3)},
            "speedup_vs_plain": round(value / plain, 2), "gpu_launches": int(launches),
            "energy_per_spin_mean": float(np.nanmean(energies))}


def run_batched(args, cfg=BATCH):
    import torch

    from paper_1006_2566_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    b = measure_batched(args.steps, args.warmup, not args.no_autotune, cfg)
    out = {
        "metric": "spin updates/ns", "value": b["value"], "unit": "spin updates/ns", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded sides and temperatures, couplings and spins from Philox",
        "config": {"workload": cfg["desc"], "lattices": b["lattices"], "sites": b["sites"],
                   "autotuned": b["autotuned"]},
        "hit_updates_per_ns": b["hit_updates_per_ns"],
        "plain_one_lattice_per_launch": b["plain_one_lattice_per_launch"],
        "speedup_vs_plain": b["speedup_vs_plain"], "gpu_launches": b["gpu_launches"],
        "energy_per_spin_mean": b["energy_per_spin_mean"],
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# Serving workload: a Poisson stream of solves through the request loop
# ---------------------------------------------------------------------------

SERVE = dict(rate=2000.0, n_overload=800, n_sub=300, n_plain=100, seed=5, budget=60 * 10 ** 9, max_slots=4096,
             desc=("serving: Poisson arrivals (mean 2000 req/s, seeded), each a fresh sample with L uniform in "
                   "{16..96 step 8}, T uniform [0.2,1.0], sweeps uniform [50,500]; per sweep 4-hit Metropolis "
                   "(ball, 0.5) + 2 OR; lattices resident in a 60 GB pool, admitted in arrival order as memory "
                   "frees; continuous batching"))


def measure_serving(n_overload: int = SERVE["n_overload"], n_sub: int = SERVE["n_sub"],
                    n_plain: int = SERVE["n_plain"], tick_sweeps=(1, 3, 30)) -> dict:
    """The serving workload on the current device: an overload trace at the
    configured rate (throughput against offered load), a sub-saturating
    trace at 0.6 x the measured capacity, and its first n_plain requests
    both served and one per launch in arrival order (p50/p99 side by side),
    then served again with each tick length in `tick_sweeps`."""
    import torch

    from paper_1006_2566_gb300 import hsg, serve

    kw = dict(kind=hsg.HSG_METROPOLIS, hits=4, proposal=hsg.HSG_PROP_BALL, step=0.5, n_or=2, renorm_every=10)
    stream = torch.cuda.Stream()
    # warm-up: a short trace (builds graphs, pages in the arena) whose pool
    # autotunes its launch configuration once; the measured traces start with
    # that configuration instead of tuning while their requests wait
    _, st_w = serve.serve(serve.poisson_trace(40, SERVE["rate"], seed=99, first_sample=10 ** 6), kw,
                          SERVE["budget"], SERVE["max_slots"], stream)
    cfg = st_w.extra["config"]
    over = serve.poisson_trace(n_overload, SERVE["rate"], seed=SERVE["seed"])
    res_o, st_o = serve.serve(over, kw, SERVE["budget"], SERVE["max_slots"], stream, config=cfg)
    capacity = st_o.completed / st_o.wall_seconds  # requests per second at saturation
    sub_rate = 0.6 * capacity
    sub = serve.poisson_trace(n_sub, sub_rate, seed=SERVE["seed"] + 1, first_sample=10 ** 5)
    res_s, st_s = serve.serve(sub, kw, SERVE["budget"], SERVE["max_slots"], stream, config=cfg)
    plain_trace = sub[:n_plain]
    res_p, st_p = serve.serve_fifo(plain_trace, kw, stream)
    res_b, st_b = serve.serve(plain_trace, kw, SERVE["budget"], SERVE["max_slots"], stream, config=cfg)
    # the same trace at other tick lengths (sweeps queued per loop iteration)
    by_tick = {}
    for tick in tick_sweeps:
        _, st_t = serve.serve(plain_trace, kw, SERVE["budget"], SERVE["max_slots"], stream, tick_sweeps=tick,
                              config=cfg)
        by_tick[str(tick)] = {"p50_ms": round(st_t.p50_ms, 2), "p99_ms": round(st_t.p99_ms, 2),
                              "ticks": st_t.ticks, "host_ms_per_tick": round(st_t.extra["host_ms_per_tick"], 3)}
    passes = 3
    offered = sum(r.L ** 3 * r.sweeps * passes for r in over) / (over[-1].arrival * 1e9)

    def block(st):
        out = {"completed": st.completed, "wall_s": round(st.wall_seconds, 3),
               "updates_per_ns": round(st.updates_per_ns, 3), "p50_ms": round(st.p50_ms, 2),
               "p99_ms": round(st.p99_ms, 2), "mean_ms": round(st.mean_ms, 2), "max_batch": st.max_batch,
               "ticks": st.ticks}
        if "host_ms_per_tick" in st.extra:
            out["host_ms_per_tick"] = round(st.extra["host_ms_per_tick"], 3)
        return out

    return {
        "overload": dict(block(st_o), offered_updates_per_ns=round(offered, 2), rate_req_per_s=SERVE["rate"],
                         requests=len(over)),
        "sub_saturating": dict(block(st_s), rate_req_per_s=round(sub_rate, 1), requests=len(sub)),
        "plain_fifo_one_per_launch": dict(block(st_p), requests=len(plain_trace), rate_req_per_s=round(sub_rate, 1)),
        "served_same_trace": dict(block(st_b), requests=len(plain_trace), tick_sweeps=10),
        "served_same_trace_by_tick_sweeps": by_tick,
        "pool_config": None if cfg is None else dict(zip(("threads", "tile_sites", "blocks_per_sm", "hits_per_pass"),
                                                         cfg)),
    }


def run_serving(args):
    import torch

    from paper_1006_2566_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    m = measure_serving()
    out = {
        "metric": "spin updates/ns", "value": m["overload"]["updates_per_ns"], "unit": "spin updates/ns",
        "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded Poisson trace; couplings and spins from Philox",
        "config": {"workload": SERVE["desc"]}, **m,
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.workload in ("batched", "l16_pooled"):
        run_batched(args, BATCH if args.workload == "batched" else BATCH_L16)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
