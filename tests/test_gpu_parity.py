"""GPU path vs the FP64 oracle, through the C ABI (needs a CUDA GPU).

The tolerances are the parity rules of tests/parity_rules.py: per site and
per half-sweep layer, 1e-5 per spin component, Metropolis sites within 1e-5
of a threshold and heat-bath sites in the frame-branch band left out, the
other colour bit-identical; whole sweeps are checked layer by layer, each
layer of the oracle starting from the GPU's own state before it.  Energies:
|E/N difference| <= 2e-6 (per-site terms are fp32).  Long runs: mean E/N
within 3 sigma (binned errors of both runs).  Every half-sweep starts the
GPU and the oracle from the same state (fp32 values, the oracle holding them
in fp64) and the same fp32-rounded J.
"""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1006_2566_gb300 import inputs  # noqa: E402
from parity_rules import (check_half_sweep, check_layer, check_or_sweep, colour_mask, frame_band,  # noqa: E402
                          record)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = 1e-5


@pytest.fixture(scope="module")
def hsg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_2566_gb300 import build

    build.build()
    oracle.build()
    from paper_1006_2566_gb300 import hsg as h

    return h


VARIANTS = [1, 2]  # HSG_KERNEL_GLOBAL, HSG_KERNEL_SLAB


def gpu_half_sweep(hsg, L, J, s32, update, colour, sched, seed=7, sample=0, replica=0, sweep=0):
    with hsg.Lattice(L, seed, sample, replica) as lat:
        lat.set_couplings(J)
        lat.set_spins(s32)
        lat.sweep_count = sweep
        lat.half_sweep(sched, update, colour)
        return lat.spins().astype(np.float64)


def oracle_state(L, seed_j, seed_s):
    J = inputs.gaussian_couplings(L, seed=seed_j)
    s32 = inputs.random_spins(L, seed=seed_s, dtype=np.float32)
    return J, s32


# ---------------------------------------------------------------------------
# Philox
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def curand_lib():
    d = tempfile.mkdtemp(prefix="hsg_curand_")
    so = os.path.join(d, "curand_philox.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-Xcompiler", "-fPIC", "-shared",
                    "-o", so, os.path.join(ROOT, "tests", "native", "curand_philox.cu")], check=True)
    lib = ctypes.CDLL(so)
    lib.curand_philox_fill.argtypes = [ctypes.c_uint32] * 6 + [ctypes.c_void_p]
    lib.curand_philox_fill.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("seed,sample,replica,c1,c2,c3", [
    (1, 0, 0, 0, (1 << 24), 0),
    (0xDEADBEEF12345678, 3, 1, 77, (3 << 24) | (1 << 16) | 5, 9),
])
def test_philox_device_matches_curand_and_oracle(hsg, curand_lib, seed, sample, replica, c1, c2, c3):
    n = 1 << 20
    mine = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    ref = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    hsg.hsg_philox(seed, sample, replica, c1, c2, c3, mine)
    k = oracle.key(seed, sample, replica)
    assert curand_lib.curand_philox_fill(k[0], k[1], c1, c2, c3, n, ref.data_ptr()) == 0
    torch.cuda.synchronize()
    a = mine.cpu().numpy().view(np.uint32).reshape(n, 4)
    b = ref.cpu().numpy().view(np.uint32).reshape(n, 4)
    assert np.array_equal(a, b)  # all 2^20 counters, bit for bit
    rng = np.random.default_rng(1)
    for t in list(range(64)) + list(rng.integers(0, n, 2000)) + [n - 1]:
        assert list(oracle.philox4x32_10((int(t), c1, c2, c3), k)) == list(b[t])


# ---------------------------------------------------------------------------
# Initial state and layout
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L,seed,sample,replica", [(4, 1, 0, 0), (16, 1, 0, 0), (24, 9, 5, 1), (66, 3, 0, 1)])
def test_initial_spins_match_oracle(hsg, L, seed, sample, replica):
    with hsg.Lattice(L, seed, sample, replica) as lat:
        got = lat.spins().astype(np.float64)
    ref = oracle.init_spins(L, seed, sample, replica)
    assert np.max(np.abs(got - ref)) < 1e-6


@pytest.mark.parametrize("L", [4, 6, 40])
def test_spin_layout_round_trip_is_exact(hsg, L):
    s = inputs.random_spins(L, seed=5, dtype=np.float32)
    with hsg.Lattice(L, 1) as lat:
        lat.set_spins(s)
        assert np.array_equal(lat.spins(), s)
        dev = torch.from_numpy(s).cuda()
        lat.set_spins(dev)
        out = torch.zeros_like(dev)
        hsg.hsg_get_spins(lat.ctx, out)
        torch.cuda.synchronize()
        assert torch.equal(out, dev)


# ---------------------------------------------------------------------------
# Half-sweeps
# ---------------------------------------------------------------------------

OR_SIZES = [4, 6, 8, 16, 24, 40, 66]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("L", OR_SIZES)
def test_over_relaxation_half_sweep_parity(hsg, variant, L):
    J, s32 = oracle_state(L, 100 + L, 200 + L)
    Jr = inputs.round_to_f32(J)
    sched = hsg.schedule(kernel=variant)
    for colour in (0, 1):
        got = gpu_half_sweep(hsg, L, J, s32, hsg.HSG_OVERRELAX, colour, sched)
        check_layer(L, Jr, s32, got, oracle.OR, colour, oracle.Params(), label=f"OR half-sweep L={L} v{variant}")


MET_CASES = [
    # (L, proposal, hits, T)
    (6, 0, 1, 1.0),
    (16, 0, 1, 1.0),
    (16, 1, 4, 0.5),
    (40, 1, 4, 0.5),
    (66, 0, 3, 0.3),
    (24, 1, 2, math.inf),
    (16, 1, 4, 0.01),  # beta = 100: exp(-beta dE) underflows for most uphill proposals
]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("case", MET_CASES)
def test_metropolis_half_sweep_parity(hsg, variant, case):
    L, proposal, hits, T = case
    J, s32 = oracle_state(L, 300 + L, 400 + L)
    Jr = inputs.round_to_f32(J)
    sched = hsg.schedule(kind=hsg.HSG_METROPOLIS, hits=hits, proposal=proposal, step=0.5, T=T, kernel=variant)
    beta = 0.0 if math.isinf(T) else 1.0 / T
    for colour in (0, 1):
        got = gpu_half_sweep(hsg, L, J, s32, hsg.HSG_METROPOLIS, colour, sched, seed=11, sweep=3)
        p = oracle.Params(key=oracle.key(11), sweep=3, beta=beta, step=0.5, hits=hits, proposal=proposal)
        check_layer(L, Jr, s32, got, oracle.MET, colour, p,
                    label=f"Metropolis half-sweep L={L} prop={proposal} hits={hits} T={T} v{variant}")
        moved = np.any(got.reshape(-1, 3) != s32.astype(np.float64).reshape(-1, 3), axis=1)
        assert moved[colour_mask(L, colour)].mean() > 0.05  # the chain does move


FUSED_CASES = [(16, 0, 1, 1.0), (24, 1, 4, 0.5), (40, 1, 2, 0.3)]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("case", FUSED_CASES)
def test_fused_metropolis_or_half_sweep_parity(hsg, variant, case):
    """The opt-in fused colour pass (Metropolis hits, then one reflection
    about the same field) against the oracle's MET_OR mode."""
    L, proposal, hits, T = case
    J, s32 = oracle_state(L, 910 + L, 920 + L)
    Jr = inputs.round_to_f32(J)
    sched = hsg.schedule(kind=hsg.HSG_METROPOLIS_OR, hits=hits, proposal=proposal, step=0.5, T=T, kernel=variant)
    for colour in (0, 1):
        got = gpu_half_sweep(hsg, L, J, s32, hsg.HSG_METROPOLIS_OR, colour, sched, seed=31, sweep=4)
        p = oracle.Params(key=oracle.key(31), sweep=4, beta=1.0 / T, step=0.5, hits=hits, proposal=proposal)
        check_layer(L, Jr, s32, got, oracle.MET_OR, colour, p,
                    label=f"fused Metropolis+OR half-sweep L={L} hits={hits} T={T} v{variant}")


def test_fused_long_run_energy_statistics_match_oracle(hsg):
    """L = 12, fused Metropolis (ball, 2 hits) + reflection at T = 0.7 for
    1200 sweeps: mean E/N agrees with the oracle's within 3 sigma."""
    L, n = 12, 1200
    J = inputs.gaussian_couplings(L, seed=33)
    with hsg.Lattice(L, 33) as lat:
        lat.set_couplings(J)
        lat.sweep(hsg.schedule(kind=hsg.HSG_METROPOLIS_OR, hits=2, proposal=1, T=0.7, energy_every=1), n)
        g = lat.energy_log()
    s = oracle.init_spins(L, 33)
    _, r = oracle.sweeps(L, inputs.round_to_f32(J), s,
                         oracle.Schedule(kind=oracle.MET_OR, hits=2, proposal=1, beta=1 / 0.7, energy_every=1),
                         oracle.key(33), n)

    def binned(x):
        b = np.array([v.mean() for v in np.array_split(x[n // 5:], 20)])
        return b.mean(), b.std(ddof=1) / np.sqrt(len(b))

    mg, eg = binned(g)
    mr, er = binned(r)
    assert abs(mg - mr) < 3 * math.hypot(eg, er) + 1e-6, (mg, eg, mr, er)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("L,T", [(6, 1.0), (16, 0.3), (40, 0.3), (66, 1.0), (16, math.inf), (16, 0.01), (40, 3.0),
                                 (66, 10.0), (40, 100.0)])
def test_heatbath_half_sweep_parity(hsg, variant, L, T):
    J, s32 = oracle_state(L, 500 + L, 600 + L)
    Jr = inputs.round_to_f32(J)
    sched = hsg.schedule(kind=hsg.HSG_HEATBATH, T=T, kernel=variant)
    beta = 0.0 if math.isinf(T) else 1.0 / T
    for colour in (0, 1):
        got = gpu_half_sweep(hsg, L, J, s32, hsg.HSG_HEATBATH, colour, sched, seed=13, sample=2, sweep=5)
        p = oracle.Params(key=oracle.key(13, 2), sweep=5, beta=beta)
        check_layer(L, Jr, s32, got, oracle.HB, colour, p, label=f"heat-bath half-sweep L={L} T={T} v{variant}")
        mask = colour_mask(L, colour)
        assert np.max(np.abs(np.linalg.norm(got.reshape(-1, 3)[mask], axis=1) - 1)) < 1e-5


@pytest.mark.parametrize("variant", VARIANTS)
def test_zero_field_half_sweeps(hsg, variant):
    """All couplings zero, so h = 0 at every site at a finite temperature
    (the degenerate case of the field): over-relaxation leaves every spin
    as it is, bit for bit; the heat-bath draws uniformly on the sphere
    (1/|h| is infinite there, not beta = 0); Metropolis accepts every
    proposal (dE = 0).  Heat-bath and Metropolis against the oracle."""
    L = 8
    J = np.zeros(3 * L ** 3)
    s32 = inputs.random_spins(L, seed=77, dtype=np.float32)
    s64 = s32.astype(np.float64)
    for colour in (0, 1):
        mask = colour_mask(L, colour)
        got = gpu_half_sweep(hsg, L, J, s32, hsg.HSG_OVERRELAX, colour, hsg.schedule(kernel=variant))
        assert np.array_equal(got, s64)

        got = gpu_half_sweep(hsg, L, J, s32, hsg.HSG_HEATBATH, colour,
                             hsg.schedule(kind=hsg.HSG_HEATBATH, T=0.5, kernel=variant), seed=19, sweep=2)
        ref = s64.copy()
        oracle.half_sweep(L, J, ref, oracle.HB, colour, oracle.Params(key=oracle.key(19), sweep=2, beta=2.0))
        assert np.max(np.abs(got - ref)) <= TOL
        assert np.all(np.any(got.reshape(-1, 3)[mask] != s64.reshape(-1, 3)[mask], axis=1))

        sched = hsg.schedule(kind=hsg.HSG_METROPOLIS, hits=2, proposal=hsg.HSG_PROP_BALL, step=0.5, T=0.5,
                             kernel=variant)
        got = gpu_half_sweep(hsg, L, J, s32, hsg.HSG_METROPOLIS, colour, sched, seed=19, sweep=2)
        ref = s64.copy()
        p = oracle.Params(key=oracle.key(19), sweep=2, beta=2.0, step=0.5, hits=2, proposal=oracle.PROP_BALL)
        margins = oracle.half_sweep(L, J, ref, oracle.MET, colour, p, want_margins=True)
        near = mask & (margins < TOL)
        assert near.sum() <= 2
        err = np.max(np.abs(got - ref).reshape(-1, 3), axis=1)
        assert np.all(err[mask & ~near] <= TOL)
        assert np.all(np.any(ref.reshape(-1, 3)[mask] != s64.reshape(-1, 3)[mask], axis=1))  # every site moved


# L = 4 .. 66: the heat-bath column march shorter than, and ragged in, its
# 6-plane chunks; the slab kernel's z chunk (chosen at launch to fill the
# GPU) is one plane up to L = 40, two at 66, and seven at 128 with a ragged
# last chunk of two planes.
@pytest.mark.parametrize("L", [4, 8, 14, 40, 66, 128])
def test_kernel_variants_are_bit_identical(hsg, L):
    J = inputs.gaussian_couplings(L, seed=3)
    out = []
    for variant in VARIANTS:
        with hsg.Lattice(L, 3) as lat:
            lat.set_couplings(J)
            lat.sweep(hsg.schedule(kind=hsg.HSG_HEATBATH, T=0.5, n_or=2, kernel=variant), 3)
            lat.sweep(hsg.schedule(kind=hsg.HSG_METROPOLIS, hits=2, proposal=1, T=0.5, n_or=1, kernel=variant), 2)
            out.append(lat.spins())
    assert np.array_equal(out[0], out[1])


# ---------------------------------------------------------------------------
# Energy and renormalisation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L", [4, 6, 16, 40, 66])
def test_energy_matches_oracle(hsg, L):
    J, s32 = oracle_state(L, 700 + L, 800 + L)
    with hsg.Lattice(L, 1) as lat:
        lat.set_couplings(J)
        lat.set_spins(s32)
        e = lat.energy()
    ref = oracle.energy(L, inputs.round_to_f32(J), s32.astype(np.float64)) / L ** 3
    assert abs(e - ref) <= 2e-6


def test_energy_closed_forms(hsg):
    L = 6
    with hsg.Lattice(L, 1) as lat:
        lat.set_couplings(inputs.uniform_couplings(L))
        lat.set_spins(inputs.aligned_spins(L, (0.0, 0.6, 0.8), dtype=np.float32))
        assert abs(lat.energy() + 3.0) < 1e-6
        for axis in range(3):
            ang = 2 * np.pi / L
            s = np.zeros((L, L, L, 3))
            coord = np.indices((L, L, L))[2 - axis]
            s[..., 0], s[..., 1] = np.cos(ang * coord), np.sin(ang * coord)
            lat.set_couplings(inputs.uniform_couplings(L, axes=(axis,)))
            lat.set_spins(s.reshape(-1).astype(np.float32))
            assert abs(lat.energy() + np.cos(ang)) < 1e-6


@pytest.mark.parametrize("scale", ["far", "near"])
def test_renorm_matches_oracle(hsg, scale):
    """Far from unit length (fp64 reciprocal square root) and within fp32
    round-off of it (the series branch): within 1 ulp of the fp64 result."""
    L = 16
    rng = np.random.default_rng(4)
    if scale == "far":
        f = rng.uniform(0.5, 2.0, size=(L ** 3, 1))
    else:
        f = 1.0 + rng.uniform(-3e-7, 3e-7, size=(L ** 3, 1))
        f[:10] = 1.0 + 0.003  # just inside the series branch
    s = (inputs.random_spins(L, seed=9).reshape(-1, 3) * f).reshape(-1)
    s32 = s.astype(np.float32)
    with hsg.Lattice(L, 1) as lat:
        lat.set_spins(s32)
        lat.renorm()
        got = lat.spins()
    ref = s32.astype(np.float64)
    oracle.renorm(L, ref)
    assert np.max(np.abs(got.astype(np.float64) - ref)) <= 2 ** -24
    assert np.max(np.abs(np.linalg.norm(got.astype(np.float64).reshape(-1, 3), axis=1) - 1)) < 2e-7


# ---------------------------------------------------------------------------
# Whole sweeps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("kind", ["HB", "MET", "METOR"])
def test_sweep_is_the_composition_of_half_sweeps(hsg, variant, kind):
    """hsg_sweep = main update on colour 0 then 1, n_or OR sweeps, counter
    advance, renormalisation, energy log: bit-identical to issuing the same
    half-sweeps one by one."""
    L = 24
    J = inputs.gaussian_couplings(L, seed=19)
    k = {"HB": hsg.HSG_HEATBATH, "MET": hsg.HSG_METROPOLIS, "METOR": hsg.HSG_METROPOLIS_OR}[kind]
    sched = hsg.schedule(kind=k, hits=3, proposal=1, T=0.8, n_or=2, renorm_every=2, energy_every=1, kernel=variant)
    with hsg.Lattice(L, 19) as a:
        a.set_couplings(J)
        a.sweep(sched, 3)
        want, want_log = a.spins(), a.energy_log()
    with hsg.Lattice(L, 19) as b:
        b.set_couplings(J)
        got_log = []
        for sw in range(3):
            b.sweep_count = sw
            for c in (0, 1):
                b.half_sweep(sched, k, c)
            for _ in range(2):
                for c in (0, 1):
                    b.half_sweep(sched, hsg.HSG_OVERRELAX, c)
            if (sw + 1) % 2 == 0:
                b.renorm()
            got_log.append(b.energy())
        assert np.array_equal(b.spins(), want)
        assert np.array_equal(np.array(got_log), want_log)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("L", [24, 40])
def test_over_relaxation_sweep_matches_oracle(hsg, variant, L):
    """One over-relaxation sweep (colour 0, then colour 1) from the same
    state through hsg_sweep, every site of both layers under the half-sweep
    rules: colour 0 against the oracle's half-sweep of the start state,
    colour 1 against the oracle's half-sweep of the GPU's own new colour 0
    (the state the GPU's colour-1 layer started from)."""
    J, s32 = oracle_state(L, 900 + L, 901 + L)
    Jr = inputs.round_to_f32(J)
    with hsg.Lattice(L, 17) as lat:
        lat.set_couplings(J)
        lat.set_spins(s32)
        lat.sweep(hsg.schedule(kind=hsg.HSG_NONE, n_or=1, kernel=variant), 1)
        got = lat.spins()
    check_or_sweep(L, Jr, s32, got, label=f"OR sweep L={L} v{variant}")


def layered_run(hsg, lat, sched, main, n_or, n_sweeps, renorm_every, energy_every):
    """The GPU's state after every layer of `n_sweeps` sweeps, issued as
    half-sweeps one by one (bit-identical to hsg_sweep, tested above):
    a list of (layer, state before, state after) and the E/N values the
    schedule logs, with the state each was computed from."""
    layers, energies = [], []
    cur = lat.spins()
    for _ in range(n_sweeps):
        sw = lat.sweep_count
        steps = ([(main, c) for c in (0, 1)] if main is not None else []) + [(hsg.HSG_OVERRELAX, c) for _ in range(n_or)
                                                                            for c in (0, 1)]
        for upd, c in steps:
            lat.half_sweep(sched, upd, c)
            nxt = lat.spins()
            layers.append(((upd, c, sw), cur, nxt))
            cur = nxt
        lat.sweep_count = sw + 1
        if renorm_every and (sw + 1) % renorm_every == 0:
            lat.renorm()
            nxt = lat.spins()
            layers.append((("renorm", None, sw), cur, nxt))
            cur = nxt
        if energy_every and (sw + 1) % energy_every == 0:
            energies.append((lat.energy(), cur))
    return layers, energies


ORACLE_UPD = {1: oracle.MET, 2: oracle.HB, 3: oracle.OR, 4: oracle.MET_OR}


def check_layers(L, Jr, layers, params_of, label):
    """Every layer of a layered_run against the oracle's same layer from the
    GPU's state before it (renormalisation: within 2^-24 of the fp64
    result)."""
    for (upd, c, sw), before, after in layers:
        if upd == "renorm":
            ref = before.astype(np.float64)
            oracle.renorm(L, ref)
            err = float(np.max(np.abs(after.astype(np.float64) - ref)))
            record(label=f"{label} renorm sweep {sw}", L=L, max_err=err)
            assert err <= 2 ** -24
            continue
        check_layer(L, Jr, before, after, ORACLE_UPD[upd], c, params_of(sw), label=f"{label} sweep {sw} upd {upd} c{c}")


@pytest.mark.parametrize("variant", VARIANTS)
def test_sweep_schedule_energy_log_matches_oracle(hsg, variant):
    """Two sweeps of heat-bath + 2 OR with renormalisation and E/N every
    sweep (12 half-sweep layers and 2 renormalisations): every layer is
    checked against the oracle's same layer from the GPU's state before it,
    every logged E/N against the oracle's energy of the state it was
    computed from (2e-6), the layered run against hsg_sweep bit for bit,
    and the log against the oracle's own two-sweep run (1e-5: its states
    differ from the GPU's by the round-off of 12 layers)."""
    L = 16
    J = inputs.gaussian_couplings(L, seed=17)
    Jr = inputs.round_to_f32(J)
    sched = hsg.schedule(kind=hsg.HSG_HEATBATH, T=0.8, n_or=2, renorm_every=1, energy_every=1, kernel=variant)
    with hsg.Lattice(L, 17) as lat:
        lat.set_couplings(J)
        s0 = lat.spins().astype(np.float64)
        lat.sweep(sched, 2)
        want = lat.spins()
        elog = lat.energy_log()
        assert lat.sweep_count == 2
    with hsg.Lattice(L, 17) as lat:
        lat.set_couplings(J)
        layers, energies = layered_run(hsg, lat, sched, hsg.HSG_HEATBATH, 2, 2, 1, 1)
        assert np.array_equal(lat.spins(), want)
    assert len(layers) == 14 and len(energies) == 2 == len(elog)
    check_layers(L, Jr, layers, lambda sw: oracle.Params(key=oracle.key(17), sweep=sw, beta=1 / 0.8),
                 f"HB+2OR schedule L={L} v{variant}")
    for (e, state), logged in zip(energies, elog):
        assert e == logged
        ref = oracle.energy(L, Jr, state.astype(np.float64)) / L ** 3
        record(label=f"energy log L={L} v{variant}", max_err=abs(e - ref))
        assert abs(e - ref) <= 2e-6
    s = s0.copy()
    sch = oracle.Schedule(kind=oracle.HB, beta=1 / 0.8, n_or=2, renorm_every=1, energy_every=1)
    sw, ref_log = oracle.sweeps(L, Jr, s, sch, oracle.key(17), 2)
    assert sw == 2
    assert np.max(np.abs(elog - ref_log)) < 1e-5


@pytest.mark.parametrize("kind", ["MET", "METOR"])
def test_metropolis_sweeps_layer_by_layer(hsg, kind):
    """Three sweeps of 3-hit ball Metropolis (or the fused pass) + 1 OR with
    renormalisation every 2 sweeps, L = 24: every layer against the oracle
    from the GPU's state before it, and the layered run equal to hsg_sweep."""
    L = 24
    J = inputs.gaussian_couplings(L, seed=29)
    Jr = inputs.round_to_f32(J)
    k = hsg.HSG_METROPOLIS if kind == "MET" else hsg.HSG_METROPOLIS_OR
    sched = hsg.schedule(kind=k, hits=3, proposal=1, step=0.5, T=0.6, n_or=1, renorm_every=2)
    with hsg.Lattice(L, 29) as lat:
        lat.set_couplings(J)
        lat.sweep(sched, 3)
        want = lat.spins()
    with hsg.Lattice(L, 29) as lat:
        lat.set_couplings(J)
        layers, _ = layered_run(hsg, lat, sched, k, 1, 3, 2, 0)
        assert np.array_equal(lat.spins(), want)
    assert len(layers) == 3 * 4 + 1
    check_layers(L, Jr, layers, lambda sw: oracle.Params(key=oracle.key(29), sweep=sw, beta=1 / 0.6, step=0.5, hits=3,
                                                         proposal=1), f"{kind}+OR sweeps L={L}")


def test_l16_workload_with_fp64_couplings_and_their_rounding_error(hsg):
    """The L = 16 workload as specified: fp64 couplings (rounded to fp32 on
    upload), 1-hit Metropolis with the uniform-sphere proposal at T = 1,
    10 sweeps.  Every layer against the oracle fed the same rounded
    couplings (the parity bar), and, separately, what the rounding alone
    changes: the oracle's layer with the raw fp64 couplings against its
    layer with the rounded ones, from the same state.  An accepted proposal
    does not depend on J, so the rounding can only flip decisions whose
    margin it crosses: at most 0.2 % of a colour's sites per layer (none is
    expected).  E/N of the final state with raw against rounded couplings is
    recorded too."""
    L, T = 16, 1.0
    J = inputs.gaussian_couplings(L, seed=1)
    Jr = inputs.round_to_f32(J)
    assert not np.array_equal(J, Jr)
    sched = hsg.schedule(kind=hsg.HSG_METROPOLIS, hits=1, proposal=hsg.HSG_PROP_SPHERE, T=T)
    with hsg.Lattice(L, 1) as lat:
        lat.set_couplings(J)
        layers, _ = layered_run(hsg, lat, sched, hsg.HSG_METROPOLIS, 0, 10, 0, 0)
        final = lat.spins()
    assert len(layers) == 20
    params_of = lambda sw: oracle.Params(key=oracle.key(1), sweep=sw, beta=1.0 / T, hits=1,  # noqa: E731
                                         proposal=hsg.HSG_PROP_SPHERE)
    check_layers(L, Jr, layers, params_of, "L=16 fp64-J Metropolis")
    worst_flips, worst_diff = 0, 0.0
    for (upd, c, sw), before, _ in layers:
        with_raw = before.astype(np.float64)
        with_rounded = with_raw.copy()
        oracle.half_sweep(L, J, with_raw, oracle.MET, c, params_of(sw))
        oracle.half_sweep(L, Jr, with_rounded, oracle.MET, c, params_of(sw))
        diff = np.max(np.abs(with_raw - with_rounded).reshape(-1, 3), axis=1)
        flips = int(np.sum(diff > 1e-5))
        assert flips <= max(2, 0.002 * L ** 3 // 2), (sw, c, flips)
        worst_flips, worst_diff = max(worst_flips, flips), max(worst_diff, float(diff.max()))
    e_raw = oracle.energy(L, J, final.astype(np.float64)) / L ** 3
    e_rounded = oracle.energy(L, Jr, final.astype(np.float64)) / L ** 3
    record(label="L=16 fp64-J rounding to fp32 (oracle raw vs rounded, per layer)", L=L,
           decision_flips_max=worst_flips, max_abs_diff=worst_diff, energy_per_spin_diff=abs(e_raw - e_rounded))
    assert abs(e_raw - e_rounded) < 1e-6


def test_long_run_energy_statistics_match_oracle(hsg):
    """L = 16, Gaussian J, Metropolis 1 hit (sphere), T = 1: the mean E/N of
    1500 sweeps agrees with the oracle's within 3 sigma."""
    L, n = 16, 1500
    J = inputs.gaussian_couplings(L, seed=1)
    with hsg.Lattice(L, 1) as lat:
        lat.set_couplings(J)
        lat.sweep(hsg.schedule(kind=hsg.HSG_METROPOLIS, hits=1, T=1.0, energy_every=1), n)
        g = lat.energy_log()
    s = oracle.init_spins(L, 1)
    _, r = oracle.sweeps(L, inputs.round_to_f32(J), s, oracle.Schedule(kind=oracle.MET, beta=1.0, energy_every=1),
                         oracle.key(1), n)

    def binned(x):
        b = np.array([v.mean() for v in np.array_split(x[n // 5:], 20)])
        return b.mean(), b.std(ddof=1) / np.sqrt(len(b))

    mg, eg = binned(g)
    mr, er = binned(r)
    assert abs(mg - mr) < 3 * math.hypot(eg, er) + 1e-6, (mg, eg, mr, er)


@pytest.mark.parametrize("kind", ["HB", "MET"])
def test_graph_replayed_sweeps_equal_direct_launches(hsg, kind):
    """On a non-default stream hsg_sweep replays captured periods of
    lcm(renorm_every, energy_every) sweeps; on the default stream it
    launches every kernel directly.  Spins, energy log, counters and the
    launch count must agree, including a call that starts mid-period, a
    counter set by hand and a cleared log."""
    L = 16
    J = inputs.gaussian_couplings(L, seed=23)
    k = hsg.HSG_HEATBATH if kind == "HB" else hsg.HSG_METROPOLIS
    sched = hsg.schedule(kind=k, hits=2, proposal=1, T=0.6, n_or=2, renorm_every=5, energy_every=2)
    outs = []
    for stream in (torch.cuda.Stream(), None):
        with hsg.Lattice(L, 23, stream=stream) as lat:
            lat.set_couplings(J)
            n0 = hsg.hsg_launch_count(lat.ctx)
            lat.sweep(sched, 3)  # not a whole period: direct launches
            lat.sweep_count = 10  # jump to a period boundary
            lat.sweep(sched, 25)  # two replayed periods + 5 direct sweeps
            log1 = lat.energy_log()
            hsg.hsg_clear_energy_log(lat.ctx)
            lat.sweep(sched, 10)
            outs.append((lat.spins(), log1, lat.energy_log(), lat.sweep_count, hsg.hsg_launch_count(lat.ctx) - n0))
    a, b = outs
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1]) and len(a[1]) == 1 + 12
    assert np.array_equal(a[2], b[2]) and len(a[2]) == 5
    assert a[3] == b[3] == 45
    assert a[4] == b[4]


def test_checkpoint_resume_is_bit_identical(hsg):
    L = 24
    J = inputs.gaussian_couplings(L, seed=5)
    sched = hsg.schedule(kind=hsg.HSG_METROPOLIS, hits=2, proposal=1, T=0.7, n_or=1, renorm_every=2)
    with hsg.Lattice(L, 5) as a:
        a.set_couplings(J)
        a.sweep(sched, 6)
        want = a.spins()
    with hsg.Lattice(L, 5) as b:
        b.set_couplings(J)
        b.sweep(sched, 3)
        mid, sw = b.spins(), b.sweep_count
    with hsg.Lattice(L, 5) as c:
        c.set_couplings(J)
        c.set_spins(mid)
        c.sweep_count = sw
        c.sweep(sched, 3)
        assert np.array_equal(c.spins(), want)


# ---------------------------------------------------------------------------
# Boundary behaviour on a device
# ---------------------------------------------------------------------------

def test_error_paths_on_device(hsg):
    with hsg.Lattice(8, 1) as lat:
        with pytest.raises(hsg.HsgError) as e:
            lat.sweep(hsg.schedule(kind=hsg.HSG_HEATBATH), 1)
        assert e.value.status == hsg.HSG_EINVAL and "couplings" in str(e.value)
        lat.set_couplings(inputs.gaussian_couplings(8, seed=1))
        bad = [dict(kind=7), dict(hits=0), dict(hits=70000), dict(proposal=3), dict(step=0.0), dict(n_or=-1),
               dict(T=0.0), dict(T=-1.0), dict(T=float("nan")), dict(renorm_every=-1), dict(kernel=9)]
        for kw in bad:
            with pytest.raises(hsg.HsgError) as e:
                lat.sweep(hsg.schedule(**kw), 1)
            assert e.value.status == hsg.HSG_EINVAL, kw
        with pytest.raises(hsg.HsgError):
            lat.sweep(hsg.schedule(), -1)
        lat.sweep(hsg.schedule(kind=hsg.HSG_HEATBATH), 0)  # no-op
        assert lat.sweep_count == 0
        with pytest.raises(hsg.HsgError):
            lat.half_sweep(hsg.schedule(), hsg.HSG_OVERRELAX, 2)
        # sampled reads and the kernel query
        for bad_sites in ([8 ** 3], [0, 2 ** 32 - 1]):
            with pytest.raises(hsg.HsgError) as e:
                hsg.hsg_get_sites(lat.ctx, np.array(bad_sites, dtype=np.uint64).astype(np.uint32))
            assert e.value.status == hsg.HSG_EINVAL
        spins, bonds = hsg.hsg_get_sites(lat.ctx, np.array([], dtype=np.uint32))
        assert spins.shape == (0, 3) and bonds.shape == (0, 3)
        with pytest.raises(hsg.HsgError) as e:
            hsg.hsg_kernel_for(lat.ctx, hsg.schedule(kernel=9))
        assert e.value.status == hsg.HSG_EINVAL
    with hsg.Lattice(8, 1) as fresh:  # bonds before couplings are set
        with pytest.raises(hsg.HsgError) as e:
            hsg.hsg_get_sites(fresh.ctx, np.array([0], dtype=np.uint32))
        assert e.value.status == hsg.HSG_EINVAL
        s, b = hsg.hsg_get_sites(fresh.ctx, np.array([0, 511], dtype=np.uint32), want_bonds=False)
        assert b is None and np.array_equal(s, fresh.spins().reshape(-1, 3)[[0, 511]])


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_injected_allocation_failure_is_reported(hsg, k):
    hsg.hsg_test_fail_alloc(k)
    try:
        with pytest.raises(hsg.HsgError) as e:
            hsg.hsg_create(16, seed=1)
        assert e.value.status == hsg.HSG_ENOMEM
    finally:
        hsg.hsg_test_fail_alloc(0)
    with hsg.Lattice(16, 1) as lat:  # the library is still usable
        lat.set_couplings(inputs.gaussian_couplings(16, seed=1))
        lat.sweep(hsg.schedule(kind=hsg.HSG_HEATBATH), 1)


def test_profiler_counts_launches(hsg):
    with hsg.Lattice(16, 1) as lat:
        lat.set_couplings(inputs.gaussian_couplings(16, seed=1))
        n0 = hsg.hsg_launch_count(lat.ctx)
        hsg.hsg_profile(lat.ctx, True)
        lat.sweep(hsg.schedule(kind=hsg.HSG_HEATBATH, n_or=4, energy_every=5, renorm_every=5), 10)
        counts = {k: hsg.hsg_profile_read(lat.ctx, k)[1] for k in range(hsg.HSG_PROF_COUNT)}
        ms = hsg.hsg_profile_read(lat.ctx, hsg.HSG_PROF_OVERRELAX)[0]
        assert counts[hsg.HSG_PROF_HEATBATH] == 20
        assert counts[hsg.HSG_PROF_OVERRELAX] == 80
        assert counts[hsg.HSG_PROF_ENERGY] == 2 and counts[hsg.HSG_PROF_RENORM] == 2
        assert ms > 0
        # 20 heat-bath + 80 OR half-sweeps, 10 counter advances, 2 energies (2 kernels), 2 renorms
        assert hsg.hsg_launch_count(lat.ctx) - n0 == 20 + 80 + 10 + 2 * 2 + 2
        hsg.hsg_profile_reset(lat.ctx)
        assert hsg.hsg_profile_read(lat.ctx, hsg.HSG_PROF_OVERRELAX)[1] == 0


def test_gpu_matches_the_golden_fixture(hsg):
    """The CUDA path against the stored oracle results of
    tests/golden/l6_seed21.json (L = 6, seed 21; the fixture's own fp32
    couplings and spins): energy, an over-relaxation, a Metropolis (3 hits,
    ball; every decision of the fixture is >= 5e-4 from its threshold) and a
    heat-bath half-sweep under the half-sweep rules, and two sweeps of
    heat-bath + 1 OR: the energy log against the stored one (1e-5, the
    states of the two runs differing by the round-off of 8 layers) and every
    layer against the oracle's same layer from the GPU's state before it."""
    import json

    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "l6_seed21.json")) as f:
        g = json.load(f)
    L, seed = g["L"], g["seed"]
    J = np.array(g["J"])
    s0 = np.array(g["s0"]).astype(np.float32)
    b64 = s0.astype(np.float64)
    with hsg.Lattice(L, seed) as lat:
        lat.set_couplings(J.astype(np.float32))
        lat.set_spins(s0)
        assert abs(lat.energy() - g["energy_s0"]) <= 2e-6
    got = gpu_half_sweep(hsg, L, J, s0, hsg.HSG_OVERRELAX, 0, hsg.schedule(), seed=seed, sweep=0)
    check_half_sweep(L, J, b64, got, np.array(g["or_colour0"]), 0)
    m = g["met_colour1"]
    assert min(m["margins"]) >= 1e-5
    sched = hsg.schedule(kind=hsg.HSG_METROPOLIS, hits=m["hits"], proposal=hsg.HSG_PROP_BALL, step=m["step"], T=m["T"])
    got = gpu_half_sweep(hsg, L, J, s0, hsg.HSG_METROPOLIS, 1, sched, seed=seed, sweep=m["sweep"])
    check_half_sweep(L, J, b64, got, np.array(m["spins"]), 1)
    h = g["hb_colour0"]
    sched = hsg.schedule(kind=hsg.HSG_HEATBATH, T=h["T"])
    got = gpu_half_sweep(hsg, L, J, s0, hsg.HSG_HEATBATH, 0, sched, seed=seed, sweep=h["sweep"])
    check_half_sweep(L, J, b64, got, np.array(h["spins"]), 0, exclude=frame_band(L, J, b64, 0))
    w = g["hb_or_two_sweeps"]
    sched = hsg.schedule(kind=hsg.HSG_HEATBATH, T=w["T"], n_or=w["n_or"], energy_every=1)
    with hsg.Lattice(L, seed) as lat:
        lat.set_couplings(J.astype(np.float32))
        lat.set_spins(s0)
        lat.sweep(sched, w["sweeps"])
        want = lat.spins()
        elog = lat.energy_log()
    assert np.max(np.abs(elog - np.array(w["energy_log"]))) < 1e-5
    with hsg.Lattice(L, seed) as lat:  # the same sweeps layer by layer, each against the oracle
        lat.set_couplings(J.astype(np.float32))
        lat.set_spins(s0)
        layers, _ = layered_run(hsg, lat, sched, hsg.HSG_HEATBATH, w["n_or"], w["sweeps"], 0, 1)
        assert np.array_equal(lat.spins(), want)
    check_layers(L, J, layers, lambda sw: oracle.Params(key=oracle.key(seed), sweep=sw, beta=1 / w["T"]),
                 f"golden HB+OR L={L}")
