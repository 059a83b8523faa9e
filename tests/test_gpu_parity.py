"""GPU path vs the FP64 oracle, through the C ABI (needs a CUDA GPU).

Tolerances (written per test):
  * half-sweeps: max |diff| <= 1e-5 per spin component at every site whose
    fp32 local field is well conditioned, 4 kappa <= 1e-5 with
    kappa = 2^-24 * sum_k |J_k| / |h| (the field's fp32 round-off relative
    to its length, which the update's direction inherits).  At the rare
    sites with a nearly cancelling field (<= 0.1 %) the difference must
    stay within 1e-5 + 64 kappa, the propagated round-off bound;
  * Metropolis: sites whose accept decisions lie within 1e-5 of their
    threshold (|u3 - exp(-beta dE)| < 1e-5, margin reported by the oracle)
    are excluded: fp32 and fp64 may decide differently there;
  * heat-bath: sites whose field is within 1e-5 (relative) of the h_z = 0
    plane are excluded: the orthonormal frame of the azimuth switches
    branch there and fp32/fp64 may pick different branches;
  * energies: |E/N difference| <= 2e-6 (per-site terms are fp32);
  * long runs: mean E/N within 3 sigma (binned errors of both runs).
Every half-sweep starts the GPU and the oracle from the same state (fp32
values, the oracle holding them in fp64) and the same fp32-rounded J.
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


U32 = 2.0 ** -24


def colour_mask(L, c):
    g = np.indices((L, L, L))
    return (((g[0] + g[1] + g[2]) % 2) == c).reshape(-1)


def bond_sums(L, J):
    """sum of |J| over the six bonds of every site."""
    a = np.abs(J.reshape(L, L, L, 3))  # [z, y, x, d]
    s = a.sum(axis=3)
    s += np.roll(a[..., 0], 1, axis=2) + np.roll(a[..., 1], 1, axis=1) + np.roll(a[..., 2], 1, axis=0)
    return s.reshape(-1)


def check_half_sweep(L, Jr, before64, got, ref, colour, exclude=None):
    """Compare one half-sweep site by site (see the module docstring).
    Returns (number of ill-conditioned sites, max err/kappa)."""
    idx = np.nonzero(colour_mask(L, colour))[0]
    h = np.array([oracle.local_field(L, Jr, before64, int(i)) for i in idx])
    hn = np.linalg.norm(h, axis=1)
    kappa = U32 * bond_sums(L, Jr)[idx] / np.maximum(hn, 1e-300)
    err = np.max(np.abs(got - ref).reshape(-1, 3)[idx], axis=1)
    skip = np.zeros(len(idx), bool) if exclude is None else exclude[idx]
    well = (4 * kappa <= TOL) & ~skip
    ill = ~well & ~skip
    assert np.all(err[well] <= TOL), float(np.max(err[well]))
    assert ill.sum() <= max(2, 0.001 * len(idx)), int(ill.sum())
    assert np.all(err[ill] <= TOL + 64 * kappa[ill])
    keep = ~skip
    return int(ill.sum()), float(np.max(err[keep] / kappa[keep])) if keep.any() else 0.0


def frame_band(L, Jr, before64, colour):
    """Sites whose field lies within 1e-5 (relative) of the h_z = 0 plane."""
    band = np.zeros(L ** 3, bool)
    for i in np.nonzero(colour_mask(L, colour))[0]:
        h = oracle.local_field(L, Jr, before64, int(i))
        band[i] = abs(h[2]) < TOL * np.linalg.norm(h)
    return band


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
        before = s32.astype(np.float64)
        ref = before.copy()
        oracle.half_sweep(L, Jr, ref, oracle.OR, colour, oracle.Params())
        check_half_sweep(L, Jr, before, got, ref, colour)
        other = ~colour_mask(L, colour)
        assert np.array_equal(got.reshape(-1, 3)[other], s32.astype(np.float64).reshape(-1, 3)[other])


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
        before = s32.astype(np.float64)
        ref = before.copy()
        p = oracle.Params(key=oracle.key(11), sweep=3, beta=beta, step=0.5, hits=hits, proposal=proposal)
        margins = oracle.half_sweep(L, Jr, ref, oracle.MET, colour, p, want_margins=True)
        mask = colour_mask(L, colour)
        near = mask & (margins < TOL)
        assert near.sum() <= max(2, 0.002 * mask.sum())
        check_half_sweep(L, Jr, before, got, ref, colour, exclude=near)
        moved = np.any(ref.reshape(-1, 3) != s32.astype(np.float64).reshape(-1, 3), axis=1)
        assert moved[mask].mean() > 0.05  # the chain does move


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
        before = s32.astype(np.float64)
        ref = before.copy()
        p = oracle.Params(key=oracle.key(31), sweep=4, beta=1.0 / T, step=0.5, hits=hits, proposal=proposal)
        margins = oracle.half_sweep(L, Jr, ref, oracle.MET_OR, colour, p, want_margins=True)
        near = colour_mask(L, colour) & (margins < TOL)
        assert near.sum() <= max(2, 0.002 * colour_mask(L, colour).sum())
        check_half_sweep(L, Jr, before, got, ref, colour, exclude=near)


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
@pytest.mark.parametrize("L,T", [(6, 1.0), (16, 0.3), (40, 0.3), (66, 1.0), (16, math.inf), (16, 0.01)])
def test_heatbath_half_sweep_parity(hsg, variant, L, T):
    J, s32 = oracle_state(L, 500 + L, 600 + L)
    Jr = inputs.round_to_f32(J)
    sched = hsg.schedule(kind=hsg.HSG_HEATBATH, T=T, kernel=variant)
    beta = 0.0 if math.isinf(T) else 1.0 / T
    for colour in (0, 1):
        s64 = s32.astype(np.float64)
        got = gpu_half_sweep(hsg, L, J, s32, hsg.HSG_HEATBATH, colour, sched, seed=13, sample=2, sweep=5)
        ref = s64.copy()
        p = oracle.Params(key=oracle.key(13, 2), sweep=5, beta=beta)
        oracle.half_sweep(L, Jr, ref, oracle.HB, colour, p)
        mask = colour_mask(L, colour)
        band = frame_band(L, Jr, s64, colour)
        assert band.sum() <= max(2, 0.001 * mask.sum())
        check_half_sweep(L, Jr, s64, got, ref, colour, exclude=band)
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


@pytest.mark.parametrize("L", [4, 8, 14, 40, 66])  # the heat-bath column march: shorter than, and ragged in, its 6-plane chunks
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
def test_over_relaxation_sweep_matches_oracle(hsg, variant):
    """One over-relaxation sweep (colour 0, then colour 1) from the same
    state through hsg_sweep.  Colour 0 is checked site by site as in the
    half-sweep tests; colour 1 is computed from colour-0 values that already
    carry fp32 round-off, so 99.5 % of its sites must agree to 1e-5 and all
    of them to 1e-3."""
    L = 24
    J, s32 = oracle_state(L, 900, 901)
    Jr = inputs.round_to_f32(J)
    with hsg.Lattice(L, 17) as lat:
        lat.set_couplings(J)
        lat.set_spins(s32)
        lat.sweep(hsg.schedule(kind=hsg.HSG_NONE, n_or=1, kernel=variant), 1)
        got = lat.spins().astype(np.float64)
    before = s32.astype(np.float64)
    mid = before.copy()
    oracle.half_sweep(L, Jr, mid, oracle.OR, 0, oracle.Params())
    ref = mid.copy()
    oracle.half_sweep(L, Jr, ref, oracle.OR, 1, oracle.Params())
    c0 = colour_mask(L, 0)
    got_mid = np.where(np.repeat(c0, 3), got, before)
    check_half_sweep(L, Jr, before, got_mid, mid, 0)
    err1 = np.max(np.abs(got - ref).reshape(-1, 3), axis=1)[~c0]
    assert np.mean(err1 <= TOL) >= 0.995
    assert np.max(err1) <= 1e-3


@pytest.mark.parametrize("variant", VARIANTS)
def test_sweep_schedule_energy_log_matches_oracle(hsg, variant):
    """Two sweeps of heat-bath + 2 OR with renormalisation and E/N every
    sweep: the energy log agrees with the oracle's to 1e-5 and the median
    spin to 1e-5 (the per-spin differences compound through the 12
    half-sweep layers; per-layer parity is checked by the half-sweep tests,
    the exact order by test_sweep_is_the_composition_of_half_sweeps)."""
    L = 16
    J = inputs.gaussian_couplings(L, seed=17)
    sched = hsg.schedule(kind=hsg.HSG_HEATBATH, T=0.8, n_or=2, renorm_every=1, energy_every=1, kernel=variant)
    with hsg.Lattice(L, 17) as lat:
        lat.set_couplings(J)
        s0 = lat.spins().astype(np.float64)
        lat.sweep(sched, 2)
        got = lat.spins().astype(np.float64)
        elog = lat.energy_log()
        assert lat.sweep_count == 2
    s = s0.copy()
    sch = oracle.Schedule(kind=oracle.HB, beta=1 / 0.8, n_or=2, renorm_every=1, energy_every=1)
    sw, ref_log = oracle.sweeps(L, inputs.round_to_f32(J), s, sch, oracle.key(17), 2)
    assert sw == 2 and len(elog) == 2
    assert np.max(np.abs(elog - ref_log)) < 1e-5
    err = np.max(np.abs(got - s).reshape(-1, 3), axis=1)
    assert np.median(err) <= TOL


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
    heat-bath half-sweep under the half-sweep rules above, and two sweeps of
    heat-bath + 1 OR under the whole-sweep rule."""
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
    with hsg.Lattice(L, seed) as lat:
        lat.set_couplings(J.astype(np.float32))
        lat.set_spins(s0)
        lat.sweep(hsg.schedule(kind=hsg.HSG_HEATBATH, T=w["T"], n_or=w["n_or"], energy_every=1), w["sweeps"])
        got = lat.spins().astype(np.float64)
        elog = lat.energy_log()
    assert np.max(np.abs(elog - np.array(w["energy_log"]))) < 1e-5
    err = np.max(np.abs(got - np.array(w["spins"])).reshape(-1, 3), axis=1)
    assert np.median(err) <= TOL
