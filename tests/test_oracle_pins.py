"""Pins of the FP64 oracle against values the mathematics fixes (CPU only).

Each test names what would break it: a dropped term, a wrong sign, a wrong
bond index or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_1006_2566_gb300 import inputs


def langevin(x):
    """Mean of cos(theta) for the density exp(x cos theta) on S^2."""
    return 1.0 / math.tanh(x) - 1.0 / x


def site(L, x, y, z):
    return x + y * L + z * L * L


# --------------------------------------------------------------------------
# Philox-4x32-10
# --------------------------------------------------------------------------

def test_philox_matches_independent_implementation(orc):
    """The oracle's Philox equals Triton's Philox-4x32-10 (run by Triton's
    CPU interpreter), an implementation written by other authors."""
    import os

    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    tl = pytest.importorskip("triton.language")
    torch = pytest.importorskip("torch")

    @triton.jit
    def _k(c_ptr, out_ptr, seed, n, BLOCK: tl.constexpr):
        offs = tl.arange(0, BLOCK)
        m = offs < n
        c0 = tl.load(c_ptr + offs * 4 + 0, mask=m)
        c1 = tl.load(c_ptr + offs * 4 + 1, mask=m)
        c2 = tl.load(c_ptr + offs * 4 + 2, mask=m)
        c3 = tl.load(c_ptr + offs * 4 + 3, mask=m)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
        tl.store(out_ptr + offs * 4 + 0, a, mask=m)
        tl.store(out_ptr + offs * 4 + 1, b, mask=m)
        tl.store(out_ptr + offs * 4 + 2, c, mask=m)
        tl.store(out_ptr + offs * 4 + 3, d, mask=m)

    rng = np.random.default_rng(11)
    n = 64
    for seed in (0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF):
        ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
        ctr[0] = 0
        ctr[1] = 0xFFFFFFFF
        out = torch.zeros(4 * n, dtype=torch.int32)
        _k[(1,)](torch.from_numpy(ctr.view(np.int32).reshape(-1).copy()), out, seed, n, BLOCK=n)
        got = out.numpy().view(np.uint32).reshape(n, 4)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for t in range(n):
            assert list(orc.philox4x32_10(ctr[t], key)) == list(got[t]), (seed, t)


def test_philox_round_structure_inverts(orc):
    """Undoing ten Philox rounds (multiplier inverses mod 2^32, Weyl key
    schedule) recovers the counter: pins constants and word order."""
    m0, m1 = 0xD2511F53, 0xCD9E8D57
    w0, w1 = 0x9E3779B9, 0xBB67AE85
    inv0, inv1 = pow(m0, -1, 2 ** 32), pow(m1, -1, 2 ** 32)
    rng = np.random.default_rng(5)
    for _ in range(50):
        ctr = [int(v) for v in rng.integers(0, 2 ** 32, size=4)]
        key = [int(v) for v in rng.integers(0, 2 ** 32, size=2)]
        o = [int(v) for v in orc.philox4x32_10(ctr, key)]
        for r in reversed(range(10)):
            k0 = (key[0] + r * w0) % 2 ** 32
            k1 = (key[1] + r * w1) % 2 ** 32
            c0 = (o[3] * inv0) % 2 ** 32
            c2 = (o[1] * inv1) % 2 ** 32
            hi0 = (m0 * c0) >> 32
            hi1 = (m1 * c2) >> 32
            c1 = o[0] ^ hi1 ^ k0
            c3 = o[2] ^ hi0 ^ k1
            o = [c0, c1, c2, c3]
        assert o == ctr


def test_u01_open_interval_and_fp32_exact(orc):
    assert orc.u01(0) == 2.0 ** -24
    assert orc.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    rng = np.random.default_rng(3)
    for r in rng.integers(0, 2 ** 32, size=2000):
        u = orc.u01(int(r))
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u  # exactly representable in fp32
    # monotone in the top 23 bits, constant in the low 9
    assert orc.u01(0x200) > orc.u01(0x1FF) == orc.u01(0)


def test_key_and_counter_layout(orc):
    k = orc.key(0x0000000500000007, sample=3, replica=1)
    assert k[0] == 7
    assert k[1] == 5 ^ ((7 * 0x9E3779B9) % 2 ** 32)
    c = orc.counter(site=12345, sweep=(9 << 32) | 77, kind=orc.KIND_HB, colour=1, hit=3)
    assert c == (12345, 77, (4 << 24) | (1 << 16) | 3, 9)


def test_key_names_each_sample_and_replica_once(orc):
    """Within replica in {0, 1} and sample < 2^31 the stream number
    2*sample + replica is one-to-one, so distinct pairs have distinct keys;
    outside that range two pairs would share a key (e.g. (s, 2) and (s+1, 0))
    and every random number, so the oracle refuses them."""
    keys = {orc.key(9, s, r) for s in list(range(64)) + [2 ** 31 - 1] for r in (0, 1)}
    assert len(keys) == 2 * 65
    for sample, replica in ((0, 2), (5, 3), (2 ** 31, 0), (2 ** 32 - 1, 1)):
        with pytest.raises(ValueError):
            orc.key(9, sample, replica)
        with pytest.raises(ValueError):
            orc.init_spins(4, 9, sample, replica)
        with pytest.raises(ValueError):
            orc.init_spin_sites([0, 1], 9, sample, replica)
    for sample in (2 ** 31, 2 ** 32 - 1):
        with pytest.raises(ValueError):
            orc.gaussian_couplings(4, 9, sample)
        with pytest.raises(ValueError):
            orc.gaussian_coupling_sites([0], 9, sample)


# --------------------------------------------------------------------------
# Initial spins
# --------------------------------------------------------------------------

def test_init_spins_unit_and_isotropic(orc):
    L = 16
    s = orc.init_spins(L, seed=1).reshape(-1, 3)
    assert np.max(np.abs(np.linalg.norm(s, axis=1) - 1.0)) < 1e-12
    # Archimedes: z uniform on [-1,1]; azimuth uniform on [0, 2pi)
    assert stats.kstest(s[:, 2], stats.uniform(-1, 2).cdf).pvalue > 1e-3
    phi = np.mod(np.arctan2(s[:, 1], s[:, 0]), 2 * np.pi)
    assert stats.kstest(phi, stats.uniform(0, 2 * np.pi).cdf).pvalue > 1e-3
    # different replicas give different, seed-reproducible states
    s2 = orc.init_spins(L, seed=1, replica=1).reshape(-1, 3)
    assert not np.allclose(s, s2)
    assert np.array_equal(s, orc.init_spins(L, seed=1).reshape(-1, 3))


# --------------------------------------------------------------------------
# Energy and local field (Eq. 1, Eq. 2)
# --------------------------------------------------------------------------

def test_ferromagnet_ground_state_energy(orc):
    """J = 1 on every bond, all spins aligned: E/N = -3 (3 bonds per site)."""
    for L in (4, 6):
        J = inputs.uniform_couplings(L)
        s = inputs.aligned_spins(L, (0.3, -0.5, 0.8))
        assert abs(orc.energy(L, J, s) / L ** 3 + 3.0) < 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_helix_energy_pins_bond_directions(orc, axis):
    """Spins rotating by 2 pi k / L per step along one axis.  With J = 1 only
    on bonds along `axis`, E/N = -cos(2 pi k/L); with J = 1 on the other two
    axes E/N = -2 (their bonds join parallel spins)."""
    L, k = 6, 1
    ang = 2 * np.pi * k / L
    s = np.zeros((L, L, L, 3))  # indexed [z, y, x]
    grid = np.indices((L, L, L))  # grid[0]=z, grid[1]=y, grid[2]=x
    coord = grid[2 - axis]
    s[..., 0] = np.cos(ang * coord)
    s[..., 1] = np.sin(ang * coord)
    s = s.reshape(-1)
    J_on = inputs.uniform_couplings(L, axes=(axis,))
    assert abs(orc.energy(L, J_on, s) / L ** 3 + np.cos(ang)) < 1e-12
    others = tuple(d for d in range(3) if d != axis)
    J_off = inputs.uniform_couplings(L, axes=others)
    assert abs(orc.energy(L, J_off, s) / L ** 3 + 2.0) < 1e-12


def test_local_field_matches_brute_force_energy_difference(orc):
    """dE = -(s' - s).h_i equals E(after) - E(before), for every site of an
    L = 4 lattice with Gaussian couplings and random proposals."""
    L = 4
    J = inputs.gaussian_couplings(L, seed=21)
    s = inputs.random_spins(L, seed=22)
    rng = np.random.default_rng(23)
    e0 = orc.energy(L, J, s)
    for i in range(L ** 3):
        h = orc.local_field(L, J, s, i)
        for _ in range(4):
            v = rng.standard_normal(3)
            v /= np.linalg.norm(v)
            t = s.copy()
            t[3 * i: 3 * i + 3] = v
            de_local = -np.dot(v - s[3 * i: 3 * i + 3], h)
            assert abs((orc.energy(L, J, t) - e0) - de_local) < 1e-12


def test_local_field_of_single_bond(orc):
    """One bond of coupling 2.5 along +y from site a: h_a = 2.5 s_b and
    h_b = 2.5 s_a, all other fields zero."""
    L = 4
    J = np.zeros(3 * L ** 3)
    a = site(L, 1, 3, 2)
    b = site(L, 1, 0, 2)  # y = 3 + 1 wraps to 0
    J[3 * a + 1] = 2.5
    s = inputs.random_spins(L, seed=3)
    assert np.allclose(orc.local_field(L, J, s, a), 2.5 * s[3 * b: 3 * b + 3], atol=1e-15)
    assert np.allclose(orc.local_field(L, J, s, b), 2.5 * s[3 * a: 3 * a + 3], atol=1e-15)
    c = site(L, 2, 3, 2)
    assert np.all(orc.local_field(L, J, s, c) == 0.0)


def test_half_sweeps_do_not_depend_on_the_thread_count(orc):
    """The OpenMP loop of a half-sweep (used to time the CPU baseline on all
    cores) gives the same state and margins as one thread."""
    L = 10
    J = inputs.gaussian_couplings(L, seed=41)
    p = orc.Params(key=orc.key(41), sweep=3, beta=1.5, hits=3, proposal=orc.PROP_BALL)
    outs = []
    for threads in (1, max(2, orc.max_threads())):
        orc.set_threads(threads)
        try:
            s = orc.init_spins(L, 41)
            m = [orc.half_sweep(L, J, s, upd, c, p, want_margins=True) for upd in (orc.MET, orc.HB, orc.OR)
                 for c in (0, 1)]
        finally:
            orc.set_threads(1)
        outs.append((s, m))
    assert np.array_equal(outs[0][0], outs[1][0])
    for a, b in zip(outs[0][1], outs[1][1]):
        assert np.array_equal(a, b, equal_nan=True)


def test_per_site_generators_are_the_lattice_generators(orc):
    """init_spin_sites / gaussian_coupling_sites (any lattice size, for
    samples) give exactly what the whole-lattice generators give."""
    L = 6
    sites = np.random.default_rng(7).permutation(L ** 3)[:100]
    s = orc.init_spins(L, 9, 2, 1)
    J = orc.gaussian_couplings(L, 9, 2)
    assert np.array_equal(orc.init_spin_sites(sites, 9, 2, 1), s.reshape(-1, 3)[sites])
    assert np.array_equal(orc.gaussian_coupling_sites(sites, 9, 2), J.reshape(-1, 3)[sites])


def test_local_field_from_explicit_neighbours_is_the_lattice_field(orc):
    """local_field_nb (six neighbours and bonds handed over) equals
    local_field on the whole lattice bit for bit, at every site of an L = 6
    lattice including the periodic wrap; a neighbour or bond in the wrong
    slot changes it."""
    L = 6
    J = inputs.gaussian_couplings(L, seed=31)
    s = inputs.random_spins(L, seed=32)
    for i in range(L ** 3):
        x, y, z = i % L, (i // L) % L, i // (L * L)
        nbs, bonds = [], []
        for d, (dx, dy, dz) in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
            up = site(L, (x + dx) % L, (y + dy) % L, (z + dz) % L)
            dn = site(L, (x - dx) % L, (y - dy) % L, (z - dz) % L)
            nbs += [s[3 * up: 3 * up + 3], s[3 * dn: 3 * dn + 3]]
            bonds += [J[3 * i + d], J[3 * dn + d]]
        h = orc.local_field_nb(np.array(nbs), np.array(bonds))
        assert np.array_equal(h, orc.local_field(L, J, s, i))
        swapped = list(bonds)
        swapped[0], swapped[1] = swapped[1], swapped[0]
        assert not np.allclose(orc.local_field_nb(np.array(nbs), np.array(swapped)), h)


# --------------------------------------------------------------------------
# Over-relaxation (Sec. 4)
# --------------------------------------------------------------------------

def test_over_relaxation_conserves_energy_and_norm(orc):
    """The paper's own correctness check: OR leaves E unchanged."""
    L = 6
    J = inputs.gaussian_couplings(L, seed=31)
    s = inputs.random_spins(L, seed=32)
    e0 = orc.energy(L, J, s)
    p = orc.Params()
    for it in range(6):
        orc.half_sweep(L, J, s, orc.OR, it % 2, p)
        assert abs(orc.energy(L, J, s) - e0) < 1e-12 * L ** 3
    assert np.max(np.abs(np.linalg.norm(s.reshape(-1, 3), axis=1) - 1)) < 1e-12


def test_over_relaxation_is_reflection_about_field(orc):
    """s' keeps its projection on h, flips the perpendicular part, and
    applying it twice gives back s."""
    rng = np.random.default_rng(4)
    p = orc.Params()
    for _ in range(200):
        s = rng.standard_normal(3)
        s /= np.linalg.norm(s)
        h = rng.standard_normal(3) * rng.uniform(0.1, 5)
        s1, _ = orc.update_site(orc.OR, s, h, p, 0, 0)
        hh = h / np.linalg.norm(h)
        assert abs(np.dot(s1, hh) - np.dot(s, hh)) < 1e-14
        perp0 = s - np.dot(s, hh) * hh
        perp1 = s1 - np.dot(s1, hh) * hh
        assert np.allclose(perp1, -perp0, atol=1e-14)
        s2, _ = orc.update_site(orc.OR, s1, h, p, 0, 0)
        assert np.allclose(s2, s, atol=1e-14)
    s = np.array([0.6, 0.0, 0.8])
    s1, _ = orc.update_site(orc.OR, s, np.zeros(3), p, 0, 0)
    assert np.array_equal(s1, s)  # h = 0: unchanged


# --------------------------------------------------------------------------
# Checkerboard
# --------------------------------------------------------------------------

@pytest.mark.parametrize("upd", [0, 1, 2])
def test_half_sweep_updates_one_colour_only(orc, upd):
    L = 6
    J = inputs.gaussian_couplings(L, seed=41)
    s0 = inputs.random_spins(L, seed=42)
    col = np.array([orc.colour(L, i) for i in range(L ** 3)])
    g = np.indices((L, L, L))
    assert np.array_equal(col, ((g[0] + g[1] + g[2]) % 2).reshape(-1))
    for c in (0, 1):
        s = s0.copy()
        p = orc.Params(key=orc.key(7), beta=1.0, hits=2)
        orc.half_sweep(L, J, s, upd, c, p)
        d = np.any(s.reshape(-1, 3) != s0.reshape(-1, 3), axis=1)
        assert not np.any(d[col != c])
        assert np.mean(d[col == c]) > 0.3


def test_sweep_order_is_main_update_then_over_relaxation(orc):
    """oracle_sweeps = MET colour 0, MET colour 1, then n_or x (OR 0, OR 1),
    then the counter advances; renormalisation and E/N on their cadence."""
    L = 4
    J = inputs.gaussian_couplings(L, seed=51)
    s = inputs.random_spins(L, seed=52)
    key = orc.key(9)
    sch = orc.Schedule(kind=orc.MET, hits=2, proposal=orc.PROP_BALL, step=0.5, n_or=2, beta=2.0,
                       renorm_every=2, energy_every=1)
    a = s.copy()
    sw, elog = orc.sweeps(L, J, a, sch, key, 3, sweep=5)
    assert sw == 8 and len(elog) == 3
    b = s.copy()
    manual = []
    for k in range(3):
        p = orc.Params(key=key, sweep=5 + k, beta=2.0, step=0.5, hits=2, proposal=orc.PROP_BALL)
        orc.half_sweep(L, J, b, orc.MET, 0, p)
        orc.half_sweep(L, J, b, orc.MET, 1, p)
        for _ in range(2):
            orc.half_sweep(L, J, b, orc.OR, 0, p)
            orc.half_sweep(L, J, b, orc.OR, 1, p)
        if (5 + k + 1) % 2 == 0:
            orc.renorm(L, b)
        manual.append(orc.energy(L, J, b) / L ** 3)
    assert np.array_equal(a, b)
    assert np.allclose(elog, manual, rtol=0, atol=0)


# --------------------------------------------------------------------------
# Metropolis
# --------------------------------------------------------------------------

@pytest.mark.parametrize("proposal", [0, 1])
def test_infinite_temperature_accepts_every_proposal(orc, proposal):
    """beta = 0: exp(-beta dE) = 1 > u3, so every hit is accepted.  With the
    sphere proposal the new spins forget the aligned start (<s_z> ~ 0);
    with the ball proposal every spin moves."""
    L = 8
    J = inputs.gaussian_couplings(L, seed=61)
    s = inputs.aligned_spins(L, (0, 0, 1))
    p = orc.Params(key=orc.key(3), beta=0.0, hits=1, proposal=proposal, step=0.5)
    orc.half_sweep(L, J, s, orc.MET, 0, p)
    col = np.array([orc.colour(L, i) for i in range(L ** 3)])
    v = s.reshape(-1, 3)[col == 0]
    assert np.all(v[:, 2] != 1.0)
    if proposal == 0:
        assert abs(np.mean(v[:, 2])) < 4 / np.sqrt(len(v))


def test_zero_temperature_limit_rejects_uphill(orc):
    """Huge beta: only moves with dE <= 0 are taken, so E never rises."""
    L = 6
    J = inputs.gaussian_couplings(L, seed=62)
    s = inputs.random_spins(L, seed=63)
    e = orc.energy(L, J, s)
    for k in range(4):
        p = orc.Params(key=orc.key(4), sweep=k, beta=1e9, hits=3, proposal=orc.PROP_BALL, step=0.5)
        orc.half_sweep(L, J, s, orc.MET, k % 2, p)
        e1 = orc.energy(L, J, s)
        assert e1 <= e + 1e-9
        e = e1


def test_metropolis_margin_reports_decision_gap(orc):
    p = orc.Params(key=orc.key(5), beta=1.0, hits=4, proposal=orc.PROP_BALL, step=0.5)
    rng = np.random.default_rng(6)
    for t in range(100):
        s = rng.standard_normal(3)
        s /= np.linalg.norm(s)
        h = rng.standard_normal(3)
        out, m = orc.update_site(orc.MET, s, h, p, t, 0)
        assert 0 <= m < math.inf
        assert abs(np.linalg.norm(out) - 1) < 1e-12


# --------------------------------------------------------------------------
# Heat-bath
# --------------------------------------------------------------------------

@pytest.mark.parametrize("x", [0.05, 1.0, 3.3, 12.0])
def test_heatbath_draws_follow_boltzmann_density(orc, x):
    """At fixed h, t = s'.h/|h| has density x e^{x t} / (2 sinh x) on [-1,1]
    (KS test), mean coth x - 1/x, and an isotropic azimuth about h."""
    rng = np.random.default_rng(int(x * 100))
    h = rng.standard_normal(3)
    h[2] = -abs(h[2])  # exercise the n_z < 0 branch of the frame
    h *= 2.0 / np.linalg.norm(h)
    beta = x / 2.0
    key = orc.key(77)
    n = 6000
    t = np.empty(n)
    perp = np.empty((n, 3))
    hh = h / 2.0
    for k in range(n):
        p = orc.Params(key=key, sweep=k // 1000, beta=beta)
        out, _ = orc.update_site(orc.HB, np.zeros(3), h, p, k % 1000, 0)
        assert abs(np.linalg.norm(out) - 1.0) < 1e-12
        t[k] = np.dot(out, hh)
        perp[k] = out - t[k] * hh

    def cdf(v):
        v = np.clip(v, -1, 1)
        return np.expm1(x * (v + 1)) / np.expm1(2 * x)

    assert stats.kstest(t, cdf).pvalue > 1e-3
    assert abs(np.mean(t) - langevin(x)) < 5 * np.std(t) / np.sqrt(n)
    # azimuth: angle of the perpendicular part in an independent frame
    a = np.cross(hh, [1.0, 0.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(hh, a)
    ang = np.mod(np.arctan2(perp @ b, perp @ a), 2 * np.pi)
    assert stats.kstest(ang, stats.uniform(0, 2 * np.pi).cdf).pvalue > 1e-3


def test_heatbath_ignores_old_spin_and_handles_zero_field(orc):
    p = orc.Params(key=orc.key(8), beta=2.0)
    h = np.array([0.3, -1.2, 0.4])
    a, _ = orc.update_site(orc.HB, np.array([1.0, 0, 0]), h, p, 5, 1)
    b, _ = orc.update_site(orc.HB, np.array([0, 0, -1.0]), h, p, 5, 1)
    assert np.array_equal(a, b)
    z, _ = orc.update_site(orc.HB, np.array([1.0, 0, 0]), np.zeros(3), p, 5, 1)
    assert abs(np.linalg.norm(z) - 1) < 1e-12
    for hz in (0.0, -0.0, 1.0, -1.0):
        hv = np.array([0.0, 0.0, hz]) if hz != 0 else np.array([1.0, 0.0, hz])
        o, _ = orc.update_site(orc.HB, np.zeros(3), hv, p, 9, 0)
        assert abs(np.linalg.norm(o) - 1) < 1e-12


# --------------------------------------------------------------------------
# Statistical closed forms of whole sweeps
# --------------------------------------------------------------------------

def _binned_mean(series, nbins=20):
    bins = np.array_split(np.asarray(series), nbins)
    m = np.array([b.mean() for b in bins])
    return m.mean(), m.std(ddof=1) / np.sqrt(len(m))


RING_CASES = [
    # (kind, proposal, hits, n_or, beta, sweeps)
    (1, 0, 1, 0, 1.0, 1200),
    (1, 1, 4, 0, 2.0, 800),
    (2, 0, 1, 0, 1.0, 800),
    (2, 0, 1, 1, 2.0, 600),
]


@pytest.mark.parametrize("case", RING_CASES)
def test_decoupled_rings_give_langevin_energy(orc, case):
    """J_x = 1, J_y = J_z = 0: L^2 independent periodic rings of L spins.  The
    bond correlation of a long classical Heisenberg ring is L(beta) =
    coth(beta) - 1/beta (ring corrections ~ L(beta)^L < 1e-4 here), so the
    equilibrium E/N = -L(beta).  A wrong sign of dE, a wrong acceptance
    exponent or a wrong heat-bath density moves the mean far outside 3 sigma."""
    kind, proposal, hits, n_or, beta, n = case
    L = 16
    J = inputs.uniform_couplings(L, axes=(0,))
    s = orc.init_spins(L, seed=2)
    sch = orc.Schedule(kind=kind, proposal=proposal, hits=hits, step=0.5, n_or=n_or, beta=beta,
                       energy_every=1)
    sw, elog = orc.sweeps(L, J, s, sch, orc.key(2), n)
    assert sw == n
    burn = n // 5
    mean, err = _binned_mean(elog[burn:])
    want = -langevin(beta)
    assert abs(mean - want) < 3 * err + 1e-4, (mean, err, want)
    assert err < 0.01


def test_high_temperature_gaussian_glass_energy(orc):
    """Gaussian J at small beta: each bond contributes -J L(beta J), so
    E/N = -beta E[J^2] + (beta^3/15) E[J^4] + O(beta^4) = -beta + 0.2 beta^3."""
    L = 8
    beta = 0.15
    J = inputs.gaussian_couplings(L, seed=71)
    s = orc.init_spins(L, seed=72)
    sch = orc.Schedule(kind=orc.HB, beta=beta, energy_every=1)
    _, elog = orc.sweeps(L, J, s, sch, orc.key(72), 1500)
    mean, err = _binned_mean(elog[100:])
    # the sample's own J moments replace the ensemble ones
    j2 = np.mean(J ** 2)
    j4 = np.mean(J ** 4)
    want = 3 * (-beta * j2 / 3 + beta ** 3 * j4 / 45)
    assert abs(mean - want) < 3 * err + 2e-4, (mean, err, want)


def test_renorm_makes_unit_and_keeps_direction(orc):
    L = 4
    rng = np.random.default_rng(9)
    s = (rng.standard_normal(3 * L ** 3) * rng.uniform(0.5, 2.0)).astype(np.float64)
    d0 = s.reshape(-1, 3) / np.linalg.norm(s.reshape(-1, 3), axis=1, keepdims=True)
    orc.renorm(L, s)
    v = s.reshape(-1, 3)
    assert np.max(np.abs(np.linalg.norm(v, axis=1) - 1)) < 1e-15
    assert np.allclose(v, d0, atol=1e-15)


def test_ball_proposal_matches_rejection_sampled_ball(orc):
    """At beta = 0 one ball hit from s = e_z gives s' = (e_z + 0.5 u)/|.|
    with u uniform in the unit ball; compare s'_z with the same map applied
    to points drawn uniform in the ball by rejection from the cube."""
    L = 8
    J = inputs.gaussian_couplings(L, seed=81)
    got = []
    for sw in range(3):
        s = inputs.aligned_spins(L, (0, 0, 1))
        p = orc.Params(key=orc.key(81), sweep=sw, beta=0.0, hits=1, proposal=orc.PROP_BALL, step=0.5)
        orc.half_sweep(L, J, s, orc.MET, 0, p)
        col = np.array([orc.colour(L, i) for i in range(L ** 3)])
        got.append(s.reshape(-1, 3)[col == 0, 2])
    got = np.concatenate(got)
    rng = np.random.default_rng(82)
    cube = rng.uniform(-1, 1, size=(40000, 3))
    ball = cube[np.sum(cube ** 2, axis=1) <= 1.0]
    v = np.array([0.0, 0.0, 1.0]) + 0.5 * ball
    ref = v[:, 2] / np.linalg.norm(v, axis=1)
    assert stats.ks_2samp(got, ref).pvalue > 1e-3


def test_gaussian_couplings_are_standard_normal(orc):
    """Philox + Box-Muller couplings: KS against N(0,1), mean 0, variance 1,
    the two members of a Box-Muller pair uncorrelated, even fourth moment 3;
    distinct samples give distinct disorder, the same sample the same."""
    L = 16
    J = orc.gaussian_couplings(L, seed=4, sample=7)
    n = J.size
    assert stats.kstest(J, stats.norm.cdf).pvalue > 1e-3
    assert abs(J.mean()) < 4 / np.sqrt(n)
    assert abs(J.var() - 1) < 4 * np.sqrt(2 / n)
    assert abs(np.mean(J ** 4) - 3) < 4 * np.sqrt(96 / n)
    Jm = J.reshape(-1, 3)
    for a, b in ((0, 1), (0, 2), (1, 2)):
        assert abs(np.corrcoef(Jm[:, a], Jm[:, b])[0, 1]) < 4 / np.sqrt(len(Jm))
    assert np.array_equal(J, orc.gaussian_couplings(L, seed=4, sample=7))
    assert not np.allclose(J, orc.gaussian_couplings(L, seed=4, sample=8))


def test_fused_metropolis_over_relaxation_keeps_the_metropolis_energy(orc):
    """The fused pass reflects the Metropolis result about the same field: the
    site energy -s.h equals that of the Metropolis result alone, the
    projection on h is kept, the perpendicular part flipped."""
    rng = np.random.default_rng(12)
    for t in range(200):
        s = rng.standard_normal(3)
        s /= np.linalg.norm(s)
        h = rng.standard_normal(3) * 2
        p = orc.Params(key=orc.key(12), sweep=t, beta=1.3, hits=3, proposal=orc.PROP_BALL, step=0.5)
        met, m1 = orc.update_site(orc.MET, s, h, p, t, t % 2)
        fused, m2 = orc.update_site(orc.MET_OR, s, h, p, t, t % 2)
        assert m1 == m2
        hh = h / np.linalg.norm(h)
        assert abs(np.dot(fused, h) - np.dot(met, h)) < 1e-13
        assert np.allclose(fused - np.dot(fused, hh) * hh, -(met - np.dot(met, hh) * hh), atol=1e-14)
        assert abs(np.linalg.norm(fused) - 1) < 1e-12


def test_fused_metropolis_over_relaxation_rings_give_langevin_energy(orc):
    """The fused chain samples the Boltzmann distribution too: decoupled
    rings at beta = 1.5 give E/N = -L(beta)."""
    L, beta, n = 16, 1.5, 800
    J = inputs.uniform_couplings(L, axes=(0,))
    s = orc.init_spins(L, seed=3)
    sch = orc.Schedule(kind=orc.MET_OR, proposal=orc.PROP_BALL, hits=2, step=0.5, beta=beta, energy_every=1)
    _, elog = orc.sweeps(L, J, s, sch, orc.key(3), n)
    mean, err = _binned_mean(elog[n // 5:])
    assert abs(mean + langevin(beta)) < 3 * err + 1e-4, (mean, err)


def test_oracle_reproduces_the_golden_fixture(orc):
    """tests/golden/l6_seed21.json holds the oracle's own results for one
    L = 6 lattice (written by tests/golden/make_golden.py, which calls only
    the oracle): the oracle must still produce every stored value exactly,
    so a change to its arithmetic cannot pass unnoticed (the fixture is then
    rewritten by that script, deliberately)."""
    import importlib.util
    import json
    import os
    import platform

    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(here, "l6_seed21.json")) as f:
        want = json.load(f)
    got = json.loads(json.dumps(mg.compute()))
    if platform.machine() in ("x86_64", "AMD64"):  # where the fixture was written: bit for bit
        assert got == want
        return
    # another libm may round exp/log/sin/cbrt an ulp differently
    def numbers(v):
        if isinstance(v, dict):
            return [x for key in sorted(v) for x in numbers(v[key])]
        if isinstance(v, list):
            return [x for e in v for x in numbers(e)]
        return [float(v)] if isinstance(v, (int, float)) else []

    assert got.keys() == want.keys() and got["source"] == want["source"]
    for k in want:
        assert np.allclose(numbers(got[k]), numbers(want[k]), rtol=0, atol=1e-12), k
