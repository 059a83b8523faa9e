"""Full-size parity: the benchmark's L = 256 lattice, schedule and launch
configuration, checked on sampled sites that the oracle computes one by one,
and on the whole-lattice energy (needs a CUDA GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1006_2566_gb300 import inputs  # noqa: E402
from parity_rules import record  # noqa: E402

TOL = 1e-5
L = 256
SEED = 3
T = 0.3


@pytest.fixture(scope="module")
def hsg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_2566_gb300 import build

    build.build()
    oracle.build()
    from paper_1006_2566_gb300 import hsg as h

    return h


U32 = 2.0 ** -24


def coords(i):
    return i % L, (i // L) % L, i // (L * L)


def site_tolerance(J, i, h):
    """1e-5 at every site (tests/parity_rules.py), and whether the site's
    fp32 field is ill-conditioned (4 kappa > 1e-5, kappa = 2^-24 sum|J| /
    |h|), which the record counts."""
    x, y, z = coords(i)
    bonds = [J[3 * i], J[3 * i + 1], J[3 * i + 2],
             J[3 * ((x - 1) % L + y * L + z * L * L)],
             J[3 * (x + ((y - 1) % L) * L + z * L * L) + 1],
             J[3 * (x + y * L + ((z - 1) % L) * L * L) + 2]]
    kappa = U32 * float(np.sum(np.abs(bonds))) / max(float(np.linalg.norm(h)), 1e-300)
    return TOL, 4 * kappa > TOL


def check_sites(label, Jd, before64, after64, sites, upd, colour, p):
    """The listed sites of one half-sweep layer against the oracle's update
    of each from `before64` (the rules of tests/parity_rules.py: 1e-5 per
    component; heat-bath sites in the frame-branch band left out, at most 3)."""
    skipped = ill = 0
    err_max = err_ill = 0.0
    for i in sites:
        i = int(i)
        h = oracle.local_field(L, Jd, before64, i)
        if upd == oracle.HB and abs(h[2]) < TOL * np.linalg.norm(h):
            skipped += 1
            continue
        want, _ = oracle.update_site(upd, before64[3 * i: 3 * i + 3], h, p, i, colour)
        tol, is_ill = site_tolerance(Jd, i, h)
        err = float(np.max(np.abs(after64[3 * i: 3 * i + 3] - want)))
        ill += is_ill
        err_max = max(err_max, err)
        if is_ill:
            err_ill = max(err_ill, err)
        assert err <= tol, (label, i, err, tol)
    record(label=label, L=L, colour=colour, sites=len(sites), excluded=skipped, ill_conditioned=ill,
           max_err=err_max, max_err_ill=err_ill)
    assert skipped <= 3


def sample_sites(rng, n_per_colour):
    """Random sites of each colour plus the lattice's and the kernels'
    tile edges."""
    cand = rng.integers(0, L ** 3, size=4 * n_per_colour)
    col = np.array([sum(coords(int(i))) % 2 for i in cand])
    extra = [0, L - 1, L * L - 1, L ** 3 - 1, L * (L - 1), (L - 1) * L * L, 63, 64, 7 * L, 8 * L, 15 * L * L,
             16 * L * L, 13 * L, 14 * L, 27 * L + 30, 28 * L + 33, (L // 3) * L * L + 14 * L + 31]
    return [[int(i) for i in cand[col == c][:n_per_colour]] + [i for i in extra if sum(coords(i)) % 2 == c]
            for c in (0, 1)]


@pytest.mark.parametrize("variant", [0, 2])  # HSG_KERNEL_AUTO (what the bench runs), HSG_KERNEL_SLAB
def test_full_size_sampled_sites_and_energy(hsg, variant):
    J = inputs.gaussian_couplings(L, seed=SEED, dtype=np.float32)
    sched = hsg.schedule(kind=hsg.HSG_HEATBATH, T=T, n_or=4, renorm_every=10, energy_every=10, kernel=variant)
    with hsg.Lattice(L, SEED) as lat:
        lat.set_couplings(J)
        lat.sweep(sched, 2)
        sweep = lat.sweep_count
        pre = lat.spins()
        lat.half_sweep(sched, hsg.HSG_HEATBATH, 0)
        mid = lat.spins()
        lat.half_sweep(sched, hsg.HSG_OVERRELAX, 1)
        post = lat.spins()
        e_gpu = lat.energy()
    Jd = J.astype(np.float64)
    pre64, mid64, post64 = (a.astype(np.float64) for a in (pre, mid, post))
    hb_sites, or_sites = sample_sites(np.random.default_rng(2024), 3000)

    p = oracle.Params(key=oracle.key(SEED), sweep=sweep, beta=1.0 / T)
    check_sites(f"L=256 heat-bath half-sweep c0 v{variant}", Jd, pre64, mid64, hb_sites, oracle.HB, 0, p)
    check_sites(f"L=256 OR half-sweep c1 v{variant}", Jd, mid64, post64, or_sites, oracle.OR, 1, p)
    # the heat-bath half-sweep touched only colour 0, the OR half-sweep only colour 1
    g = np.indices((L, L, L)).sum(axis=0).reshape(-1) % 2
    assert np.array_equal(pre.reshape(-1, 3)[g == 1], mid.reshape(-1, 3)[g == 1])
    assert np.array_equal(mid.reshape(-1, 3)[g == 0], post.reshape(-1, 3)[g == 0])
    e_ref = oracle.energy(L, Jd, post64) / L ** 3
    assert abs(e_gpu - e_ref) <= 2e-6


def test_full_size_wave_sweep_sampled_sites(hsg):
    """The benchmark's dominant kernel, the temporally blocked OR sweep, at
    L = 256 on a stream as the benchmark runs it: 3000+ sampled sites of
    each colour (random, lattice edges, tile edges), each layer under the
    strict rule -- colour 0 against the oracle's update from the state
    before the sweep, colour 1 against the oracle's update from the GPU's own
    new colour 0 beside the old colour 1 -- and the energy conserved."""
    J = inputs.gaussian_couplings(L, seed=SEED, dtype=np.float32)
    stream = torch.cuda.Stream()
    with hsg.Lattice(L, SEED, stream=stream) as lat:
        lat.set_couplings(J)
        lat.sweep(hsg.schedule(kind=hsg.HSG_HEATBATH, T=T, n_or=4, renorm_every=10, energy_every=10), 2)
        pre = lat.spins()
        e0 = lat.energy()
        sched = hsg.schedule(kind=hsg.HSG_NONE, n_or=1, kernel=hsg.HSG_KERNEL_AUTO)
        assert hsg.hsg_kernel_for(lat.ctx, sched) == hsg.HSG_KERNEL_WAVE
        lat.sweep(sched, 1)
        post = lat.spins()
        e1 = lat.energy()
    Jd = J.astype(np.float64)
    pre64, post64 = pre.astype(np.float64), post.astype(np.float64)
    g = (np.indices((L, L, L)).sum(axis=0).reshape(-1) % 2 == 0).repeat(3)
    mid64 = np.where(g, post64, pre64)  # the GPU's new colour 0 beside the old colour 1
    s0, s1 = sample_sites(np.random.default_rng(2025), 3000)
    p = oracle.Params()
    check_sites("L=256 wave OR sweep c0", Jd, pre64, post64, s0, oracle.OR, 0, p)
    check_sites("L=256 wave OR sweep c1", Jd, mid64, post64, s1, oracle.OR, 1, p)
    assert len(s0) + len(s1) >= 6000
    record(label="L=256 wave OR sweep energy change", L=L, max_err=abs(e1 - e0))
    assert abs(e1 - e0) <= 2e-6
