"""The largest lattice the library accepts, L = 1624 (N = 4.28e9 sites, site
indices just below 2^32, N/2 just below 2^31), checked on sampled sites that
the oracle computes one by one (needs a CUDA GPU with ~190 GB free).

A whole copy of this lattice would be 51 GB per array, so the sites and
their six neighbours come back through hsg_get_sites, and the oracle's
local_field_nb forms Eq. 2 from them.  Covered: device couplings and spin
initialisation, a global over-relaxation and heat-bath half-sweep, a
temporally blocked over-relaxation sweep, FP64 energies (an over-relaxation
half-sweep conserves E to round-off), at sites spread over the lattice and at
its corners, its last plane and the indices around 2^31.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from parity_rules import record  # noqa: E402

TOL = 1e-5
U32 = 2.0 ** -24
L = 1624
N = L ** 3
SEED = 11
T = 0.5


@pytest.fixture(scope="module")
def hsg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 200 * 2 ** 30:
        pytest.skip(f"needs ~190 GB of free device memory, {free / 2 ** 30:.0f} GiB free")
    from paper_1006_2566_gb300 import build

    build.build()
    oracle.build()
    from paper_1006_2566_gb300 import hsg as h

    return h


def coords(i):
    return i % L, (i // L) % L, i // (L * L)


def idx(x, y, z):
    return (x % L) + (y % L) * L + (z % L) * L * L


def neighbour_sites(i):
    """+x, -x, +y, -y, +z, -z neighbours (local_field_nb's order)."""
    x, y, z = coords(i)
    return [idx(x + 1, y, z), idx(x - 1, y, z), idx(x, y + 1, z), idx(x, y - 1, z), idx(x, y, z + 1),
            idx(x, y, z - 1)]


def samples(colour, rng, n=1500):
    cand = rng.integers(0, N, size=6 * n, dtype=np.int64)
    x, y, z = cand % L, (cand // L) % L, cand // (L * L)
    pick = [int(i) for i in cand[(x + y + z) % 2 == colour][:n]]
    edges = [0, 1, L - 1, L * L - 1, L * L, N - 1, N - 2, N - L, N - L * L, 2 ** 31 - 1, 2 ** 31, 2 ** 31 + 1,
             (N // 2) - 1, N // 2, idx(L - 1, L - 1, L // 2), idx(0, L - 1, L - 1)]
    return pick + [i for i in edges if sum(coords(i)) % 2 == colour]


def state_of(hsg, lat, sites):
    """Spins of the sites, and for each its neighbours' spins and six bonds."""
    allsites = []
    for i in sites:
        allsites += [i] + neighbour_sites(i)
    s, b = hsg.hsg_get_sites(lat.ctx, np.array(allsites, dtype=np.uint32))
    s = s.astype(np.float64).reshape(len(sites), 7, 3)
    b = b.astype(np.float64).reshape(len(sites), 7, 3)
    own = s[:, 0]
    nb = s[:, 1:]
    # bonds: +d from the site itself, -d from the -d neighbour's +d bond
    bonds = np.stack([b[:, 0, 0], b[:, 2, 0], b[:, 0, 1], b[:, 4, 1], b[:, 0, 2], b[:, 6, 2]], axis=1)
    return own, nb, bonds


def tolerance(bonds, h):
    """1e-5 at every site (tests/parity_rules.py), and whether the site's
    fp32 field is ill-conditioned (4 kappa > 1e-5), which the record counts."""
    kappa = U32 * float(np.sum(np.abs(bonds))) / max(float(np.linalg.norm(h)), 1e-300)
    return TOL, 4 * kappa > TOL


def check_half_sweep(hsg, lat, sites, upd, colour, params, before):
    """`before` = state_of the sites before the half-sweep; compare the
    sites' new spins with the oracle's update from the same inputs."""
    own0, nb0, bonds0 = before
    after, _ = hsg.hsg_get_sites(lat.ctx, np.array(sites, dtype=np.uint32), want_bonds=False)
    skipped = ill = 0
    err_max = 0.0
    for k, i in enumerate(sites):
        h = oracle.local_field_nb(nb0[k], bonds0[k])
        if upd == oracle.HB and abs(h[2]) < TOL * np.linalg.norm(h):
            skipped += 1  # frame-branch band (tests/parity_rules.py)
            continue
        want, _ = oracle.update_site(upd, own0[k], h, params, i, colour)
        tol, is_ill = tolerance(bonds0[k], h)
        ill += is_ill
        err = float(np.max(np.abs(after[k].astype(np.float64) - want)))
        err_max = max(err_max, err)
        assert err <= tol, (i, after[k], want)
    record(label=f"L=1624 sampled half-sweep upd {upd} c{colour}", L=L, colour=colour, sites=len(sites),
           excluded=skipped, ill_conditioned=ill, max_err=err_max)
    assert skipped <= 3


def test_max_size_lattice_sampled_sites(hsg):
    rng = np.random.default_rng(1624)
    s0, s1 = samples(0, rng), samples(1, rng)
    with hsg.Lattice(L, SEED, stream=torch.cuda.Stream()) as lat:
        lat.generate_couplings()
        # initial spins and device couplings against the oracle's Philox maps
        probe = np.array(s0[:300] + s1[:300], dtype=np.uint32)
        spins, bonds = hsg.hsg_get_sites(lat.ctx, probe)
        assert np.max(np.abs(spins - oracle.init_spin_sites(probe, SEED))) < 1e-6
        ref = oracle.gaussian_coupling_sites(probe, SEED).astype(np.float32)
        np.testing.assert_array_max_ulp(bonds, ref, maxulp=1)
        e0 = lat.energy()
        assert abs(e0) < 1e-3  # random spins: E/N ~ N^-1/2

        p = oracle.Params(key=oracle.key(SEED), sweep=0, beta=1.0 / T)
        sched = hsg.schedule(kind=hsg.HSG_HEATBATH, T=T, kernel=hsg.HSG_KERNEL_GLOBAL)
        # over-relaxation on colour 0 (global kernel): per site, and E conserved
        before = state_of(hsg, lat, s0)
        lat.half_sweep(sched, hsg.HSG_OVERRELAX, 0)
        check_half_sweep(hsg, lat, s0, oracle.OR, 0, p, before)
        e1 = lat.energy()
        assert abs(e1 - e0) <= 2e-6
        # heat-bath on colour 1 at sweep 0
        before = state_of(hsg, lat, s1)
        lat.half_sweep(sched, hsg.HSG_HEATBATH, 1)
        check_half_sweep(hsg, lat, s1, oracle.HB, 1, p, before)

        # one temporally blocked over-relaxation sweep: colour 0 from the old
        # colour 1, then colour 1 from the new colour 0
        before0 = state_of(hsg, lat, s0)
        own1_old, _ = hsg.hsg_get_sites(lat.ctx, np.array(s1, dtype=np.uint32), want_bonds=False)
        e2 = lat.energy()
        lat.sweep(hsg.schedule(kind=hsg.HSG_NONE, n_or=1, kernel=hsg.HSG_KERNEL_WAVE), 1)
        check_half_sweep(hsg, lat, s0, oracle.OR, 0, p, before0)
        own1_new, nb_new, bonds1 = state_of(hsg, lat, s1)  # neighbours: the new colour 0
        ill = 0
        err_max = 0.0
        for k, i in enumerate(s1):
            h = oracle.local_field_nb(nb_new[k], bonds1[k])
            want, _ = oracle.update_site(oracle.OR, own1_old[k].astype(np.float64), h, p, i, 1)
            tol, is_ill = tolerance(bonds1[k], h)
            ill += is_ill
            err = float(np.max(np.abs(own1_new[k] - want)))
            err_max = max(err_max, err)
            assert err <= tol, (i, own1_new[k], want)
        record(label="L=1624 sampled wave OR sweep c1", L=L, colour=1, sites=len(s1), excluded=0,
               ill_conditioned=ill, max_err=err_max)
        e3 = lat.energy()
        assert abs(e3 - e2) <= 4e-6
        assert lat.sweep_count == 1
