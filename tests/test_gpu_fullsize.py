"""Full-size parity: the benchmark's L = 256 lattice, schedule and launch
configuration, checked on sampled sites that the oracle computes one by one,
and on the whole-lattice energy (needs a CUDA GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1006_2566_gb300 import inputs  # noqa: E402

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
    """1e-5 where the fp32 field is well conditioned (4 kappa <= 1e-5,
    kappa = 2^-24 sum|J| / |h|), else 1e-5 + 64 kappa (see test_gpu_parity)."""
    x, y, z = coords(i)
    bonds = [J[3 * i], J[3 * i + 1], J[3 * i + 2],
             J[3 * ((x - 1) % L + y * L + z * L * L)],
             J[3 * (x + ((y - 1) % L) * L + z * L * L) + 1],
             J[3 * (x + y * L + ((z - 1) % L) * L * L) + 2]]
    kappa = U32 * float(np.sum(np.abs(bonds))) / max(float(np.linalg.norm(h)), 1e-300)
    return (TOL, False) if 4 * kappa <= TOL else (TOL + 64 * kappa, True)


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
    rng = np.random.default_rng(2024)
    cand = rng.integers(0, L ** 3, size=12000)
    col = np.array([sum(coords(int(i))) % 2 for i in cand])
    # edges of the lattice and of the kernels' tiles are in the sample too
    extra = [0, L - 1, L * L - 1, L ** 3 - 1, L * (L - 1), (L - 1) * L * L, 63, 64, 7 * L, 8 * L, 15 * L * L,
             16 * L * L]
    hb_sites = list(cand[col == 0][:3000]) + [i for i in extra if sum(coords(i)) % 2 == 0]
    or_sites = list(cand[col == 1][:3000]) + [i for i in extra if sum(coords(i)) % 2 == 1]

    p = oracle.Params(key=oracle.key(SEED), sweep=sweep, beta=1.0 / T)
    skipped = ill = 0
    for i in hb_sites:
        i = int(i)
        h = oracle.local_field(L, Jd, pre64, i)
        if abs(h[2]) < TOL * np.linalg.norm(h):
            skipped += 1  # frame-branch band, see the tolerance notes of test_gpu_parity
            continue
        want, _ = oracle.update_site(oracle.HB, pre64[3 * i: 3 * i + 3], h, p, i, 0)
        tol, is_ill = site_tolerance(Jd, i, h)
        ill += is_ill
        assert float(np.max(np.abs(mid64[3 * i: 3 * i + 3] - want))) <= tol, i
    assert skipped <= 3
    for i in or_sites:
        i = int(i)
        h = oracle.local_field(L, Jd, mid64, i)
        want, _ = oracle.update_site(oracle.OR, mid64[3 * i: 3 * i + 3], h, p, i, 1)
        tol, is_ill = site_tolerance(Jd, i, h)
        ill += is_ill
        assert float(np.max(np.abs(post64[3 * i: 3 * i + 3] - want))) <= tol, i
    assert ill <= 10
    # the heat-bath half-sweep touched only colour 0, the OR half-sweep only colour 1
    g = np.indices((L, L, L)).sum(axis=0).reshape(-1) % 2
    assert np.array_equal(pre.reshape(-1, 3)[g == 1], mid.reshape(-1, 3)[g == 1])
    assert np.array_equal(mid.reshape(-1, 3)[g == 0], post.reshape(-1, 3)[g == 0])
    e_ref = oracle.energy(L, Jd, post64) / L ** 3
    assert abs(e_gpu - e_ref) <= 2e-6
