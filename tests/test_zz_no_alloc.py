"""hsg_energy_noalloc: the energy entry point for callers that cannot let a
library allocate device memory (their own arena owns it all, or an
allocation's synchronisation is too costly for them).  Its result must match
hsg_energy of a context on the same state, call after call, although the
fixed scratch array keeps each call's partial sums (needs a CUDA GPU).

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1006_2566_gb300 import inputs  # noqa: E402

TOL = 2e-6  # the energy tolerance of the other parity tests


@pytest.fixture(scope="module")
def hsg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_2566_gb300 import build

    build.build()
    from paper_1006_2566_gb300 import hsg as h

    return h


def test_energy_without_allocation_matches_context_energy(hsg):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    sched = hsg.schedule(kind=hsg.HSG_HEATBATH, T=0.5, n_or=1)
    # successive calls on different sizes: a smaller lattice after a larger
    # one must not pick up the larger call's leftover partial sums
    for call, (L, seed) in enumerate([(40, 5), (8, 6), (40, 7), (64, 8)]):
        J = inputs.gaussian_couplings(L, seed=seed, dtype=np.float32)
        with hsg.Lattice(L, seed) as lat:
            lat.set_couplings(J)
            lat.sweep(sched, 2)
            e_ref = lat.energy()
            spins = torch.empty(3 * L ** 3, dtype=torch.float32, device="cuda")
            hsg.hsg_get_spins(lat.ctx, spins)
            torch.cuda.synchronize()
        Jd = torch.from_numpy(J).cuda()
        hsg.hsg_energy_noalloc(L, spins, Jd, out)
        torch.cuda.synchronize()
        got = out.item()
        assert abs(got - e_ref) <= TOL, (call, L, got, e_ref)
        out.fill_(float("nan"))


def test_energy_without_allocation_rejects_bad_sizes(hsg):
    d = torch.zeros(3 * 8 ** 3, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for L in (1626, 2000, 7, 2):
        with pytest.raises(hsg.HsgError) as e:
            hsg.hsg_energy_noalloc(L, d, d, out)
        assert e.value.status == hsg.HSG_EINVAL
        assert "L must be even" in hsg.hsg_last_error(None)
