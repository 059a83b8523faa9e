"""hsg_energy_noalloc: the energy entry point for callers that cannot let a
library allocate device memory (their own arena owns it all, or an
allocation's synchronisation is too costly for them).  Its result must match
the FP64 oracle's energy of the same state, and hsg_energy of a context on
that state, call after call, although the fixed scratch array keeps each
call's partial sums (needs a CUDA GPU).

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1006_2566_gb300 import inputs  # noqa: E402

TOL = 2e-6  # the energy tolerance of the other parity tests


@pytest.fixture(scope="module")
def hsg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_2566_gb300 import build

    build.build()
    oracle.build()
    from paper_1006_2566_gb300 import hsg as h

    return h


def test_energy_without_allocation_matches_oracle_and_context(hsg):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    sched = hsg.schedule(kind=hsg.HSG_HEATBATH, T=0.5, n_or=1)
    # successive calls on different sizes: a smaller lattice after a larger
    # one must not pick up the larger call's leftover partial sums
    for call, (L, seed) in enumerate([(40, 5), (8, 6), (40, 7), (64, 8)]):
        J = inputs.gaussian_couplings(L, seed=seed, dtype=np.float32)
        with hsg.Lattice(L, seed) as lat:
            lat.set_couplings(J)
            lat.sweep(sched, 2)
            e_ctx = lat.energy()
            spins = torch.empty(3 * L ** 3, dtype=torch.float32, device="cuda")
            hsg.hsg_get_spins(lat.ctx, spins)
            torch.cuda.synchronize()
        e_ref = oracle.energy(L, J.astype(np.float64), spins.cpu().numpy().astype(np.float64)) / L ** 3
        Jd = torch.from_numpy(J).cuda()
        for repeat in range(2):  # two calls in a row on the same state
            hsg.hsg_energy_noalloc(L, spins, Jd, out)
            torch.cuda.synchronize()
            got = out.item()
            assert abs(got - e_ref) <= TOL, (call, repeat, L, got, e_ref)
            assert abs(got - e_ctx) <= TOL, (call, repeat, L, got, e_ctx)
            out.fill_(float("nan"))


def test_energy_without_allocation_rejects_bad_sizes(hsg):
    d = torch.zeros(3 * 8 ** 3, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for L in (1626, 2000, 7, 2):
        with pytest.raises(hsg.HsgError) as e:
            hsg.hsg_energy_noalloc(L, d, d, out)
        assert e.value.status == hsg.HSG_EINVAL
        assert "L must be even" in hsg.hsg_last_error(None)


def test_energy_without_allocation_rejects_bad_arrays_before_any_launch(hsg):
    """Wrong dtypes, arrays too short for L and host memory are refused on the
    host: by the binding (it knows the tensors' lengths) and, for a host
    pointer handed to the C entry point directly, by the library."""
    L = 8
    n = 3 * L ** 3
    spins = torch.zeros(n, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    bad = [
        (spins.double(), spins, out),  # fp64 spins
        (spins, spins.double(), out),  # fp64 J
        (spins, spins, torch.zeros(1, dtype=torch.float32, device="cuda")),  # fp32 output
        (spins[: n - 1], spins, out),  # one element short
        (spins, spins[: n - 3], out),
        (spins, spins, out[:0]),  # empty output
        (spins.cpu(), spins, out),  # host tensor
    ]
    for args in bad:
        with pytest.raises(ValueError):
            hsg.hsg_energy_noalloc(L, *args)
    host = np.zeros(n, dtype=np.float32)
    host_out = np.zeros(1, dtype=np.float64)
    lib = hsg._lib
    dptr, optr = ctypes.c_void_p(spins.data_ptr()), ctypes.c_void_p(out.data_ptr())
    for args in [(host.ctypes.data, dptr, optr), (dptr, host.ctypes.data, optr), (dptr, dptr, host_out.ctypes.data)]:
        assert lib.hsg_energy_noalloc(L, *args, None) == hsg.HSG_EINVAL
        assert "device" in hsg.hsg_last_error(None)
    # the library is still usable afterwards
    hsg.hsg_energy_noalloc(L, spins, spins, out)
    torch.cuda.synchronize()
    assert out.item() == 0.0
