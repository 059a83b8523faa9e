"""The packed spin layout (HSG_LAYOUT_PACKED: three fp32 arrays per colour,
12 bytes a spin) through the C ABI (needs a CUDA GPU).

The packed global kernel hands the site code the same float4 values as the
float4 layout, so every result must be bit-identical to the float4 lattice:
initial spins, spin upload and read-back, all update kinds, whole sweeps
with renormalisation and energy log, graph replay, sampled site reads.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import parity_rules  # noqa: E402
from paper_1006_2566_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def hsg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_2566_gb300 import build

    build.build()
    oracle.build()
    from paper_1006_2566_gb300 import hsg as h

    return h


def run(hsg, L, layout, sched_kw, n, stream=None, spins=None):
    with hsg.Lattice(L, 13, stream=stream, layout=layout) as lat:
        lat.generate_couplings()
        if spins is not None:
            lat.set_spins(spins)
        s0 = lat.spins()
        lat.sweep(hsg.schedule(**sched_kw), n)
        sites = np.array([0, L ** 3 - 1, L * L + 3, (L ** 3) // 2 + 1], dtype=np.uint32)
        return s0, lat.spins(), lat.energy_log(), lat.energy(), hsg.hsg_get_sites(lat.ctx, sites)


KINDS = {"HB": dict(kind=2, T=0.4), "MET": dict(kind=1, hits=3, proposal=1, step=0.5, T=0.6),
         "METOR": dict(kind=4, hits=2, proposal=0, T=0.9), "OR": dict(kind=0)}


@pytest.mark.parametrize("L", [4, 6, 16, 34, 66])
@pytest.mark.parametrize("kind", sorted(KINDS))
def test_packed_layout_is_bit_identical_to_float4(hsg, L, kind):
    kw = dict(KINDS[kind], n_or=2, renorm_every=2, energy_every=1)
    a = run(hsg, L, hsg.HSG_LAYOUT_FLOAT4, kw, 3)
    b = run(hsg, L, hsg.HSG_LAYOUT_PACKED, kw, 3)
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    assert np.array_equal(a[4][0], b[4][0]) and np.array_equal(a[4][1], b[4][1])


def test_packed_graph_replay_and_uploaded_spins(hsg):
    L = 24
    s_in = inputs.random_spins(L, seed=3, dtype=np.float32)
    kw = dict(kind=hsg.HSG_HEATBATH, T=0.5, n_or=4, renorm_every=5, energy_every=5)
    a = run(hsg, L, hsg.HSG_LAYOUT_FLOAT4, kw, 12, stream=None, spins=s_in)
    b = run(hsg, L, hsg.HSG_LAYOUT_PACKED, kw, 12, stream=torch.cuda.Stream(), spins=s_in)
    assert np.array_equal(a[0], s_in) and np.array_equal(b[0], s_in)
    for x, y in zip(a[1:4], b[1:4]):
        assert np.array_equal(x, y)


def test_packed_half_sweep_matches_oracle(hsg):
    """Over-relaxation and heat-bath half-sweeps of a packed lattice, both
    colours, against the oracle layer by layer under the parity rules of
    the float4 tests (every site within 1e-5, the other colour unchanged)."""
    L = 16
    J = inputs.gaussian_couplings(L, seed=5)
    Jr = inputs.round_to_f32(J)
    s32 = inputs.random_spins(L, seed=6, dtype=np.float32)
    params = oracle.Params(key=oracle.key(1), beta=1.0 / 0.5)
    with hsg.Lattice(L, 1, layout=hsg.HSG_LAYOUT_PACKED) as lat:
        lat.set_couplings(J)
        lat.set_spins(s32)
        before = lat.spins()
        for upd, kind in ((oracle.OR, hsg.HSG_OVERRELAX), (oracle.HB, hsg.HSG_HEATBATH)):
            for colour in (0, 1):
                lat.half_sweep(hsg.schedule(T=0.5), kind, colour)
                after = lat.spins()
                parity_rules.check_layer(L, Jr, before, after, upd, colour, params, label=f"packed {upd} c{colour}")
                before = after


def test_packed_layout_rejects_staged_kernels(hsg):
    with hsg.Lattice(8, 1, layout=hsg.HSG_LAYOUT_PACKED) as lat:
        lat.generate_couplings()
        assert hsg.hsg_kernel_for(lat.ctx, hsg.schedule(n_or=1)) == hsg.HSG_KERNEL_GLOBAL
        for k in (hsg.HSG_KERNEL_SLAB, hsg.HSG_KERNEL_WAVE):
            with pytest.raises(hsg.HsgError) as e:
                lat.sweep(hsg.schedule(n_or=1, kernel=k), 1)
            assert e.value.status == hsg.HSG_EINVAL
    with pytest.raises(hsg.HsgError) as e:
        hsg.Lattice(8, 1, layout=7)
    assert e.value.status == hsg.HSG_EINVAL
