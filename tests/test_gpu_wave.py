"""Temporally blocked over-relaxation (HSG_KERNEL_WAVE) through the C ABI
(needs a CUDA GPU).

The wave kernel runs colour 0 and colour 1 of an over-relaxation sweep in one
pass, reading one spin buffer and writing the other; the main update of each
sweep stays two half-sweeps.  It evaluates every site with the same device
code as the half-sweep kernels, in the same order of colours, so the results
must be bit-identical to HSG_KERNEL_GLOBAL: spins, energy log, counters.
Sizes cover lattices smaller than one 16 x 14 tile, ragged edge tiles, a
single z chunk and several chunks; one case is also checked against the FP64
oracle directly.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1006_2566_gb300 import inputs  # noqa: E402
from parity_rules import check_or_sweep  # noqa: E402


@pytest.fixture(scope="module")
def hsg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_2566_gb300 import build

    build.build()
    oracle.build()
    from paper_1006_2566_gb300 import hsg as h

    return h


def run(hsg, L, sched_kw, n, kernel, stream=None, seed=31, J=None, spins=None):
    with hsg.Lattice(L, seed, stream=stream) as lat:
        if J is None:
            lat.generate_couplings()
        else:
            lat.set_couplings(J)
        if spins is not None:
            lat.set_spins(spins)
        lat.sweep(hsg.schedule(kernel=kernel, **sched_kw), n)
        return lat.spins(), lat.energy_log(), lat.sweep_count, lat.energy()


SIZES = [4, 6, 8, 10, 16, 18, 34, 66, 72, 130]


@pytest.mark.parametrize("L", SIZES)
@pytest.mark.parametrize("kind", ["HB", "OR"])
def test_wave_sweeps_are_bit_identical_to_half_sweeps(hsg, L, kind):
    kw = dict(T=0.7, n_or=2, renorm_every=2, energy_every=1)
    kw["kind"] = hsg.HSG_HEATBATH if kind == "HB" else hsg.HSG_NONE
    want = run(hsg, L, kw, 3, hsg.HSG_KERNEL_GLOBAL)
    got = run(hsg, L, kw, 3, hsg.HSG_KERNEL_WAVE)
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[1], want[1]) and len(got[1]) == 3
    assert got[2] == want[2] == 3
    assert got[3] == want[3]


@pytest.mark.parametrize("L", [8, 34])
def test_wave_with_metropolis_main_update(hsg, L):
    """Metropolis main updates stay half-sweeps in place; the OR sweeps after
    them go through the wave kernel and the buffer swaps."""
    kw = dict(kind=hsg.HSG_METROPOLIS, hits=3, proposal=hsg.HSG_PROP_BALL, step=0.5, T=0.5, n_or=1,
              renorm_every=3, energy_every=2)
    want = run(hsg, L, kw, 5, hsg.HSG_KERNEL_GLOBAL)
    got = run(hsg, L, kw, 5, hsg.HSG_KERNEL_WAVE)
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[1], want[1])


@pytest.mark.parametrize("n_or", [1, 3, 4])
def test_wave_graph_replay_with_odd_and_even_buffer_swaps(hsg, n_or):
    """Heat-bath + n_or OR is n_or buffer swaps per sweep.  On a stream
    the sweeps replay captured periods (doubled when a period would swap an
    odd number of times); on the default stream they launch directly.  Both
    must equal the global kernel, across calls that start mid-period."""
    L = 24
    kw = dict(kind=hsg.HSG_HEATBATH, T=0.4, n_or=n_or, renorm_every=5, energy_every=5)
    outs = []
    for kernel, stream in [(hsg.HSG_KERNEL_GLOBAL, None), (hsg.HSG_KERNEL_WAVE, torch.cuda.Stream()),
                           (hsg.HSG_KERNEL_WAVE, None)]:
        with hsg.Lattice(L, 8, stream=stream) as lat:
            lat.generate_couplings()
            sched = hsg.schedule(kernel=kernel, **kw)
            lat.sweep(sched, 3)
            lat.sweep(sched, 27)
            e_mid = lat.energy()
            lat.sweep(sched, 12)
            outs.append((lat.spins(), lat.energy_log(), e_mid, lat.sweep_count))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0])
        assert np.array_equal(o[1], outs[0][1]) and len(o[1]) == 8
        assert o[2] == outs[0][2]
        assert o[3] == 42


def test_wave_state_follows_the_current_buffer(hsg):
    """After an odd number of swaps the state lives in the second buffer:
    reading, writing, renormalising, half-sweeps and energies must all see
    it."""
    L = 16
    J = inputs.gaussian_couplings(L, seed=4)
    s_in = inputs.random_spins(L, seed=5, dtype=np.float32)
    one_hb = dict(kind=hsg.HSG_HEATBATH, T=0.9, n_or=1)
    results = []
    for kernel in (hsg.HSG_KERNEL_GLOBAL, hsg.HSG_KERNEL_WAVE):
        with hsg.Lattice(L, 3) as lat:
            lat.set_couplings(J)
            lat.sweep(hsg.schedule(kernel=kernel, **one_hb), 1)  # one swap (the OR sweep)
            a = lat.spins()
            e_a = lat.energy()
            lat.half_sweep(hsg.schedule(kernel=kernel), hsg.HSG_OVERRELAX, 1)
            lat.renorm()
            b = lat.spins()
            lat.set_spins(s_in)
            lat.sweep(hsg.schedule(kernel=kernel, **one_hb), 2)
            results.append((a, e_a, b, lat.spins(), lat.energy()))
    for x, y in zip(*results):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("L", [24, 40])
def test_wave_over_relaxation_sweep_matches_oracle(hsg, L):
    """One wave OR sweep from a random state, every site of both layers
    under the half-sweep rules: colour 0 against the oracle's half-sweep of
    the start state, colour 1 against the oracle's half-sweep of the GPU's
    own new colour 0 (what the kernel's colour-1 stage read from shared
    memory); energy conserved to round-off."""
    J, s32 = inputs.gaussian_couplings(L, seed=77), inputs.random_spins(L, seed=78, dtype=np.float32)
    Jr = inputs.round_to_f32(J)
    with hsg.Lattice(L, 2) as lat:
        lat.set_couplings(J)
        lat.set_spins(s32)
        e0 = lat.energy()
        lat.sweep(hsg.schedule(kind=hsg.HSG_NONE, n_or=1, kernel=hsg.HSG_KERNEL_WAVE), 1)
        got = lat.spins()
        e1 = lat.energy()
    check_or_sweep(L, Jr, s32, got, label=f"wave OR sweep L={L}")
    assert abs(e1 - e0) <= 2e-6


def test_wave_heatbath_energy_statistics_match_oracle(hsg):
    """Heat-bath + 1 OR at T = 0.5, L = 12: mean E/N over 600 wave sweeps
    within 3 sigma of the oracle's."""
    L, n = 12, 600
    J = inputs.gaussian_couplings(L, seed=12)
    with hsg.Lattice(L, 12) as lat:
        lat.set_couplings(J)
        lat.sweep(hsg.schedule(kind=hsg.HSG_HEATBATH, T=0.5, n_or=1, energy_every=1, renorm_every=10,
                               kernel=hsg.HSG_KERNEL_WAVE), n)
        g = lat.energy_log()
    s = oracle.init_spins(L, 12)
    _, r = oracle.sweeps(L, inputs.round_to_f32(J), s,
                         oracle.Schedule(kind=oracle.HB, beta=2.0, n_or=1, energy_every=1), oracle.key(12), n)

    def binned(x):
        b = np.array([v.mean() for v in np.array_split(x[n // 5:], 20)])
        return b.mean(), b.std(ddof=1) / np.sqrt(len(b))

    mg, eg = binned(g)
    mr, er = binned(r)
    assert abs(mg - mr) < 3 * math.hypot(eg, er) + 1e-6, (mg, eg, mr, er)


def test_wave_profiler_counts_one_launch_per_full_sweep(hsg):
    L = 32
    with hsg.Lattice(L, 1) as lat:
        lat.generate_couplings()
        hsg.hsg_profile(lat.ctx, 1)
        lat.sweep(hsg.schedule(kind=hsg.HSG_HEATBATH, T=0.3, n_or=4, kernel=hsg.HSG_KERNEL_WAVE), 2)
        _, n_or = hsg.hsg_profile_read(lat.ctx, hsg.HSG_PROF_OVERRELAX)
        _, n_hb = hsg.hsg_profile_read(lat.ctx, hsg.HSG_PROF_HEATBATH)
    assert (n_or, n_hb) == (8, 4)  # one launch per OR sweep; the heat-bath stays two half-sweeps


def test_wave_full_size_l256_is_bit_identical(hsg):
    """The timed L = 256 workload (heat-bath at T = 0.3 + 4 OR sweeps, FP64
    renormalisation and energy every sweep here) in the launch configuration
    the benchmark uses: two sweeps, wave vs global kernel, bit for bit."""
    L = 256
    kw = dict(kind=hsg.HSG_HEATBATH, T=0.3, n_or=4, renorm_every=1, energy_every=1)
    stream = torch.cuda.Stream()
    want = run(hsg, L, kw, 2, hsg.HSG_KERNEL_GLOBAL, stream=stream, seed=3)
    got = run(hsg, L, kw, 2, hsg.HSG_KERNEL_WAVE, stream=stream, seed=3)
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[1], want[1]) and len(got[1]) == 2


def test_auto_picks_the_wave_kernel_only_beyond_three_quarters_of_l2(hsg):
    """HSG_KERNEL_AUTO resolves to the temporally blocked sweep once the
    28 N bytes of spins and bonds exceed three quarters of L2, else to the
    global kernel."""
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    sched = hsg.schedule(kind=hsg.HSG_HEATBATH, n_or=4)
    for L in (16, 128, 144, 152, 256):
        with hsg.Lattice(L, 1) as lat:
            want = hsg.HSG_KERNEL_WAVE if 4 * 28 * L ** 3 > 3 * l2 else hsg.HSG_KERNEL_GLOBAL
            assert hsg.hsg_kernel_for(lat.ctx, sched) == want
            for k in (hsg.HSG_KERNEL_GLOBAL, hsg.HSG_KERNEL_SLAB, hsg.HSG_KERNEL_WAVE):
                assert hsg.hsg_kernel_for(lat.ctx, hsg.schedule(n_or=1, kernel=k)) == k


def test_wave_fuses_the_renormalisation_into_the_last_over_relaxation_sweep(hsg):
    """With the wave kernel a renormalisation due after a sweep is done by
    that sweep's last over-relaxation launch (no launch of its own); with
    half-sweeps it stays a launch.  Results are the same bit for bit (the
    tests above run renormalising schedules on both kernels)."""
    L = 32
    counts = {}
    for kernel in (hsg.HSG_KERNEL_WAVE, hsg.HSG_KERNEL_GLOBAL):
        with hsg.Lattice(L, 1) as lat:
            lat.generate_couplings()
            hsg.hsg_profile(lat.ctx, 1)
            lat.sweep(hsg.schedule(kind=hsg.HSG_HEATBATH, T=0.3, n_or=2, renorm_every=2, kernel=kernel), 4)
            counts[kernel] = [hsg.hsg_profile_read(lat.ctx, k)[1]
                              for k in (hsg.HSG_PROF_OVERRELAX, hsg.HSG_PROF_OVERRELAX_RENORM, hsg.HSG_PROF_RENORM)]
    assert counts[hsg.HSG_KERNEL_WAVE] == [6, 2, 0]  # the last OR sweep of sweeps 2 and 4 renormalises
    assert counts[hsg.HSG_KERNEL_GLOBAL] == [16, 0, 2]


@pytest.mark.parametrize("source", ["f32", "f64", "generated"])
def test_new_couplings_after_wave_sweeps(hsg, source):
    """From L = 32 the temporally blocked sweep reads its bonds from a
    halo-padded copy of the couplings, made by its first sweep.  New
    couplings after that -- uploaded (fp32 or fp64: the upload writes the
    copy too) or generated on the device (the copy rebuilt before the next
    sweep) -- must read back exactly and sweep bit for bit as with the
    global kernel."""
    L = 40
    J1 = inputs.gaussian_couplings(L, seed=41, dtype=np.float32)
    J2 = inputs.gaussian_couplings(L, seed=42)
    sched = dict(kind=hsg.HSG_HEATBATH, T=0.6, n_or=2, renorm_every=2)
    outs = []
    for kernel in (hsg.HSG_KERNEL_GLOBAL, hsg.HSG_KERNEL_WAVE):
        with hsg.Lattice(L, 9, 3) as lat:
            lat.set_couplings(J1)
            lat.sweep(hsg.schedule(kernel=kernel, **sched), 1)
            if source == "generated":
                lat.generate_couplings()
                want_J = oracle.gaussian_couplings(L, 9, 3).astype(np.float32)
                np.testing.assert_array_max_ulp(lat.couplings(), want_J, maxulp=1)
            else:
                lat.set_couplings(J2.astype(np.float32) if source == "f32" else J2)
                assert np.array_equal(lat.couplings(), J2.astype(np.float32))
            lat.sweep(hsg.schedule(kernel=kernel, **sched), 2)
            outs.append((lat.spins(), lat.couplings()))
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][0], outs[1][0])


@pytest.mark.parametrize("which", [1, 2, 3])
def test_tensor_load_waits_run_out_and_are_reported(hsg, which):
    """The waits of the temporally blocked sweep for its loads are bounded
    (0.2 s): for the couplings' tensor boxes (which = 1), for the colour-1
    planes' barriers (2), or both (3).  With the test switch each such wait
    expects more than its loads deliver, so it runs out: the sweep still
    ends, hsg_energy reports HSG_ETIMEOUT (once), and the context stays
    usable -- with the switch off, the same sweep from the same state equals
    the global kernel's bit for bit."""
    import time

    L = 40
    J = inputs.gaussian_couplings(L, seed=51, dtype=np.float32)
    sched = hsg.schedule(kind=hsg.HSG_NONE, n_or=1, kernel=hsg.HSG_KERNEL_WAVE)
    with hsg.Lattice(L, 51) as lat:  # the default stream: launches issued directly, no captured graph
        lat.set_couplings(J)
        lat.sweep(sched, 1)  # makes the padded copy: tensor loads from here on
        lat.energy()
        s0 = lat.spins()
        hsg.hsg_test_stall_tensor_loads(which)
        try:
            t0 = time.perf_counter()
            lat.sweep(sched, 1)
            with pytest.raises(hsg.HsgError) as e:
                lat.energy()
            assert e.value.status == hsg.HSG_ETIMEOUT
            assert time.perf_counter() - t0 < 10.0
        finally:
            hsg.hsg_test_stall_tensor_loads(False)
        lat.energy()  # reported once
        lat.set_spins(s0)
        lat.sweep(sched, 1)
        got = lat.spins()
    with hsg.Lattice(L, 51) as ref:
        ref.set_couplings(J)
        ref.set_spins(s0)
        ref.sweep(hsg.schedule(kind=hsg.HSG_NONE, n_or=1, kernel=hsg.HSG_KERNEL_GLOBAL), 1)
        assert np.array_equal(got, ref.spins())


def test_register_bonds_when_the_padded_copy_cannot_be_allocated(hsg):
    """Without memory for the halo-padded couplings (the sweep's second
    allocation made to fail) the temporally blocked sweep keeps its other
    kernel, which loads each site's bonds into registers; its results are
    the global kernel's bit for bit too."""
    L = 72
    kw = dict(kind=hsg.HSG_HEATBATH, T=0.7, n_or=2, renorm_every=2, energy_every=1)
    want = run(hsg, L, kw, 3, hsg.HSG_KERNEL_GLOBAL)
    with hsg.Lattice(L, 31) as lat:
        lat.generate_couplings()
        hsg.hsg_test_fail_alloc(2)  # the first sweep allocates the second spin buffer, then the padded copy
        try:
            lat.sweep(hsg.schedule(kernel=hsg.HSG_KERNEL_WAVE, **kw), 3)
        finally:
            hsg.hsg_test_fail_alloc(0)
        got = lat.spins(), lat.energy_log()
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[1], want[1])
