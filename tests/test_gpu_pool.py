"""Device coupling generator and pools of lattices (needs a CUDA GPU).

A lattice swept inside a pool must be bit-identical to the same lattice
(same key, temperature, couplings) swept alone through a context, whatever
else is admitted or retired around it and whatever launch configuration the
pool uses: same device code, same random numbers.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
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


# ---------------------------------------------------------------------------
# Couplings on the device
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L,seed,sample", [(8, 4, 7), (24, 1, 0), (40, 9, 3)])
def test_generated_couplings_match_oracle(hsg, L, seed, sample):
    """Both sides evaluate Box-Muller in fp64 from the same Philox words;
    the device rounds once to fp32, so the values agree to the last bit
    except where the two fp64 results straddle an fp32 rounding boundary."""
    with hsg.Lattice(L, seed, sample, replica=1) as lat:
        lat.generate_couplings()
        got = lat.couplings()
    ref = oracle.gaussian_couplings(L, seed, sample).astype(np.float32)
    assert np.mean(got == ref) > 0.9999
    np.testing.assert_array_max_ulp(got, ref, maxulp=1)


def test_coupling_upload_round_trip(hsg):
    L = 12
    J = inputs.gaussian_couplings(L, 3, dtype=np.float32)
    with hsg.Lattice(L, 1) as lat:
        lat.set_couplings(J)
        assert np.array_equal(lat.couplings(), J)
        lat.set_couplings(J.astype(np.float64))
        assert np.array_equal(lat.couplings(), J)


# ---------------------------------------------------------------------------
# Pools
# ---------------------------------------------------------------------------

SPECS = [  # (L, seed, sample, replica, T)
    (4, 11, 0, 0, 0.5),
    (6, 11, 0, 1, 0.5),
    (16, 11, 1, 0, 1.0),
    (24, 11, 2, 0, 0.3),
    (8, 11, 3, 1, math.inf),
    (40, 11, 4, 0, 0.7),
]


def base_schedule(hsg, kind):
    k = {"MET": hsg.HSG_METROPOLIS, "HB": hsg.HSG_HEATBATH, "METOR": hsg.HSG_METROPOLIS_OR}[kind]
    return dict(kind=k, hits=3, proposal=hsg.HSG_PROP_BALL, step=0.5, n_or=2, renorm_every=2)


def run_alone(hsg, spec, sched_kw, n, J=None):
    L, seed, sample, replica, T = spec
    with hsg.Lattice(L, seed, sample, replica) as lat:
        if J is None:
            lat.generate_couplings()
        else:
            lat.set_couplings(J)
        lat.sweep(hsg.schedule(T=T, **sched_kw), n)
        return lat.spins(), lat.energy()


@pytest.mark.parametrize("kind", ["MET", "HB", "METOR"])
@pytest.mark.parametrize("use_stream", [True, False])
def test_pool_lattices_are_bit_identical_to_lattices_alone(hsg, kind, use_stream):
    kw = base_schedule(hsg, kind)
    stream = torch.cuda.Stream() if use_stream else None  # graph replay / direct launches
    with hsg.Pool(1 << 28, 16, stream) as pool:
        slots = [pool.admit(*spec) for spec in SPECS]
        pool.sweep(hsg.schedule(**kw), 3)
        late = pool.admit(12, 11, 9, 0, 0.9)  # admitted mid-run: the work list changes
        pool.retire(slots[1])  # and one retired
        pool.sweep(hsg.schedule(**kw), 2)
        e = pool.energies()
        assert math.isnan(e[slots[1]])
        for slot, spec in zip(slots, SPECS):
            if slot == slots[1]:
                continue
            want, want_e = run_alone(hsg, spec, kw, 5)
            assert np.array_equal(pool.spins(slot), want), spec
            assert abs(e[slot] - want_e) <= 2e-6
            assert pool.sweep_count(slot) == 5
        want, _ = run_alone(hsg, (12, 11, 9, 0, 0.9), kw, 2)
        assert np.array_equal(pool.spins(late), want)
        assert pool.sweep_count(late) == 2


def test_pool_with_host_couplings(hsg):
    kw = base_schedule(hsg, "MET")
    J = inputs.gaussian_couplings(10, seed=5)
    with hsg.Pool(1 << 24, 4, torch.cuda.Stream()) as pool:
        s = pool.admit(10, 5, 0, 0, 0.6, J=J)
        pool.sweep(hsg.schedule(**kw), 3)
        got = pool.spins(s)
    want, _ = run_alone(hsg, (10, 5, 0, 0, 0.6), kw, 3, J=J)
    assert np.array_equal(got, want)


def test_pool_results_do_not_depend_on_launch_configuration(hsg):
    kw = base_schedule(hsg, "HB")
    outs = []
    for cfg in [(64, 64, 2, 0), (256, 2048, 16, 0), (128, 384, 5, 0)]:
        with hsg.Pool(1 << 28, 8, torch.cuda.Stream()) as pool:
            hsg.hsg_pool_config(pool.pool, *cfg)
            slots = [pool.admit(*spec) for spec in SPECS]
            pool.sweep(hsg.schedule(**kw), 3)
            outs.append([pool.spins(s) for s in slots])
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    for a, b in zip(outs[0], outs[2]):
        assert np.array_equal(a, b)


def test_pool_autotune_restores_state_and_keeps_results(hsg):
    kw = base_schedule(hsg, "MET")
    with hsg.Pool(1 << 28, 8, torch.cuda.Stream()) as pool:
        slots = [pool.admit(*spec) for spec in SPECS]
        pool.sweep(hsg.schedule(**kw), 2)
        before = [pool.spins(s) for s in slots]
        cfg = hsg.hsg_pool_autotune(pool.pool, hsg.schedule(**kw))
        assert cfg[0] in (128, 256) and cfg[1] % cfg[0] == 0 and cfg[2] >= 1 and cfg[3] in (0, 1, 2)
        for s, b in zip(slots, before):
            assert np.array_equal(pool.spins(s), b)
            assert pool.sweep_count(s) == 2
        pool.sweep(hsg.schedule(**kw), 2)
        for s, spec in zip(slots, SPECS):
            want, _ = run_alone(hsg, spec, kw, 4)
            assert np.array_equal(pool.spins(s), want)


def test_pool_admission_by_budget_and_slots(hsg):
    per = 28 * 16 ** 3  # bytes of one L = 16 lattice (a multiple of 256)
    with hsg.Pool(2 * per, 3, torch.cuda.Stream()) as pool:
        a = pool.admit(16, 1, 0)
        b = pool.admit(16, 1, 1)
        assert pool.usage() == (2 * per, 2 * per, 2)
        with pytest.raises(hsg.HsgError) as e:
            pool.admit(16, 1, 2)
        assert e.value.status == hsg.HSG_EBUSY
        pool.retire(a)
        c = pool.admit(8, 1, 3)
        d = pool.admit(8, 1, 4)  # two small ones fit in the freed block
        with pytest.raises(hsg.HsgError) as e:
            pool.admit(4, 1, 5)  # no free slot left (3 of 3)
        assert e.value.status == hsg.HSG_EBUSY
        pool.sweep(hsg.schedule(kind=hsg.HSG_HEATBATH, n_or=1), 1)
        for bad in (dict(L=7), dict(L=2), dict(L=2000), dict(T=0.0)):
            args = dict(L=8, seed=1, sample=9, replica=0, T=1.0)
            args.update(bad)
            with pytest.raises(hsg.HsgError) as e:
                pool.admit(**args)
            assert e.value.status in (hsg.HSG_EINVAL, hsg.HSG_EBUSY)
        with pytest.raises(hsg.HsgError) as e:
            pool.sweep(hsg.schedule(kind=hsg.HSG_HEATBATH, energy_every=1), 1)
        assert e.value.status == hsg.HSG_EINVAL
        assert c == a  # the freed slot index is reused
        pool.retire(d)
        with pytest.raises(hsg.HsgError):
            pool.retire(d)  # already free
        with pytest.raises(hsg.HsgError):
            pool.retire(7)  # no such slot
        assert len({b, c, d}) == 3


def test_pool_energies_queued_before_a_retirement_survive_reuse_of_the_memory(hsg):
    """hsg_pool_energies_async + hsg_pool_retire do not wait: a lattice's
    E/N queued before its retirement is its final value even when a new
    lattice is admitted into the freed block and swept before the read;
    the new lattice is unaffected, and so is a lattice running alongside."""
    kw = base_schedule(hsg, "MET")
    per = 28 * 16 ** 3
    with hsg.Pool(2 * per, 4, torch.cuda.Stream()) as pool:
        a = pool.admit(16, 3, 0, 0, 0.5)
        b = pool.admit(16, 3, 1, 0, 0.8)
        pool.sweep(hsg.schedule(**kw), 4)
        pool.energies_async(0)
        pool.retire(a)
        c = pool.admit(16, 3, 2, 0, 0.6)  # into a's block (the budget holds two)
        pool.sweep(hsg.schedule(**kw), 3)
        pool.energies_async(1)
        pool.retire(b)
        e0 = pool.energies_read(0)
        e1 = pool.energies_read(1)
        got_c = pool.spins(c)
        _, ea = run_alone(hsg, (16, 3, 0, 0, 0.5), kw, 4)
        _, eb4 = run_alone(hsg, (16, 3, 1, 0, 0.8), kw, 4)
        _, eb7 = run_alone(hsg, (16, 3, 1, 0, 0.8), kw, 7)
        want_c, ec = run_alone(hsg, (16, 3, 2, 0, 0.6), kw, 3)
        assert abs(e0[a] - ea) <= 2e-6 and abs(e0[b] - eb4) <= 2e-6
        assert abs(e1[b] - eb7) <= 2e-6 and abs(e1[c] - ec) <= 2e-6
        assert np.array_equal(got_c, want_c)
        assert math.isnan(e1[3]) and math.isnan(e0[2])  # free slots
        # the finished slot alone: the same value, NaN elsewhere
        pool.energies_async(0, [c])
        e2 = pool.energies_read(0)
        assert e2[c] == e1[c] and np.isnan(np.delete(e2, c)).all()
        for bad in (lambda: pool.energies_read(0),  # nothing queued any more
                    lambda: pool.energies_async(2), lambda: hsg.hsg_pool_energies_read(pool.pool, -1, 4),
                    lambda: pool.energies_async(0, [b])):  # b is retired
            with pytest.raises(hsg.HsgError) as err:
                bad()
            assert err.value.status == hsg.HSG_EINVAL


@pytest.mark.parametrize("kind", ["MET", "METOR"])
def test_pool_metropolis_hits_split_over_passes_give_the_same_result(hsg, kind):
    """A colour's k Metropolis hits in passes of h hits (h = 1, 2, k - 1)
    equal all k in one pass bit for bit, and the lattice swept alone: the
    field is fixed for the half-sweep and hit j is keyed by j; the fused
    reflection follows the last hit."""
    kw = dict(base_schedule(hsg, kind), hits=5)
    outs = []
    for h in (0, 1, 2, 4):
        with hsg.Pool(1 << 28, 8, torch.cuda.Stream()) as pool:
            hsg.hsg_pool_config(pool.pool, 256, 512, 8, h)
            slots = [pool.admit(*spec) for spec in SPECS]
            n0 = hsg.hsg_pool_launch_count(pool.pool)
            pool.sweep(hsg.schedule(**kw), 3)
            launches = hsg.hsg_pool_launch_count(pool.pool) - n0
            outs.append([pool.spins(s) for s in slots])
        passes = 1 if h == 0 else -(-5 // h)
        assert launches == 3 * (2 * passes + 2 * kw["n_or"] + 1 + 1)  # + counter advance + renormalisation
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)
    for got, spec in zip(outs[0], SPECS):
        want, _ = run_alone(hsg, spec, kw, 3)
        assert np.array_equal(got, want)


# ---------------------------------------------------------------------------
# Pools against the FP64 oracle
# ---------------------------------------------------------------------------

ORACLE_SPECS = [  # (L, seed, sample, replica, T, couplings from the host?)
    (4, 21, 0, 0, 0.5, True),
    (6, 21, 1, 1, 0.8, False),
    (24, 21, 2, 0, 0.3, True),
    (40, 21, 3, 1, 1.0, False),
    (16, 21, 4, 0, math.inf, True),
]


def oracle_couplings(L, seed, sample, host):
    """The fp32 couplings a pooled lattice holds: the host array uploaded
    (rounded to fp32), or the device generator's, which equal the oracle's
    Box-Muller values rounded to fp32 to within 1 ulp (test above); the
    oracle is fed the same fp32 values as fp64."""
    if host:
        return inputs.round_to_f32(inputs.gaussian_couplings(L, seed=seed + 100 * sample))
    return oracle.gaussian_couplings(L, seed, sample).astype(np.float32).astype(np.float64)


def test_pool_sweeps_match_oracle_layer_by_layer(hsg):
    """Lattices of uneven L at distinct temperatures in one pool (several
    tiles for the larger ones, less than one for the smallest, a non-default
    launch shape): each pool sweep of one update kind -- Metropolis (ball,
    3 hits), over-relaxation, heat-bath, the fused pass -- checked on every
    site of every lattice, layer by layer, against the oracle's half-sweeps
    from that lattice's state before the layer, with its own key, counter
    and temperature.  A lattice admitted mid-run (next to lattices three
    sweeps ahead) and the hole left by a retired one are covered, and a
    composite sweep (Metropolis + 1 OR) in a second pool equals the two
    checked single-kind sweeps bit for bit."""
    from parity_rules import check_one_sweep, check_or_sweep

    met = dict(kind=hsg.HSG_METROPOLIS, hits=3, proposal=hsg.HSG_PROP_BALL, step=0.5)
    kinds = [("MET", met, oracle.MET), ("OR", dict(kind=hsg.HSG_NONE, n_or=1), oracle.OR),
             ("HB", dict(kind=hsg.HSG_HEATBATH), oracle.HB),
             ("METOR", dict(met, kind=hsg.HSG_METROPOLIS_OR, hits=2), oracle.MET_OR)]
    Js = {spec: oracle_couplings(spec[0], spec[1], spec[2], spec[5]) for spec in ORACLE_SPECS}
    late = (12, 21, 9, 0, 0.6, False)
    Js[late] = oracle_couplings(*late[:3], late[5])

    def admit(pool, spec):
        L, seed, sample, replica, T, host = spec
        return pool.admit(L, seed, sample, replica, T, J=Js[spec] if host else None)

    def check(pool, slots, before, name, kw, upd, sweep_of):
        for spec, slot in slots.items():
            L, seed, sample, replica, T, _ = spec
            after = pool.spins(slot)
            label = f"pool {name} L={L} T={T} slot {slot}"
            if upd == oracle.OR:
                check_or_sweep(L, Js[spec], before[slot], after, label=label)
            else:
                p = oracle.Params(key=oracle.key(seed, sample, replica), sweep=sweep_of[slot],
                                  beta=0.0 if math.isinf(T) else 1.0 / T, step=0.5, hits=kw.get("hits", 1),
                                  proposal=hsg.HSG_PROP_BALL)
                check_one_sweep(L, Js[spec], before[slot], after, upd, p, label=label)

    with hsg.Pool(1 << 26, 8, torch.cuda.Stream()) as pool, hsg.Pool(1 << 26, 8, torch.cuda.Stream()) as twin:
        hsg.hsg_pool_config(pool.pool, 128, 384, 6, 0)
        slots = {spec: admit(pool, spec) for spec in ORACLE_SPECS}
        twin_slots = {spec: admit(twin, spec) for spec in ORACLE_SPECS}
        for spec, slot in slots.items():  # the initial spins: the oracle's Philox map, to fp32 round-off
            L, seed, sample, replica = spec[:4]
            assert np.max(np.abs(pool.spins(slot) - oracle.init_spins(L, seed, sample, replica))) < 1e-6
        twin.sweep(hsg.schedule(**dict(met, n_or=1)), 1)  # one composite sweep
        for n, (name, kw, upd) in enumerate(kinds):
            if n == 2:  # retire one lattice and admit a new one into the pool mid-run
                pool.retire(slots.pop(ORACLE_SPECS[1]))
                slots[late] = admit(pool, late)
            before = {slot: pool.spins(slot) for slot in slots.values()}
            sweep_of = {slot: pool.sweep_count(slot) for slot in slots.values()}
            pool.sweep(hsg.schedule(**kw), 1)
            check(pool, slots, before, name, kw, upd, sweep_of)
            if n == 1:  # Metropolis then OR == the composite sweep of the twin pool
                for spec, slot in slots.items():
                    assert np.array_equal(pool.spins(slot), twin.spins(twin_slots[spec])), spec
        assert pool.sweep_count(slots[late]) == 2 and pool.sweep_count(slots[ORACLE_SPECS[0]]) == 4
        e = pool.energies()
        for spec, slot in slots.items():  # E/N of each lattice against the oracle's energy of its state
            L = spec[0]
            ref = oracle.energy(L, Js[spec], pool.spins(slot).astype(np.float64)) / L ** 3
            assert abs(e[slot] - ref) <= 2e-6, spec


def test_pooled_l16_metropolis_matches_oracle_layer_by_layer(hsg):
    """The L = 16 single-lattice workload (1-hit Metropolis, uniform-sphere
    proposal, T = 1) run as the benchmark pools it: independent samples in
    one pool under the autotuned launch shape.  Two sweeps of every lattice
    are checked on every site, layer by layer, against the oracle's
    half-sweeps from the lattice's state before the layer."""
    from parity_rules import check_one_sweep

    kw = dict(kind=hsg.HSG_METROPOLIS, hits=1, proposal=hsg.HSG_PROP_SPHERE, step=0.5)
    specs = [(16, 1, s, 0, 1.0, s % 2 == 0) for s in range(8)]
    Js = {spec: oracle_couplings(spec[0], spec[1], spec[2], spec[5]) for spec in specs}
    with hsg.Pool(1 << 26, len(specs), torch.cuda.Stream()) as pool:
        slots = {spec: pool.admit(*spec[:5], J=Js[spec] if spec[5] else None) for spec in specs}
        hsg.hsg_pool_autotune(pool.pool, hsg.schedule(**kw))
        for n in range(2):
            before = {slot: pool.spins(slot) for slot in slots.values()}
            pool.sweep(hsg.schedule(**kw), 1)
            for spec, slot in slots.items():
                L, seed, sample, replica, T, _ = spec
                p = oracle.Params(key=oracle.key(seed, sample, replica), sweep=n, beta=1.0 / T, step=0.5, hits=1,
                                  proposal=hsg.HSG_PROP_SPHERE)
                check_one_sweep(L, Js[spec], before[slot], pool.spins(slot), oracle.MET, p,
                                label=f"pooled L=16 sample {sample} sweep {n}")
