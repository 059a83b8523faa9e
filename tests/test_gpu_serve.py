"""The continuous-batching request loop (needs a CUDA GPU): every result is
the same alone and in the mix; requests wait for memory and are admitted in
arrival order; served results agree with the FP64 oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1006_2566_gb300 import serve  # noqa: E402
from parity_rules import check_one_sweep, check_or_sweep, record  # noqa: E402


@pytest.fixture(scope="module")
def hsg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_2566_gb300 import build

    build.build()
    oracle.build()
    from paper_1006_2566_gb300 import hsg as h

    return h


def test_each_result_is_the_same_alone_and_in_the_mix(hsg):
    reqs = serve.poisson_trace(14, rate_per_s=300.0, seed=8, sides=(8, 12, 16, 20, 24), sweep_range=(4, 30))
    kw = dict(kind=hsg.HSG_METROPOLIS, hits=4, proposal=hsg.HSG_PROP_BALL, step=0.5, n_or=2, renorm_every=10)
    budget = 3 * 28 * 24 ** 3  # room for three of the largest lattices: later arrivals must wait
    res, st = serve.serve(reqs, kw, budget, 6, torch.cuda.Stream(), tick_sweeps=4, keep_spins=True, autotune=False)
    assert st.completed == len(reqs)
    assert st.max_batch >= 2  # requests overlapped on the device
    by_id = {r.rid: r for r in res}
    admitted = [by_id[q.rid].admitted for q in sorted(reqs, key=lambda q: q.arrival)]
    assert all(a <= b for a, b in zip(admitted, admitted[1:]))  # arrival order
    for q in reqs:
        r = by_id[q.rid]
        assert r.arrival <= r.admitted + 1e-9 <= r.finished + 1e-9
        with hsg.Lattice(q.L, q.seed, q.sample, 0) as lat:
            lat.generate_couplings()
            lat.sweep(hsg.schedule(T=q.T, **kw), q.sweeps)
            assert np.array_equal(r.spins, lat.spins()), q
            assert abs(r.energy - lat.energy()) <= 2e-6
    fifo, fst = serve.serve_fifo(reqs, kw, keep_spins=True)
    assert fst.completed == len(reqs)
    for f in fifo:
        assert np.array_equal(f.spins, by_id[f.rid].spins)
        assert abs(f.energy - by_id[f.rid].energy) <= 2e-6


def test_withdrawn_requests_leave_the_others_unchanged(hsg):
    """Clients withdraw two requests (one while it runs, one before it is
    admitted); every other result is still bit-identical to its request run
    alone, and the withdrawn lattice's memory goes to the next admission."""
    reqs = serve.poisson_trace(10, rate_per_s=200.0, seed=9, sides=(8, 16, 24), sweep_range=(10, 40))
    kw = dict(kind=hsg.HSG_HEATBATH, n_or=1, renorm_every=5)
    budget = 2 * 28 * 24 ** 3
    first, last = reqs[0].rid, reqs[-1].rid
    res, st = serve.serve(reqs, kw, budget, 4, torch.cuda.Stream(), tick_sweeps=2, keep_spins=True,
                          autotune=False, cancels={first: reqs[0].arrival + 1e-4, last: 0.0})
    assert sorted(st.extra["cancelled"]) == sorted([first, last])
    assert st.completed == len(reqs) - 2
    for r in res:
        q = next(x for x in reqs if x.rid == r.rid)
        with hsg.Lattice(q.L, q.seed, q.sample, 0) as lat:
            lat.generate_couplings()
            lat.sweep(hsg.schedule(T=q.T, **kw), q.sweeps)
            assert np.array_equal(r.spins, lat.spins()), q


@pytest.mark.parametrize("kind", ["MET", "HB", "OR"])
def test_served_requests_match_oracle_layer_by_layer(hsg, kind):
    """Small requests (L <= 16) of one sweep each, of one update kind,
    arriving faster than they are served, with memory for three of the
    largest at a time (so that they queue, share ticks and are admitted into
    freed memory): every request's final spins on every site, layer by
    layer, against the oracle's half-sweeps from the request's initial state
    with its own key and temperature, and its E/N against the oracle's
    energy of its final state.  The oracle is fed the initial spins and
    device-generated couplings of the request's key as a lone context holds
    them -- the same generator kernels as the pool's -- after they are
    checked against the oracle's own Philox maps (1e-6, 1 ulp)."""
    kw, upd = {
        "MET": (dict(kind=hsg.HSG_METROPOLIS, hits=4, proposal=hsg.HSG_PROP_BALL, step=0.5), oracle.MET),
        "HB": (dict(kind=hsg.HSG_HEATBATH), oracle.HB),
        "OR": (dict(kind=hsg.HSG_NONE, n_or=1), oracle.OR),
    }[kind]
    reqs = serve.poisson_trace(12, rate_per_s=20000.0, seed=40 + len(kind), sides=(4, 6, 8, 12, 16),
                               sweep_range=(1, 1))
    budget = 3 * 28 * 16 ** 3
    res, st = serve.serve(reqs, kw, budget, 6, torch.cuda.Stream(), tick_sweeps=1, keep_spins=True, autotune=False)
    assert st.completed == len(reqs) and st.max_batch >= 2
    by_id = {q.rid: q for q in reqs}
    for r in res:
        q = by_id[r.rid]
        with hsg.Lattice(q.L, q.seed, q.sample, 0) as lat:
            lat.generate_couplings()
            s0, J = lat.spins(), lat.couplings()
        assert np.max(np.abs(s0 - oracle.init_spins(q.L, q.seed, q.sample, 0))) < 1e-6
        np.testing.assert_array_max_ulp(J, oracle.gaussian_couplings(q.L, q.seed, q.sample).astype(np.float32),
                                        maxulp=1)
        Jd = J.astype(np.float64)
        label = f"served {kind} L={q.L} T={q.T:.3f} request {q.rid}"
        if upd == oracle.OR:
            check_or_sweep(q.L, Jd, s0, r.spins, label=label)
        else:
            p = oracle.Params(key=oracle.key(q.seed, q.sample), sweep=0, beta=1.0 / q.T, step=0.5,
                              hits=kw.get("hits", 1), proposal=hsg.HSG_PROP_BALL)
            check_one_sweep(q.L, Jd, s0, r.spins, upd, p, label=label)
        e_ref = oracle.energy(q.L, Jd, r.spins.astype(np.float64)) / q.L ** 3
        record(label=f"{label} E/N", max_err=abs(r.energy - e_ref))
        assert abs(r.energy - e_ref) <= 2e-6 and math.isfinite(r.energy)
