"""Host logic of the serving loop: the request trace and latency statistics
(CPU only)."""
import numpy as np
import pytest

from paper_1006_2566_gb300 import serve


def test_poisson_trace_shape_and_distributions():
    n, rate = 4000, 2000.0
    tr = serve.poisson_trace(n, rate, seed=5)
    assert [r.rid for r in tr] == list(range(n))
    arr = np.array([r.arrival for r in tr])
    assert arr[0] == 0.0 and np.all(np.diff(arr) >= 0)
    gaps = np.diff(arr)
    assert abs(gaps.mean() * rate - 1) < 4 / np.sqrt(n)  # exponential gaps, mean 1/rate
    assert abs(gaps.std() / gaps.mean() - 1) < 0.1  # coefficient of variation 1
    Ls = np.array([r.L for r in tr])
    assert set(Ls) <= set(range(16, 97, 8)) and len(set(Ls)) == 11
    Ts = np.array([r.T for r in tr])
    assert Ts.min() >= 0.2 and Ts.max() <= 1.0
    sw = np.array([r.sweeps for r in tr])
    assert sw.min() >= 50 and sw.max() <= 500
    assert len({r.sample for r in tr}) == n  # a fresh disorder sample per request
    # mean work per request: E[L^3] E[sweeps] = 283,136 * 275 site-sweeps
    assert abs(np.mean(Ls.astype(float) ** 3) / 283136 - 1) < 0.05
    assert serve.poisson_trace(10, rate, seed=5)[3] == tr[3]  # seeded, prefix-stable


def test_latency_statistics():
    res = [serve.Result(k, 0.0, arrival=0.0, admitted=0.0, finished=(k + 1) / 1000.0) for k in range(100)]
    p50, p99, mean = serve.latency_stats(res)
    assert p50 == pytest.approx(50.5)
    assert p99 == pytest.approx(99.01)
    assert mean == pytest.approx(50.5)
    assert all(np.isnan(v) for v in serve.latency_stats([]))


class FakePool:
    """A pool with the hsg.Pool interface and no GPU: each admitted lattice
    takes L^3 bytes of the budget; every sweep adds k to its counter;
    energies are -(sweeps done)/1000 per slot, so results show how far each
    lattice ran.  Records admissions and retirements."""

    def __init__(self, budget, max_slots, stream=None):
        self.budget, self.max_slots = budget, max_slots
        self.slots = {}  # slot -> [L, sweeps]
        self.log = []
        FakePool.last = self

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.closed = True

    def admit(self, L, seed, sample, replica, T):
        from paper_1006_2566_gb300 import hsg

        used = sum(v[0] ** 3 for v in self.slots.values())
        if used + L ** 3 > self.budget or len(self.slots) >= self.max_slots:
            raise hsg.HsgError(hsg.HSG_EBUSY, "busy")
        slot = min(set(range(self.max_slots)) - set(self.slots))
        self.slots[slot] = [L, 0]
        self.log.append(("admit", sample, slot))
        return slot

    def retire(self, slot):
        self.log.append(("retire", slot))
        del self.slots[slot]

    def sweep(self, sched, k):
        for v in self.slots.values():
            v[1] += k

    def energies(self):
        return np.array([-self.slots[s][1] / 1000.0 if s in self.slots else np.nan for s in range(self.max_slots)])

    def energies_async(self, buffer, slots=None):
        assert buffer in (0, 1) and buffer not in getattr(self, "queued", {})  # read before reuse
        self.queued = getattr(self, "queued", {})
        e = self.energies()
        if slots is not None:
            e[[s for s in range(self.max_slots) if s not in slots]] = np.nan
        self.queued[buffer] = e

    def energies_read(self, buffer):
        return self.queued.pop(buffer)

    def spins(self, slot):
        return np.zeros(3 * self.slots[slot][0] ** 3, dtype=np.float32)


class SyncStream:
    """Stands in for a CUDA stream whose work is already done."""

    def synchronize(self):
        pass

    def record_event(self):
        return self


def reqs(spec):
    return [serve.Request(k, t, L, 1, k, 0.5, sw) for k, (t, L, sw) in enumerate(spec)]


def test_serve_loop_admits_in_order_under_the_budget_and_runs_each_to_its_sweeps():
    pytest.importorskip("torch")
    rq = reqs([(0.0, 8, 30), (0.0, 8, 20), (0.0, 8, 40), (0.0, 6, 10)])
    res, st = serve.serve(rq, dict(kind=1, n_or=1), budget_bytes=2 * 8 ** 3, max_slots=4, stream=SyncStream(),
                          autotune=False, pool_factory=FakePool)
    by = {r.rid: r for r in res}
    assert sorted(by) == [0, 1, 2, 3] and st.completed == 4
    for r in rq:
        assert by[r.rid].energy == -r.sweeps / 1000.0  # each ran exactly its sweeps
    admits = [e[1] for e in FakePool.last.log if e[0] == "admit"]
    assert admits == [0, 1, 2, 3]  # arrival order; request 2 waited for memory
    assert st.max_batch == 2 and st.extra["cancelled"] == [] and st.extra["rejected"] == []
    assert st.extra["config"] is None and st.extra["host_ms_per_tick"] >= 0.0


class ConfigPool(FakePool):
    """Counts its sweep calls; is its own handle for hsg_pool_config."""

    def __init__(self, *a):
        super().__init__(*a)
        self.pool = self
        self.sweeps = 0

    def sweep(self, sched, k):
        self.sweeps += 1
        super().sweep(sched, k)


def test_serve_loop_sets_a_given_launch_configuration_before_the_first_sweep(monkeypatch):
    pytest.importorskip("torch")
    from paper_1006_2566_gb300 import hsg

    calls = []
    monkeypatch.setattr(hsg, "hsg_pool_config", lambda pool, *cfg: calls.append((pool.sweeps, cfg)))
    monkeypatch.setattr(hsg, "hsg_pool_autotune", lambda *a: pytest.fail("autotuned although a config was given"))
    rq = reqs([(0.0, 6, 5)] * 9)
    res, st = serve.serve(rq, dict(kind=1, n_or=1), budget_bytes=9 * 6 ** 3, max_slots=16, stream=SyncStream(),
                          pool_factory=ConfigPool, config=(256, 1024, 8, 4))
    assert st.completed == 9 and st.extra["config"] == (256, 1024, 8, 4)
    assert calls == [(0, (256, 1024, 8, 4))]  # set once, before the first sweep
    assert ConfigPool.last.sweeps > 0


class SlowPool(FakePool):
    """2 ms per pool sweep call, so that wall-clock withdrawals land mid-run."""

    def sweep(self, sched, k):
        import time

        time.sleep(0.002)
        super().sweep(sched, k)


def test_serve_loop_withdraws_waiting_and_running_requests():
    pytest.importorskip("torch")
    # request 0 needs 40 ticks (>= 80 ms) and is withdrawn at 50 ms; 1 and 2
    # finish within ~20 ms; 3 is withdrawn before it arrives; 99 is unknown
    rq = reqs([(0.0, 8, 400), (0.0, 8, 50), (0.0, 8, 30), (0.2, 6, 10)])
    res, st = serve.serve(rq, dict(kind=1, n_or=1), budget_bytes=2 * 8 ** 3, max_slots=4, stream=SyncStream(),
                          tick_sweeps=10, autotune=False, pool_factory=SlowPool,
                          cancels={0: 0.05, 3: 0.0, 99: 0.0})
    by = {r.rid: r for r in res}
    assert sorted(by) == [1, 2]  # 0 withdrawn while running, 3 before it arrived
    assert by[1].energy == -0.05 and by[2].energy == -0.03
    assert sorted(st.extra["cancelled"]) == [0, 3]
    retired = [e[1] for e in FakePool.last.log if e[0] == "retire"]
    assert len(retired) == 3  # the withdrawn lattice freed its slot too


def test_serve_loop_rejects_a_request_larger_than_the_pool_and_propagates_errors():
    pytest.importorskip("torch")
    rq = reqs([(0.0, 8, 10), (0.0, 16, 10)])
    res, st = serve.serve(rq, dict(kind=1), budget_bytes=8 ** 3, max_slots=2, stream=SyncStream(),
                          autotune=False, pool_factory=FakePool)
    assert [r.rid for r in res] == [0] and st.extra["rejected"] == [1]

    class Failing(FakePool):
        def sweep(self, sched, k):
            raise RuntimeError("injected device error")

    with pytest.raises(RuntimeError, match="injected"):
        serve.serve(reqs([(0.0, 8, 10)]), dict(kind=1), budget_bytes=8 ** 3, max_slots=1, stream=SyncStream(),
                    autotune=False, pool_factory=Failing)
    assert FakePool.last.closed  # the pool is released on the way out
