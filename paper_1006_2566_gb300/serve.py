"""Continuous-batching request loop over a pool of lattices.

Requests are independent Monte Carlo solves (a fresh disorder sample, side
L, temperature T, a number of sweeps).  They arrive over time; the loop
admits waiting requests into the pool in arrival order whenever a slot and
enough arena memory are free (the arena is the HBM budget), runs the pool so
that every admitted lattice advances together -- requests that arrive while
others are on the GPU join the running batch -- and retires each lattice the
moment its sweeps are done, returning its final E/N.  Lattices and their
random-number counters stay resident on the device from admission to
retirement.

Because each lattice in a pool is updated exactly as it would be alone (same
key, counters and device code), every result is the same alone and in any
mix.

`serve_fifo` is the comparison without batching: one request at a time on
its own context, in arrival order.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float  # seconds after the start of the run
    L: int
    seed: int
    sample: int
    T: float
    sweeps: int


@dataclass
class Result:
    rid: int
    energy: float
    arrival: float
    admitted: float
    finished: float
    spins: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class ServeStats:
    completed: int
    wall_seconds: float
    site_updates: int
    p50_ms: float
    p99_ms: float
    mean_ms: float
    max_batch: int
    ticks: int
    extra: dict = field(default_factory=dict)

    @property
    def updates_per_ns(self) -> float:
        return self.site_updates / (self.wall_seconds * 1e9) if self.wall_seconds > 0 else 0.0


def poisson_trace(n: int, rate_per_s: float, seed: int, sides=tuple(range(16, 97, 8)), t_range=(0.2, 1.0),
                  sweep_range=(50, 500), first_sample: int = 0) -> list[Request]:
    """n requests with exponential inter-arrival gaps (mean 1/rate), L
    uniform in `sides`, T uniform in `t_range`, sweeps uniform in the
    inclusive `sweep_range`; request k is disorder sample first_sample + k."""
    # one row of four uniforms per request, so a trace is a prefix of any longer one
    u = np.random.default_rng([int(seed), 0x5E]).random((n, 4))
    gaps = -np.log1p(-u[:, 0]) / rate_per_s
    arrivals = np.cumsum(gaps) - gaps[0]
    sides = np.asarray(sides)
    Ls = sides[np.minimum((u[:, 1] * len(sides)).astype(int), len(sides) - 1)]
    Ts = t_range[0] + (t_range[1] - t_range[0]) * u[:, 2]
    span = sweep_range[1] - sweep_range[0] + 1
    sw = sweep_range[0] + np.minimum((u[:, 3] * span).astype(int), span - 1)
    return [Request(k, float(arrivals[k]), int(Ls[k]), int(seed), first_sample + k, float(Ts[k]), int(sw[k]))
            for k in range(n)]


def latency_stats(results: list[Result]) -> tuple[float, float, float]:
    """(p50, p99, mean) latency in milliseconds."""
    if not results:
        return math.nan, math.nan, math.nan
    lat = np.array([r.latency for r in results]) * 1e3
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99)), float(lat.mean())


def _updates(req: Request, passes: int) -> int:
    return req.L ** 3 * req.sweeps * passes


def _marker(stream):
    """An event recorded on `stream` after the work queued so far."""
    if stream is None:
        import torch

        return torch.cuda.current_stream().record_event()
    return stream.record_event()


def serve(requests: list[Request], sched_kw: dict, budget_bytes: int, max_slots: int, stream=None,
          tick_sweeps: int = 10, keep_spins: bool = False, autotune: bool = True,
          cancels: dict[int, float] | None = None, pool_factory=None,
          config: tuple | None = None) -> tuple[list[Result], ServeStats]:
    """Run the request loop in real time (arrivals are honoured on the wall
    clock from the call).  sched_kw: the schedule of every request
    (hsg.schedule keywords without T).  cancels: request id -> time (seconds
    from the start) at which its client withdraws it -- a request still
    waiting is dropped, an admitted one is retired at the next tick (its
    memory freed for the next admission); the other lattices are untouched.
    pool_factory(budget_bytes, max_slots, stream) makes the pool (hsg.Pool by
    default).  config: a pool launch configuration (threads, tile_sites,
    blocks_per_sm, hits_per_pass), e.g. the one a previous run's autotuner
    chose, set before the first sweep; with it the loop does not autotune.
    Otherwise, with autotune, the loop tunes once, when eight lattices are
    first resident -- every admitted request then waits for the tuning
    sweeps, so a server tunes at start-up and passes the result here.
    Returns per-request results in completion order and summary statistics
    (ids of withdrawn requests in stats.extra["cancelled"], of requests
    larger than the whole pool in stats.extra["rejected"], the launch
    configuration used in stats.extra["config"], None if the default).

    The host knows when every lattice finishes (its sweep count), so it
    schedules tick n+1 -- retirements, admissions into the freed memory,
    the next sweeps -- as soon as tick n is queued, and only then waits for
    tick n-1 to finish and hands out the results finished there (their
    energies were queued into one of two pinned buffers before their
    slots were retired).  The device always has the next tick queued while
    the host does its bookkeeping."""
    from . import hsg

    sched = hsg.schedule(**sched_kw)
    make_pool = pool_factory or hsg.Pool
    cancel_at = dict(cancels or {})
    cancelled: list[int] = []
    rejected: list[int] = []  # larger than the whole pool
    passes = (1 if sched_kw.get("kind", hsg.HSG_NONE) != hsg.HSG_NONE else 0) + sched_kw.get("n_or", 0)
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    waiting: collections.deque[Request] = collections.deque()
    active: dict[int, list] = {}  # slot -> [request, sweeps left, admitted at]
    results: list[Result] = []
    ticks = max_batch = 0
    tuned = not autotune or config is not None
    used_config = tuple(config) if config is not None else None
    prev = None  # the tick in flight: (marker, energy buffer or None, [(slot, request, admitted, spins)])
    buf = 0
    waited = 0.0  # seconds the host spent waiting (for the device or for arrivals)
    with make_pool(budget_bytes, max_slots, stream) as pool:
        if config is not None:
            hsg.hsg_pool_config(pool.pool, *config)
        t0 = time.perf_counter()
        while pending or waiting or active or prev is not None:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            if cancel_at:  # withdrawals that are due
                due = {rid for rid, tc in cancel_at.items() if tc <= now}
                for rid in due:
                    del cancel_at[rid]
                    for q in (pending, waiting):
                        hit = [r for r in q if r.rid == rid]
                        for r in hit:
                            q.remove(r)
                            cancelled.append(rid)
                    for slot in [sl for sl, a in active.items() if a[0].rid == rid]:
                        pool.retire(slot)
                        del active[slot]
                        cancelled.append(rid)
            while waiting:  # admit in arrival order while a slot and memory are free
                r = waiting[0]
                try:
                    slot = pool.admit(r.L, r.seed, r.sample, 0, r.T)
                except hsg.HsgError as e:
                    if e.status == hsg.HSG_EBUSY:
                        break
                    raise
                waiting.popleft()
                active[slot] = [r, r.sweeps, time.perf_counter() - t0]
            cur = None
            if active:
                if not tuned and len(active) >= 8:
                    used_config = hsg.hsg_pool_autotune(pool.pool, sched)
                    tuned = True
                k = min(tick_sweeps, min(a[1] for a in active.values()))
                pool.sweep(sched, k)
                ticks += 1
                max_batch = max(max_batch, len(active))
                done = []
                for slot, a in active.items():
                    a[1] -= k
                    if a[1] == 0:
                        done.append(slot)
                finished = []
                if done:
                    pool.energies_async(buf, done)  # the finished lattices' final E/N, before their slots go
                    for slot in done:
                        r, _, t_adm = active.pop(slot)
                        spins = pool.spins(slot) if keep_spins else None
                        finished.append((slot, r, t_adm, spins))
                        pool.retire(slot)
                cur = (_marker(stream), buf if done else None, finished)
                if done:
                    buf ^= 1
            elif prev is None:
                if waiting:  # an empty pool refused it: it can never be admitted
                    rejected.append(waiting.popleft().rid)
                elif pending:
                    tw = time.perf_counter()
                    time.sleep(max(0.0, min(pending[0].arrival - (tw - t0), 0.01)))
                    waited += time.perf_counter() - tw
                continue
            if prev is not None:  # wait for the tick before this one and hand out its results
                marker, b, finished = prev
                tw = time.perf_counter()
                marker.synchronize()
                waited += time.perf_counter() - tw
                if finished:
                    energies = pool.energies_read(b)
                    t_done = time.perf_counter() - t0
                    for slot, r, t_adm, spins in finished:
                        results.append(Result(r.rid, float(energies[slot]), r.arrival, t_adm, t_done, spins))
            prev = cur
        wall = time.perf_counter() - t0
    p50, p99, mean = latency_stats(results)
    by_id = {q.rid: q for q in requests}
    upd = sum(_updates(by_id[r.rid], passes) for r in results)
    return results, ServeStats(len(results), wall, upd, p50, p99, mean, max_batch, ticks,
                               extra={"cancelled": cancelled, "rejected": rejected, "config": used_config,
                                      "host_ms_per_tick": (wall - waited) * 1e3 / ticks if ticks else math.nan})


def serve_fifo(requests: list[Request], sched_kw: dict, stream=None, keep_spins: bool = False):
    """The comparison without batching: each request on its own context,
    one at a time in arrival order (wall-clock arrivals honoured)."""
    import torch

    from . import hsg

    passes = (1 if sched_kw.get("kind", hsg.HSG_NONE) != hsg.HSG_NONE else 0) + sched_kw.get("n_or", 0)
    results: list[Result] = []
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda q: q.arrival):
        wait = r.arrival - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        t_start = time.perf_counter() - t0
        with hsg.Lattice(r.L, r.seed, r.sample, 0, stream) as lat:
            lat.generate_couplings()
            lat.sweep(hsg.schedule(T=r.T, **sched_kw), r.sweeps)
            e = lat.energy()  # synchronises
            spins = lat.spins() if keep_spins else None
        results.append(Result(r.rid, e, r.arrival, t_start, time.perf_counter() - t0, spins))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    p50, p99, mean = latency_stats(results)
    upd = sum(_updates(r, passes) for r in requests)
    return results, ServeStats(len(results), wall, upd, p50, p99, mean, 1, len(results))
