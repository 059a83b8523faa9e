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
