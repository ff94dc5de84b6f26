"""Host-side logic of the serving driver (no GPU): the Poisson request stream
and the latency summary that bench.py reports for the engine and for the
one-request-at-a-time form."""
import numpy as np

from paper_2606_11402_gb300 import serve as sv


def test_poisson_stream_statistics():
    """Arrivals of a Poisson process of rate r over T seconds: the count is
    Poisson(rT) (within 5 standard deviations), the gaps exponential with mean
    1/r, arrivals increasing inside [0, T), instances and operations uniform
    over their ranges."""
    rate, T, n_inst = 2000.0, 5.0, 64
    reqs = sv.poisson_stream(n_inst, rate, T, seed=8)
    n = len(reqs)
    assert abs(n - rate * T) <= 5 * np.sqrt(rate * T)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < T
    gaps = np.diff(np.r_[0.0, t])
    assert abs(gaps.mean() * rate - 1.0) <= 5 / np.sqrt(n)
    # exponential gaps: P(gap > 1/r) = e^-1
    assert abs(np.mean(gaps > 1 / rate) - np.exp(-1)) <= 5 * np.sqrt(np.exp(-1) * (1 - np.exp(-1)) / n)
    inst = np.array([r.inst for r in reqs])
    ops = np.array([r.op for r in reqs])
    assert inst.min() >= 0 and inst.max() < n_inst
    assert set(ops.tolist()) == set(sv.OPS)
    for o in sv.OPS:
        assert abs(np.mean(ops == o) - 1 / len(sv.OPS)) <= 5 * np.sqrt(0.25 * 0.75 / n)
    counts = np.bincount(inst, minlength=n_inst)
    expect = n / n_inst
    assert np.all(np.abs(counts - expect) <= 6 * np.sqrt(expect))


def test_poisson_stream_is_seeded():
    a = sv.poisson_stream(16, 500.0, 1.0, seed=3)
    b = sv.poisson_stream(16, 500.0, 1.0, seed=3)
    c = sv.poisson_stream(16, 500.0, 1.0, seed=4)
    assert [(r.inst, r.op, r.arrival) for r in a] == [(r.inst, r.op, r.arrival) for r in b]
    assert [(r.inst, r.op, r.arrival) for r in a] != [(r.inst, r.op, r.arrival) for r in c]
    only = sv.poisson_stream(4, 500.0, 1.0, seed=3, ops=(sv.LOGDET,))
    assert {r.op for r in only} == {sv.LOGDET}


def test_latency_percentiles():
    """p50 / p99 / p99.9 / mean / max in milliseconds of latencies given in seconds,
    against the order statistics of 1..100 ms (linear interpolation)."""
    lat = np.arange(1, 101) * 1e-3
    rng = np.random.default_rng(0)
    rng.shuffle(lat)
    p = sv._percentiles(lat)
    assert np.isclose(p["p50_ms"], 50.5)
    assert np.isclose(p["p99_ms"], 99.01)
    assert np.isclose(p["p999_ms"], 99.901)
    assert np.isclose(p["mean_ms"], 50.5)
    assert np.isclose(p["max_ms"], 100.0)
