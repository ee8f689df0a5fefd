"""The seeded workload generators: reproducible, within their stated ranges, and
shaped as stated (log-uniform positions, uniform precision choice, Poisson
arrivals at the requested rate, the long query first)."""

import math
import statistics

import workloads


def test_batched_queries_are_seeded_and_in_range():
    a = workloads.batched_queries(4096, seed=0)
    b = workloads.batched_queries(4096, seed=0)
    c = workloads.batched_queries(4096, seed=1)
    assert a == b and a != c
    ns, Ps = a
    assert len(ns) == len(Ps) == 4096
    assert all(10**4 <= n < 10**10 for n in ns)
    assert set(Ps) == {64, 128, 256}
    # log-uniform: log10 n is spread evenly over [4, 10)
    logs = [math.log10(n) for n in ns]
    assert abs(statistics.mean(logs) - 7.0) < 0.1
    quarters = [sum(1 for v in logs if 4 + 1.5 * i <= v < 4 + 1.5 * (i + 1)) for i in range(4)]
    assert all(abs(q - 1024) < 120 for q in quarters)
    assert all(abs(Ps.count(p) - 4096 / 3) < 130 for p in (64, 128, 256))


def test_expected_terms_is_seven_tenths_of_n():
    assert workloads.expected_terms([10, 100]) == 0.7 * 110


def test_serving_arrivals_shape():
    rate = 3.0
    tr = workloads.serving_arrivals(2000, rate, seed=1, long_query=(10**13 + 1, 256))
    assert tr[0] == (0.0, 10**13 + 1, 256)
    times = [t for t, _, _ in tr[1:]]
    assert times == sorted(times) and times[0] > 0
    gaps = [b - a for a, b in zip([0.0] + times[:-1], times)]
    assert abs(statistics.mean(gaps) - 1 / rate) < 0.05 / rate * 3     # exponential gaps, mean 1 / rate
    assert abs(statistics.pstdev(gaps) - 1 / rate) < 0.1 / rate * 3    # exponential: sd = mean
    assert all(10**6 <= n < 10**11 for _, n, _ in tr[1:])
    assert {P for _, _, P in tr[1:]} == {64, 256}
    assert tr == workloads.serving_arrivals(2000, rate, seed=1, long_query=(10**13 + 1, 256))
    assert workloads.serving_arrivals(5, 1.0)[0][0] > 0                 # no long query: first arrival after 0
