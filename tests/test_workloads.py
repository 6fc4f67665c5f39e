"""The seeded synthetic workloads are reproducible (CPU only): the instances
the bench and the design notes quote are the ones the generators draw."""
import numpy as np

import oracle
from paper_2407_20474_gb300 import workloads


def test_config2_instance():
    g = workloads.config2_generators(0)
    assert tuple(g) == (56, 90, 96, 127, 146, 178)
    n = workloads.find_n(oracle.count_upto, g, workloads.CONFIG2_TARGET, 4096)
    assert n == 39064
    assert oracle.count(g, n) == 500_108_275
    assert oracle.count(g, n - 1) < workloads.CONFIG2_TARGET


def test_config3_instance():
    g = workloads.config3_generators(1)
    assert tuple(g) == (4, 20, 22, 31, 39)
    counts = oracle.count_upto(g, workloads.CONFIG3_N)
    assert int(np.sum(np.asarray(counts, dtype=np.float64))) == 35_967_533


def test_config4_and_config5_draws_are_seeded():
    a = workloads.config4_instances(2, 64)
    b = workloads.config4_instances(2, 64)
    assert [x.g for x in a] == [x.g for x in b]
    assert [x.target for x in a] == [x.target for x in b]
    for x in a:
        assert 3 <= len(x.g) <= 8 and all(2 <= v <= 300 for v in x.g)
        assert np.gcd.reduce(np.asarray(x.g)) == 1
        assert 1e2 <= x.target <= 1e6
    s1 = workloads.config5_stream(3, duration_s=1.0)
    s2 = workloads.config5_stream(3, duration_s=1.0)
    assert np.array_equal(s1.arrivals_s, s2.arrivals_s)
    assert len(s1.sets) == 64
