"""Workload definitions (CPU): the configurations bench.py times have the
sizes they are named for, and every sweep point is a valid context."""
import math

import numpy as np

from paper_2504_06067_gb300 import workloads as wl


def _das_dennis(m, p1, p2=0):
    return math.comb(p1 + m - 1, m - 1) + (math.comb(p2 + m - 1, m - 1) if p2 else 0)


def test_named_configs_match_their_sizes():
    assert wl.SCALE.w == _das_dennis(5, 20) == 10626 and wl.SCALE.N == 10628
    assert wl.LARGE.w == _das_dennis(10, 3, 2) == 275 and wl.LARGE.N == 100000
    assert wl.SMALL.w == 91 and wl.KNAPSACK.w == _das_dennis(3, 158)


def test_largest_p_fits_and_is_largest():
    for m in (3, 6, 16, 512):
        for N in (50, 800, 12800):
            p = wl.largest_p(m, N)
            assert _das_dennis(m, p) <= N or p == 1
            assert _das_dennis(m, p + 1) > N


def test_objective_sweep_is_table_two_shape():
    cfgs = wl.objective_sweep()
    assert [c.m for c in cfgs] == [4, 8, 16, 32, 64, 128, 256, 512]
    for c in cfgs:
        assert c.N == 800 and c.d == 1000 and c.d >= c.m - 1 and c.w <= c.N
        assert c.N % 2 == 0


def test_population_sweep_is_table_one_shape():
    cfgs = wl.population_sweep()
    assert [c.N for c in cfgs] == [50, 100, 200, 400, 800, 1600, 3200, 6400, 12800]
    for c in cfgs:
        assert c.m == 6 and c.d == 500 and c.w <= c.N and c.N % 2 == 0


def test_objective_inputs_are_seeded_and_finite():
    for kind in wl.KINDS:
        a = wl.objectives(kind, 64, 7, seed=3)
        b = wl.objectives(kind, 64, 7, seed=3)
        assert a.dtype == np.float32 and a.shape == (64, 7)
        assert np.array_equal(a, b) and np.isfinite(a).all()
