"""Second workload, 0-1 multi-objective knapsack: every step is integer or
bit arithmetic, so the GPU runs must equal the oracle's bit for bit -- the
initial population, the children of a generation (uniform crossover,
bit-flip mutation, repair, objectives) and whole runs."""
import ctypes as C

import numpy as np
import pytest

from paper_2504_06067_gb300 import workloads as wl

from gpu_util import Run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def n():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_2504_06067_gb300 import native
    return native


def _kp_run(n, m, d, N, p, seed, inst):
    profit, weight, cap = inst
    return Run(n, m, d, N, p, seed=seed, problem=1, kp_profit=profit.ctypes.data,
               kp_weight=weight.ctypes.data, kp_capacity=cap.ctypes.data)


CASES = [(2, 40, 100, 9), (3, 120, 300, 14), (5, 60, 200, 4)]


@pytest.mark.parametrize("m,d,N,p", CASES)
def test_kp_init_matches_oracle(n, orc, m, d, N, p):
    inst = wl.knapsack_instance(m, d, seed=m)
    with _kp_run(n, m, d, N, p, 3, inst) as r:
        r.check(n.nsga3_init(r.ctx, None))
        X, F, rank = r.population()
    Xo, Fo = orc.kp_eval(orc.kp_init(N, d, 3), *inst)
    assert np.array_equal(X, Xo) and np.array_equal(F, Fo) and (rank == 0).all()


@pytest.mark.parametrize("m,d,N,p", CASES)
def test_kp_children_match_oracle(n, orc, m, d, N, p):
    inst = wl.knapsack_instance(m, d, seed=m + 1)
    X = (wl.population(N, d, seed=2) < 0.6).astype(np.float32)
    X, F = orc.kp_eval(X, *inst)
    rank = wl.parent_ranks(N, 3, seed=1)
    with _kp_run(n, m, d, N, p, 5, inst) as r:
        r.set_population(X, F, rank)
        r.check(n.nsga3_set_counter(r.ctx, 7, None))
        r.check(n.nsga3_vary(r.ctx, None))
        Xc, Fc = r.children()
    Xo, Fo = orc.kp_eval(orc.kp_vary(X, rank, seed=5, gen=7), *inst)
    assert np.array_equal(Xc, Xo) and np.array_equal(Fc, Fo)


@pytest.mark.parametrize("m,d,N,p", CASES)
def test_kp_runs_equal_oracle(n, orc, m, d, N, p):
    inst = wl.knapsack_instance(m, d, seed=10 + m)
    gens = 25
    with _kp_run(n, m, d, N, p, 8, inst) as r:
        r.check(n.nsga3_init(r.ctx, None))
        r.check(n.nsga3_run(r.ctx, gens, None))
        assert r.sync() == 0
        X, F, rank = r.population()
    Z = orc.refdirs(m, p)
    Xo, Fo, ro = orc.kp_run(N, d, *inst, Z, seed=8, generations=gens)
    assert np.array_equal(X, Xo) and np.array_equal(F, Fo) and np.array_equal(rank, ro)
    # repaired populations are feasible
    W = inst[1].astype(np.int64)
    assert np.all(W @ X.T.astype(np.int64) <= inst[2][:, None])


def test_kp_rejects_bad_instances(n):
    profit, weight, cap = wl.knapsack_instance(3, 20, seed=0)
    bad = profit.copy()
    bad[1, 3] = 0
    o = n.default_opts(problem=1, kp_profit=bad.ctypes.data, kp_weight=weight.ctypes.data,
                       kp_capacity=cap.ctypes.data)
    h = C.c_void_p()
    assert n.nsga3_create(3, 20, 40, 5, C.byref(o), C.byref(h)) == n.EINVAL
    o = n.default_opts(problem=2)
    assert n.nsga3_create(3, 20, 40, 5, C.byref(o), C.byref(h)) == n.EINVAL
