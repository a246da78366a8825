"""The run server (continuous batching): every run's result equals the same
run executed alone through nsga3_init + nsga3_run, bit for bit; admission
respects the memory budget; a request larger than the budget fails cleanly."""
import time

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


def _alone(n, c, W, gens):
    with Run(n, c.m, c.d, c.N, c.p1, p2=c.p2, seed=c.seed, W=W) as r:
        r.check(n.nsga3_init(r.ctx, None))
        r.check(n.nsga3_run(r.ctx, gens, None))
        assert r.sync() == 0
        return r.population()


def _collect(n, srv, ids, cfgs, timeout_s=300):
    out = {}
    t_end = time.time() + timeout_s
    while len(out) < len(ids) and time.time() < t_end:
        rid = srv.wait(1000)
        if rid < 0:
            continue
        c = cfgs[rid]
        X = np.zeros((c.N, c.d), np.float32)
        F = np.zeros((c.N, c.m), np.float32)
        R = np.zeros(c.N, np.int32)
        st, info = srv.fetch(rid, X.ctypes.data, F.ctypes.data, R.ctypes.data)
        out[rid] = (st, info, (X, F, R))
    assert len(out) == len(ids), "server did not finish in time"
    return out


def test_results_same_alone_and_in_the_mix(n):
    """Uneven runs arriving while others are on the GPU: each final population
    equals the run alone."""
    rng = np.random.default_rng(5)
    cfgs, Ws, gens = {}, {}, {}
    with n.Server(4 << 30, max_active=6, gens_per_launch=3) as srv:
        ids = []
        for i in range(10):
            m = int(rng.choice([3, 5, 8]))
            N = int(rng.choice([100, 228, 640, 1500, 3000]))
            c = wl.RunConfig("srv%d" % i, m=m, d=m + 9, N=N, p1=wl.largest_p(m, N), seed=100 + i)
            g = int(rng.integers(4, 25))
            W = wl.objective_weights(m, c.seed)
            rid = srv.submit(c.m, c.d, c.N, c.p1, g, W, seed=c.seed)
            cfgs[rid], Ws[rid], gens[rid] = c, W, g
            ids.append(rid)
            time.sleep(0.005 * (i % 3))
        got = _collect(n, srv, ids, cfgs)
        stats = srv.stats()
    assert stats["completed"] == 10 and stats["peak_active"] >= 2
    for rid in ids:
        st, info, pop = got[rid]
        assert st == n.OK, info.message
        assert info.t_submit <= info.t_admit <= info.t_done
        exp = _alone(n, cfgs[rid], Ws[rid], gens[rid])
        for a, b in zip(pop, exp):
            assert np.array_equal(a, b), rid


def test_admission_respects_the_memory_budget(n):
    m, d, N = 5, 30, 2000
    p = wl.largest_p(m, N)
    need = n.workspace_bytes(m, d, N, p)
    W = wl.objective_weights(m, 0)
    with n.Server(int(2.5 * need), max_active=8, gens_per_launch=4) as srv:
        ids = [srv.submit(m, d, N, p, 12, W, seed=s) for s in range(5)]
        cfgs = {i: wl.RunConfig("b", m=m, d=d, N=N, p1=p) for i in ids}
        got = _collect(n, srv, ids, cfgs)
        stats = srv.stats()
    assert all(got[i][0] == n.OK for i in ids)
    assert stats["peak_active"] <= 2
    assert stats["peak_bytes"] <= int(2.5 * need)
    assert stats["bytes_in_use"] == 0


def test_request_above_the_budget_fails_cleanly(n):
    W3 = wl.objective_weights(3, 0)
    small = n.workspace_bytes(3, 12, 92, 12)
    with n.Server(4 * small, max_active=4, gens_per_launch=4) as srv:
        big = srv.submit(3, 12, 4000, 20, 5, W3, seed=1)
        ok = srv.submit(3, 12, 92, 12, 5, W3, seed=2)
        cfgs = {big: wl.RunConfig("x", m=3, d=12, N=4000, p1=20),
                ok: wl.RunConfig("y", m=3, d=12, N=92, p1=12)}
        got = _collect(n, srv, [big, ok], cfgs)
    assert got[big][0] == n.ENOMEM and got[big][1].t_admit < 0
    assert got[ok][0] == n.OK
    with n.Server(1 << 28, max_active=2) as srv:
        with pytest.raises(n.NSGA3Error):
            srv.submit(1, 12, 92, 12, 5, W3)
        with pytest.raises(n.NSGA3Error):
            srv.submit(3, 12, 91, 12, 5, W3)
