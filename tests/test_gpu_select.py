"""GPU parity of the environmental selection against the FP64 oracle.

The bar is bit-exact: ranks, selected indices, the normalization (ideal
point, intercepts, extremes) and the association (pi, d) must equal the
oracle's on identical FP32 objectives.
"""
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


def _compare(orc, run, F, Z, seed, gen, check_assoc=True):
    st, rank, sel = run.select(F, gen=gen)
    assert st == 0, "device status %d" % st
    ref = orc.select(F, run.N, Z, seed=seed, gen=gen)
    info = run.info()
    assert info["l"] == ref["l"] and info["nS"] == ref["nS"] and info["nFl"] == ref["nFl"]
    assert np.array_equal(rank, ref["rank"])
    if ref["niche"] and check_assoc:
        z, a, e = run.normalization()
        zs, aa, ee, fb = orc.normalize(F, ref["rank"], ref["l"])
        assert np.array_equal(z, zs) and np.array_equal(a, aa) and np.array_equal(e, ee)
        assert bool(info["fallback"]) == fb
        pi, dist = run.association()
        T = (ref["rank"] >= 0) & (ref["rank"] <= ref["l"])
        assert np.array_equal(pi[T], ref["pi"][T])
        assert np.array_equal(dist[T], ref["dist"][T])
    assert np.array_equal(sel, ref["selected"])
    return info, ref


def test_refdirs_bit_exact(n, orc):
    for m, p1, p2 in ((3, 12, 0), (5, 20, 0), (10, 3, 2), (2, 7, 0), (8, 5, 3)):
        with Run(n, m, m + 2, 64, p1, p2=p2) as r:
            Z = r.refs()
            assert np.array_equal(Z, orc.refdirs(m, p1, p2, 0.5))


@pytest.mark.parametrize("kind", wl.KINDS)
@pytest.mark.parametrize("shape", [(3, 92, 12, 0), (5, 300, 6, 0), (10, 500, 3, 2), (2, 70, 9, 0)])
def test_select_parity(n, orc, kind, shape):
    m, N, p1, p2 = shape
    Z = orc.refdirs(m, p1, p2, 0.5)
    with Run(n, m, m + 1, N, p1, p2=p2, seed=11) as r:
        for s in range(2):
            F = wl.objectives(kind, 2 * N, m, seed=s)
            _compare(orc, r, F, Z, seed=11, gen=s + 1)


def test_select_parity_ragged_sizes(n, orc):
    """Sizes that are not multiples of the 32/128/256 tiles (ragged tails)."""
    for m, N in ((3, 2), (4, 6), (3, 130), (6, 258), (7, 514)):
        p = wl.largest_p(m, N)
        Z = orc.refdirs(m, p)
        with Run(n, m, m + 1, N, p, seed=5) as r:
            for kind in ("early", "late", "dups"):
                F = wl.objectives(kind, 2 * N, m, seed=N)
                _compare(orc, r, F, Z, seed=5, gen=7)


def test_select_parity_scale_shape(n, orc):
    """m = 5, p = 20 (10,626 directions), N = 10,628: the plain-at-scale shape."""
    cfg = wl.SCALE
    Z = orc.refdirs(cfg.m, cfg.p1)
    with Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, seed=0) as r:
        for kind in ("late", "early"):
            F = wl.objectives(kind, 2 * cfg.N, cfg.m, seed=3)
            info, ref = _compare(orc, r, F, Z, seed=0, gen=4)
            assert info["overflow"] == 0


def test_full_sort_ranks_everyone(n, orc):
    m, N = 4, 200
    Z = orc.refdirs(m, 5)
    with Run(n, m, m + 1, N, 5, full_sort=1) as r:
        for kind in ("early", "chain", "grid"):
            F = wl.objectives(kind, 2 * N, m, seed=2)
            st, rank, sel = r.select(F, gen=1)
            assert st == 0
            ref = orc.select(F, N, Z, seed=0, gen=1, full_sort=True)
            assert np.array_equal(rank, ref["rank"]) and (rank >= 0).all()
            assert np.array_equal(sel, ref["selected"])


def test_debug_recheck_finds_no_miss(n, orc):
    m, N = 5, 2000
    p = 9
    Z = orc.refdirs(m, p)
    with Run(n, m, m + 1, N, p, debug_recheck_all=1) as r:
        for kind in ("late", "simplex", "uniform"):
            F = wl.objectives(kind, 2 * N, m, seed=9)
            info, _ = _compare(orc, r, F, Z, seed=0, gen=2)
            if info["niche"]:
                assert info["recheck_miss"] == 0


def test_nonfinite_objectives_rejected(n, orc):
    m, N = 3, 64
    with Run(n, m, m + 1, N, 6) as r:
        F = wl.objectives("late", 2 * N, m)
        for bad in (np.nan, np.inf, -np.inf):
            G = F.copy()
            G[17, 1] = bad
            st, _, _ = r.select(G)
            assert st == n.ENONFINITE
        # the context recovers: the status is cleared by the sync
        st, rank, sel = r.select(F, gen=0)
        assert st == 0
        ref = orc.select(F, N, orc.refdirs(m, 6), seed=0, gen=0)
        assert np.array_equal(sel, ref["selected"])


def test_bad_arguments(n):
    import ctypes as C
    h = C.c_void_p()
    o = n.default_opts()
    for args in ((1, 3, 10, 4), (513, 3, 10, 4), (3, 3, 9, 4), (3, 3, 10, 0), (3, 3, 0, 4)):
        assert n.nsga3_create(*args, C.byref(o), C.byref(h)) == n.EINVAL
        assert h.value is None
    # streaming and the knapsack workload stop at m = 10
    for o in (n.default_opts(streaming=1), n.default_opts(problem=1)):
        assert n.nsga3_create(11, 12, 10, 1, C.byref(o), C.byref(h)) == n.EINVAL
        assert h.value is None


def test_wait_budget_expires_cleanly(n, orc):
    """Failure detection without a fault: a device wait on a word nothing
    sets gives up after opts.wait_ms of device time and records
    NSGA3_ETIMEOUT; nsga3_sync reports it once, and the same context then
    selects like the oracle."""
    import time
    m, N, p = 3, 92, 12
    Z = orc.refdirs(m, p)
    with Run(n, m, m + 1, N, p, seed=2, wait_ms=300) as r:
        t0 = time.time()
        r.check(n.nsga3_wait_probe(r.ctx, None))
        assert r.sync() == n.ETIMEOUT
        assert 0.25 <= time.time() - t0 < 30.0
        assert r.sync() == n.OK
        F = wl.objectives("early", 2 * N, m, seed=1)
        st, rank, sel = r.select(F, gen=1)
        assert st == 0
        ref = orc.select(F, N, Z, seed=2, gen=1)
        assert np.array_equal(rank, ref["rank"]) and np.array_equal(sel, ref["selected"])


def test_phase_timing_levels(n):
    """opts.phase_timing: 0 records no timing events in the graphs (phase
    times are refused), 1 times the dominance build and the peel, 2 every
    phase; the event nodes change nothing in the results."""
    import ctypes as C
    import os
    m, d, N, p = 3, 4, 92, 12
    W = wl.objective_weights(m, 1)
    pops = []
    for lv in (0, 1, 2):
        with Run(n, m, d, N, p, seed=3, W=W, phase_timing=lv) as r:
            r.check(n.nsga3_init(r.ctx, None))
            for _ in range(3):
                r.check(n.nsga3_step(r.ctx, None))
            assert r.sync() == 0
            ms = (C.c_float * 7)()
            st = n.nsga3_phase_times(r.ctx, ms, 7)
            v = list(ms)
            if lv == 0:
                if os.environ.get("NSGA3_EAGER") != "1":  # eager execution times every phase
                    assert st == n.EINVAL
            else:
                assert st == n.OK and v[2] > 0 and v[3] > 0
                if lv == 1:
                    assert all(v[t] == -1.0 for t in (0, 1, 4, 5, 6))
                else:
                    assert min(v) >= 0 and v[6] >= v[2] + v[3] - 1e-3
            pops.append(r.population())
    for P in pops[1:]:
        for a, b in zip(pops[0], P):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("dc,pc", [(1, 0), (2, 1), (3, 2), (0, 1)])
def test_launch_shapes_change_nothing(n, orc, dc, pc):
    """The launch-shape options (persistent CTAs per SM of the dominance
    build, cooperative CTAs per SM of the peel) change no result: selections
    of several shapes equal the oracle's."""
    for m, N, p1, p2, kind in ((10, 3000, 3, 2, "early"), (5, 2000, 6, 0, "late"), (3, 4000, 40, 0, "dups")):
        Z = orc.refdirs(m, p1, p2, 0.5)
        with Run(n, m, m + 1, N, p1, p2=p2, seed=4, dom_ctas_per_sm=dc, peel_ctas_per_sm=pc) as r:
            F = wl.objectives(kind, 2 * N, m, seed=dc + 3 * pc)
            _compare(orc, r, F, Z, seed=4, gen=2)


@pytest.mark.parametrize("m", list(range(2, 11)))
def test_dominance_entry_paths_every_m(n, orc, m):
    """Every specialised dominance kernel (m = 2 ... 10): odd m takes the
    scalar subtraction for its last objective in the live-column loop, m > 6
    the early end after five objectives; early (many fronts), late and
    simplex objective sets give entries with and without live rows and
    columns, packed and unpacked row pairs.  Ranks and selections equal the
    oracle's."""
    N = 2500
    p = wl.largest_p(m, N)
    Z = orc.refdirs(m, p)
    with Run(n, m, m + 1, N, p, seed=6) as r:
        for s, kind in enumerate(("early", "late", "simplex")):
            F = wl.objectives(kind, 2 * N, m, seed=40 + s)
            _compare(orc, r, F, Z, seed=6, gen=s + 1)
