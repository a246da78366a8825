"""GPU parity of the generation around the selection: initial population,
variation + objective (tolerance), the next population (bit-exact given the
GPU's own children), determinism, resume, and the IGD of full runs."""
import numpy as np
import pytest

from paper_2504_06067_gb300 import workloads as wl

from gpu_util import Run

pytestmark = pytest.mark.gpu

# Children are FP32 in [0, 1].  The GPU evaluates SBX and polynomial
# mutation in FP32 (powf for the spread factor beta, expm1/log for the
# mutation step), the oracle in FP64.  The error of beta (an ulp or two of a
# value up to 2.14) reaches a child as 0.5 |y2 - y1| d(beta), an ABSOLUTE
# error that does not shrink with the child: SBX forms a child near 0 as the
# difference of two terms near |y2 - y1|.  So the children are held to 1e-6
# relative where |x| >= X_FLOOR and to the absolute bound 1e-6 X_FLOOR below
# it.  Measured on the GB300 over 15 variations (m = 3 ... 10, up to 4 M
# children): at most 1 ulp (1.2e-7 in [0.5, 1), 6e-8 below 0.5), so at most
# 6e-7 relative from 0.1 up, and 6e-8 absolute below.  The objective is
# evaluated in FP64 on both sides and rounded to FP32.
X_RTOL = 1e-6
X_FLOOR = 0.1
F_RTOL = 1e-6


def assert_children_close(Xc, Xo):
    """|Xc - Xo| <= X_RTOL max(|Xo|, X_FLOOR), element by element."""
    Xc = np.asarray(Xc, np.float64)
    Xo = np.asarray(Xo, np.float64)
    err = np.abs(Xc - Xo)
    bound = X_RTOL * np.maximum(np.abs(Xo), X_FLOOR)
    bad = np.flatnonzero(err > bound)
    assert len(bad) == 0, ("%d children outside the bound; worst err %.3g at |x| = %.3g; max abs err %.3g"
                           % (len(bad), err.flat[bad[np.argmax(err.flat[bad])]],
                              abs(Xo.flat[bad[np.argmax(err.flat[bad])]]), err.max()))


@pytest.fixture(scope="module")
def n():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_2504_06067_gb300 import native
    return native


CFGS = [wl.SMALL, wl.RunConfig("m5_N1000_d100", m=5, d=100, N=1000, p1=7),
        wl.RunConfig("m10_N600_d60", m=10, d=60, N=600, p1=3, p2=2)]


@pytest.mark.parametrize("cfg", CFGS, ids=lambda c: c.name)
def test_init_matches_oracle(n, orc, cfg):
    W = wl.objective_weights(cfg.m, 0)
    with Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, p2=cfg.p2, seed=cfg.seed, W=W) as r:
        r.check(n.nsga3_init(r.ctx, None))
        X, F, rank = r.population()
        Xo = orc.init_population(cfg.N, cfg.d, cfg.seed)
        assert np.array_equal(X, Xo)
        Fo = orc.evaluate(Xo, W)
        np.testing.assert_allclose(F, Fo, rtol=F_RTOL, atol=0)
        assert (rank == 0).all() and r.counter() == 0


@pytest.mark.parametrize("cfg", CFGS, ids=lambda c: c.name)
@pytest.mark.parametrize("gen", [0, 17])
def test_variation_matches_oracle(n, orc, cfg, gen):
    W = wl.objective_weights(cfg.m, 1)
    X = wl.population(cfg.N, cfg.d, seed=gen)
    F = orc.evaluate(X, W)
    rank = wl.parent_ranks(cfg.N, 4, seed=gen)
    with Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, p2=cfg.p2, seed=3, W=W) as r:
        r.set_population(X, F, rank)
        r.check(n.nsga3_set_counter(r.ctx, gen, None))
        r.check(n.nsga3_vary(r.ctx, None))
        Xc, Fc = r.children()
    Xo = orc.vary(X, rank, seed=3, gen=gen)
    assert_children_close(Xc, Xo)
    # objective of the GPU's own children, evaluated by the oracle
    np.testing.assert_allclose(Fc, orc.evaluate(Xc, W), rtol=F_RTOL, atol=0)


@pytest.mark.parametrize("cfg", CFGS, ids=lambda c: c.name)
def test_step_selects_like_oracle(n, orc, cfg):
    """After one generation the next population equals the oracle's
    selection over (parents u the GPU's children), bit for bit."""
    W = wl.objective_weights(cfg.m, 2)
    Z = orc.refdirs(cfg.m, cfg.p1, cfg.p2, cfg.tau)
    with Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, p2=cfg.p2, seed=9, W=W) as r:
        r.check(n.nsga3_init(r.ctx, None))
        for g in range(4):
            X, F, rank = r.population()
            r.check(n.nsga3_step(r.ctx, None))
            assert r.sync() == 0
            Xc, Fc = r.children()
            Xn, Fn, rn = r.population()
            RX = np.vstack([X, Xc])
            RF = np.vstack([F, Fc])
            ref = orc.select(RF, cfg.N, Z, seed=9, gen=g)
            sel = ref["selected"]
            assert np.array_equal(Xn, RX[sel]) and np.array_equal(Fn, RF[sel])
            assert np.array_equal(rn, ref["rank"][sel])
        assert r.counter() == 4


def test_bench_workload_generations_match_oracle(n, orc):
    """The default bench workload (m = 5, N = 10,628, d = 100, 10,626
    directions) in the configuration bench.py times (its seed and weights,
    events around the dominance build and the peel): the initial population
    equals the oracle's, the children are within X_RTOL relative (above
    X_FLOOR) of the oracle's variation of the same parents and their
    objectives within F_RTOL, and
    two generations select exactly the oracle's next populations."""
    cfg = wl.SCALE
    W = wl.objective_weights(cfg.m, cfg.seed)
    Z = orc.refdirs(cfg.m, cfg.p1, cfg.p2, cfg.tau)
    with Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, p2=cfg.p2, tau=cfg.tau, seed=cfg.seed, W=W,
             phase_timing=1) as r:
        r.check(n.nsga3_init(r.ctx, None))
        X, F, rank = r.population()
        assert np.array_equal(X, orc.init_population(cfg.N, cfg.d, cfg.seed))
        np.testing.assert_allclose(F, orc.evaluate(X, W), rtol=F_RTOL, atol=0)
        for g in range(2):
            X, F, rank = r.population()
            r.check(n.nsga3_step(r.ctx, None))
            assert r.sync() == 0
            Xc, Fc = r.children()
            Xo = orc.vary(X, rank, seed=cfg.seed, gen=g)
            assert_children_close(Xc, Xo)
            np.testing.assert_allclose(Fc, orc.evaluate(Xc, W), rtol=F_RTOL, atol=0)
            Xn, Fn, rn = r.population()
            RX, RF = np.vstack([X, Xc]), np.vstack([F, Fc])
            ref = orc.select(RF, cfg.N, Z, seed=cfg.seed, gen=g)
            sel = ref["selected"]
            assert np.array_equal(Xn, RX[sel]) and np.array_equal(Fn, RF[sel])
            assert np.array_equal(rn, ref["rank"][sel])


def test_runs_are_deterministic_and_resume(n, orc):
    cfg = CFGS[1]
    W = wl.objective_weights(cfg.m, 0)
    with Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, seed=4, W=W) as a, \
            Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, seed=4, W=W) as b:
        a.check(n.nsga3_init(a.ctx, None))
        a.check(n.nsga3_run(a.ctx, 20, None))
        pa = a.population()
        # 10 generations, checkpoint through the host, resume in a new context
        b.check(n.nsga3_init(b.ctx, None))
        b.check(n.nsga3_run(b.ctx, 10, None))
        X, F, rank = b.population()
        gen = b.counter()
    with Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, seed=4, W=W) as c:
        c.set_population(X, F, rank)
        c.check(n.nsga3_set_counter(c.ctx, gen, None))
        c.check(n.nsga3_run(c.ctx, 10, None))
        pc = c.population()
    for u, v in zip(pa, pc):
        assert np.array_equal(u, v)


def _igd(orc, F, rank, W, m):
    y = wl.front_sample(m, 10000)
    Xf = np.full((len(y), m - 1), 0.0, dtype=np.float32)
    Xf[:, :] = y
    R = orc.evaluate(np.hstack([Xf, np.full((len(y), 1), 0.5, np.float32)]), W).astype(np.float64)
    return orc.igd(F[rank == 0], R)


def test_igd_matches_oracle_median(n, orc):
    """m = 3, N = 92, p = 12, d = 12, 100 generations: the median IGD of the
    GPU runs is within 2% of the oracle runs' median.  GPU and oracle runs of
    one seed separate after a few generations (FP32 vs FP64 variation
    arithmetic), so the medians compare two samples of one distribution whose
    seed-to-seed spread is ~1.6%; 16 seeds keep the medians' noise near 0.5%
    (5 seeds would fail a correct implementation about one time in eight)."""
    cfg = wl.SMALL
    W = wl.objective_weights(cfg.m, 0)
    Z = orc.refdirs(cfg.m, cfg.p1)
    gi, oi = [], []
    for seed in range(16):
        with Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, seed=seed, W=W) as r:
            r.check(n.nsga3_init(r.ctx, None))
            r.check(n.nsga3_run(r.ctx, cfg.generations, None))
            assert r.sync() == 0
            X, F, rank = r.population()
        gi.append(_igd(orc, F, rank, W, cfg.m))
        Xo, Fo, ro = orc.run(cfg.N, cfg.d, W, Z, seed, cfg.generations)
        oi.append(_igd(orc, Fo, ro, W, cfg.m))
    g, o = float(np.median(gi)), float(np.median(oi))
    assert abs(g - o) <= 0.02 * o, (gi, oi)


def test_batched_runs_equal_single_runs(n, orc):
    """Several uneven runs advanced by one batched graph per generation give
    the same populations as each run stepped alone."""
    cfgs = wl.batched_configs(n_runs=6, generations=5)
    cfgs = [c for c in cfgs if c.N <= 4000][:4]
    runs = []
    try:
        for c in cfgs:
            W = wl.objective_weights(c.m, c.seed)
            r = Run(n, c.m, c.d, c.N, c.p1, seed=c.seed, W=W)
            r.check(n.nsga3_init(r.ctx, None))
            runs.append((c, W, r))
        n.check(n.run_batch([r.ctx for _, _, r in runs], 5, None))
        for c, W, r in runs:
            assert r.sync() == 0
            got = r.population()
            with Run(n, c.m, c.d, c.N, c.p1, seed=c.seed, W=W) as alone:
                alone.check(n.nsga3_init(alone.ctx, None))
                alone.check(n.nsga3_run(alone.ctx, 5, None))
                exp = alone.population()
            for u, v in zip(got, exp):
                assert np.array_equal(u, v)
    finally:
        for _, _, r in runs:
            r.close()


def test_batched_graphs_follow_context_identity_not_address(n, orc):
    """The batched graphs are cached by the runs' creation serials: after a
    member is destroyed and a new context takes its place in the list (at the
    same host address or not), the next call rebuilds the graphs before any
    launch (checked with generations = 0, which launches nothing), and the
    populations then equal each run stepped alone.  A list naming one context
    twice is rejected without any launch."""
    cfgs = [c for c in wl.batched_configs(n_runs=8, generations=3) if c.N <= 2000][:3]
    assert len(cfgs) == 3
    Ws = [wl.objective_weights(c.m, c.seed) for c in cfgs]
    runs = [Run(n, c.m, c.d, c.N, c.p1, seed=c.seed, W=W) for c, W in zip(cfgs, Ws)]
    try:
        for r in runs:
            r.check(n.nsga3_init(r.ctx, None))
        lead = runs[0]
        n.check(n.run_batch([r.ctx for r in runs], 2, None), lead.ctx)
        assert n.batch_graph_builds(lead.ctx) == 1
        n.check(n.run_batch([r.ctx for r in runs], 0, None), lead.ctx)
        assert n.batch_graph_builds(lead.ctx) == 1  # same list: graphs reused
        assert n.run_batch([runs[0].ctx, runs[1].ctx, runs[0].ctx], 1, None) == n.EINVAL
        assert b"more than once" in n.nsga3_last_error(lead.ctx)
        for r in runs:
            assert r.sync() == 0
        # replace member 1 by a new context of the same sizes and seed
        old_addr = runs[1].ctx
        runs[1].close()
        c, W = cfgs[1], Ws[1]
        runs[1] = Run(n, c.m, c.d, c.N, c.p1, seed=c.seed, W=W)
        runs[1].check(n.nsga3_init(runs[1].ctx, None))
        runs[1].check(n.nsga3_run(runs[1].ctx, 2, None))  # catch up with the others
        same_address = runs[1].ctx == old_addr
        n.check(n.run_batch([r.ctx for r in runs], 0, None), lead.ctx)
        assert n.batch_graph_builds(lead.ctx) == 2, "graphs not rebuilt (same address: %s)" % same_address
        n.check(n.run_batch([r.ctx for r in runs], 3, None), lead.ctx)
        for (c, W), r in zip(zip(cfgs, Ws), runs):
            assert r.sync() == 0
            got = r.population()
            with Run(n, c.m, c.d, c.N, c.p1, seed=c.seed, W=W) as alone:
                alone.check(n.nsga3_init(alone.ctx, None))
                alone.check(n.nsga3_run(alone.ctx, 5, None))
                exp = alone.population()
            for u, v in zip(got, exp):
                assert np.array_equal(u, v)
    finally:
        for r in runs:
            r.close()


def test_igd_matches_oracle_median_m5(n, orc):
    """m = 5, N = 212, p = 6 (210 directions), d = 24, 60 generations: the
    median IGD of the GPU runs is within 2% of the oracle runs' median.  One
    run's IGD varies by about 3.6% (std / mean) from seed to seed here, so
    each median takes 128 seeds (the difference of two medians then has a
    standard deviation near 0.6%, and a correct implementation stays inside
    2% but for about one time in two thousand)."""
    m, N, d, p, G = 5, 212, 24, 6, 60
    W = wl.objective_weights(m, 0)
    Z = orc.refdirs(m, p)
    gi, oi = [], []
    for seed in range(128):
        with Run(n, m, d, N, p, seed=seed, W=W) as r:
            r.check(n.nsga3_init(r.ctx, None))
            r.check(n.nsga3_run(r.ctx, G, None))
            assert r.sync() == 0
            X, F, rank = r.population()
        gi.append(_igd(orc, F, rank, W, m))
        Xo, Fo, ro = orc.run(N, d, W, Z, seed, G)
        oi.append(_igd(orc, Fo, ro, W, m))
    g, o = float(np.median(gi)), float(np.median(oi))
    assert abs(g - o) <= 0.02 * o, (g, o)
