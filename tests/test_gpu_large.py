"""Parity at the full large-population size: m = 10, N = 100,000 (merged
2N = 200,000, a 5.0 GB bit matrix), two-layer directions p1 = 3, p2 = 2
(w = 275), d = 200, in the launch configuration bench.py times.

The ranks of all 200,000 merged points are compared element by element with
the oracle's non-dominated sort (Alg. 1; O((2N)^2 m), run on every host core
through the oracle's OpenMP loops, about a minute).  The sampled checks of
the front definition stay as an independent cross-check (a point of front
k is dominated by no point of front >= k nor of F_drop and, for k > 0, by
some point of front k-1; a point of F_drop is dominated by some point of
F_l).  Given those ranks, the oracle computes the rest of the selection in
full (normalization, association of every point of S u F_l, niching) and
the GPU must match it bit for bit."""
import numpy as np
import pytest

from paper_2504_06067_gb300 import workloads as wl

from gpu_util import Run

pytestmark = pytest.mark.gpu

CFG = wl.LARGE
SAMPLES = 300


@pytest.fixture(scope="module")
def large(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_2504_06067_gb300 import native as n
    c = CFG
    W = wl.objective_weights(c.m, c.seed)
    out = {"n": n}
    with Run(n, c.m, c.d, c.N, c.p1, p2=c.p2, tau=c.tau, seed=c.seed, W=W) as r:
        r.check(n.nsga3_init(r.ctx, None))
        r.check(n.nsga3_run(r.ctx, 2, None))
        X, F, rank = r.population()
        gen = r.counter()
        r.check(n.nsga3_step(r.ctx, None))
        assert r.sync() == 0
        Xc, Fc = r.children()
        out["next"] = r.population()
        RF = np.vstack([F, Fc])
        out["RX"] = np.vstack([X, Xc])
        out["RF"] = RF
        # the same merged objectives through nsga3_select, same counter
        st, rank2, sel = r.select(RF, gen=gen)
        assert st == 0
        out.update(rank=rank2, sel=sel, info=r.info(), gen=gen)
        out["norm"] = r.normalization()
        out["assoc"] = r.association()
        out["Z"] = r.refs()
    return out


def _dominators(RF, i):
    f = RF[i]
    return np.all(RF <= f, axis=1) & np.any(RF < f, axis=1)


def test_step_equals_select(large):
    """The generation's selection (graph) and nsga3_select on the same merged
    objectives and counter pick the same individuals."""
    Xn, Fn, rn = large["next"]
    sel = large["sel"]
    assert np.all(np.diff(sel) > 0)
    assert np.array_equal(Xn, large["RX"][sel]) and np.array_equal(Fn, large["RF"][sel])
    assert np.array_equal(rn, large["rank"][sel])


def test_front_sizes_and_l(large):
    rank, info = large["rank"], large["info"]
    l = info["l"]
    sizes = np.bincount(rank[rank >= 0])
    assert len(sizes) == l + 1
    cum = np.cumsum(sizes)
    assert cum[-1] >= CFG.N and (l == 0 or cum[-2] < CFG.N)
    assert info["nS"] == (cum[-2] if l > 0 else 0) and info["nFl"] == sizes[-1]


def test_all_ranks_equal_the_oracle(large, orc):
    """Every one of the 2N = 200,000 ranks (front index, -1 for F_drop)
    equals the oracle's sort of the same FP32 objectives."""
    rank, info = large["rank"], large["info"]
    ref, l = orc.nds(large["RF"], CFG.N)
    assert l == info["l"]
    bad = np.flatnonzero(rank != ref)
    assert len(bad) == 0, (len(bad), bad[:10], rank[bad[:10]], ref[bad[:10]])


def test_sampled_ranks_satisfy_the_front_definition(large):
    RF, rank = large["RF"], large["rank"]
    l = large["info"]["l"]
    rng = np.random.default_rng(0)
    idx = rng.choice(len(RF), size=SAMPLES, replace=False)
    # make sure every kind of point is sampled
    for k in (0, l, -1):
        pool = np.flatnonzero(rank == k)
        if len(pool):
            idx = np.concatenate([idx, rng.choice(pool, size=min(20, len(pool)), replace=False)])
    for i in idx:
        dom = _dominators(RF, i)
        r = rank[i]
        if r >= 0:
            later = (rank >= r) | (rank < 0)
            assert not np.any(dom & later), i
            if r > 0:
                assert np.any(dom & (rank == r - 1)), i
        else:
            assert np.any(dom & (rank == l)), i


def test_normalization_matches_oracle(large, orc):
    rank, l = large["rank"], large["info"]["l"]
    zstar, a, ext, fb = orc.normalize(large["RF"], rank, l)
    z, ag, eg = large["norm"]
    assert np.array_equal(z, zstar) and np.array_equal(ag, a) and np.array_equal(eg, ext)
    assert bool(large["info"]["fallback"]) == fb


def test_association_matches_oracle(large, orc):
    rank, l = large["rank"], large["info"]["l"]
    z, a, _ = large["norm"]
    Z = orc.refdirs(CFG.m, CFG.p1, CFG.p2, CFG.tau)
    assert np.array_equal(large["Z"], Z)
    pi, dist = orc.associate(large["RF"], rank, l, z, a, Z)
    gpi, gdist = large["assoc"]
    T = (rank >= 0) & (rank <= l)
    assert np.array_equal(gpi[T], pi[T])
    assert np.array_equal(gdist[T], dist[T])


def test_niching_matches_oracle(large, orc):
    rank, info, gen = large["rank"], large["info"], large["gen"]
    l, K = info["l"], info["K"]
    pi, dist = large["assoc"]
    w = large["Z"].shape[0]
    sel = large["sel"]
    S = np.flatnonzero((rank >= 0) & (rank < l))
    if info["niche"]:
        picked = orc.niche(rank, l, K, pi, dist, w, CFG.seed, gen)
        exp = np.sort(np.concatenate([S, np.flatnonzero(picked)]))
    else:
        exp = np.flatnonzero((rank >= 0) & (rank <= l))
    assert np.array_equal(sel, exp)


def test_full_sort_many_fronts_at_full_size(large, orc):
    """2N = 200,000 points with many fronts (m = 3, full_sort): every rank
    equals the oracle's full sort, and sampled ranks of every depth satisfy
    the front definition."""
    n = large["n"]
    N = CFG.N
    RF = wl.objectives("early", 2 * N, 3, seed=7)
    with Run(n, 3, 3, N, 12, full_sort=1) as r:
        st, rank, sel = r.select(RF)
        assert st == 0
    assert rank.min() == 0 and rank.max() > 10
    ref, _ = orc.nds(RF, N, full_sort=True)
    assert np.array_equal(rank, ref), int(np.count_nonzero(rank != ref))
    sizes = np.bincount(rank)
    assert sizes.sum() == 2 * N and np.all(sizes > 0)
    rng = np.random.default_rng(1)
    idx = rng.choice(2 * N, size=SAMPLES, replace=False)
    for i in idx:
        dom = _dominators(RF, i)
        assert not np.any(dom & (rank >= rank[i])), i
        if rank[i] > 0:
            assert np.any(dom & (rank == rank[i] - 1)), i
