"""Streaming dominance (opts.streaming = 1: no dominance matrix; the peel
recomputes the dominance of each front's members from the objectives).

The bar is the same as for the matrix path: ranks and selected indices
bit-exact against the oracle, identical generations to the matrix path, and
at a size whose matrix would not be stored (2N = 600,000: a 45 GB matrix),
sampled ranks that satisfy the definition of the fronts."""
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


@pytest.mark.parametrize("kind", wl.KINDS)
@pytest.mark.parametrize("shape", [(3, 92, 12, 0), (5, 300, 6, 0), (10, 500, 3, 2), (2, 70, 9, 0)])
def test_streaming_select_parity(n, orc, kind, shape):
    m, N, p1, p2 = shape
    Z = orc.refdirs(m, p1, p2, 0.5)
    with Run(n, m, m + 1, N, p1, p2=p2, seed=11, streaming=1) as r:
        for s in range(2):
            F = wl.objectives(kind, 2 * N, m, seed=s)
            st, rank, sel = r.select(F, gen=s + 1)
            assert st == 0
            ref = orc.select(F, N, Z, seed=11, gen=s + 1)
            assert np.array_equal(rank, ref["rank"])
            assert np.array_equal(sel, ref["selected"])


def test_streaming_full_sort_matches_matrix(n, orc):
    """Many fronts (chain, early) and ragged sizes, every front ranked."""
    for m, N in ((3, 130), (5, 1000), (8, 2050)):
        p = wl.largest_p(m, N)
        Z = orc.refdirs(m, p)
        with Run(n, m, m + 1, N, p, full_sort=1, streaming=1) as s_run, \
                Run(n, m, m + 1, N, p, full_sort=1) as m_run:
            for kind in ("early", "chain", "grid", "dups"):
                F = wl.objectives(kind, 2 * N, m, seed=N)
                st, rs, ss = s_run.select(F, gen=2)
                st2, rm, sm = m_run.select(F, gen=2)
                assert st == 0 and st2 == 0
                assert np.array_equal(rs, rm) and np.array_equal(ss, sm)
                if N <= 1000:
                    ref = orc.select(F, N, Z, seed=0, gen=2, full_sort=True)
                    assert np.array_equal(rs, ref["rank"])


def test_streaming_generations_equal_matrix(n):
    cfg = wl.RunConfig("m5_N1000_d100", m=5, d=100, N=1000, p1=7)
    W = wl.objective_weights(cfg.m, 0)
    pops = []
    for streaming in (0, 1):
        with Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, seed=4, W=W, streaming=streaming) as r:
            r.check(n.nsga3_init(r.ctx, None))
            r.check(n.nsga3_run(r.ctx, 12, None))
            assert r.sync() == 0
            pops.append(r.population())
    for a, b in zip(*pops):
        assert np.array_equal(a, b)


def test_streaming_workspace_is_linear(n):
    o = n.default_opts(streaming=1)
    small = n.workspace_bytes(3, 3, 300000, 12, o)
    full = n.workspace_bytes(3, 3, 300000, 12)
    assert full > 40e9 and small < 1e9


def test_streaming_at_a_size_without_matrix(n):
    """2N = 600,000 (m = 3): the matrix would take 45 GB; sampled ranks of
    every depth satisfy the front definition against all points."""
    N = 300000
    F = wl.objectives("early", 2 * N, 3, seed=9)
    with Run(n, 3, 3, N, 12, full_sort=1, streaming=1) as r:
        st, rank, sel = r.select(F, gen=1)
        assert st == 0
    assert rank.min() == 0 and rank.max() > 10 and (rank >= 0).all()
    rng = np.random.default_rng(3)
    for i in rng.choice(2 * N, size=200, replace=False):
        f = F[i]
        dom = np.all(F <= f, axis=1) & np.any(F < f, axis=1)
        assert not np.any(dom & (rank >= rank[i])), i
        if rank[i] > 0:
            assert np.any(dom & (rank == rank[i] - 1)), i
