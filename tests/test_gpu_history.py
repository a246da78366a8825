"""Normalization with history (opts.norm_history = 1): a running ideal point
and remembered extreme points carried from selection to selection.  Every
selection of a sequence must equal the oracle's with the same history:
ranks, selected indices, ideal point, intercepts and extreme indices
(2N + r for a remembered vector), bit for bit."""
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


def _check(orc, r, F, Z, h, seed, gen):
    st, rank, sel = r.select(F, gen=gen)
    assert st == 0
    ref = orc.select(F, r.N, Z, seed=seed, gen=gen, history=h)
    assert np.array_equal(rank, ref["rank"]) and np.array_equal(sel, ref["selected"])
    if ref["niche"]:
        z, a, e = r.normalization()
        assert np.array_equal(z, h["z"])
        return z, a, e, ref
    return None, None, None, ref


@pytest.mark.parametrize("m,N,p", [(3, 92, 12), (5, 300, 6), (8, 400, 3)])
def test_history_sequence_matches_oracle(n, orc, m, N, p):
    Z = orc.refdirs(m, p)
    h = orc.new_history(m)
    with Run(n, m, m + 1, N, p, seed=3, norm_history=1) as r:
        for g in range(6):
            kind = ("early", "late", "uniform")[g % 3]
            # later generations drift upwards: the running ideal must hold
            F = (wl.objectives(kind, 2 * N, m, seed=g) + np.float32(0.02 * g)).astype(np.float32)
            prev = {k: v.copy() for k, v in h.items()}
            z, a, e, ref = _check(orc, r, F, Z, h, seed=3, gen=g + 1)
            if z is not None:
                rank, l = ref["rank"], ref["l"]
                zz, aa, ee, fb = orc.normalize_hist(F, rank, l, prev)
                assert np.array_equal(z, zz) and np.array_equal(a, aa) and np.array_equal(e, ee)


def test_remembered_axis_extremes_on_gpu(n, orc):
    """The closed-form case of the oracle pin: axis points in generation 1,
    interior points later; the GPU picks the remembered vectors (2N + q)."""
    m, N = 3, 10
    rng = np.random.default_rng(0)
    F1 = rng.dirichlet(np.ones(m), size=2 * N).astype(np.float32)
    F1[:3] = np.eye(m, dtype=np.float32)
    F2 = (0.1 + 0.3 * rng.dirichlet(np.ones(m), size=2 * N)).astype(np.float32)
    Z = orc.refdirs(m, 3)
    h = orc.new_history(m)
    with Run(n, m, m + 1, N, 3, seed=1, norm_history=1) as r:
        _check(orc, r, F1, Z, h, seed=1, gen=1)
        z, a, e, ref = _check(orc, r, F2, Z, h, seed=1, gen=2)
    if ref["niche"]:
        assert np.array_equal(z, np.zeros(m)) and np.array_equal(e, 2 * N + np.arange(m))
        assert np.array_equal(a, np.ones(m))


def test_history_generations_and_init_reset(n, orc):
    """nsga3_step with history selects like the oracle with history on the
    GPU's own children; nsga3_init starts a fresh history."""
    cfg = wl.RunConfig("m5_N300", m=5, d=20, N=300, p1=6)
    W = wl.objective_weights(cfg.m, 2)
    Z = orc.refdirs(cfg.m, cfg.p1)
    with Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, seed=9, W=W, norm_history=1) as r:
        for rep in range(2):
            h = orc.new_history(cfg.m)
            r.check(n.nsga3_init(r.ctx, None))
            for g in range(5):
                X, F, rank = r.population()
                r.check(n.nsga3_step(r.ctx, None))
                assert r.sync() == 0
                Xc, Fc = r.children()
                Xn, Fn, rn = r.population()
                RF = np.vstack([F, Fc])
                ref = orc.select(RF, cfg.N, Z, seed=9, gen=g, history=h)
                sel = ref["selected"]
                assert np.array_equal(Fn, RF[sel]) and np.array_equal(rn, ref["rank"][sel])
