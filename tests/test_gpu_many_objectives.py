"""Many objectives (m > 10, up to the m = 512 of the paper's Table II).

Above m = 10 the kernels take m at run time: chunked dominance tiles, the
extreme-point search by entry keys, the intercept system solved by one warp
(m <= 32) or by a cooperative grid (m > 32), and the association without
cone pruning.  The bar is the same as for m <= 10: ranks, selected indices,
normalization and association bit-exact against the oracle.
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


def corners(n2, m, seed):
    """Points near the unit simplex plus one point close to each vertex, so
    that the extreme points are distinct and the intercept system is
    regular (the elimination runs to the end instead of the fallback)."""
    rng = np.random.default_rng([seed, n2, m, 99])
    F = rng.dirichlet(np.ones(m), size=n2) * (1.0 + rng.exponential(0.05, size=(n2, 1)))
    k = min(m, n2)
    C = 0.02 * rng.random((k, m)) / m
    C[np.arange(k), np.arange(k)] = 0.9 + 0.05 * rng.random(k)
    F[rng.permutation(n2)[:k]] = C
    return F.astype(np.float32)


def _inputs(kind, n2, m, seed):
    return corners(n2, m, seed) if kind == "corners" else wl.objectives(kind, n2, m, seed=seed)


def _compare(orc, run, F, Z, seed, gen, history=None):
    st, rank, sel = run.select(F, gen=gen)
    assert st == 0, "device status %d" % st
    ref = orc.select(F, run.N, Z, seed=seed, gen=gen, history=history)
    info = run.info()
    assert info["l"] == ref["l"] and info["nFl"] == ref["nFl"]
    assert np.array_equal(rank, ref["rank"])
    if ref["niche"]:
        z, a, e = run.normalization()
        if history is None:
            zs, aa, ee, fb = orc.normalize(F, ref["rank"], ref["l"])
            assert np.array_equal(z, zs) and np.array_equal(e, ee)
            assert np.array_equal(a, aa)
            assert bool(info["fallback"]) == fb
        pi, dist = run.association()
        T = (ref["rank"] >= 0) & (ref["rank"] <= ref["l"])
        assert np.array_equal(pi[T], ref["pi"][T])
        assert np.array_equal(dist[T], ref["dist"][T])
    assert np.array_equal(sel, ref["selected"])
    return info, ref


# (m, N, p1, p2): warp-solved m <= 32 and grid-solved m > 32, up to 512
SHAPES = [(11, 120, 2, 0), (16, 200, 2, 1), (24, 160, 2, 0), (32, 300, 2, 0),
          (33, 200, 1, 1), (64, 300, 1, 1), (128, 200, 1, 0)]


@pytest.mark.parametrize("kind", ["early", "late", "uniform", "corners", "dups", "chain"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "m%d_N%d" % (s[0], s[1]))
def test_select_parity_many(n, orc, kind, shape):
    m, N, p1, p2 = shape
    Z = orc.refdirs(m, p1, p2, 0.5)
    with Run(n, m, m + 1, N, p1, p2=p2, seed=5) as r:
        for s in range(2):
            _compare(orc, r, _inputs(kind, 2 * N, m, s), Z, seed=5, gen=s + 1)


@pytest.mark.parametrize("kind", ["corners", "late", "uniform"])
def test_select_parity_m512(n, orc, kind):
    """m = 512, N = 600 (Table II's largest objective count)."""
    m, N = 512, 600
    Z = orc.refdirs(m, 1)
    with Run(n, m, m + 1, N, 1, seed=2) as r:
        info, ref = _compare(orc, r, _inputs(kind, 2 * N, m, 0), Z, seed=2, gen=7)
    if kind == "corners":
        assert ref["niche"] and info["fallback"] == 0  # the 512 x 512 system was eliminated


@pytest.mark.parametrize("m", [20, 64])
def test_corners_solve_without_fallback(n, orc, m):
    N = 4 * m
    Z = orc.refdirs(m, 1, 1, 0.5)
    with Run(n, m, m + 1, N, 1, p2=1, seed=1) as r:
        info, ref = _compare(orc, r, corners(2 * N, m, 3), Z, seed=1, gen=2)
    assert ref["niche"] and info["fallback"] == 0


@pytest.mark.parametrize("m", [20, 40])
def test_history_many(n, orc, m):
    """Normalization with history: warp solver (m = 20) and grid (m = 40)."""
    N = 3 * m
    Z = orc.refdirs(m, 1, 1, 0.5)
    h = orc.new_history(m)
    with Run(n, m, m + 1, N, 1, p2=1, seed=4, norm_history=1) as r:
        for g in range(5):
            kind = ("corners", "late", "early", "uniform", "corners")[g]
            F = (_inputs(kind, 2 * N, m, g) + np.float32(0.01 * g)).astype(np.float32)
            prev = {k: v.copy() for k, v in h.items()}
            info, ref = _compare(orc, r, F, Z, seed=4, gen=g + 1, history=h)
            if ref["niche"]:
                z, a, e = r.normalization()
                zz, aa, ee, fb = orc.normalize_hist(F, ref["rank"], ref["l"], prev)
                assert np.array_equal(z, zz) and np.array_equal(a, aa) and np.array_equal(e, ee)


def test_debug_recheck_many(n, orc):
    """Every point rechecked over all references in FP64: no miss."""
    m, N = 48, 200
    Z = orc.refdirs(m, 1, 1, 0.5)
    with Run(n, m, m + 1, N, 1, p2=1, seed=8, debug_recheck_all=1) as r:
        for kind in ("early", "corners"):
            info, _ = _compare(orc, r, _inputs(kind, 2 * N, m, 1), Z, seed=8, gen=3)
            assert info["recheck_miss"] == 0


@pytest.mark.parametrize("cfg", [wl.RunConfig("m16_N200_d40", m=16, d=40, N=200, p1=2),
                                 wl.RunConfig("m40_N240_d60", m=40, d=60, N=240, p1=1, p2=1)],
                         ids=lambda c: c.name)
def test_generations_many(n, orc, cfg):
    """nsga3_step: children's objectives match the oracle's evaluation and
    the next population is the oracle's selection, bit for bit; the launch
    count of a generation includes the extra normalization kernels."""
    W = wl.objective_weights(cfg.m, 2)
    Z = orc.refdirs(cfg.m, cfg.p1, cfg.p2, cfg.tau)
    with Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, p2=cfg.p2, seed=9, W=W) as r:
        r.check(n.nsga3_init(r.ctx, None))
        X, F, rank = r.population()
        np.testing.assert_allclose(F, orc.evaluate(X, W), rtol=1e-6, atol=0)
        for g in range(3):
            X, F, rank = r.population()
            r.check(n.nsga3_step(r.ctx, None))
            assert r.sync() == 0
            Xc, Fc = r.children()
            np.testing.assert_allclose(Fc, orc.evaluate(Xc, W), rtol=1e-6, atol=0)
            Xn, Fn, rn = r.population()
            RX, RF = np.vstack([X, Xc]), np.vstack([F, Fc])
            ref = orc.select(RF, cfg.N, Z, seed=9, gen=g)
            sel = ref["selected"]
            assert np.array_equal(Xn, RX[sel]) and np.array_equal(Fn, RF[sel])
            assert np.array_equal(rn, ref["rank"][sel])
        import ctypes as C
        import torch
        k = C.c_int32()
        r.check(n.nsga3_last_launches(r.ctx, C.byref(k)))
        # + ideal point, entry keys and their reduction, |f'|, candidate
        # distances; + the cooperative elimination (m > 32);
        # + the finishing kernel of a split dominance build (fewer tiles than
        # two per SM and more than one objective chunk)
        T = -(-2 * cfg.N // 256)
        split = T * (T + 1) // 2 < 2 * torch.cuda.get_device_properties(0).multi_processor_count \
            and cfg.m > 16
        # + the objective's dot-product kernel
        assert k.value == 21 + 5 + (1 if cfg.m > 32 else 0) + (1 if split else 0) + 1


@pytest.mark.parametrize("m,N", [(11, 2), (33, 2), (64, 6), (512, 4)])
def test_tiny_population_many_objectives(n, orc, m, N):
    """Fewer merged points than objectives (the extreme-point system is then
    singular and falls back to the nadir): same results as the oracle."""
    Z = orc.refdirs(m, 1)
    with Run(n, m, m + 1, N, 1, seed=6) as r:
        for s, kind in enumerate(("uniform", "early", "corners")):
            _compare(orc, r, _inputs(kind, 2 * N, m, s), Z, seed=6, gen=s + 1)
