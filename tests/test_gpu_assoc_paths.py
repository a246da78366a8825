"""GPU parity of the two association scans for more than 512 directions
(m <= 10): the tiled scan (every FP32 cosine, per-block candidate lists)
and the pruned scan (cone bounds per block of 32 directions).  Each is
chosen for the contexts a process creates by NSGA3_ASSOC=tile|scan; both
must give the oracle's association (pi, d) and selection bit for bit,
including points whose lists overflow to the FP64 scan (many directions at
the same distance) and points at the ideal point (|f'| = 0)."""
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


def _check(orc, r, F, Z, seed, gen):
    st, rank, sel = r.select(F, gen=gen)
    assert st == 0, "device status %d" % st
    ref = orc.select(F, r.N, Z, seed=seed, gen=gen)
    assert np.array_equal(rank, ref["rank"])
    info = r.info()
    if ref["niche"]:
        pi, dist = r.association()
        T = (ref["rank"] >= 0) & (ref["rank"] <= ref["l"])
        assert np.array_equal(pi[T], ref["pi"][T])
        assert np.array_equal(dist[T], ref["dist"][T])
    assert np.array_equal(sel, ref["selected"])
    return info, ref


# (m, N, p1, p2): w = 666, 715, 792, 1716, 715 and a two-layer set of 660
SHAPES = [(3, 700, 35, 0), (5, 800, 9, 0), (6, 900, 7, 0), (8, 1000, 6, 0), (10, 700, 4, 0),
          (4, 600, 14, 5)]


@pytest.mark.parametrize("path", ["tile", "scan"])
@pytest.mark.parametrize("shape", SHAPES)
def test_assoc_paths_parity(n, orc, monkeypatch, path, shape):
    m, N, p1, p2 = shape
    monkeypatch.setenv("NSGA3_ASSOC", path)
    Z = orc.refdirs(m, p1, p2, 0.5)
    assert len(Z) > 512
    with Run(n, m, m + 1, N, p1, p2=p2, seed=4) as r:
        for kind in wl.KINDS:
            F = wl.objectives(kind, 2 * N, m, seed=m + N)
            _check(orc, r, F, Z, seed=4, gen=3)


@pytest.mark.parametrize("debug", [0, 1])
@pytest.mark.parametrize("path", ["tile", "scan"])
def test_assoc_paths_near_ties(n, orc, monkeypatch, path, debug):
    """Points near the centroid direction, which is equidistant from 28
    directions (m = 8, p = 6: every direction with six ones and two zeros,
    spread over many blocks), and duplicated points.  With
    debug_recheck_all every point also takes the FP64 scan over all
    directions, which must find no other minimum."""
    m, N, p1 = 8, 600, 6
    monkeypatch.setenv("NSGA3_ASSOC", path)
    Z = orc.refdirs(m, p1)
    rng = np.random.default_rng(8)
    F = wl.objectives("simplex", 2 * N, m, seed=8).astype(np.float64)
    c = np.full(m, 1.0 / m)
    F[:60] = c + rng.normal(0.0, 1e-7, (60, m))
    F[:60] /= F[:60].sum(axis=1, keepdims=True)
    F[60:120] = F[120:180]
    F = F.astype(np.float32)
    with Run(n, m, m + 1, N, p1, seed=2, debug_recheck_all=debug) as r:
        info, ref = _check(orc, r, F, Z, seed=2, gen=1)
        if ref["niche"] and debug:
            assert info["recheck_miss"] == 0


def test_assoc_paths_scale_shape_agree(n, monkeypatch):
    """m = 5, 10,626 directions, N = 10,628 (late and early objectives): the
    two scans give the same ranks, selection and association."""
    cfg = wl.SCALE
    out = {}
    for path in ("tile", "scan"):
        monkeypatch.setenv("NSGA3_ASSOC", path)
        with Run(n, cfg.m, cfg.d, cfg.N, cfg.p1, seed=0) as r:
            res = []
            for kind in ("late", "early"):
                F = wl.objectives(kind, 2 * cfg.N, cfg.m, seed=3)
                st, rank, sel = r.select(F, gen=4)
                assert st == 0
                res.append((rank, sel) + r.association())
            out[path] = res
    for a, b in zip(out["tile"], out["scan"]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
