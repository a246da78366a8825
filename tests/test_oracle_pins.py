"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with a
published known answer, a closed form, an invariant of the definition, a
hand-written example or a different construction of the same quantity.
"""
import itertools
import math
import os

import numpy as np
import pytest

from paper_2504_06067_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ Philox --
def test_philox_known_answers(orc):
    """Published Philox4x32-10 known-answer vectors (Salmon et al., SC'11)."""
    for row in _read_golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = orc.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_priorities_are_distinct_streams(orc):
    # ref and member priorities come from different counters: same index,
    # different stream word -> (almost surely) different words.
    a = [orc.ref_priority(0, 3, j) for j in range(64)]
    b = [orc.member_priority(0, 3, j) for j in range(64)]
    assert a != b and len(set(a)) == 64


# ------------------------------------------------------------- Das-Dennis --
@pytest.mark.parametrize("m,p,w", [(3, 12, 91), (5, 20, 10626), (10, 3, 220), (10, 2, 55),
                                   (2, 7, 8), (4, 1, 4)])
def test_das_dennis_count_closed_form(orc, m, p, w):
    """w = C(p+m-1, m-1) (the lattice of compositions of p into m parts)."""
    assert orc.das_dennis_count(m, p) == w == math.comb(p + m - 1, m - 1)
    Z = orc.refdirs(m, p)
    assert Z.shape == (w, m)
    # every row on the unit simplex, entries multiples of 1/p, rows distinct
    assert np.allclose(Z.sum(1), 1.0, atol=1e-12)
    k = Z * p
    assert np.allclose(k, np.round(k), atol=1e-9)
    assert len({tuple(np.round(r).astype(int)) for r in k}) == w


def test_das_dennis_golden_m3_p2(orc):
    Z = orc.refdirs(3, 2)
    G = np.array([[float(x) for x in r] for r in _read_golden("das_dennis_m3_p2.txt")])
    assert np.array_equal(Z, G)


def test_das_dennis_two_layer(orc):
    """Two layers: 220 outer (p1=3) + 55 inner (p2=2) = 275 for m = 10;
    the inner layer is shrunk toward the centroid and still sums to 1."""
    Z = orc.refdirs(10, 3, 2, 0.5)
    assert Z.shape == (275, 10)
    assert np.allclose(Z.sum(1), 1.0, atol=1e-12)
    inner = Z[220:]
    assert inner.min() >= 0.05 - 1e-15  # (1 - tau)/m = 0.05
    # the vertices e_q are in the outer layer
    for q in range(10):
        e = np.zeros(10)
        e[q] = 1.0
        assert np.any(np.all(Z[:220] == e, axis=1))


# --------------------------------------------------------------- dominance --
def test_dominance_examples(orc):
    assert orc.dominates([1, 2], [2, 3])
    assert orc.dominates([1, 2], [1, 3])
    assert not orc.dominates([1, 2], [1, 2])          # equal: no dominance
    assert not orc.dominates([1, 3], [2, 2])          # incomparable
    assert not orc.dominates([2, 2], [1, 3])
    assert not orc.dominates([-0.0, 1.0], [0.0, 1.0])  # -0 == +0
    assert not orc.dominates([0.0, 1.0], [-0.0, 1.0])
    assert orc.dominates([-1.0, 0.0], [-0.0, 0.0])


def test_dominance_is_product_order_on_grid(orc):
    """On the integer grid {0,1,2}^m, a dominates b iff b - a is a nonzero
    vector of N^m (closed form of the Pareto order), checked exhaustively."""
    for m in (2, 3):
        pts = list(itertools.product(range(3), repeat=m))
        for a in pts:
            for b in pts:
                diff = [y - x for x, y in zip(a, b)]
                expect = all(t >= 0 for t in diff) and any(t > 0 for t in diff)
                assert orc.dominates(a, b) == expect


def test_dominance_strict_partial_order(orc):
    F = wl.objectives("grid", 40, 3, seed=1)
    D = np.array([[orc.dominates(F[i], F[j]) for j in range(40)] for i in range(40)])
    assert not D.diagonal().any()                 # irreflexive
    assert not (D & D.T).any()                    # antisymmetric
    D2 = (D.astype(int) @ D.astype(int)) > 0
    assert not (D2 & ~D).any()                    # transitive


# ---------------------------------------------------------------- sorting --
def _front_invariants(orc, F, rank, N, full):
    n2 = F.shape[0]
    l = rank.max()
    fronts = [np.flatnonzero(rank == k) for k in range(l + 1)]
    assert sum(len(f) for f in fronts) == (n2 if full else int((rank >= 0).sum()))
    for k, f in enumerate(fronts):
        assert len(f) > 0
        for i in f:              # mutually non-dominated
            for j in f:
                assert not orc.dominates(F[i], F[j])
        if k > 0:                # dominated by some member of the previous front
            for j in f:
                assert any(orc.dominates(F[i], F[j]) for i in fronts[k - 1])
        # no member of a later (or dropped) set dominates a member of front k
        later = np.flatnonzero((rank > k) | (rank < 0))
        for j in f:
            for i in later:
                assert not orc.dominates(F[i], F[j])
    if not full:
        cum = np.cumsum([len(f) for f in fronts])
        assert cum[-1] >= N and (l == 0 or cum[-2] < N)


@pytest.mark.parametrize("kind", wl.KINDS)
def test_nds_invariants(orc, kind):
    N = 30
    F = wl.objectives(kind, 2 * N, 3, seed=2)
    for full in (False, True):
        rank, l = orc.nds(F, N, full_sort=full)
        cum = np.cumsum(np.bincount(rank[rank >= 0]))
        assert l == int(np.argmax(cum >= N))
        if not full:
            assert l == rank.max()
        _front_invariants(orc, F, rank, N, full)


def test_nds_grid_closed_form(orc):
    """On the full grid {0..a}^m the front index of x is sum(x) (anti-diagonals)."""
    for m, a in ((2, 5), (3, 3)):
        pts = np.array(list(itertools.product(range(a + 1), repeat=m)), dtype=np.float32)
        n2 = len(pts) - len(pts) % 2
        pts = pts[:n2]
        rank, _ = orc.nds(pts, n2 // 2, full_sort=True)
        assert np.array_equal(rank, pts.sum(1).astype(int))


def test_nds_chain_and_equal(orc):
    F = wl.objectives("chain", 20, 4)
    rank, l = orc.nds(F, 10, full_sort=True)
    assert sorted(rank.tolist()) == list(range(20))
    rank, l = orc.nds(F, 10)
    assert l == 9 and (rank >= 0).sum() == 10
    F = wl.objectives("equal", 20, 4)
    rank, l = orc.nds(F, 10)
    assert l == 0 and (rank == 0).all()


# ---------------------------------------------------------- normalization --
def test_normalize_axis_extremes_closed_form(orc):
    """Extremes on the axes: z* = 0 and the hyperplane through A_q e_q has
    intercepts exactly A_q."""
    A = np.array([2.0, 3.0, 5.0, 0.5], dtype=np.float32)
    m = 4
    rng = np.random.default_rng(0)
    inner = rng.random((12, m)).astype(np.float32) * 0.1 + 0.05
    ext = np.diag(A)
    F = np.vstack([inner[:6], ext, inner[6:]]).astype(np.float32)
    n2 = F.shape[0]
    F = np.vstack([F, F[:(n2 % 2)]])  # even
    F[:, :] = np.where(F == 0.0, 0.0, F)
    # make the ideal exactly 0: zeros in every column come from the axis points
    rank = np.zeros(F.shape[0], dtype=np.int32)
    zstar, a, extremes, fb = orc.normalize(F, rank, 0)
    assert np.array_equal(zstar, np.zeros(m))
    assert not fb
    assert np.allclose(a, A.astype(np.float64), rtol=1e-12)
    for q in range(m):
        assert np.array_equal(F[extremes[q]], ext[q])


def test_normalize_extremes_on_hyperplane(orc):
    """When the solve succeeds, every extreme point lies on the normalised
    hyperplane: sum_r (f_er - z*_r) / a_r = 1."""
    for seed in range(5):
        F = wl.objectives("late", 200, 5, seed=seed)
        rank, l = orc.nds(F, 100)
        zstar, a, ext, fb = orc.normalize(F, rank, l)
        if fb:
            continue
        for q in range(5):
            s = np.sum((F[ext[q]].astype(np.float64) - zstar) / a)
            assert abs(s - 1.0) < 1e-9
        # ideal point is the column minimum over S u F_l
        T = (rank >= 0) & (rank <= l)
        assert np.array_equal(zstar, F[T].min(0).astype(np.float64))


def test_normalize_singular_fallback(orc):
    """All members identical in every column but one: the extreme matrix is
    singular; intercepts fall back to the maximum translated objective, and to
    1 where that maximum is 0."""
    m = 3
    F = np.zeros((8, m), dtype=np.float32)
    F[:, 0] = np.arange(8, dtype=np.float32)
    F[:, 1] = 2.0
    F[:, 2] = 7.0 - np.arange(8, dtype=np.float32)
    rank = np.zeros(8, dtype=np.int32)
    zstar, a, ext, fb = orc.normalize(F, rank, 0)
    assert fb
    assert np.array_equal(a, np.array([7.0, 1.0, 7.0]))


def _corner_points(n2, m, seed):
    """Points near the unit simplex and one near each vertex (distinct
    extremes, a regular intercept system)."""
    rng = np.random.default_rng([seed, n2, m, 99])
    F = rng.dirichlet(np.ones(m), size=n2) * (1.0 + rng.exponential(0.05, size=(n2, 1)))
    C = 0.02 * rng.random((m, m)) / m
    C[np.arange(m), np.arange(m)] = 0.9 + 0.05 * rng.random(m)
    F[rng.permutation(n2)[:m]] = C
    return F.astype(np.float32)


@pytest.mark.parametrize("m", [64, 200, 512])
def test_normalize_many_objectives_matches_lapack(orc, m):
    """Up to the m = 512 of Table II: the intercepts from the elimination
    equal 1 / (LAPACK's solution of (E - z*) b = 1) to rounding, the ideal is
    the column minimum and the m extremes are distinct."""
    F = _corner_points(2 * m + 100, m, 1)
    rank = np.zeros(len(F), dtype=np.int32)
    zstar, a, ext, fb = orc.normalize(F, rank, 0)
    assert not fb and len(set(ext.tolist())) == m
    assert np.array_equal(zstar, F.min(0).astype(np.float64))
    b = np.linalg.solve(F[ext].astype(np.float64) - zstar, np.ones(m))
    np.testing.assert_allclose(a, 1.0 / b, rtol=1e-12, atol=0)


# ------------------------------------------- normalization with history --
def test_normalize_hist_first_call_equals_stateless(orc):
    """Without history the running ideal over all 2N points equals the ideal
    over S u F_l (a minimum of every objective is attained by a non-dominated
    point), so the first call reproduces the stateless normalization."""
    for kind, seed in (("early", 1), ("late", 2), ("uniform", 3), ("grid", 4)):
        F = wl.objectives(kind, 200, 4, seed=seed)
        rank, l = orc.nds(F, 100)
        h = orc.new_history(4)
        z1, a1, e1, fb1 = orc.normalize_hist(F, rank, l, h)
        z0, a0, e0, fb0 = orc.normalize(F, rank, l)
        assert np.array_equal(z1, z0) and np.array_equal(a1, a0) and np.array_equal(e1, e0)
        assert fb1 == fb0 and h["valid"][0] == 1
        assert np.array_equal(h["z"], z0)
        assert np.array_equal(h["e"], F[e0])


def test_normalize_hist_keeps_ideal_and_axis_extremes(orc):
    """Generation 1 holds the three axis points (1 on one axis, 0 elsewhere):
    z* = 0 and E = I, so a = (1, 1, 1).  Generation 2 holds interior points
    only (every objective >= 0.1): the running ideal stays 0, the remembered
    axis points (ASF 1) beat every interior point (ASF >= 0.1 / 1e-6), so the
    extremes are the remembered vectors (indices 2N + q) and a = (1, 1, 1)
    again, where the stateless normalization would move both."""
    m = 3
    rng = np.random.default_rng(0)
    F1 = rng.dirichlet(np.ones(m), size=20).astype(np.float32)
    F1[:3] = np.eye(m, dtype=np.float32)
    rank1, l1 = orc.nds(F1, 10)
    h = orc.new_history(m)
    z, a, e, fb = orc.normalize_hist(F1, rank1, l1, h)
    assert np.array_equal(z, np.zeros(m)) and np.array_equal(a, np.ones(m)) and not fb
    F2 = (0.1 + 0.3 * rng.dirichlet(np.ones(m), size=20)).astype(np.float32)
    rank2, l2 = orc.nds(F2, 10)
    z2, a2, e2, fb2 = orc.normalize_hist(F2, rank2, l2, h)
    assert np.array_equal(z2, np.zeros(m))
    assert np.array_equal(e2, 20 + np.arange(m)) and np.array_equal(a2, np.ones(m)) and not fb2
    zs, as_, es, _ = orc.normalize(F2, rank2, l2)
    assert np.all(zs >= 0.1) and np.all(es < 20)


def test_normalize_hist_ideal_is_a_running_minimum(orc):
    m = 4
    h = orc.new_history(m)
    running = np.full(m, np.inf)
    for g in range(4):
        F = wl.objectives("early", 100, m, seed=10 + g) + np.float32(g * 0.05)
        rank, l = orc.nds(F, 50)
        z, a, e, fb = orc.normalize_hist(F, rank, l, h)
        running = np.minimum(running, F.astype(np.float64).min(axis=0))
        assert np.array_equal(z, running + 0.0)


def test_select_hist_without_niching_leaves_history(orc):
    """A selection whose fronts fill N exactly computes no normalization."""
    m, N = 3, 4
    F = np.array([[0, 3, 3], [3, 0, 3], [3, 3, 0], [1, 1, 1],
                  [5, 5, 5], [6, 6, 6], [7, 7, 7], [8, 8, 8]], dtype=np.float32)
    Z = orc.refdirs(m, 2)
    h = orc.new_history(m)
    r = orc.select(F, N, Z, seed=0, gen=0, history=h)
    assert r["niche"] == 0 and h["valid"][0] == 0


# ------------------------------------------------------------ association --
def test_associate_point_on_direction(orc):
    """A point on direction j (after normalisation) has d = 0 and pi = j."""
    Z = orc.refdirs(3, 4)
    m = 3
    zstar = np.zeros(m)
    a = np.ones(m)
    # choose interior directions (no ties with others along the ray)
    js = [4, 7, 11]
    F = np.array([Z[j] * s for j, s in zip(js, (0.5, 1.0, 3.0))] + [Z[0]], dtype=np.float32)
    rank = np.zeros(4, dtype=np.int32)
    pi, dist = orc.associate(F, rank, 0, zstar, a, Z)
    assert pi[:3].tolist() == js
    assert np.all(dist[:3] < 1e-7)


def test_associate_matches_vector_rejection(orc):
    """Eq. 2 with cos^2 equals the length of the rejection of f' from the
    direction (a different construction of the perpendicular distance)."""
    m = 4
    Z = orc.refdirs(m, 5)
    F = wl.objectives("late", 300, m, seed=3)
    rank, l = orc.nds(F, 150)
    zstar, a, _, _ = orc.normalize(F, rank, l)
    pi, dist = orc.associate(F, rank, l, zstar, a, Z)
    T = np.flatnonzero((rank >= 0) & (rank <= l))
    Zh = Z / np.linalg.norm(Z, axis=1, keepdims=True)
    for i in T:
        fp = (F[i].astype(np.float64) - zstar) / a
        proj = fp @ Zh.T
        rej = np.linalg.norm(fp[None, :] - proj[:, None] * Zh, axis=1)
        j = int(np.argmin(rej))
        srt = np.sort(rej)
        if srt[1] - srt[0] > 1e-9:
            assert pi[i] == j
        assert abs(dist[i] - rej[pi[i]]) < 1e-9 * max(1.0, np.linalg.norm(fp))
    assert np.all(pi[rank < 0] == -1)


def test_associate_many_objectives_vector_rejection(orc):
    """m = 100: the association equals the nearest direction by the length
    of the rejection of f' (computed with numpy)."""
    m = 100
    Z = orc.refdirs(m, 1, 1, 0.5)
    F = _corner_points(300, m, 2)
    rank = np.zeros(300, dtype=np.int32)
    zstar, a, _, _ = orc.normalize(F, rank, 0)
    pi, dist = orc.associate(F, rank, 0, zstar, a, Z)
    Zh = Z / np.linalg.norm(Z, axis=1, keepdims=True)
    fp = (F.astype(np.float64) - zstar) / a
    proj = fp @ Zh.T
    rej = np.sqrt(np.maximum(0.0, np.sum(fp * fp, 1)[:, None] - proj * proj))
    for i in range(len(F)):
        srt = np.sort(rej[i])
        if srt[1] - srt[0] > 1e-9:
            assert pi[i] == int(np.argmin(rej[i]))
        assert abs(dist[i] - rej[i, pi[i]]) < 1e-9 * max(1.0, np.linalg.norm(fp[i]))


def test_nds_many_objectives_invariants(orc):
    """m = 300: fronts are antichains and every member of a later front is
    dominated by some member of the front before."""
    N = 40
    for kind in ("early", "chain"):
        F = wl.objectives(kind, 2 * N, 300, seed=5)
        rank, l = orc.nds(F, N, full_sort=True)
        _front_invariants(orc, F, rank, N, True)


def test_associate_2d_angle(orc):
    """m = 2: perpendicular distance = |f'| |sin(theta_f - theta_z)|."""
    Z = orc.refdirs(2, 9)
    F = wl.objectives("uniform", 60, 2, seed=4)
    rank = np.zeros(60, dtype=np.int32)
    zstar = F.min(0).astype(np.float64)
    a = (F.max(0).astype(np.float64) - zstar)
    pi, dist = orc.associate(F, rank, 0, zstar, a, Z)
    for i in range(60):
        fp = (F[i].astype(np.float64) - zstar) / a
        r = np.hypot(*fp)
        th = math.atan2(fp[1], fp[0])
        d = [r * abs(math.sin(th - math.atan2(z[1], z[0]))) for z in Z]
        assert abs(dist[i] - min(d)) < 1e-12 * max(1.0, r)


# ------------------------------------------------------------------ niching --
def _niche_case(orc, kind, N, m, p, seed):
    F = wl.objectives(kind, 2 * N, m, seed=seed)
    Z = orc.refdirs(m, p)
    rank, l = orc.nds(F, N)
    nS = int(((rank >= 0) & (rank < l)).sum())
    nFl = int((rank == l).sum())
    K = N - nS
    zstar, a, _, _ = orc.normalize(F, rank, l)
    pi, dist = orc.associate(F, rank, l, zstar, a, Z)
    return F, Z, rank, l, K, nFl, pi, dist


@pytest.mark.parametrize("kind", ["early", "late", "uniform", "simplex", "dups", "grid"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_niche_alg1_equals_alg2(orc, kind, seed):
    """The Alg. 1 while-loop and the Alg. 2 cached batched loop (with the
    last batch truncated in shuffled-reference order) pick identical sets."""
    # (30, 3, 12): more directions (91) than N, so the first batch (the
    # references without a member in S) is itself truncated
    for N, m, p in ((40, 3, 6), (64, 5, 3), (30, 4, 4), (30, 3, 12)):
        F, Z, rank, l, K, nFl, pi, dist = _niche_case(orc, kind, N, m, p, seed)
        if K == nFl:
            continue
        for gen in (0, 5):
            a = orc.niche(rank, l, K, pi, dist, Z.shape[0], seed, gen, 0)
            b = orc.niche(rank, l, K, pi, dist, Z.shape[0], seed, gen, 1)
            assert a.sum() == K
            assert np.array_equal(a, b)


def test_niche_water_filling_and_nearest(orc):
    """Properties of the loop: (1) final niche levels are filled evenly --
    every reference with members left over ends with a count no lower than
    the last count taken from any reference; (2) a reference with no member
    in S that receives a pick receives its nearest member first."""
    for seed in range(6):
        F, Z, rank, l, K, nFl, pi, dist = _niche_case(orc, "early", 60, 3, 8, seed)
        if K == nFl:
            continue
        w = Z.shape[0]
        picked = orc.niche(rank, l, K, pi, dist, w, seed, 1, 0)
        rho = np.bincount(pi[(rank >= 0) & (rank < l)], minlength=w)
        rhop = np.bincount(pi[rank == l], minlength=w)
        took = np.bincount(pi[picked], minlength=w)
        final = rho + took
        top_taken = max(final[j] - 1 for j in range(w) if took[j] > 0)
        left = [final[j] for j in range(w) if rhop[j] > took[j]]
        assert all(v >= top_taken for v in left)
        for j in range(w):
            if rho[j] == 0 and took[j] > 0:
                mem = np.flatnonzero((rank == l) & (pi == j))
                nearest = mem[np.argmin(dist[mem])]
                assert picked[nearest]


def test_niche_single_ref_nearest(orc):
    """Hand example: one reference, no member in S, two F_l members, K = 1:
    the nearest one is taken whatever the priorities."""
    rank = np.array([0, 0], dtype=np.int32)
    pi = np.array([0, 0], dtype=np.int32)
    for dist in ([0.3, 0.1], [0.1, 0.3]):
        d = np.array(dist)
        for variant in (0, 1):
            picked = orc.niche(rank, 0, 1, pi, d, 1, 0, 0, variant)
            assert picked.tolist() == [d[0] < d[1], d[1] < d[0]]


# ------------------------------------------------------------------ select --
@pytest.mark.parametrize("kind", wl.KINDS)
def test_select_invariants(orc, kind):
    N, m = 48, 4
    F = wl.objectives(kind, 2 * N, m, seed=7)
    Z = orc.refdirs(m, 5)
    r = orc.select(F, N, Z, seed=3, gen=2)
    sel = r["selected"]
    assert len(sel) == N and np.all(np.diff(sel) > 0)
    rank, l = r["rank"], r["l"]
    S = np.flatnonzero((rank >= 0) & (rank < l))
    assert set(S) <= set(sel)
    assert set(sel) <= set(np.flatnonzero((rank >= 0) & (rank <= l)))
    r1 = orc.select(F, N, Z, seed=3, gen=2, variant=1)
    assert np.array_equal(r1["selected"], sel)


# --------------------------------------------------------------- variation --
def test_sbx_conserves_parent_mean(orc):
    """SBX children average to the parents' average (c1 + c2 = x1 + x2) when
    no clipping and no mutation happen; with eta -> inf children = parents."""
    N, d = 64, 10
    X = (wl.population(N, d, seed=1) * 0.2 + 0.4).astype(np.float32)
    rank = np.zeros(N, dtype=np.int32)
    C = orc.vary(X, rank, seed=5, gen=0, eta_c=20.0, p_m=0.0)
    # ranks equal -> tournament keeps the first drawn index; recover parents
    for q in range(N // 2):
        c1, c2 = C[2 * q].astype(np.float64), C[2 * q + 1].astype(np.float64)
        # each variable: either copied or crossed; in both cases sums match
        s = c1 + c2
        # parents are rows of X: find a pair whose sums match
        found = False
        for a_ in range(N):
            for b_ in range(N):
                if np.allclose(X[a_].astype(np.float64) + X[b_], s, atol=2e-7):
                    found = True
                    break
            if found:
                break
        assert found
    C2 = orc.vary(X, rank, seed=5, gen=0, eta_c=1e9, p_m=0.0)
    assert np.all(np.isin(C2.round(5), X.round(5)))


def test_variation_bounds_and_identity(orc):
    N, d = 50, 13
    X = wl.population(N, d, seed=2)
    rank = wl.parent_ranks(N, 3)
    C = orc.vary(X, rank, seed=1, gen=4)
    assert C.min() >= 0.0 and C.max() <= 1.0
    # p_c = 0 and p_m = 0: children are copies of tournament winners
    C0 = orc.vary(X, rank, seed=1, gen=4, p_c=0.0, p_m=0.0)
    rows = {tuple(r) for r in X}
    assert all(tuple(r) in rows for r in C0)
    # the tournament prefers the lower front: the winners' mean rank is lower
    idx = [next(i for i in range(N) if np.array_equal(X[i], r)) for r in C0]
    assert rank[idx].mean() < rank.mean()


def test_mutation_changes_about_pm_fraction(orc):
    N, d = 400, 50
    X = wl.population(N, d, seed=3)
    rank = np.zeros(N, dtype=np.int32)
    C0 = orc.vary(X, rank, seed=2, gen=0, p_m=0.0)
    C1 = orc.vary(X, rank, seed=2, gen=0, p_m=0.1)
    frac = np.mean(C0 != C1)
    assert 0.08 < frac < 0.12


# --------------------------------------------------------------- objective --
def test_objective_front_sums_to_one(orc):
    """g = 0 (x_v = 0.5 for v >= m-1): sum_j f_j = 1 (the closed-form front)."""
    m, d = 5, 20
    W = wl.objective_weights(m, 0)
    X = wl.population(100, d, seed=4)
    X[:, m - 1:] = 0.5
    F = orc.evaluate(X, W)
    assert np.allclose(F.astype(np.float64).sum(1), 1.0, atol=1e-6)
    # W = 0: every objective equals (1 + g) / m
    X2 = wl.population(10, d, seed=5)
    F2 = orc.evaluate(X2, np.zeros_like(W))
    g = ((X2[:, m - 1:].astype(np.float64) - 0.5) ** 2).sum(1)
    assert np.allclose(F2, ((1 + g) / m)[:, None], rtol=1e-6)


def test_init_uniform(orc):
    X = orc.init_population(200, 30, seed=9)
    assert X.min() >= 0 and X.max() < 1
    assert abs(X.mean() - 0.5) < 0.01
    assert not np.array_equal(X, orc.init_population(200, 30, seed=10))


# --------------------------------------------------------------------- IGD --
def test_igd_closed_forms(orc):
    R = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert orc.igd(R.astype(np.float32), R) == 0.0
    P = np.array([[0.0, 0.0]], dtype=np.float32)
    assert abs(orc.igd(P, R) - 1.0) < 1e-15
    P = np.array([[0.0, 1.0], [3.0, 4.0]], dtype=np.float32)
    assert abs(orc.igd(P, R) - (0.0 + math.sqrt(2.0)) / 2) < 1e-15


# -------------------------------------------------------------- full runs --
def test_small_run_approaches_closed_form_front(orc):
    """m = 3, N = 92, p = 12, d = 12: after 100 generations the rank-0 set
    sits near the closed-form front (sum f = 1) and its IGD to a sample of
    the true front is small."""
    cfg = wl.SMALL
    W = wl.objective_weights(cfg.m, cfg.seed)
    Z = orc.refdirs(cfg.m, cfg.p1)
    X, F, rank = orc.run(cfg.N, cfg.d, W, Z, cfg.seed, 100)
    P = F[rank == 0].astype(np.float64)
    assert np.mean(np.abs(P.sum(1) - 1.0)) < 0.05
    y = wl.front_sample(cfg.m, 2000)
    Xf = np.full((len(y), cfg.d), 0.5, dtype=np.float32)
    Xf[:, :cfg.m - 1] = y
    R = orc.evaluate(Xf, W).astype(np.float64)
    igd_end = orc.igd(F[rank == 0], R)
    X0 = orc.init_population(cfg.N, cfg.d, cfg.seed)
    igd_start = orc.igd(orc.evaluate(X0, W), R)
    assert igd_end < 0.1 * igd_start


# ------------------------------------------------------ 0-1 knapsack -------
def test_kp_repair_hand_example(orc):
    """Two knapsacks, four items.  Best ratios: item 0 max(10/5, 1/1) = 2,
    item 1 max(1/10, 2/10) = 0.2, item 2 max(6/6, 6/2) = 3, item 3
    max(4/8, 5/5) = 1, so items leave in the order 1, 3, 0, 2.  With every
    item chosen the loads (29, 18) exceed the capacities (15, 12): item 1
    leaves (19, 8), still over in knapsack 0; item 3 leaves (11, 3): done."""
    profit = np.array([[10, 1, 6, 4], [1, 2, 6, 5]], dtype=np.int32)
    weight = np.array([[5, 10, 6, 8], [1, 10, 2, 5]], dtype=np.int32)
    cap = np.array([15, 12], dtype=np.int32)
    assert np.array_equal(orc.kp_order(profit, weight), [1, 3, 0, 2])
    X, F = orc.kp_eval(np.ones((1, 4), dtype=np.float32), profit, weight, cap)
    assert np.array_equal(X[0], [1, 0, 1, 0])
    # f_j = P_j - profit kept: P = (21, 14), kept (16, 7)
    assert np.array_equal(F[0], [5, 7])


def test_kp_repair_is_feasible_and_minimal(orc):
    profit, weight, cap = wl.knapsack_instance(4, 60, seed=1)
    order = orc.kp_order(profit, weight)
    X0 = orc.kp_init(40, 60, seed=2)
    X, F = orc.kp_eval(X0, profit, weight, cap, order)
    W = weight.astype(np.int64)
    for x0, x in zip(X0, X):
        assert np.all(W @ x.astype(np.int64) <= cap)               # feasible
        removed = np.flatnonzero(x0 != x)
        assert np.all(x0[removed] == 1)                             # only removals
        if len(removed):
            pos = {int(v): k for k, v in enumerate(order)}
            last = max(pos[int(v)] for v in removed)
            # every chosen item before the last removed one in the order left
            assert all(x[order[k]] == 0 for k in range(last + 1))
            back = x.copy()
            back[order[last]] = 1                                    # minimal prefix
            assert np.any(W @ back.astype(np.int64) > cap)
    # objectives: total profit minus profit kept (exact integers)
    assert np.array_equal(F, (profit.sum(1)[None, :] - X.astype(np.int64) @ profit.T).astype(np.float32))


def test_kp_uniform_crossover_conserves_bits(orc):
    N, d = 40, 64
    X = orc.kp_init(N, d, seed=3)
    rank = np.zeros(N, dtype=np.int32)
    Xc = orc.kp_vary(X, rank, seed=4, gen=0, p_m=0.0)
    # without mutation every child pair carries, item by item, the bits of
    # two parents: the pair's column sums are 0, 1 or 2 and appear in X
    s = Xc[0::2] + Xc[1::2]
    assert set(np.unique(s).tolist()) <= {0.0, 1.0, 2.0}
    assert np.array_equal(np.unique(Xc), [0.0, 1.0])


def test_kp_bit_flip_rate(orc):
    N, d = 200, 100
    X = np.zeros((N, d), dtype=np.float32)
    rank = np.zeros(N, dtype=np.int32)
    Xc = orc.kp_vary(X, rank, seed=5, gen=1, p_c=0.0)
    rate = Xc.mean()
    assert abs(rate - 1.0 / d) < 0.3 / d


def test_hv_closed_forms(orc):
    assert orc.hv([[1, 2]], [4, 5]) == 3 * 3
    # staircase: two boxes minus the overlap
    assert orc.hv([[1, 3], [2, 1]], [4, 5]) == 3 * 2 + 2 * 4 - 2 * 2
    assert orc.hv([[5, 1]], [4, 5]) == 0.0          # outside the box
    assert orc.hv([[1, 2, 3]], [2, 4, 7]) == 1 * 2 * 4
    # two 3-D boxes: inclusion-exclusion
    a, b, r = np.array([0, 2, 1.0]), np.array([2, 0, 3.0]), np.array([4, 4, 4.0])
    inter = np.prod(r - np.maximum(a, b))
    assert abs(orc.hv([a, b], r) - (np.prod(r - a) + np.prod(r - b) - inter)) < 1e-12


def test_normalized_hv_app_e(orc):
    """App. E: ref = 1.01 f_max, ideal = 0.9 f_min; a single point at the
    ideal-side corner f_min gives prod(1.01 f_max - f_min) / prod(1.01 f_max - 0.9 f_min)."""
    fmin, fmax = np.array([2.0, 4.0]), np.array([10.0, 20.0])
    v = orc.normalized_hv([fmin], fmin, fmax)
    expect = np.prod(1.01 * fmax - fmin) / np.prod(1.01 * fmax - 0.9 * fmin)
    assert abs(v - expect) < 1e-12 and 0 < v < 1


# -------------------------------------- pins that planted mistakes need --
# Each of these closes a gap that a planted mistake in the oracle
# (tests/test_oracle_mutants.py) slipped through.

@pytest.mark.parametrize("seed", [0, 1])
def test_normalize_with_row_exchanges_matches_lapack(orc, seed):
    """Members spread over the inside of the simplex (m = 12, Dirichlet(2))
    give extreme vectors whose matrix is not diagonally dominant, so partial
    pivoting exchanges rows (LAPACK's LU permutation is not the identity);
    the intercepts still equal 1 / LAPACK's solution of (E - z*) b = 1."""
    sl = pytest.importorskip("scipy.linalg")
    m = 12
    rng = np.random.default_rng([m, seed])
    F = rng.dirichlet(np.full(m, 2.0), size=300).astype(np.float32)
    rank = np.zeros(len(F), dtype=np.int32)
    zstar, a, ext, fb = orc.normalize(F, rank, 0)
    E = F[ext].astype(np.float64) - zstar
    P, _, _ = sl.lu(E)
    assert not np.array_equal(P, np.eye(m))  # the system needs row exchanges
    assert not fb and len(set(ext.tolist())) == m
    np.testing.assert_allclose(a, 1.0 / np.linalg.solve(E, np.ones(m)), rtol=1e-9, atol=0)


def test_sbx_spread_factor_distribution(orc):
    """SBX's spread factor beta = |c1 - c2| / |x1 - x2| has the published
    density (Deb and Agrawal, 1995) 0.5 (eta+1) beta^eta on [0, 1] and
    0.5 (eta+1) beta^-(eta+2) above 1, i.e. the distribution function
    beta^(eta+1) / 2 below 1 and 1 - beta^-(eta+1) / 2 above.  Two parents
    0.45 and 0.55 in every variable (children clip only for beta > 10);
    crossed variables of the pairs whose parents differ; Kolmogorov-Smirnov
    distance against that law."""
    eta, d = 2.0, 400
    X = np.empty((2, d), dtype=np.float32)
    X[0], X[1] = 0.45, 0.55
    rank = np.zeros(2, dtype=np.int32)
    gap = float(X[1, 0]) - float(X[0, 0])
    betas = []
    for gen in range(80):
        C = orc.vary(X, rank, seed=11, gen=gen, eta_c=eta, p_m=0.0).astype(np.float64)
        diff = np.abs(C[0] - C[1])
        if not diff.any():
            continue  # both parents are the same individual
        crossed = diff != gap
        inside = (C[0] > 0) & (C[0] < 1) & (C[1] > 0) & (C[1] < 1)
        betas.append(diff[crossed & inside] / gap)
    beta = np.sort(np.concatenate(betas))
    n = len(beta)
    assert n > 4000
    law = np.where(beta <= 1.0, 0.5 * beta ** (eta + 1), 1.0 - 0.5 * beta ** -(eta + 1))
    ecdf_hi = np.arange(1, n + 1) / n
    ks = max(np.max(ecdf_hi - law), np.max(law - (ecdf_hi - 1.0 / n)))
    assert ks < 1.95 / math.sqrt(n)  # the 0.1 % critical value


def test_polynomial_mutation_symmetric_at_centre(orc):
    """Bounded polynomial mutation of y = 0.5 on [0, 1]: the two branches
    mirror each other (the distances to both bounds are equal), so the
    mutated values rise as often as they fall, by the same amounts in law,
    and stay inside [0, 1]."""
    N, d = 200, 100
    X = np.full((N, d), 0.5, dtype=np.float32)
    rank = np.zeros(N, dtype=np.int32)
    C = orc.vary(X, rank, seed=4, gen=1, p_c=0.0, p_m=0.3).astype(np.float64)
    dlt = (C - 0.5)[C != 0.5]
    assert len(dlt) > 0.25 * N * d and C.min() >= 0.0 and C.max() <= 1.0
    assert abs(np.mean(dlt > 0) - 0.5) < 0.03
    up, down = np.sort(dlt[dlt > 0]), np.sort(-dlt[dlt < 0])
    # two-sample Kolmogorov-Smirnov distance between rises and falls
    grid = np.concatenate([up, down])
    ks = np.max(np.abs(np.searchsorted(up, grid, side="right") / len(up)
                       - np.searchsorted(down, grid, side="right") / len(down)))
    assert ks < 1.95 * math.sqrt(1.0 / len(up) + 1.0 / len(down))


def test_tournament_winner_distribution(orc):
    """Binary tournament on two uniform draws: with half the parents in
    front 0 and half in front 1 a winner is in front 0 with probability
    1 - (1/2)^2 = 3/4, for the first and for the second parent of a pair;
    with one front every parent is equally likely to win.  Without
    crossover and mutation the children are copies of the winners."""
    N, d = 400, 3
    X = np.tile(((np.arange(N) + 0.5) / N)[:, None], (1, d)).astype(np.float32)
    rng = np.random.default_rng(5)
    two = rng.permutation(np.repeat([0, 1], N // 2)).astype(np.int32)
    one = np.zeros(N, dtype=np.int32)
    front0 = [0, 0]
    upper = 0
    for gen in range(10):
        C = orc.vary(X, two, seed=21, gen=gen, p_c=0.0, p_m=0.0)
        idx = np.rint(C[:, 0].astype(np.float64) * N - 0.5).astype(int)
        assert np.array_equal(C, X[idx])
        for h in (0, 1):
            front0[h] += int(np.sum(two[idx[h::2]] == 0))
        C = orc.vary(X, one, seed=22, gen=gen, p_c=0.0, p_m=0.0)
        idx = np.rint(C[:, 0].astype(np.float64) * N - 0.5).astype(int)
        upper += int(np.sum(idx >= N // 2))
    for h in (0, 1):
        assert abs(front0[h] / (10 * N // 2) - 0.75) < 0.04
    assert abs(upper / (10 * N) - 0.5) < 0.04


def test_objective_hand_example(orc):
    """m = 3, k = 2 with W's rows e_0, e_1 and 0: W x[:2] = (x_0, x_1, 0), so
    f = (1 + g) (e^x0, e^x1, 1) / (e^x0 + e^x1 + 1) with g the squared
    distance of x[2:] to 0.5."""
    W = np.array([[1, 0], [0, 1], [0, 0]], dtype=np.float32)
    X = np.array([[0.25, 0.75, 0.5, 0.5, 0.5],
                  [1.0, 0.0, 0.0, 0.5, 1.0]], dtype=np.float32)
    F = orc.evaluate(X, W).astype(np.float64)
    g = np.array([0.0, 0.25 + 0.25])
    for x, f, gi in zip(X.astype(np.float64), F, g):
        e = np.array([math.exp(x[0]), math.exp(x[1]), 1.0])
        np.testing.assert_allclose(f, (1.0 + gi) * e / e.sum(), rtol=1e-6, atol=0)


def test_kp_repair_keeps_an_exact_fit(orc):
    """The hand example's four items with capacities equal to their full
    loads (29, 18): every knapsack is exactly full, which is feasible, so
    the repair removes nothing and nothing is left over."""
    profit = np.array([[10, 1, 6, 4], [1, 2, 6, 5]], dtype=np.int32)
    weight = np.array([[5, 10, 6, 8], [1, 10, 2, 5]], dtype=np.int32)
    X, F = orc.kp_eval(np.ones((1, 4), dtype=np.float32), profit, weight,
                       np.array([29, 18], dtype=np.int32))
    assert np.array_equal(X[0], [1, 1, 1, 1]) and np.array_equal(F[0], [0, 0])


def test_kp_bit_flip_flips_ones_and_zeros(orc):
    """Bit-flip mutation changes a one as often as a zero: all-zero and
    all-one populations both change in about a p_m fraction of their bits."""
    N, d, pm = 200, 100, 0.1
    rank = np.zeros(N, dtype=np.int32)
    for v in (0.0, 1.0):
        X = np.full((N, d), v, dtype=np.float32)
        C = orc.kp_vary(X, rank, seed=3, gen=1, p_c=0.0, p_m=pm)
        assert abs(np.mean(C != X) - pm) < 0.01


def test_associate_ties_go_to_the_first_direction(orc):
    """A point on the bisector of two directions is equally far from both
    (the two distances are the same rounded operations); pi takes the first
    of the minimal distances, in either order of the directions."""
    F = np.array([[1.0, 1.0], [2.0, 2.0]], dtype=np.float32)
    rank = np.zeros(2, dtype=np.int32)
    for Z in (np.array([[1.0, 0.0], [0.0, 1.0]]), np.array([[0.0, 1.0], [1.0, 0.0]])):
        pi, dist = orc.associate(F, rank, 0, np.zeros(2), np.ones(2), Z)
        assert pi.tolist() == [0, 0]
        np.testing.assert_allclose(dist, [1.0, 2.0], rtol=1e-15)


def test_polynomial_mutation_bounded_form_stays_inside(orc):
    """The bounded polynomial mutation scales its perturbation to the
    distances from y to the bounds, so from y = 0.1 or 0.9 a mutated value
    reaches 0 or 1 only for u = 0 exactly: none lands on a bound."""
    N, d = 200, 100
    rank = np.zeros(N, dtype=np.int32)
    for y in (0.1, 0.9):
        X = np.full((N, d), y, dtype=np.float32)
        C = orc.vary(X, rank, seed=6, gen=2, p_c=0.0, p_m=0.5)
        moved = C[C != X]
        assert len(moved) > 0.4 * N * d
        assert moved.min() > 0.0 and moved.max() < 1.0


def test_kp_uniform_crossover_mixes_parents(orc):
    """Uniform crossover takes each item from either parent with
    probability 1/2: from an all-ones and an all-zeros parent, a pair with
    different parents gets complementary children with about half their
    bits set."""
    d = 400
    X = np.zeros((2, d), dtype=np.float32)
    X[0] = 1.0
    rank = np.zeros(2, dtype=np.int32)
    mixed = 0
    for gen in range(40):
        C = orc.kp_vary(X, rank, seed=7, gen=gen, p_c=1.0, p_m=0.0)
        if np.all(C[0] + C[1] == 1.0):
            mixed += 1
            assert abs(C[0].mean() - 0.5) < 0.1
        else:
            assert np.array_equal(C[0], C[1])  # both children of one parent
    assert mixed >= 10


def test_kp_init_fair_bits(orc):
    """Initial knapsack bits are fair coins."""
    X = orc.kp_init(200, 100, seed=8)
    assert set(np.unique(X).tolist()) <= {0.0, 1.0}
    assert abs(X.mean() - 0.5) < 0.01


def _closed_form_niche(orc, rank, l, K, pi, dist, w, seed, gen):
    """The closed form of the niching loop, written from its definition: a
    reference j with rho_j members in S orders its F_l members (the nearest
    first, ties to the lower index, when rho_j = 0; the rest by member
    priority, then index); the member at position t has level rho_j + t;
    L* is the K-th smallest level; every member below L* is taken and, at
    L*, the members of the references of smallest (priority, j)."""
    S = (rank >= 0) & (rank < l)
    rho = np.bincount(pi[S], minlength=w)
    Fl = np.flatnonzero(rank == l)
    mp = {int(i): orc.member_priority(seed, gen, int(i)) for i in Fl}
    levels = []
    for j in range(w):
        mem = [int(i) for i in Fl if pi[i] == j]
        order = sorted(mem, key=lambda i: (mp[i], i))
        if rho[j] == 0 and mem:
            near = min(mem, key=lambda i: (dist[i], i))
            order = [near] + [i for i in order if i != near]
        levels += [(int(rho[j]) + t, j, i) for t, i in enumerate(order)]
    Lstar = sorted(L for L, _, _ in levels)[K - 1]
    taken = [i for L, _, i in levels if L < Lstar]
    at = sorted((orc.ref_priority(seed, gen, j), j, i) for L, j, i in levels if L == Lstar)
    taken += [i for _, _, i in at[:K - len(taken)]]
    picked = np.zeros(len(rank), dtype=bool)
    picked[taken] = True
    return picked


@pytest.mark.parametrize("case", range(60))
def test_niche_closed_form_equals_the_loops(orc, case):
    """Random niching problems (few references, tied distances, S members
    stacked on some references, every K from 1 to |F_l|): the closed form
    of the batched loop that the kernels compute picks the same set as the
    literal Alg. 1 loop and the Alg. 2 cached loop."""
    rng = np.random.default_rng([case, 77])
    n2 = int(rng.integers(6, 70))
    w = int(rng.integers(1, 14))
    l = int(rng.integers(0, 4))
    rank = rng.integers(0, l + 2, size=n2).astype(np.int32)
    rank[rng.random(n2) < 0.1] = -1
    rank[int(rng.integers(n2))] = l  # F_l is never empty
    pi = rng.integers(0, max(1, w // 2) if case % 3 == 0 else w, size=n2).astype(np.int32)
    dist = rng.integers(0, 4, size=n2) * 0.25
    nFl = int((rank == l).sum())
    seed, gen = int(rng.integers(1 << 30)), int(rng.integers(100))
    for K in sorted({1, nFl, int(rng.integers(1, nFl + 1))}):
        want = _closed_form_niche(orc, rank, l, K, pi, dist, w, seed, gen)
        assert want.sum() == K
        for variant in (0, 1):
            assert np.array_equal(orc.niche(rank, l, K, pi, dist, w, seed, gen, variant), want)
