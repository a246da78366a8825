"""nsga3_rank_noalloc (workspace in a static device array, no allocation)
against the context-based entry point and the oracle: the front index of
every point from nsga3_rank_noalloc equals the ranks nsga3_select returns
with full_sort = 1 and the oracle's non-dominated sort (Alg. 1), over two
calls in a row that share the static workspace.

Collected last on purpose: it must pass both alone in a fresh process and
after every other GPU test has run in the same process."""
import numpy as np
import pytest

from paper_2504_06067_gb300 import workloads as wl

from gpu_util import Run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_2504_06067_gb300 import native
    return torch, native


def _select_ranks(native, F):
    """Front index of every row from the context-based nsga3_select."""
    n2, m = F.shape
    with Run(native, m, m, n2 // 2, 4, full_sort=1) as r:
        st, rank, _ = r.select(F)
        assert st == 0
    return rank


def _noalloc_ranks(torch, native, F, poison=True):
    n, m = F.shape
    dF = torch.from_numpy(np.ascontiguousarray(F, np.float32)).cuda()
    dr = torch.full((n,), -7 if poison else 0, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    native.rank_noalloc(dF.data_ptr(), n, m, dr.data_ptr(), stream)
    torch.cuda.synchronize()
    return dr.cpu().numpy()


# Two calls in a row per case: the second one starts from the first one's
# leftover workspace (a larger n first, then a smaller one, then larger).
PAIRS = [
    (("early", 2048, 5), ("chain", 1000, 3)),
    (("dups", 512, 4), ("early", 2048, 10)),
    (("late", 1996, 3), ("grid", 2048, 2)),
]


@pytest.mark.parametrize("pair", PAIRS, ids=lambda p: "%s%d-then-%s%d" % (p[0][0], p[0][1], p[1][0], p[1][1]))
def test_two_calls_match_select(env, orc, pair):
    torch, native = env
    for kind, n, m in pair:
        F = wl.objectives(kind, n, m, seed=n + m).astype(np.float32)
        got = _noalloc_ranks(torch, native, F)
        exp = _select_ranks(native, F)
        assert np.array_equal(got, exp), (kind, n, m)
        ora, _ = orc.nds(F, n // 2, full_sort=True)
        assert np.array_equal(got, ora), (kind, n, m)


def test_repeated_call_same_input(env, orc):
    torch, native = env
    F = wl.objectives("early", 2048, 3, seed=5).astype(np.float32)
    a = _noalloc_ranks(torch, native, F)
    b = _noalloc_ranks(torch, native, F)
    assert np.array_equal(a, b)
    assert np.array_equal(a, _select_ranks(native, F))
    assert np.array_equal(a, orc.nds(F, 1024, full_sort=True)[0])


def _fronts_by_rule(F):
    """Front index of every row by the stated rule, brute force in numpy:
    i dominates j iff f_i <= f_j everywhere and < somewhere (IEEE, so a NaN
    in either row makes both comparisons false); fronts are peeled one by
    one from the rows no remaining row dominates."""
    n = len(F)
    le = np.all(F[:, None, :] <= F[None, :, :], axis=2)
    lt = np.any(F[:, None, :] < F[None, :, :], axis=2)
    dom = le & lt
    rank = np.full(n, -1, np.int32)
    k = 0
    while (rank < 0).any():
        rem = rank < 0
        front = rem & ~np.any(dom & rem[:, None], axis=0)
        assert front.any()
        rank[front] = k
        k += 1
    return rank


def test_nan_rows_neither_dominate_nor_are_dominated(env, orc):
    """Rows holding a NaN objective form part of the first front and never
    push another row back, as the header states; checked against the rule
    written out in numpy and against the oracle's sort."""
    torch, native = env
    n, m = 33, 3
    F = wl.objectives("early", 34, m, seed=2)[:n].astype(np.float32)
    nan_rows = [0, 5, 17, 32]
    F[nan_rows[0], 1] = np.nan
    F[nan_rows[1], :] = np.nan
    F[nan_rows[2], 0] = np.nan
    F[nan_rows[3], 2] = np.nan
    got = _noalloc_ranks(torch, native, F)
    rule = _fronts_by_rule(F)
    assert np.array_equal(got, rule)
    assert np.all(got[nan_rows] == 0)
    assert np.array_equal(got, orc.nds(F, n, full_sort=True)[0])
    # without the NaN rows the other rows keep the ranks of the finite set
    keep = np.setdiff1d(np.arange(n), nan_rows)
    assert np.array_equal(got[keep], _fronts_by_rule(F[keep]))


def test_ragged_sizes_against_oracle(env, orc):
    """Sizes the context API does not take (odd n, n = 1): the oracle's
    non-dominated sort gives the reference ranks."""
    torch, native = env
    for kind, n, m in [("early", 1, 3), ("uniform", 33, 4), ("early", 2047, 6)]:
        F = wl.objectives(kind, max(n, 2), m, seed=1)[:n].astype(np.float32)
        got = _noalloc_ranks(torch, native, F)
        exp, _ = orc.nds(F, n, full_sort=True)
        assert np.array_equal(got, exp), (kind, n, m)


def test_rejects_sizes_beyond_the_maximum(env):
    torch, native = env
    n = native.NOALLOC_MAX_N + 1
    dF = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    dr = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    assert native.nsga3_rank_noalloc(dF.data_ptr(), n, 3, dr.data_ptr(), None) == native.EINVAL
    assert native.nsga3_rank_noalloc(dF.data_ptr(), 0, 3, dr.data_ptr(), None) == native.EINVAL
    assert native.nsga3_rank_noalloc(dF.data_ptr(), 8, 11, dr.data_ptr(), None) == native.EINVAL
    with pytest.raises(native.NSGA3Error, match="n <= 2048"):
        native.rank_noalloc(dF.data_ptr(), n, 3, dr.data_ptr())
    torch.cuda.synchronize()
    assert (dr == -7).all()  # nothing was enqueued
