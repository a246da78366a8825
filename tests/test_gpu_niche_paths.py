"""GPU parity of the niching kernels' capacity paths (Alg. 1 niching loop,
Alg. 2 cached batched form, read as the closed form of the level threshold).

The level and pick kernels keep their working sets in shared memory up to
fixed capacities and switch to other code beyond them: niche counts read
from global memory when more than 12,288 references cannot be staged, a
binary search for the level threshold L* from 4,096 on, a generic select
when more than 4,096 references hold a level-L* member, a block-wide member
selection for partial takes from references of more than 32 members, and
8-bit radix passes in that selection for more than 1,024 candidates.  Each
case below drives one or more of those paths, asserts through
nsga3_get_selection_paths that they were taken, and requires the ranks and
selected indices to equal the oracle's (the literal sequential niching
loop) bit for bit.  The radix passes that only hundreds of thousands of
members on one reference would reach are driven through the selection
routine's own self-test entry point on crafted keys."""
import ctypes as C

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


# (id, m, p, N, objective kind, paths that must be taken)
CASES = [
    # w = C(162, 2) = 13,041 references (> 12,288): counts from global memory;
    # one front of 2N points spread over the simplex puts about 7,700
    # references at level L* = 1 (> 4,096 staged keys)
    ("wide_simplex", 3, 160, 13044, "simplex", ("UNSTAGED", "CKOVER")),
    ("wide_late", 3, 160, 13044, "late", ("UNSTAGED",)),
    # all 2N points identical: one front, every point on the first nearest
    # reference, L* = N - 1 >= 4,096 on the unstaged path, a partial take
    # from one reference of 2N members (radix pass over member keys)
    ("wide_equal", 3, 160, 13044, "equal", ("UNSTAGED", "DEEP", "LARGE", "RADIX")),
    # three references (the simplex vertices) and one front of 32,000 points:
    # L* about 5,300 on the staged path, partial takes of about 10,000 members
    ("deep_simplex", 3, 1, 16000, "simplex", ("DEEP", "LARGE", "RADIX")),
    ("deep_late", 3, 1, 16000, "late", ("DEEP", "LARGE", "RADIX")),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_capacity_path_matches_oracle(n, orc, case):
    _, m, p, N, kind, want = case
    F = wl.objectives(kind, 2 * N, m, seed=N + p)
    Z = orc.refdirs(m, p)
    gen = 5
    with Run(n, m, m + 1, N, p, seed=13) as r:
        assert r.w == len(Z)
        st, rank, sel = r.select(F, gen=gen)
        assert st == 0, "device status %d" % st
        info = r.info()
        paths = r.paths()
    ref = orc.select(F, N, Z, seed=13, gen=gen, variant=0)
    assert ref["niche"] and info["niche"]
    for name in want:
        bit = getattr(n, "PATH_" + name)
        assert paths & bit, "path %s not taken (paths = %#x, L* = %d)" % (name, paths, info["Lstar"])
    assert np.array_equal(rank, ref["rank"])
    assert np.array_equal(sel, ref["selected"])


def _probe(n, torch, keys, need):
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    marks = torch.full((len(keys),), 7, dtype=torch.int32, device="cuda")
    paths = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = n.nsga3_select_smallest_probe(dk.data_ptr(), len(keys), need, marks.data_ptr(),
                                       paths.data_ptr(), None)
    assert st == n.OK
    torch.cuda.synchronize()
    return marks.cpu().numpy(), int(paths.cpu().numpy()[0])


@pytest.mark.parametrize("shared_bits,n_keys", [(0, 600), (8, 5000), (16, 3000), (40, 2048), (56, 200)])
def test_select_routine_radix_passes(n, shared_bits, n_keys):
    """The `need` smallest of unique keys whose top `shared_bits` bits are
    equal: the routine must narrow through several 8-bit radix passes (one
    per shared byte while more than 1,024 candidates remain) and still mark
    exactly the smallest keys, for every need from 0 to n."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(shared_bits * 7919 + n_keys)
    low_bits = 64 - shared_bits
    low = rng.choice(np.uint64(1) << np.uint64(min(low_bits, 62)), size=n_keys, replace=False).astype(np.uint64)
    top = np.uint64(0xA5C3F00DDEADBEEF) >> np.uint64(low_bits) << np.uint64(low_bits) if shared_bits else np.uint64(0)
    keys = (top | low).astype(np.uint64)
    if shared_bits == 0:
        keys = rng.choice(np.iinfo(np.int64).max, size=n_keys, replace=False).astype(np.uint64)
    assert len(np.unique(keys)) == n_keys
    order = np.argsort(keys, kind="stable")
    saw = 0
    for need in sorted({0, 1, n_keys // 3, n_keys // 2 + 1, n_keys - 1, n_keys}):
        marks, paths = _probe(n, torch, keys, need)
        exp = np.zeros(n_keys, np.int32)
        exp[order[:need]] = 1
        assert np.array_equal(marks, exp), (shared_bits, n_keys, need)
        saw |= paths
    if n_keys > 1024 and shared_bits >= 8:
        assert saw & n.PATH_RADIX and saw & n.PATH_RADIX2, hex(saw)
    elif n_keys > 1024:
        assert saw & n.PATH_RADIX


def test_select_probe_rejects_bad_arguments(n):
    torch = pytest.importorskip("torch")
    dk = torch.zeros(4, dtype=torch.int64, device="cuda")
    dm = torch.zeros(4, dtype=torch.int32, device="cuda")
    dp = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert n.nsga3_select_smallest_probe(dk.data_ptr(), 4, 5, dm.data_ptr(), dp.data_ptr(), None) == n.EINVAL
    assert n.nsga3_select_smallest_probe(dk.data_ptr(), 0, 0, dm.data_ptr(), dp.data_ptr(), None) == n.EINVAL
    assert n.nsga3_select_smallest_probe(None, 4, 1, dm.data_ptr(), dp.data_ptr(), None) == n.EINVAL
