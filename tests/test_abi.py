"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/nsga3.h declares (no compute calls here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nsga3.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nsga3_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_06067_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("nsga3_create", "nsga3_select", "nsga3_step", "nsga3_run", "nsga3_destroy",
                     "nsga3_get_population", "nsga3_set_counter", "nsga3_last_error",
                     "nsga3_run_batch"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [nm for nm in _declared() if not hasattr(lib, nm)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2504_06067_gb300 import build
    build.build()
    from paper_2504_06067_gb300 import native
    for nm in _declared():
        assert hasattr(native, nm), nm


def test_create_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2504_06067_gb300 import native as n
    h = C.c_void_p()
    o = n.default_opts()
    st = n.nsga3_create(3, 12, 92, 12, C.byref(o), C.byref(h))
    assert st == n.ECUDA and h.value is None
    assert b"device" in n.nsga3_last_error(None)
    # argument errors are reported before any device work
    assert n.nsga3_create(1, 12, 92, 12, C.byref(o), C.byref(h)) == n.EINVAL
    assert n.nsga3_create(3, 12, 91, 12, C.byref(o), C.byref(h)) == n.EINVAL


def test_workspace_bytes_without_gpu(lib):
    """The sizing pass touches no device: the bit matrix dominates at scale,
    the count grows with N and bad arguments are rejected like nsga3_create."""
    from paper_2504_06067_gb300 import native as n
    prev = 0
    for N in (92, 1000, 10628, 100000):
        b = n.workspace_bytes(5, 100, N, 4)
        ld = -(-2 * N // 256) * 256
        assert b >= ld * ld // 8 + 2 * N * 100 * 4
        assert b > prev
        prev = b
    big = n.workspace_bytes(10, 200, 100000, 3, n.default_opts(p2=2))
    assert 5.0e9 < big < 5.6e9
    out = C.c_uint64()
    o = n.default_opts()
    assert n.nsga3_workspace_bytes(1, 12, 92, 12, C.byref(o), C.byref(out)) == n.EINVAL
    assert n.nsga3_workspace_bytes(3, 12, 91, 12, C.byref(o), C.byref(out)) == n.EINVAL


def test_many_objectives_workspace(lib):
    """m up to 512 is accepted (Table II's sweep); m > 32 adds the m x (m+1)
    elimination matrix; streaming and the knapsack stop at m = 10."""
    from paper_2504_06067_gb300 import native as n
    b32 = n.workspace_bytes(32, 1000, 800, 2)
    b512 = n.workspace_bytes(512, 1000, 800, 1)
    assert b512 > 512 * 513 * 8 and b32 > 0
    out = C.c_uint64()
    for m, o in ((513, n.default_opts()), (11, n.default_opts(streaming=1)),
                 (11, n.default_opts(problem=1))):
        assert n.nsga3_workspace_bytes(m, 1000, 800, 1, C.byref(o), C.byref(out)) == n.EINVAL


def test_phase_timing_option(lib):
    """opts.phase_timing defaults to 0 (no timing events in the graphs) and
    takes 0, 1 or 2."""
    from paper_2504_06067_gb300 import native as n
    assert n.default_opts().phase_timing == 0
    out = C.c_uint64()
    for lv, want in ((0, n.OK), (1, n.OK), (2, n.OK), (-1, n.EINVAL), (3, n.EINVAL)):
        o = n.default_opts(phase_timing=lv)
        assert n.nsga3_workspace_bytes(3, 12, 92, 12, C.byref(o), C.byref(out)) == want


def test_server_create_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2504_06067_gb300 import native as n
    h = C.c_void_p()
    assert n.nsga3_server_create(1 << 20, 4, 8, C.byref(h)) == n.ECUDA and h.value is None
    assert n.nsga3_server_create(1 << 20, 0, 8, C.byref(h)) == n.EINVAL


def test_streaming_workspace_has_no_matrix(lib):
    from paper_2504_06067_gb300 import native as n
    N = 100000
    full = n.workspace_bytes(10, 200, N, 3, n.default_opts(p2=2))
    stream = n.workspace_bytes(10, 200, N, 3, n.default_opts(p2=2, streaming=1))
    ld = -(-2 * N // 256) * 256
    NW = ld // 32
    bitmap = -(-NW * (-(-NW // 8)) // 256) * 256  # one bit per 32 x 32 block of the matrix
    assert full - stream == ld * ld // 8 - 256 + bitmap


def test_launch_shape_options(lib):
    """opts.dom_ctas_per_sm and opts.peel_ctas_per_sm default to 0 (every CTA
    that fits at once) and take 0 ... 64."""
    from paper_2504_06067_gb300 import native as n
    o = n.default_opts()
    assert o.dom_ctas_per_sm == 0 and o.peel_ctas_per_sm == 0
    out = C.c_uint64()
    for dc, pc, want in ((0, 0, n.OK), (1, 2, n.OK), (64, 64, n.OK), (-1, 0, n.EINVAL), (0, 65, n.EINVAL)):
        o = n.default_opts(dom_ctas_per_sm=dc, peel_ctas_per_sm=pc)
        assert n.nsga3_workspace_bytes(10, 12, 500, 3, C.byref(o), C.byref(out)) == want
