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
