"""ctypes binding of libnsga3.so with the entry-point names of include/nsga3.h.

Argument marshalling only: every computation runs in the CUDA library.
Pointers are passed as integers (``tensor.data_ptr()`` for torch tensors,
``array.ctypes.data`` for numpy arrays); streams as ``cudaStream_t`` values
(``torch.cuda.current_stream().cuda_stream``).  Importing this module raises
if the library has not been built, and there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnsga3.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libnsga3.so is not built (run __graft_entry__.build() or "
                      "python -m paper_2504_06067_gb300.build); there is no CPU fallback")

_lib = C.CDLL(LIB_PATH)

NOALLOC_MAX_N = 2048  # NSGA3_NOALLOC_MAX_N

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ESTATE, EINTERNAL = range(8)
# NSGA3_PATH_* bits of nsga3_get_selection_paths
PATH_UNSTAGED, PATH_DEEP, PATH_CKOVER, PATH_BINOVER, PATH_LARGE, PATH_RADIX, PATH_RADIX2 = (
    1, 2, 4, 8, 16, 32, 64)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENONFINITE",
                5: "ETIMEOUT", 6: "ESTATE", 7: "EINTERNAL"}


class nsga3_opts(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64),
        ("p2", C.c_int),
        ("tau", C.c_double),
        ("eta_c", C.c_float),
        ("eta_m", C.c_float),
        ("p_c", C.c_float),
        ("p_m", C.c_float),
        ("full_sort", C.c_int),
        ("debug_recheck_all", C.c_int),
        ("W", C.c_void_p),
        ("streaming", C.c_int),
        ("norm_history", C.c_int),
        ("problem", C.c_int),
        ("kp_profit", C.c_void_p),
        ("kp_weight", C.c_void_p),
        ("kp_capacity", C.c_void_p),
        ("wait_ms", C.c_int),
        ("phase_timing", C.c_int),
        ("dom_ctas_per_sm", C.c_int),
        ("peel_ctas_per_sm", C.c_int),
    ]


class nsga3_request(C.Structure):
    _fields_ = [("m", C.c_int), ("d", C.c_int), ("N", C.c_int), ("ref_divisions", C.c_int),
                ("generations", C.c_int), ("opts", nsga3_opts)]


class nsga3_run_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("m", C.c_int32), ("d", C.c_int32), ("N", C.c_int32),
                ("generations", C.c_int32), ("workspace_bytes", C.c_uint64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("message", C.c_char * 256)]


class nsga3_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("active", C.c_int64), ("pending", C.c_int64), ("peak_active", C.c_int64),
                ("launches", C.c_int64), ("budget_bytes", C.c_uint64), ("bytes_in_use", C.c_uint64),
                ("peak_bytes", C.c_uint64)]


_P = C.c_void_p
_CTX = C.c_void_p
_I = C.c_int
_SIGS = {
    "nsga3_default_opts": (None, [C.POINTER(nsga3_opts)]),
    "nsga3_create": (_I, [_I, _I, _I, _I, C.POINTER(nsga3_opts), C.POINTER(_CTX)]),
    "nsga3_destroy": (None, [_CTX]),
    "nsga3_last_error": (C.c_char_p, [_CTX]),
    "nsga3_num_refs": (_I, [_CTX]),
    "nsga3_get_refs": (_I, [_CTX, _P]),
    "nsga3_select": (_I, [_CTX, _P, _P, _P, _P]),
    "nsga3_init": (_I, [_CTX, _P]),
    "nsga3_vary": (_I, [_CTX, _P]),
    "nsga3_step": (_I, [_CTX, _P]),
    "nsga3_run": (_I, [_CTX, _I, _P]),
    "nsga3_run_batch": (_I, [C.POINTER(_CTX), _I, _I, _P]),
    "nsga3_batch_graph_builds": (_I, [_CTX, C.POINTER(C.c_int64)]),
    "nsga3_get_population": (_I, [_CTX, _P, _P, _P, _P]),
    "nsga3_set_population": (_I, [_CTX, _P, _P, _P, _P]),
    "nsga3_get_children": (_I, [_CTX, _P, _P, _P]),
    "nsga3_set_counter": (_I, [_CTX, C.c_uint64, _P]),
    "nsga3_get_counter": (_I, [_CTX, C.POINTER(C.c_uint64), _P]),
    "nsga3_sync": (_I, [_CTX, _P]),
    "nsga3_wait_probe": (_I, [_CTX, _P]),
    "nsga3_get_selection_info": (_I, [_CTX, _P]),
    "nsga3_get_normalization": (_I, [_CTX, _P, _P, _P]),
    "nsga3_get_selection_paths": (_I, [_CTX, C.POINTER(C.c_uint32)]),
    "nsga3_get_dominance_stats": (_I, [_CTX, _P]),
    "nsga3_select_smallest_probe": (_I, [_P, _I, _I, _P, _P, _P]),
    "nsga3_issue_probe": (_I, [_I, _I, _I, C.POINTER(C.c_double), C.POINTER(C.c_float), _P, _P]),
    "nsga3_get_association": (_I, [_CTX, _P, _P]),
    "nsga3_phase_times": (_I, [_CTX, _P, _I]),
    "nsga3_last_launches": (_I, [_CTX, _P]),
    "nsga3_total_launches": (_I, [_CTX, _P]),
    "nsga3_rank_noalloc": (_I, [_P, _I, _I, _P, _P]),
    "nsga3_workspace_bytes": (_I, [_I, _I, _I, _I, C.POINTER(nsga3_opts), C.POINTER(C.c_uint64)]),
    "nsga3_server_create": (_I, [C.c_uint64, _I, _I, C.POINTER(_P)]),
    "nsga3_server_submit": (_I, [_P, C.POINTER(nsga3_request), C.POINTER(C.c_int64)]),
    "nsga3_server_wait": (_I, [_P, _I, C.POINTER(C.c_int64)]),
    "nsga3_server_fetch": (_I, [_P, C.c_int64, _P, _P, _P, C.POINTER(nsga3_run_info)]),
    "nsga3_server_get_stats": (_I, [_P, C.POINTER(nsga3_server_stats)]),
    "nsga3_server_now": (C.c_double, [_P]),
    "nsga3_server_last_error": (C.c_char_p, [_P]),
    "nsga3_server_destroy": (None, [_P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class NSGA3Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def check(status, ctx=None):
    """Raise NSGA3Error for a non-OK status (message from nsga3_last_error)."""
    if status != OK:
        msg = nsga3_last_error(ctx)
        raise NSGA3Error(status, msg.decode() if msg else "")
    return status


def default_opts(**kw) -> nsga3_opts:
    o = nsga3_opts()
    nsga3_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def create(m, d, N, ref_divisions, opts=None):
    """nsga3_create; returns the context handle (an int)."""
    if opts is None:
        opts = default_opts()
    h = _CTX()
    check(nsga3_create(m, d, N, ref_divisions, C.byref(opts), C.byref(h)))
    return h.value


def run_batch(ctxs, generations, stream=0):
    arr = (_CTX * len(ctxs))(*ctxs)
    return nsga3_run_batch(arr, len(ctxs), generations, stream)


def batch_graph_builds(ctx):
    """nsga3_batch_graph_builds: times ctx built its batched graphs."""
    b = C.c_int64()
    check(nsga3_batch_graph_builds(ctx, C.byref(b)), ctx)
    return b.value


def issue_probe(scratch_ptr, blocks_per_sm=8, iters=20000, reps=5, stream=0):
    """nsga3_issue_probe: (thread-instructions per second, best launch ms)."""
    r = C.c_double()
    ms = C.c_float()
    st = nsga3_issue_probe(blocks_per_sm, iters, reps, C.byref(r), C.byref(ms), scratch_ptr, stream)
    if st != OK:
        raise NSGA3Error(st, "nsga3_issue_probe failed")
    return r.value, ms.value


def rank_noalloc(objs_ptr, n, m, ranks_ptr, stream=0):
    """nsga3_rank_noalloc with a descriptive error; pointers are device
    addresses of n x m FP32 objectives and n int32 ranks."""
    st = nsga3_rank_noalloc(objs_ptr, n, m, ranks_ptr, stream)
    if st == EINVAL:
        raise NSGA3Error(st, "nsga3_rank_noalloc takes 1 <= n <= %d points (got %d), "
                             "2 <= m <= 10 (got %d) and non-NULL pointers"
                         % (NOALLOC_MAX_N, n, m))
    if st != OK:
        raise NSGA3Error(st, "nsga3_rank_noalloc: CUDA device lookup or launch failed")
    return st


def workspace_bytes(m, d, N, ref_divisions, opts=None):
    """nsga3_workspace_bytes: device bytes nsga3_create would allocate."""
    if opts is None:
        opts = default_opts()
    b = C.c_uint64()
    check(nsga3_workspace_bytes(m, d, N, ref_divisions, C.byref(opts), C.byref(b)))
    return b.value


class Server:
    """Thin owner of an nsga3_server handle (calls map one to one)."""

    def __init__(self, memory_budget, max_active=64, gens_per_launch=8):
        h = C.c_void_p()
        st = nsga3_server_create(int(memory_budget), max_active, gens_per_launch, C.byref(h))
        if st != OK:
            raise NSGA3Error(st, "nsga3_server_create failed")
        self.h = h.value
        self._keep = {}

    def submit(self, m, d, N, ref_divisions, generations, W, **opts):
        import numpy as np
        W = np.ascontiguousarray(W, dtype=np.float32)
        o = default_opts(W=W.ctypes.data, **opts)
        req = nsga3_request(m, d, N, ref_divisions, generations, o)
        i = C.c_int64()
        st = nsga3_server_submit(self.h, C.byref(req), C.byref(i))
        if st != OK:
            msg = nsga3_server_last_error(self.h)
            raise NSGA3Error(st, msg.decode() if msg else "")
        return i.value

    def wait(self, timeout_ms=-1):
        i = C.c_int64()
        check(nsga3_server_wait(self.h, timeout_ms, C.byref(i)))
        return i.value

    def fetch(self, rid, X=0, F=0, rank=0):
        info = nsga3_run_info()
        st = nsga3_server_fetch(self.h, rid, X, F, rank, C.byref(info))
        return st, info

    def stats(self):
        s = nsga3_server_stats()
        check(nsga3_server_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def now(self):
        return nsga3_server_now(self.h)

    def close(self):
        if self.h:
            nsga3_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
