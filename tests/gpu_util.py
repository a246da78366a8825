"""Helpers for the GPU tests: a context wrapper over the C ABI binding."""
import ctypes as C

import numpy as np


class Run:
    """Owns one nsga3 context; all transfers go through host numpy arrays."""

    def __init__(self, n, m, d, N, p1, p2=0, tau=0.5, seed=0, W=None, **opts):
        self.n = n
        self.m, self.d, self.N = m, d, N
        self._W = None if W is None else np.ascontiguousarray(W, dtype=np.float32)
        o = n.default_opts(seed=seed, p2=p2, tau=tau,
                           W=None if self._W is None else self._W.ctypes.data, **opts)
        self.ctx = n.create(m, d, N, p1, o)
        self.w = n.nsga3_num_refs(self.ctx)

    def close(self):
        if self.ctx:
            self.n.nsga3_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def check(self, st):
        return self.n.check(st, self.ctx)

    def sync(self):
        return self.n.nsga3_sync(self.ctx, None)

    def refs(self):
        Z = np.zeros((self.w, self.m))
        self.check(self.n.nsga3_get_refs(self.ctx, Z.ctypes.data))
        return Z

    def select(self, F, gen=0):
        F = np.ascontiguousarray(F, dtype=np.float32)
        rank = np.zeros(2 * self.N, np.int32)
        sel = np.zeros(self.N, np.int32)
        self.check(self.n.nsga3_set_counter(self.ctx, gen, None))
        self.check(self.n.nsga3_select(self.ctx, F.ctypes.data, rank.ctypes.data, sel.ctypes.data, None))
        st = self.sync()
        return st, rank, sel

    def info(self):
        a = np.zeros(13, np.int32)
        self.check(self.n.nsga3_get_selection_info(self.ctx, a.ctypes.data))
        keys = ["l", "nS", "K", "nFl", "niche", "fallback", "passes", "nT", "Lstar", "rlev",
                "overflow", "recheck_miss", "peel_rows"]
        return dict(zip(keys, (int(x) for x in a)))

    def paths(self):
        p = C.c_uint32()
        self.check(self.n.nsga3_get_selection_paths(self.ctx, C.byref(p)))
        return p.value

    def normalization(self):
        z = np.zeros(self.m)
        a = np.zeros(self.m)
        e = np.zeros(self.m, np.int32)
        self.check(self.n.nsga3_get_normalization(self.ctx, z.ctypes.data, a.ctypes.data, e.ctypes.data))
        return z, a, e

    def association(self):
        pi = np.zeros(2 * self.N, np.int32)
        dist = np.zeros(2 * self.N)
        self.check(self.n.nsga3_get_association(self.ctx, pi.ctypes.data, dist.ctypes.data))
        return pi, dist

    def set_population(self, X, F, rank):
        self._keep = [np.ascontiguousarray(X, np.float32), np.ascontiguousarray(F, np.float32),
                      np.ascontiguousarray(rank, np.int32)]
        self.check(self.n.nsga3_set_population(self.ctx, *(a.ctypes.data for a in self._keep), None))
        self.check(self.sync())

    def population(self):
        X = np.zeros((self.N, self.d), np.float32)
        F = np.zeros((self.N, self.m), np.float32)
        r = np.zeros(self.N, np.int32)
        self.check(self.n.nsga3_get_population(self.ctx, X.ctypes.data, F.ctypes.data, r.ctypes.data, None))
        self.check(self.sync())
        return X, F, r

    def children(self):
        X = np.zeros((self.N, self.d), np.float32)
        F = np.zeros((self.N, self.m), np.float32)
        self.check(self.n.nsga3_get_children(self.ctx, X.ctypes.data, F.ctypes.data, None))
        self.check(self.sync())
        return X, F

    def counter(self):
        g = C.c_uint64()
        self.check(self.n.nsga3_get_counter(self.ctx, C.byref(g), None))
        return g.value
