"""FP64 CPU oracle for NSGA-III environmental selection (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's cpu_baseline /
reference leg may import this package.  The product path (the CUDA library
and its Python binding) never touches it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module only builds that file with gcc and
marshals numpy arrays through ctypes.  Each wrapper names the paper passage
its C routine follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, EINVAL, ENOMEM = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no FMA contraction),
    with OpenMP when the compiler has it (the parallel loops give the same
    results bit for bit; without OpenMP the build is single-threaded)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def threads() -> int:
    """Host threads the oracle's parallel loops use (1 without OpenMP)."""
    return int(_load().orc_threads())


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # NSGA3_ORACLE_LIB names another build of oracle.c: the planted-mistake
    # tests load copies with one error each this way
    other = os.environ.get("NSGA3_ORACLE_LIB")
    if other:
        lib = C.CDLL(other)
    else:
        build()
        lib = C.CDLL(_LIB)
    P = C.c_void_p
    i32, u32, u64, i64, f64, f32 = C.c_int, C.c_uint32, C.c_uint64, C.c_int64, C.c_double, C.c_float
    sig = {
        "orc_philox4x32_10": (None, [P, P, P]),
        "orc_ref_priority": (u32, [u64, u32, u32]),
        "orc_member_priority": (u32, [u64, u32, u32]),
        "orc_binom": (i64, [i32, i32]),
        "orc_das_dennis_count": (i64, [i32, i32]),
        "orc_refdirs": (i64, [i32, i32, i32, f64, P]),
        "orc_dominates": (i32, [P, P, i32]),
        "orc_nds": (i32, [P, i32, i32, i32, i32, P]),
        "orc_threads": (i32, []),
        "orc_normalize": (i32, [P, P, i32, i32, i32, P, P, P, P]),
        "orc_associate": (None, [P, P, i32, i32, i32, P, P, P, i32, P, P]),
        "orc_niche_sequential": (i32, [P, i32, i32, i32, P, P, i32, u64, u32, P]),
        "orc_niche_batched": (i32, [P, i32, i32, i32, P, P, i32, u64, u32, P]),
        "orc_select": (i32, [P, i32, i32, P, i32, u64, u32, i32, i32, P, P, P, P, P]),
        "orc_select_hist": (i32, [P, i32, i32, P, i32, u64, u32, i32, i32, P, P, P, P, P, P, P, P]),
        "orc_normalize_hist": (i32, [P, P, i32, i32, i32, P, P, P, P, P, P, P]),
        "orc_vary": (None, [P, P, i32, i32, u64, u32, f64, f64, f32, f32, P]),
        "orc_eval": (None, [P, i32, i32, i32, P, P]),
        "orc_init": (None, [i32, i32, u64, P]),
        "orc_generation": (i32, [P, P, P, i32, i32, i32, P, P, i32, u64, u32, f64, f64,
                                 f32, f32, i32]),
        "orc_igd": (f64, [P, i32, i32, P, i32]),
        "orc_kp_order": (None, [P, P, i32, i32, P]),
        "orc_kp_eval": (None, [P, i32, i32, i32, P, P, P, P, P]),
        "orc_kp_init": (None, [i32, i32, u64, P]),
        "orc_kp_vary": (None, [P, P, i32, i32, u64, u32, f32, f32, P]),
        "orc_kp_generation": (i32, [P, P, P, i32, i32, i32, P, P, P, P, P, i32, u64, u32, f32, f32]),
        "orc_hv": (f64, [P, i32, i32, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- Philox ----
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al., SC'11) for a 4-word counter, 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def ref_priority(seed: int, gen: int, j: int) -> int:
    return int(_load().orc_ref_priority(seed, gen, j))


def member_priority(seed: int, gen: int, i: int) -> int:
    return int(_load().orc_member_priority(seed, gen, i))


# ----------------------------------------------------- reference points -----
def das_dennis_count(m: int, p: int) -> int:
    """C(p+m-1, m-1): size of the Das-Dennis lattice (Sec. II-C)."""
    return int(_load().orc_das_dennis_count(m, p))


def refdirs(m: int, p1: int, p2: int = 0, tau: float = 0.5) -> np.ndarray:
    """Das-Dennis directions, outer layer p1 then optional inner layer p2 (w x m, FP64)."""
    lib = _load()
    w = das_dennis_count(m, p1) + (das_dennis_count(m, p2) if p2 > 0 else 0)
    Z = np.zeros((w, m), dtype=np.float64)
    got = lib.orc_refdirs(m, p1, p2, tau, _p(Z))
    if got != w:
        raise ValueError("refdirs: bad arguments")
    return Z


# ------------------------------------------------------------ selection -----
def dominates(a, b) -> bool:
    a = _f32(a)
    b = _f32(b)
    return bool(_load().orc_dominates(_p(a), _p(b), a.shape[0]))


def nds(F, N: int, full_sort: bool = False):
    """Non-dominated sorting of the 2N x m objectives (Alg. 1).  Returns (rank, l)."""
    F = _f32(F)
    n2, m = F.shape
    rank = np.zeros(n2, dtype=np.int32)
    l = _load().orc_nds(_p(F), n2, m, N, int(full_sort), _p(rank))
    if l < 0 and n2 > 0:
        raise MemoryError("orc_nds failed")
    return rank, int(l)


def normalize(F, rank, l: int):
    """Ideal point, ASF extremes and intercepts over S u F_l (the normalization of Alg. 2)."""
    F = _f32(F)
    rank = _i32(rank)
    n2, m = F.shape
    zstar = np.zeros(m)
    a = np.zeros(m)
    ext = np.zeros(m, dtype=np.int32)
    fb = np.zeros(1, dtype=np.int32)
    rc = _load().orc_normalize(_p(F), _p(rank), n2, m, l, _p(zstar), _p(a), _p(ext), _p(fb))
    if rc != OK:
        raise ValueError("normalize: empty normalization set")
    return zstar, a, ext, bool(fb[0])


def new_history(m: int) -> dict:
    """Empty normalization history: running ideal z[m], remembered extreme
    vectors e[m][m] (FP32), valid flag.  Updated in place by the *_hist calls."""
    return {"valid": np.zeros(1, dtype=np.int32), "z": np.zeros(m), "e": np.zeros((m, m), dtype=np.float32)}


def normalize_hist(F, rank, l: int, history: dict):
    """Normalization with a running ideal point and remembered extreme points
    (an option; the paper defines no history).  Extreme indices >= 2N name the
    remembered vectors.  Updates `history`."""
    F = _f32(F)
    rank = _i32(rank)
    n2, m = F.shape
    zstar = np.zeros(m)
    a = np.zeros(m)
    ext = np.zeros(m, dtype=np.int32)
    fb = np.zeros(1, dtype=np.int32)
    rc = _load().orc_normalize_hist(_p(F), _p(rank), n2, m, l, _p(history["valid"]), _p(history["z"]),
                                    _p(history["e"]), _p(zstar), _p(a), _p(ext), _p(fb))
    if rc != OK:
        raise ValueError("normalize_hist: empty normalization set")
    return zstar, a, ext, bool(fb[0])


def associate(F, rank, l: int, zstar, a, Z):
    """pi = argmin_j D_ij and d = min_j D_ij with D from Eq. (2) (Alg. 2)."""
    F = _f32(F)
    rank = _i32(rank)
    Z = _f64(Z)
    n2, m = F.shape
    pi = np.zeros(n2, dtype=np.int32)
    dist = np.zeros(n2)
    _load().orc_associate(_p(F), _p(rank), n2, m, l, _p(_f64(zstar)), _p(_f64(a)), _p(Z),
                          Z.shape[0], _p(pi), _p(dist))
    return pi, dist


def niche(rank, l: int, K: int, pi, dist, w: int, seed: int, gen: int, variant: int = 0):
    """Niche selection of K members of F_l: variant 0 = Alg. 1 loop, 1 = Alg. 2 cached loop."""
    rank = _i32(rank)
    pi = _i32(pi)
    dist = _f64(dist)
    picked = np.zeros(rank.shape[0], dtype=np.uint8)
    fn = _load().orc_niche_sequential if variant == 0 else _load().orc_niche_batched
    rc = fn(_p(rank), rank.shape[0], l, K, _p(pi), _p(dist), w, seed, gen, _p(picked))
    if rc != OK:
        raise ValueError("niche selection failed (rc=%d)" % rc)
    return picked.astype(bool)


def select(F, N: int, Z, seed: int, gen: int, variant: int = 0, full_sort: bool = False,
           history: dict | None = None):
    """Full environmental selection of N out of the 2N x m objectives.

    With `history` (see new_history) the normalization keeps a running ideal
    point and remembered extreme points, and `history` is updated in place.
    Returns dict(rank, selected, pi, dist, l, nS, K, nFl, niche, fallback).
    """
    F = _f32(F)
    Z = _f64(Z)
    n2, m = F.shape
    assert n2 == 2 * N
    rank = np.zeros(n2, dtype=np.int32)
    sel = np.zeros(N, dtype=np.int32)
    pi = np.zeros(n2, dtype=np.int32)
    dist = np.zeros(n2)
    info = np.zeros(6, dtype=np.int32)
    if history is None:
        rc = _load().orc_select(_p(F), N, m, _p(Z), Z.shape[0], seed, gen, variant, int(full_sort),
                                _p(rank), _p(sel), _p(pi), _p(dist), _p(info))
    else:
        rc = _load().orc_select_hist(_p(F), N, m, _p(Z), Z.shape[0], seed, gen, variant,
                                     int(full_sort), _p(rank), _p(sel), _p(pi), _p(dist), _p(info),
                                     _p(history["valid"]), _p(history["z"]), _p(history["e"]))
    if rc != OK:
        raise ValueError("orc_select failed (rc=%d)" % rc)
    keys = ["l", "nS", "K", "nFl", "niche", "fallback"]
    out = dict(zip(keys, (int(v) for v in info)))
    out.update(rank=rank, selected=sel, pi=pi, dist=dist)
    return out


# ------------------------------------------------- variation / problem -----
def vary(X, rank, seed: int, gen: int, eta_c=20.0, eta_m=20.0, p_c=1.0, p_m=None):
    """Tournament + SBX + polynomial mutation: N x d parents -> N x d children."""
    X = _f32(X)
    rank = _i32(rank)
    N, d = X.shape
    if p_m is None:
        p_m = float(np.float32(1.0) / np.float32(d))
    Xc = np.zeros_like(X)
    _load().orc_vary(_p(X), _p(rank), N, d, seed, gen, float(eta_c), float(eta_m), float(p_c),
                     float(p_m), _p(Xc))
    return Xc


def evaluate(X, W):
    """Softmax-simplex objective f = (1+g) softmax(W x[:m-1]) (FP64, rounded to FP32)."""
    X = _f32(X)
    W = _f32(W)
    n, d = X.shape
    m = W.shape[0]
    F = np.zeros((n, m), dtype=np.float32)
    _load().orc_eval(_p(X), n, d, m, _p(W), _p(F))
    return F


def init_population(N: int, d: int, seed: int):
    X = np.zeros((N, d), dtype=np.float32)
    _load().orc_init(N, d, seed, _p(X))
    return X


def generation(X, F, rank, W, Z, seed: int, gen: int, eta_c=20.0, eta_m=20.0, p_c=1.0,
               p_m=None, variant: int = 0):
    """One NSGA-III generation (Alg. 1) in place on copies; returns (X, F, rank)."""
    X = _f32(X).copy()
    F = _f32(F).copy()
    rank = _i32(rank).copy()
    W = _f32(W)
    Z = _f64(Z)
    N, d = X.shape
    m = F.shape[1]
    if p_m is None:
        p_m = float(np.float32(1.0) / np.float32(d))
    rc = _load().orc_generation(_p(X), _p(F), _p(rank), N, d, m, _p(W), _p(Z), Z.shape[0], seed,
                                gen, float(eta_c), float(eta_m), float(p_c), float(p_m), variant)
    if rc != OK:
        raise ValueError("orc_generation failed (rc=%d)" % rc)
    return X, F, rank


def run(N: int, d: int, W, Z, seed: int, generations: int, **kw):
    """Init (Philox stream 6) + evaluate + ranks 0, then `generations` generations."""
    X = init_population(N, d, seed)
    F = evaluate(X, W)
    rank = np.zeros(N, dtype=np.int32)
    for g in range(generations):
        X, F, rank = generation(X, F, rank, W, Z, seed, g, **kw)
    return X, F, rank


def igd(P, R) -> float:
    """Inverted generational distance of population objectives P to reference front R."""
    P = _f32(P)
    R = _f64(R)
    return float(_load().orc_igd(_p(P), P.shape[0], P.shape[1], _p(R), R.shape[0]))


# ---------------------------------------------- 0-1 knapsack workload -----
def kp_order(profit, weight):
    """Repair order: items by ascending best profit/weight ratio (exact), ties lower index."""
    profit = _i32(profit)
    weight = _i32(weight)
    m, d = profit.shape
    order = np.zeros(d, dtype=np.int32)
    _load().orc_kp_order(_p(profit), _p(weight), m, d, _p(order))
    return order


def kp_eval(X, profit, weight, cap, order=None):
    """Repair (in a copy) and evaluate: returns (X repaired, F) with
    f_j = P_j - sum_v p[j][v] x_v (minimised, integer-valued)."""
    X = _f32(X).copy()
    profit, weight, cap = _i32(profit), _i32(weight), _i32(cap)
    if order is None:
        order = kp_order(profit, weight)
    n, d = X.shape
    m = profit.shape[0]
    F = np.zeros((n, m), dtype=np.float32)
    _load().orc_kp_eval(_p(X), n, d, m, _p(profit), _p(weight), _p(cap), _p(_i32(order)), _p(F))
    return X, F


def kp_init(N: int, d: int, seed: int):
    X = np.zeros((N, d), dtype=np.float32)
    _load().orc_kp_init(N, d, seed, _p(X))
    return X


def kp_vary(X, rank, seed: int, gen: int, p_c=1.0, p_m=None):
    """Tournament + uniform crossover + bit-flip mutation (N x d bits -> N x d)."""
    X = _f32(X)
    rank = _i32(rank)
    N, d = X.shape
    if p_m is None:
        p_m = float(np.float32(1.0) / np.float32(d))
    Xc = np.zeros_like(X)
    _load().orc_kp_vary(_p(X), _p(rank), N, d, seed, gen, float(p_c), float(p_m), _p(Xc))
    return Xc


def kp_generation(X, F, rank, profit, weight, cap, order, Z, seed: int, gen: int, p_c=1.0, p_m=None):
    """One knapsack generation on copies; returns (X, F, rank)."""
    X, F, rank = _f32(X).copy(), _f32(F).copy(), _i32(rank).copy()
    profit, weight, cap, order, Z = _i32(profit), _i32(weight), _i32(cap), _i32(order), _f64(Z)
    N, d = X.shape
    m = F.shape[1]
    if p_m is None:
        p_m = float(np.float32(1.0) / np.float32(d))
    rc = _load().orc_kp_generation(_p(X), _p(F), _p(rank), N, d, m, _p(profit), _p(weight), _p(cap),
                                   _p(order), _p(Z), Z.shape[0], seed, gen, float(p_c), float(p_m))
    if rc != OK:
        raise ValueError("orc_kp_generation failed (rc=%d)" % rc)
    return X, F, rank


def kp_run(N: int, d: int, profit, weight, cap, Z, seed: int, generations: int, p_c=1.0, p_m=None):
    """Init + repair/evaluate + ranks 0, then `generations` knapsack generations."""
    profit, weight, cap = _i32(profit), _i32(weight), _i32(cap)
    order = kp_order(profit, weight)
    m = profit.shape[0]
    if p_m is None:
        p_m = float(np.float32(1.0) / np.float32(d))
    X, F = kp_eval(kp_init(N, d, seed), profit, weight, cap, order)
    rank = np.zeros(N, dtype=np.int32)
    Z = _f64(Z)
    for g in range(generations):
        rc = _load().orc_kp_generation(_p(X), _p(F), _p(rank), N, d, m, _p(profit), _p(weight), _p(cap),
                                       _p(order), _p(Z), Z.shape[0], seed, g, float(p_c), float(p_m))
        if rc != OK:
            raise ValueError("orc_kp_generation failed (rc=%d)" % rc)
    return X, F, rank


def hv(P, ref) -> float:
    """Hypervolume (minimisation) of P inside the box below ref, exact for m = 2, 3."""
    P = _f32(P)
    ref = _f64(ref)
    v = float(_load().orc_hv(_p(P), P.shape[0], P.shape[1], _p(ref)))
    if v < 0:
        raise ValueError("hv: m must be 2 or 3")
    return v


def normalized_hv(P, fmin, fmax) -> float:
    """App. E: ref = 1.01 f_max, ideal = 0.9 f_min, HV / prod(ref - ideal)."""
    ref = 1.01 * _f64(fmax)
    ideal = 0.9 * _f64(fmin)
    return hv(P, ref) / float(np.prod(ref - ideal))


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB)
