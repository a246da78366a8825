"""Seeded synthetic inputs shared by tests, bench.py and smoke().

This module holds no arithmetic of the selection method or of variation:
it only draws numbers (numpy's PCG64 generator) and lays them out in the
shapes of the workloads.  The paper's own workloads (DTLZ, MNK-landscape,
MOKnapsack, Brax, Sec. IV) are not available here; the softmax-simplex
family below stands in for them with the same shape parameters (m
objectives, d variables, population N, Das-Dennis divisions p).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class RunConfig:
    """One plain NSGA-III run: m objectives, d variables, population N."""
    name: str
    m: int
    d: int
    N: int
    p1: int          # outer Das-Dennis divisions
    p2: int = 0      # inner layer divisions (0 = single layer)
    tau: float = 0.5  # inner layer shrink factor
    generations: int = 100
    seed: int = 0

    @property
    def w(self) -> int:
        w = math.comb(self.p1 + self.m - 1, self.m - 1)
        if self.p2 > 0:
            w += math.comb(self.p2 + self.m - 1, self.m - 1)
        return w


# Plain single run, small: m=3, p=12 (91 directions), N=92, d=12, 100 generations.
SMALL = RunConfig("m3_N92_d12_p12", m=3, d=12, N=92, p1=12, generations=100)
# Plain single run at scale: m=5, p=20 (10,626 directions), N=10,628, d=100, 500 generations.
SCALE = RunConfig("m5_N10628_d100_p20", m=5, d=100, N=10628, p1=20, generations=500)
# Large population: m=10, two layers p1=3 + p2=2 (tau 0.5; 275 directions), N=100,000, d=200.
LARGE = RunConfig("m10_N100000_d200_p3+2", m=10, d=200, N=100000, p1=3, p2=2, tau=0.5,
                  generations=200)
# Beyond the dominance matrix (streaming only): m=10, N = 1,000,000 (merged
# 2N = 2,000,000 would need a 500 GB matrix), same directions as LARGE.
HUGE = RunConfig("m10_N1000000_d200_p3+2", m=10, d=200, N=1000000, p1=3, p2=2, tau=0.5,
                 generations=20)
PLAIN_CONFIGS = (SMALL, SCALE, LARGE)
# 0-1 knapsack workload (binary variables): m = 3 knapsacks, d = 500 items,
# N = 12,800 (the largest population of the paper's discrete runs), p = 158
# (12,720 directions).
KNAPSACK = RunConfig("kp_m3_N12800_d500_p158", m=3, d=500, N=12800, p1=158, generations=100)


# Objective sweep in the shape of the paper's Table II (N = 800, d = 1000,
# m = 4 ... 512; its runs use DTLZ3, here the softmax-simplex objective):
# single-layer Das-Dennis directions with the largest p whose set fits N.
SWEEP_M = (4, 8, 16, 32, 64, 128, 256, 512)


def objective_sweep(N: int = 800, d: int = 1000, generations: int = 100):
    return [RunConfig("sweep_m%d_N%d_d%d_p%d" % (m, N, d, largest_p(m, N)), m=m, d=d, N=N,
                      p1=largest_p(m, N), generations=generations) for m in SWEEP_M]


# Population sweep in the shape of the paper's Table I (m = 6, d = 500,
# N = 50 ... 12,800; its runs use DTLZ3, here the softmax-simplex objective).
POP_SWEEP_N = (50, 100, 200, 400, 800, 1600, 3200, 6400, 12800)


def population_sweep(m: int = 6, d: int = 500, generations: int = 100):
    return [RunConfig("popsweep_m%d_N%d_d%d_p%d" % (m, N, d, largest_p(m, N)), m=m, d=d, N=N,
                      p1=largest_p(m, N), generations=generations) for N in POP_SWEEP_N]


def knapsack_instance(m: int, d: int, seed: int = 0):
    """Integer profits and weights uniform in [10, 100] (m x d) and capacities
    of half the total weight per knapsack: the usual random 0-1 multi-
    objective knapsack instance.  Returns (profit, weight, capacity) int32."""
    rng = np.random.default_rng([seed, 13, m, d])
    profit = rng.integers(10, 101, size=(m, d)).astype(np.int32)
    weight = rng.integers(10, 101, size=(m, d)).astype(np.int32)
    capacity = (weight.astype(np.int64).sum(axis=1) // 2).astype(np.int32)
    return profit, weight, capacity


def objective_weights(m: int, seed: int) -> np.ndarray:
    """W ~ N(0,1), m x (m-1), FP32: the parameters of the softmax-simplex problem."""
    rng = np.random.default_rng([seed, 7, m])
    return rng.standard_normal((m, m - 1)).astype(np.float32)


def front_sample(m: int, n: int = 10000, seed: int = 2**32 - 1) -> np.ndarray:
    """y ~ U[0,1]^(m-1): the decision points whose images sample the true front."""
    rng = np.random.default_rng([seed, 8, m])
    return rng.random((n, m - 1))


def largest_p(m: int, N: int) -> int:
    """Largest single-layer p with C(p+m-1, m-1) <= N (w close to n, Sec. II-C)."""
    p = 1
    while math.comb(p + 1 + m - 1, m - 1) <= N:
        p += 1
    return p


def batched_configs(n_runs: int = 64, seed: int = 0, generations: int = 300):
    """Uneven independent runs: N log-uniform in [100, 20000] (multiple of 4),
    m in {3, 5, 8}, d = m + 19, seeds 0..n_runs-1."""
    rng = np.random.default_rng([seed, 9])
    out = []
    for r in range(n_runs):
        N = int(math.exp(rng.uniform(math.log(100), math.log(20000))))
        N = (N + 3) // 4 * 4
        m = int(rng.choice([3, 5, 8]))
        out.append(RunConfig("batch%02d" % r, m=m, d=m + 19, N=N, p1=largest_p(m, N),
                             generations=generations, seed=r))
    return out


def served_requests(n_req: int = 2000, rate_hz: float = 40.0, seed: int = 0,
                    n_max: int = 50000, gens_max: int = 1000):
    """Poisson arrivals of run requests: N log-uniform [100, n_max], m in 3..10,
    generations uniform [50, gens_max], d = m + 29, request i has seed i."""
    rng = np.random.default_rng([seed, 10])
    t = 0.0
    out = []
    for i in range(n_req):
        t += rng.exponential(1.0 / rate_hz)
        N = int(math.exp(rng.uniform(math.log(100), math.log(n_max))))
        N = (N + 3) // 4 * 4
        m = int(rng.integers(3, 11))
        g = int(rng.integers(50, gens_max + 1))
        out.append((t, RunConfig("req%04d" % i, m=m, d=m + 29, N=N, p1=largest_p(m, N),
                                 generations=g, seed=i)))
    return out


# ------------------------------------------------ objective matrices --------
def objectives(kind: str, n2: int, m: int, seed: int = 0) -> np.ndarray:
    """2N x m FP32 objective matrices with the structures the selection meets.

    kind:
      "early"      points near a scaled simplex with a wide spread of the
                   distance factor: many fronts (first generations);
      "late"       points close to the unit simplex: one or two large fronts;
      "uniform"    i.i.d. U[0,1] in every objective;
      "simplex"    exactly on a simplex with distinct points: a single front;
      "chain"      a totally ordered chain: one member per front;
      "equal"      all rows identical: a single front of size 2N;
      "dups"       few distinct rows repeated many times, with ties per column;
      "grid"       small integer grid values: many exact ties;
      "signedzero" rows mixing -0.0 and +0.0 and equal values.
    """
    rng = np.random.default_rng([seed, n2, m, sum(map(ord, kind))])
    if kind == "early":
        s = rng.dirichlet(np.ones(m), size=n2)
        g = 1.0 + rng.gamma(2.0, 2.0, size=(n2, 1))
        F = s * g
    elif kind == "late":
        s = rng.dirichlet(np.ones(m), size=n2)
        g = 1.0 + rng.exponential(0.01, size=(n2, 1))
        F = s * g
    elif kind == "uniform":
        F = rng.random((n2, m))
    elif kind == "simplex":
        F = rng.dirichlet(np.ones(m), size=n2)
        F = F / F.sum(axis=1, keepdims=True)
    elif kind == "chain":
        base = rng.random(m)
        step = rng.random(m) + 0.1
        order = rng.permutation(n2)
        F = base[None, :] + order[:, None] * step[None, :]
    elif kind == "equal":
        F = np.tile(rng.random(m), (n2, 1))
    elif kind == "dups":
        k = max(2, n2 // 16)
        pool = rng.integers(0, 5, size=(k, m)).astype(np.float64)
        F = pool[rng.integers(0, k, size=n2)]
    elif kind == "grid":
        F = rng.integers(0, 4, size=(n2, m)).astype(np.float64)
    elif kind == "signedzero":
        F = rng.integers(0, 3, size=(n2, m)).astype(np.float64) - 1.0
        F[F == 0.0] = np.where(rng.random(np.sum(F == 0.0)) < 0.5, -0.0, 0.0)
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(F, dtype=np.float32)


KINDS = ("early", "late", "uniform", "simplex", "chain", "equal", "dups", "grid", "signedzero")


def population(N: int, d: int, seed: int = 0) -> np.ndarray:
    """N x d decision vectors, U[0,1], FP32."""
    rng = np.random.default_rng([seed, N, d, 11])
    return rng.random((N, d), dtype=np.float32)


def parent_ranks(N: int, n_fronts: int, seed: int = 0) -> np.ndarray:
    """Front indices in [0, n_fronts) for N parents."""
    rng = np.random.default_rng([seed, N, 12])
    return rng.integers(0, n_fronts, size=N).astype(np.int32)
