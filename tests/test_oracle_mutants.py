"""Planted mistakes in the oracle (CPU only).

Each mutant is a copy of oracle/oracle.c with one plausible error planted by
a textual substitution: a flipped comparison, a dropped term, a transposed
operand, a wrong constant, exponent or index.  The copy is built with gcc
and the oracle pins (tests/test_oracle_pins.py) run against it in a child
process; every mutant must make at least one pin fail.  A control build of
the unmodified source must pass, so that a failing mutant means the pins
saw the mistake and not that the harness broke.  Nothing here touches the
CUDA library.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (name, text of oracle.c, planted replacement, occurrences of the text)
MUTANTS = [
    # Philox4x32-10 and the uniform / bounded draws
    ("philox_multiplier", "orc_mulhilo(0xD2511F53u, x0, &hi0, &lo0);",
     "orc_mulhilo(0xD2511F35u, x0, &hi0, &lo0);", 1),
    ("philox_weyl_constant", "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE58u;", 1),
    ("philox_output_word", "uint32_t y1 = lo1;", "uint32_t y1 = lo0;", 1),
    ("uniform_bits", "return (double)(w >> 8) * (1.0 / 16777216.0);",
     "return (double)(w >> 9) * (1.0 / 16777216.0);", 1),
    ("bounded_half_range", "return (uint32_t)(((uint64_t)w * (uint64_t)n) >> 32);",
     "return (uint32_t)(((uint64_t)w * (uint64_t)n) >> 33);", 1),
    # Das-Dennis directions (Sec. II-C)
    ("das_dennis_step", "double z = (double)k[r] / (double)p;",
     "double z = (double)k[r] / (double)(p + 1);", 1),
    ("das_dennis_inner_centroid", "double a = (1.0 - tau) / (double)m;",
     "double a = (1.0 - tau) / (double)(m - 1);", 1),
    # dominance (Eq. 1) and the non-dominated sort
    ("dominance_not_strict", "if (x < y) any_lt = 1;", "if (x <= y) any_lt = 1;", 1),
    ("dominance_maximises", "if (!(x <= y)) all_le = 0;", "if (!(x >= y)) all_le = 0;", 1),
    ("last_front_off_by_one", "if (l < 0 && cum >= N) l = k;", "if (l < 0 && cum > N) l = k;", 1),
    ("front_sweep_clears_count",
     "if (orc_dominates(F + (size_t)front[t] * m, F + (size_t)j * m, m)) cnt[j]--;",
     "if (orc_dominates(F + (size_t)front[t] * m, F + (size_t)j * m, m)) cnt[j] = 0;", 1),
    ("dominator_count_one_sided", "for (int i = 0; i < n2; ++i)\n            if (orc_dominates(",
     "for (int i = 0; i < j; ++i)\n            if (orc_dominates(", 1),
    ("das_dennis_no_inner_layer", "if (p2 > 0) orc_dd_rec(m, p2, 0, p2, k, Z, &row, 1, tau);", "", 1),
    # normalization
    ("asf_weights_swapped", "double wq = (r == q) ? 1.0 : 1e-6;",
     "double wq = (r == q) ? 1e-6 : 1.0;", 2),
    ("extremes_not_translated", "AQ(q, r) = (double)F[(size_t)extremes[q] * m + r] - zstar[r];",
     "AQ(q, r) = (double)F[(size_t)extremes[q] * m + r];", 1),
    ("pivot_swap_misses_rhs", "double t = rhs[c]; rhs[c] = rhs[p]; rhs[p] = t;", "", 2),
    ("elimination_factor_transposed", "double factor = AQ(r, c) / AQ(c, c);",
     "double factor = AQ(c, r) / AQ(c, c);", 2),
    ("back_substitution_transposed", "double prod = AQ(r, cc) * b[cc];",
     "double prod = AQ(cc, r) * b[cc];", 2),
    ("intercept_not_inverted", "a[q] = 1.0 / b[q];", "a[q] = b[q];", 2),
    ("fallback_zero_span", "a[q] = (mx == 0.0) ? 1.0 : mx;", "a[q] = mx;", 2),
    # normalization with history
    ("history_not_kept", "*hvalid = 1;", "*hvalid = 0;", 1),
    ("history_ideal_restarts", "for (int q = 0; q < m; ++q) zstar[q] = *hvalid ? hz[q] : INFINITY;",
     "for (int q = 0; q < m; ++q) zstar[q] = INFINITY;", 1),
    ("history_vectors_ignored", "const int ncand = n2 + (*hvalid ? m : 0);", "const int ncand = n2;", 1),
    # association (Eq. 2)
    ("cosine_not_squared", "double cc = c * c;", "double cc = c;", 1),
    ("point_not_normalised", "fp[q] = ft / a[q];", "fp[q] = ft;", 1),
    ("direction_norm_squared", "nz[j] = sqrt(s);", "nz[j] = s;", 1),
    ("association_last_minimum", "if (D < best) { best = D; arg = j; }",
     "if (D <= best) { best = D; arg = j; }", 1),
    # niching (Alg. 1 loop and Alg. 2 cached loop)
    ("niche_farthest_member", "if (t < 0 || dist[i] < dist[t]) t = i;",
     "if (t < 0 || dist[i] > dist[t]) t = i;", 2),
    ("niche_largest_count", "if (v < 0 || rho[j] < rho[v] ||", "if (v < 0 || rho[j] > rho[v] ||", 1),
    ("niche_member_priority_max", "if (t < 0 || pr < bp) { t = i; bp = pr; }",
     "if (t < 0 || pr > bp) { t = i; bp = pr; }", 1),
    ("batched_first_batch_unsorted", "orc_sort_batch(B, nb, rprio);\n    int keep = nb < K ? nb : K;",
     "int keep = nb < K ? nb : K;", 1),
    ("batched_queue_reversed", "while (y >= lo && (mprio[Q[y]] > mprio[v] ||",
     "while (y >= lo && (mprio[Q[y]] < mprio[v] ||", 1),
    ("selection_one_short", "int K = N - nS;", "int K = N - nS - 1;", 1),
    # variation (Sec. III-A): tournament, SBX, polynomial mutation
    ("tournament_prefers_worse", "uint32_t p1 = rank[b1] < rank[a1] ? b1 : a1;",
     "uint32_t p1 = rank[b1] > rank[a1] ? b1 : a1;", 2),
    ("sbx_children_equal", "c2 = 0.5 * ((1.0 - beta) * x1 + (1.0 + beta) * x2);",
     "c2 = 0.5 * ((1.0 + beta) * x1 + (1.0 - beta) * x2);", 1),
    ("sbx_spread_exponent", "double e = 1.0 / (eta_c + 1.0);", "double e = 1.0 / eta_c;", 1),
    ("sbx_upper_branch", "pow(1.0 / (2.0 * (1.0 - u)), e)", "pow(1.0 / (2.0 * u), e)", 1),
    ("mutation_upper_sign", "dq = 1.0 - pow(val, mp);", "dq = pow(val, mp) - 1.0;", 1),
    ("sbx_never_swapped", "if ((float)orc_uniform(s[2]) < 0.5f) { double tt = c1; c1 = c2; c2 = tt; }",
     "", 1),
    ("mutation_lower_distance", "double xy = 1.0 - d1;", "double xy = 1.0 - d2;", 1),
    # objective
    ("softmax_not_divided", "double sj = e[j] / den;", "double sj = e[j];", 1),
    ("softmax_without_exp", "e[j] = exp(s);", "e[j] = s;", 1),
    ("distance_not_centred", "double t = (double)x[v] - 0.5;", "double t = (double)x[v];", 1),
    ("distance_skips_first", "for (int v = k; v < d; ++v) {", "for (int v = k + 1; v < d; ++v) {", 1),
    ("weights_transposed", "double pr = (double)W[j * k + v] * (double)x[v];",
     "double pr = (double)W[v * m + j] * (double)x[v];", 1),
    # 0-1 knapsack
    ("repair_order_reversed", "if (na * db != nb * da) return na * db < nb * da;",
     "if (na * db != nb * da) return na * db > nb * da;", 1),
    ("repair_at_capacity", "if (load[j] > cap[j]) over = 1;", "if (load[j] >= cap[j]) over = 1;", 1),
    ("knapsack_objective_taken", "if (x[v] == 0.0f) left += p[(size_t)j * d + v];",
     "if (x[v] != 0.0f) left += p[(size_t)j * d + v];", 1),
    ("bit_set_not_flipped", "if ((float)orc_uniform(pm[0]) < p_m) c1 = 1.0f - c1;",
     "if ((float)orc_uniform(pm[0]) < p_m) c1 = 1.0f;", 1),
    ("uniform_crossover_missing",
     "if (cross && (float)orc_uniform(s[0]) < 0.5f) { float tt = c1; c1 = c2; c2 = tt; }", "", 1),
    ("knapsack_init_biased", "X[(size_t)i * d + v] = ((float)orc_uniform(o[0]) < 0.5f) ? 1.0f : 0.0f;",
     "X[(size_t)i * d + v] = ((float)orc_uniform(o[0]) < 0.25f) ? 1.0f : 0.0f;", 1),
    # indicators
    ("hv_full_height", "area += (ref[0] - x) * (best - y);", "area += (ref[0] - x) * (ref[1] - y);", 1),
    ("igd_squared", "acc = acc + sqrt(best);", "acc = acc + best;", 1),
    ("hv_slice_height", "double top = ref[2];", "double top = lev[t];", 1),
    ("igd_over_population", "return nr > 0 ? acc / (double)nr : 0.0;",
     "return nr > 0 ? acc / (double)np : 0.0;", 1),
]


def _build(text, out_dir, name):
    c = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, name + ".so")
    with open(c, "w") as fh:
        fh.write(text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-o", so, c, "-lm"], check=True, capture_output=True)
    return so


def _run_pins(so):
    # one BLAS thread per child: the children already run side by side
    env = dict(os.environ, NSGA3_ORACLE_LIB=so, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, (r.stdout + r.stderr)[-1500:]


def test_mutants_apply_once():
    text = open(SRC).read()
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, old, new, count in MUTANTS:
        assert text.count(old) == count, name
        assert old != new, name


@pytest.mark.slow
def test_planted_mistakes_fail_the_pins(orc, tmp_path):
    text = open(SRC).read()
    jobs = [("control", text)] + [(name, text.replace(old, new)) for name, old, new, _ in MUTANTS]

    def one(job):
        name, src = job
        return name, _run_pins(_build(src, str(tmp_path), name))

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        res = dict(ex.map(one, jobs))
    rc, out = res.pop("control")
    assert rc == 0, out
    # pytest exits 1 when a test failed; anything else (a crash, an
    # interrupted run) would not show that a pin caught the mistake
    survivors = {name: r for name, r in res.items() if r[0] != 1}
    assert not survivors, "mutants not caught: %s" % sorted(survivors)
