"""bench.py's roofline bookkeeping on CPU: the dominance build's units are
the pairs the kernel reports testing (nsga3_get_dominance_stats), and the
committed ncu summaries it quotes describe the committed kernel source."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b
    return b


def test_dominance_roofline_counts_the_tested_pairs(bench):
    """frac = tested pairs x 2m compares / launch time / issue peak, with the
    tested pairs taken from stats[6]; the block-pair and live-pair fractions
    sit beside it."""
    from paper_2504_06067_gb300 import workloads as wl
    cfg = wl.LARGE
    n2 = 2 * cfg.N
    pairs = n2 * (n2 - 1) / 2
    domstat = [100.0, 10.0, 20.0, 0.0, 1.0, 5.0, 0.01 * pairs, 0.005 * pairs]
    probe = {"instr_per_s": 35.0e12}
    roof = bench.roofline_of(cfg, {"dominance": 1.0, "peel": 0.1}, 0.0, probe, {}, "measured", domstat)
    ops = 0.01 * pairs * 2 * cfg.m
    assert roof["bound"] == "alu"
    assert roof["achieved"] == pytest.approx(ops / 1e-3 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 35.0)
    assert roof["pairs_tested_frac"] == pytest.approx(0.01)
    assert roof["live_pairs_frac"] == pytest.approx(0.005)
    assert roof["block_pair_pairs_frac"] == pytest.approx(1024.0 * 31 / pairs)
    assert roof["block_pairs"]["zero"] == pytest.approx(100.0 / 131.0)


def test_committed_summaries_name_the_current_kernel(bench):
    """profiles/traffic.txt and profiles/issue.txt carry the dominance
    build's source hash; both resolve for the headline configuration, so
    the bench line quotes them (a kernel edit without a new capture shows up
    here before it turns the fields to null)."""
    src = os.path.join(ROOT, "paper_2504_06067_gb300", "csrc", "k_dominance.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for name in ("traffic.txt", "issue.txt"):
        lines = [l for l in open(os.path.join(ROOT, "profiles", name))
                 if l.startswith("k_dominance ")]
        assert lines and all(l.split()[3] == "k_dominance.cu:" + h for l in lines), name
    assert bench.ncu_traffic("k_dominance", "m10_N100000_d200_p3+2") > 0
    assert bench.ncu_issue_active("k_dominance")["value"] > 0
