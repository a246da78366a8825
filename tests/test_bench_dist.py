"""bench.py's multi-rank bookkeeping on CPU: two gloo ranks, a barrier, the
max-over-ranks time and the whole-job rate (N GPUs are replicas: units of
every rank over the slowest rank's time)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_env()
    dist = bench.dist_init(w, "gloo")
    bench.barrier(dist)
    rate, tmax = bench.job_rate(dist, w, 1000, 1.0 + r, "cpu")
    q.put((r, w, rate, tmax))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    ps = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, rate, tmax in res:
        assert w == 2 and tmax == 2.0 and rate == 2 * 1000 / 2.0


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1, "gloo") is None
    assert bench.job_rate(None, 1, 50, 2.0) == (25.0, 2.0)


def test_reference_arm_line_on_cpu():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the contract's keys; no GPU is involved."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "small", "--steps", "2", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "sols/s"
    assert line["steps"] == 2 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"] == "m3_N92_d12_p12"


def test_default_workload_is_the_large_configuration():
    """With no flags bench.py measures m = 10, N = 100,000 (the largest
    single-GPU configuration), and the reference arm times the oracle on that
    same configuration with the same config keys."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2504_06067_gb300 import workloads as wl
    args = bench.parse_args([])
    assert args.workload == "headline" and args.warmup >= 3
    assert bench.reference_cfg(args) is wl.LARGE
    assert bench.cfg_dict(wl.LARGE)["workload"] == "m10_N100000_d200_p3+2"
    assert wl.LARGE.N == 100000 and wl.LARGE.m == 10 and wl.LARGE.generations == 200
