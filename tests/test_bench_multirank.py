"""Multi-rank host logic of bench.py on CPU: two gloo ranks under
torch.distributed.run (the launcher the GPU runs use), and the weak-scaling
shards of the headline workload."""
import json
import os
import socket
import subprocess
import sys

import numpy as np

import bench
from paper_2007_15385_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_report_the_slowest_rank_time():
    env = dict(os.environ)
    env.pop("WORLD_SIZE", None)
    env.pop("RANK", None)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "tests", "multirank_probe.py")]
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, "only rank 0 prints"
    r = json.loads(lines[0])
    assert r["world"] == 2
    assert sorted(s["rank"] for s in r["seen"]) == [0, 1]
    assert all(s["slowest"] == 15.0 for s in r["seen"])
    # 1e9 units per rank, two ranks, 15 ms: 2e9 / 0.015 s = 133.3 G units/s
    assert abs(r["rate"] - 2e9 / 0.015 / 1e9) < 1e-9


def test_single_rank_helpers():
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.whole_job_rate(5e8, 1, 10.0) == 50.0
    assert bench.whole_job_rate(5e8, 4, 10.0) == 200.0


def test_shards_share_the_footprint_but_not_the_points():
    a = wl.vehicle_footprint(m=2000)
    a0 = wl.vehicle_footprint(m=2000, shard=0)
    b = wl.vehicle_footprint(m=2000, shard=1)
    c = wl.vehicle_footprint(m=2000, shard=2)
    np.testing.assert_array_equal(a.vertices, a0.vertices)
    np.testing.assert_array_equal(a.points, a0.points)
    np.testing.assert_array_equal(a.vertices, b.vertices)
    np.testing.assert_array_equal(a.vertices, c.vertices)
    assert not np.array_equal(a.points, b.points)
    assert not np.array_equal(b.points, c.points)


def test_cpu_baseline_reports_one_thread_all_cores_and_plain_fp64():
    w = wl.vehicle_footprint(m=1 << 14)
    r = bench.cpu_baseline_run(w, 1 << 13)
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["value"] > 0
    assert r["all_cores"]["cores"] == (os.cpu_count() or 1) and r["all_cores"]["value"] > 0
    assert r["plain_fp64_alg5"]["cores"] == 1 and r["plain_fp64_alg5"]["value"] > 0
    assert isinstance(r["cpu_model"], str) and r["cpu_model"]
