"""The N > 1 path of the benchmark (replicas: each rank runs its own copy of
the workload, no collective on the data path; the slowest rank's timed region
counts) on CPU: two gloo ranks over 127.0.0.1, and the reference arm's rank
rule (rank 0 alone works and prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # the ranks' timed regions differ; every rank must see the slowest
    slowest = bench.max_over_ranks(10.0 + 7.5 * rank, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump({"slowest_ms": slowest,
                   "rate": bench.whole_job_rate(1000, world, slowest / 1e3)}, f)


def test_two_gloo_ranks_take_the_slowest_region(tmp_path):
    port = _free_port()
    torch.multiprocessing.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    for g in got:
        assert g["slowest_ms"] == 17.5
        assert abs(g["rate"] - 2 * 1000 / 0.0175) < 1e-6


def test_reference_arm_rank_rule():
    """--impl reference: rank 0 runs the oracle and prints one JSON line;
    other ranks exit 0 without work or output."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "smooth",
           "--steps", "2", "--warmup", "1"]
    env1 = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r1 = subprocess.run(cmd, env=env1, capture_output=True, text=True, timeout=300)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    env0 = dict(os.environ, RANK="0", WORLD_SIZE="2")
    r0 = subprocess.run(cmd, env=env0, capture_output=True, text=True, timeout=300)
    assert r0.returncode == 0, r0.stderr[-2000:]
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
