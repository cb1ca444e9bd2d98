"""The multi-process path of bench.py on the host: one process per rank
(gloo on 127.0.0.1, world size 2). The plain build is replicated, each rank
on its own seeded input, and the job's time is the slowest rank's."""
from __future__ import annotations

import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, values, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(values[rank], dist, torch.device("cpu"))
    finally:
        dist.destroy_process_group()


def test_the_job_time_is_the_slowest_ranks():
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    values = [12.5, 71.25]
    mp.start_processes(_rank_main, args=(2, _free_port(), values, out), nprocs=2, start_method="spawn")
    assert dict(out) == {0: 71.25, 1: 71.25}


def test_without_a_process_group_the_value_is_kept():
    import bench
    assert bench.max_over_ranks(3.5, None, torch.device("cpu")) == 3.5


def test_each_rank_builds_its_own_seeded_input():
    import bench
    s0, kw0 = bench.workload("c3", 0)
    s1, kw1 = bench.workload("c3", 1)
    assert (s0.n, s0.d, s0.r, kw0) == (s1.n, s1.d, s1.r, kw1)
    assert s0.seed != s1.seed and s0.sid_seed != s1.sid_seed


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_prints_its_line_on_rank_zero():
    """The reference arm at N = 1 (the oracle on the host cores, a bounded
    sample of the small profiling workload): one JSON line carrying the arm's
    name, the metric, a cpu_baseline record with the line's value, and an
    end-to-end record with no host-device copies."""
    import json
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c3s",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["n_gpus"] == 1 and j["steps"] == 1 and j["warmup"] == 3
    assert j["metric"] == "build points×levels/s" and j["unit"] == "points*levels/s"
    assert j["higher_is_better"] is True and j["value"] > 0
    assert j["config"]["workload"].startswith("plain_studentt_n4194304_d8")
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == j["value"]
    e = j["e2e"]
    assert e["value"] == j["value"] and e["unit"] == j["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
