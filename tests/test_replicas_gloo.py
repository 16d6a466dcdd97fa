"""The N>1 bench path on CPU: two gloo ranks stand in for two GPUs.

A heap belongs to one device, so N GPUs run N independent replicas (weak
scaling): each rank draws its own seeded batch and times it; the whole-job
value is every rank's operations over the slowest rank's time.  These tests
check that host logic (seeds, max over ranks, aggregation) and that the
reference arm prints on rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist

    import bench
    from paper_2504_18211_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        sizes = W.sweep_sizes(4096, seed=bench.replica_seed(rank))
        local_ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        total = bench.max_over_ranks(dist, local_ms, "cpu")
        value = bench.whole_job_value(ws, 4, 2 * sizes.size, total)
        q.put((rank, sizes.tobytes(), total, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_whole_job_value():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(ws):
        rank, sz, total, value = q.get(timeout=120)
        got[rank] = (np.frombuffer(sz, np.uint32), total, value)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s0, s1 = got[0][0], got[1][0]
    assert s0.size == s1.size == 4096
    assert not np.array_equal(s0, s1)                      # each replica its own requests
    for rank in range(ws):
        assert got[rank][1] == 15.0                        # the slowest rank's time, on every rank
        # 2 ranks x 4 steps x 8192 ops over 15 ms
        assert got[rank][2] == pytest.approx(2 * 4 * 8192 / 15e-3 / 1e6)


def test_replica_seeds_and_single_process_identity():
    import bench
    from paper_2504_18211_gb300 import workloads as W
    assert bench.replica_seed(0) == W.SEED_BASE + 1        # rank 0 runs the single-GPU workload
    assert len({bench.replica_seed(r) for r in range(8)}) == 8
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.whole_job_value(1, 20, 2 << 20, 1000.0) == pytest.approx(20 * (2 << 20) / 1e6)


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line():
    pytest.importorskip("numpy")
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    # the line states what ran: the headline workload itself, on a stated host
    cfg, cb = line["config"], line["cpu_baseline"]
    assert cfg["threads"] == 1 << 20 and cfg["heap_bytes"] == 8 << 30 and cfg["chunk_bytes"] == 8192
    assert cb["host_cpus"] == os.cpu_count() and cb["cpu_model"] and cb["cores"] == 1
    assert "1048576 requests" in cb["sample"] and "pinned to core" in cb["sample"]
