"""bench.py's multi-rank logic on CPU (gloo, world size 2).

A replicas run on N GPUs reports the whole-job throughput from the slowest
rank's time (max over ranks), and only rank 0 prints.  Here two CPU processes
play the ranks: the combine and the throughput formula are checked on known
numbers, and the reference arm is run as rank 1 (silent) and rank 0 (one JSON
line).  No GPU is used.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [40.0, 50.0][rank]      # timed-region ms of each replica
        e2e = [0.9, 0.7][rank]       # end-to-end seconds of each replica
        got = bench.combine_ranks(ms, e2e, world, "cpu")
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump(list(got), f)
    finally:
        dist.destroy_process_group()


def test_combine_takes_the_slowest_rank(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        ms, e2e = json.load(open(tmp_path / f"r{r}.json"))
        assert ms == 50.0 and e2e == 0.9
    sys.path.insert(0, ROOT)
    import bench
    # 2 replicas x 30,720 unknowns x 10 steps in 50 ms
    assert bench.job_value(2, 30720, 10, 50.0) == pytest.approx(2 * 30720 * 10 / 0.05)
    assert bench.combine_ranks(3.0, 4.0, 1, "cpu") == (3.0, 4.0)


def _reference(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1", OMP_WAIT_POLICY="PASSIVE")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
           "lossy-sphere-480", "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.5"]
    return subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_only_rank0_prints():
    r1 = _reference(1, 2)
    assert r1.returncode == 0, r1.stderr
    assert r1.stdout.strip() == ""
    r0 = _reference(0, 2)
    assert r0.returncode == 0, r0.stderr
    lines = [ln for ln in r0.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
