"""The N > 1 host path of bench.py on CPU: two gloo ranks, no GPU.

The path shards as independent replicas (every rank matches its own volume,
no data-path collective); the only collective is the timing reduction: the
job's time is the slowest rank's, and the whole-job rate counts the units of
all ranks.  Under torchrun the reference arm runs on rank 0 alone."""

import json
import os
import socket
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
ms = [12.5, 20.0, 7.0, 15.0][rank]
t = bench.max_over_ranks(ms, dist, "cpu")
print(json.dumps(dict(rank=rank, t_max=t, rate=bench.job_rate(1000, 4, world, t))), flush=True)
dist.destroy_process_group()
"""


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _env(rank: int, world: int, port: int) -> dict:
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), REPO_ROOT=ROOT)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    return env


def test_slowest_rank_sets_the_job_time():
    world = 2
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", WORKER], env=_env(r, world, port),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(world)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    slowest = max([12.5, 20.0, 7.0, 15.0][:world])
    for o in outs:
        assert o["t_max"] == slowest
        # 1000 units per rank and step, 4 steps, every rank: per second of the slowest
        assert o["rate"] == pytest.approx(1000 * 4 * world / (slowest * 1e-3))


def test_single_process_needs_no_collective():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(10, 2, 1, 4.0) == pytest.approx(5000.0)


def test_reference_arm_runs_on_rank_zero_only():
    # rank 1 of 2 leaves without work and without output
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=_env(1, 2, _free_port()), capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
