"""The multi-rank logic of bench.py on CPU: two gloo ranks, max-over-ranks
timing, whole-job throughput, and the reference arm running on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
value = bench.job_throughput(1000, world, ms / 2)
print(json.dumps({"rank": rank, "ms": ms, "value": value}), flush=True)
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_rank():
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    import json
    lines = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    for d in lines:
        assert d["ms"] == 15.0  # the slower rank's time on every rank
        assert d["value"] == pytest.approx(2 * 1000 / (7.5 / 1e3))


def test_reference_arm_prints_on_rank_zero_only():
    base = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "c0", "--steps", "1",
            "--warmup", "0"]
    for rank, expect_line in ((1, False), (0, True)):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2")
        r = subprocess.run(base + ["--gpus", "2"], env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        out = [l for l in r.stdout.splitlines() if l.startswith("{")]
        assert bool(out) == expect_line
        if out:
            import json
            d = json.loads(out[0])
            assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
