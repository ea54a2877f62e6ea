"""The multi-process path of the benchmark on the CPU: two gloo ranks, as torchrun launches them on one node.

The path shards into independent replicas (one block per GPU, no data-path collective); the only cross-rank
operations are the timing barrier and the max-reduce of the elapsed time, from which rank 0 reports the
whole-job rate.  The reference arm runs on rank 0 alone; the other ranks exit without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, sys
sys.path.insert(0, ROOT_DIR)
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
world, rank, local = bench.dist_env()
bench.barrier(world)
ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)
print(json.dumps({"rank": rank, "world": world, "ms": ms, "rate": bench.replica_rate(world, 1000, 2, ms)}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    return dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")


def test_two_ranks_take_the_slowest_time_and_sum_the_replicas():
    port = _free_port()
    code = WORKER.replace("ROOT_DIR", repr(ROOT))
    procs = [subprocess.Popen([sys.executable, "-c", code], env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, cwd=ROOT) for r in range(2)]
    outs = [p.communicate(timeout=180) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err[-2000:]
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o, _ in outs), key=lambda d: d["rank"])
    assert [d["rank"] for d in res] == [0, 1]
    for d in res:
        assert d["world"] == 2 and d["ms"] == 15.0  # the slower rank's time
        assert d["rate"] == pytest.approx(2 * 1000 * 4 * 2 / 15e-3)


def test_reference_arm_runs_on_rank_zero_only():
    port = _free_port()
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--n", "16", "--steps", "1", "--warmup", "0"]
    r1 = subprocess.run(cmd, env=_env(1, 2, port), capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r1.returncode == 0 and r1.stdout.strip() == "", r1.stderr[-2000:]
    r0 = subprocess.run(cmd, env=_env(0, 2, port), capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r0.returncode == 0, r0.stderr[-2000:]
    d = json.loads(r0.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "zone-updates/s"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
