"""Host logic of the multi-rank bench: replicas on two gloo ranks (CPU, no GPU).

Each rank runs its own independent copy of the workload; the job's time per step is the
maximum over ranks and the whole-job throughput counts every rank's cell updates.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank, world, local = bench.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=world)
bench.barrier(world)
t, v = bench.aggregate(1.0 + rank, world, 1000.0)   # rank r takes 1 + r seconds per step
m = bench.reduce_max(-3.5 * (rank + 1), world)
bench.barrier(world)
dist.destroy_process_group()
print(json.dumps({{"rank": rank, "t": t, "v": v, "m": m}}), flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(code, world, extra_env=None, timeout=120):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_replica_aggregation_two_ranks():
    outs = _launch(_CHILD.format(root=ROOT), 2)
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o in outs), key=lambda d: d["rank"])
    for d in res:
        assert d["t"] == 2.0                 # slowest rank
        assert d["v"] == 2 * 1000.0 / 2.0    # both ranks' units over the slowest time
        assert d["m"] == -3.5


def test_single_rank_aggregate_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(0.5, 1, 100.0) == (0.5, 200.0)
    assert bench.reduce_max(7.0, 1) == 7.0


def test_reference_arm_runs_on_rank_zero_only():
    # rank 1 of a two-rank reference run exits 0 at once and prints nothing
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
