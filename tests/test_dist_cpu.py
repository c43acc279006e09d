"""Host logic of bench.py's multi-rank mode on CPU (gloo, world_size 2).

Every GPU machine of this pool has one GPU, so N > 1 runs N independent replicas
(the workload is one system; ranks exchange nothing on the data path). What
must hold is the bookkeeping: a barrier before and after the timed region, the
time taken as the maximum over ranks, and the work summed over ranks. Two
processes check exactly that with the same helpers bench.py uses.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json, time
sys.path.insert(0, os.environ["NB_ROOT"])
import bench
import torch.distributed as dist
ws, rank = bench.dist_init("gloo")
assert ws == 2 and dist.is_initialized()
bench.dist_barrier()
local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
local_work = 100.0 * (rank + 1)
t = bench.dist_max(local_ms)
w = bench.dist_sum(local_work)
bench.dist_barrier()
print(json.dumps({"rank": rank, "max_ms": t, "sum_work": w}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_max_time_and_summed_work():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, NB_ROOT=ROOT, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out.strip().splitlines()[-1])
    import json
    rows = [json.loads(o) for o in outs]
    for r in rows:
        assert r["max_ms"] == 15.0          # the slower rank's time
        assert r["sum_work"] == 300.0       # all ranks' work


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 runs the CPU reference; rank 1 returns at once."""
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        args = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                "--steps", "1", "--warmup", "3", "--ref-t-end", "0.0009765625"]
        procs.append(subprocess.Popen(args, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=600)
        assert p.returncode == 0, err
        outs.append(out.strip())
    import json
    line = json.loads(outs[0].splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert outs[1] == ""
