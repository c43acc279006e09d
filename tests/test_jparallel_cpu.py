"""The j-parallel block step of Sect. 3 (its Flowchart) across two gloo ranks on CPU.

paper_0711_0643_gb300/jparallel.py drives the step: every rank holds the whole system,
rank g sums the block's forces over its share of j, the partial forces are all-gathered
and added in rank order, and every rank corrects identically. Here its block-step
operations are the oracle stand-in of tests/jp_oracle_ops.py (there is no GPU on CPU
ranks). Workload: Plummer N = 1024 (the C1 initial conditions), 16 block steps.
  * Both ranks end with bitwise identical states and schedules (replicated correction).
  * The two-rank run selects the same blocks (t_next, s, active list) as the one-rank run
    for all 16 steps, with forces within 1e-12 of its forces (FP64 partial sums).
  * A second two-rank run is bitwise identical to the first (sums in rank order).
  * The shares of j are whole tiles and cover [0, n) without overlap, for several p.
A rank whose replica diverges is reported by the driver's per-step agreement check: a
rank made to start from a perturbed state raises on both ranks. Perturber lists of binaries
(Sect. 3.1) found per share and merged in rank order equal the serial scan's.
"""
import json
import os
import socket
import subprocess
import sys
import zlib

import numpy as np
import pytest

import ics

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json, zlib
sys.path.insert(0, os.environ["NB_ROOT"])
import numpy as np
import torch.distributed as dist
import ics, oracle
from tests.jp_oracle_ops import OracleOps
from paper_0711_0643_gb300.jparallel import JParallel
dist.init_process_group("gloo")
rank = dist.get_rank()
if os.environ.get("NB_PERTLIST"):
    snap = ics.plummer_binaries(1024, 100, 20071106 + 48, 1.0 / 256, a_lo=1e-3, a_hi=3e-2)
    jp = JParallel(OracleOps(oracle, snap))
    lists, counts = jp.perturbers(snap.meta["pairs"], gamma=1e-7, nmax=32)
    print(json.dumps({"lists": lists.tolist(), "counts": counts.tolist(), "j": [jp.j0, jp.j1]}))
    dist.destroy_process_group()
    sys.exit(0)
ops = OracleOps(oracle, ics.config(1))
if os.environ.get("NB_PERTURB") and rank == 1:
    ops.st["dt"] *= 0.5             # this replica's schedule differs from rank 0's
jp = JParallel(ops)
rows, forces = [], []
try:
    for _ in range(16):
        tn, s = jp.step()
        rows.append([tn, s, zlib.crc32(np.ascontiguousarray(ops.idx, dtype=np.int32).tobytes())])
        forces.append(ops.last_forces.tolist())
    out = {"rows": rows, "j": [jp.j0, jp.j1], "forces": forces,
           "state": {k: v.tolist() for k, v in ops.st.items()}}
except RuntimeError as e:
    out = {"error": str(e)}
print(json.dumps(out))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _two_ranks(perturb=False, pertlist=False):
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, NB_ROOT=ROOT, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
        if perturb:
            env["NB_PERTURB"] = "1"
        if pertlist:
            env["NB_PERTLIST"] = "1"
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=600)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    return outs


def _one_rank(orc):
    from tests.jp_oracle_ops import OracleOps
    from paper_0711_0643_gb300.jparallel import JParallel
    ops = OracleOps(orc, ics.config(1))
    jp = JParallel(ops)
    assert jp.world == 1 and (jp.j0, jp.j1) == (0, 1024)
    rows, forces = [], []
    for _ in range(16):
        tn, s = jp.step()
        rows.append([tn, s, zlib.crc32(np.ascontiguousarray(ops.idx, dtype=np.int32).tobytes())])
        forces.append(ops.last_forces)
    return rows, forces


def test_two_ranks_match_one_rank_and_rerun(orc):
    pytest.importorskip("torch")
    a = _two_ranks()
    b = _two_ranks()
    ref_rows, ref_forces = _one_rank(orc)
    assert a[0]["j"] == [0, 512] and a[1]["j"] == [512, 1024]
    for key in ("m", "x", "v", "a", "k", "t", "dt"):
        assert a[0]["state"][key] == a[1]["state"][key], key          # replicas identical
        assert a[0]["state"][key] == b[0]["state"][key], key          # rerun identical
    assert a[0]["rows"] == a[1]["rows"] == b[0]["rows"]
    assert a[0]["rows"] == ref_rows                                    # same blocks as one rank
    for f2, f1 in zip(a[0]["forces"], ref_forces):
        f2 = np.array(f2)
        scale = np.abs(f1).max(axis=0)
        assert np.all(np.abs(f2 - f1) <= 1e-12 * scale), np.abs(f2 - f1).max()


def test_two_rank_perturber_lists_are_the_serial_lists(orc):
    """Sect. 3.1: each rank finds the perturbers in its share of the stars; the lists merged
    in rank order and cut at N_pert are the serial scan's lists on both ranks, counts summed
    (Plummer N = 1024 with 100 binaries, N_pert = 32 so that some lists are cut)."""
    pytest.importorskip("torch")
    outs = _two_ranks(pertlist=True)
    snap = ics.plummer_binaries(1024, 100, ics.BASE_SEED + 48, 1.0 / 256, a_lo=1e-3, a_hi=3e-2)
    ref_l, ref_c = orc.perturbers(snap.m, snap.x, snap.meta["pairs"], gamma=1e-7, nmax=32)
    assert outs[0]["j"] == [0, 512] and outs[1]["j"] == [512, 1024]
    assert np.any(ref_c > 32) and np.any((ref_c > 0) & (ref_c < 32))
    for o in outs:
        assert np.array_equal(np.array(o["lists"]), ref_l)
        assert np.array_equal(np.array(o["counts"]), ref_c)


def test_diverged_replica_is_reported():
    pytest.importorskip("torch")
    outs = _two_ranks(perturb=True)
    for o in outs:
        assert "error" in o and "diverged" in o["error"], o


@pytest.mark.parametrize("n,world", [(1024, 2), (1000, 3), (16384, 8), (300, 4), (65536, 7)])
def test_shares_are_whole_tiles_covering_n(n, world):
    from tests.jp_oracle_ops import TILE, OracleOps
    ops = OracleOps.__new__(OracleOps)
    ops.n = n
    shares = [ops.j_range(r, world) for r in range(world)]
    assert shares[0][0] == 0 and shares[-1][1] == n
    for (b0, e0), (b1, e1) in zip(shares, shares[1:]):
        assert e0 == b1
    for b, e in shares:
        assert b % TILE == 0 and (e % TILE == 0 or e == n) and b <= e
