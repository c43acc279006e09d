"""The library side of the j-parallel block step (Sect. 3, Flowchart) on one GPU.

* Partial forces over rank shares (nb_j_range, nb_force_jerk_range), added in rank order,
  equal the whole force sum within the mixed tolerance; an empty share gives zeros; a share
  that does not start on a tile boundary is refused.
* nb_correct_forces with the forces of nb_force_jerk gives the same state, bit for bit, as
  nb_correct.
* Two processes, each with its own context on this GPU, run the driver
  (paper_0711_0643_gb300/jparallel.py) with their partial forces exchanged over gloo through
  host memory (no kernel of one process waits on the other's): 16 block steps of the Plummer
  N = 1024 workload leave both replicas identical, and identical bit for bit to one process
  that computes both shares itself and adds them in the same order.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import ics
from tests.nbtools import condition_scales, rel_scalar

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nb():
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody
    nbody.load()
    return nbody


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_rank_shares_add_up_to_the_whole_sum(nb, world):
    snap = ics.plummer(3000, seed=41, eps=1.0 / 256)
    with nb.Context(precision=0) as c:
        c.init(snap)
        nb.nb_predict(c.ctx, 0.0)
        idx = np.arange(0, snap.n, 5, dtype=np.int32)
        a, k, phi = nb.nb_force_jerk(c.ctx, idx)
        tot = np.zeros((idx.size, 7))
        for r in range(world):
            j0, j1 = nb.nb_j_range(c.ctx, r, world)
            pa, pk, pp = nb.nb_force_jerk_range(c.ctx, idx, None, j0, j1)
            tot += np.concatenate([pa, pk, pp[:, None]], axis=1)
        xp, vp = nb.nb_get_predicted(c.ctx, snap.n)
        A, K = condition_scales(snap.m, xp, vp, snap.eps2, idx)
        assert (np.linalg.norm(tot[:, 0:3] - a, axis=1) / A).max() < 1e-6
        assert (np.linalg.norm(tot[:, 3:6] - k, axis=1) / K).max() < 1e-6
        assert rel_scalar(tot[:, 6], phi).max() < 1e-6
        if world == 1:
            np.testing.assert_array_equal(tot[:, 0:3], a)   # the whole range is the same launch
        # an empty share, and a share that does not start on a tile boundary
        za, zk, zp = nb.nb_force_jerk_range(c.ctx, idx, None, 512, 512)
        assert not za.any() and not zk.any() and not zp.any()
        with pytest.raises(nb.NbError) as e:
            nb.nb_force_jerk_range(c.ctx, idx, None, 100, 512)
        assert e.value.status == nb.NB_ERR_ARG


def test_correct_with_given_forces_equals_correct(nb):
    snap = ics.config(1)
    states = []
    for given in (False, True):
        with nb.Context(precision=0) as c:
            c.init(snap)
            for _ in range(5):
                nb.nb_step(c.ctx)
            for _ in range(4):
                tn, s = nb.nb_next_block(c.ctx)
                nb.nb_predict(c.ctx, tn)
                a, k, _ = nb.nb_force_jerk(c.ctx, None, s)
                if given:
                    nb.nb_correct_forces(c.ctx, tn, a, k)
                else:
                    nb.nb_correct(c.ctx, tn)
            states.append(c.state())
    for key in ("x", "v", "a", "k", "t", "dt"):
        np.testing.assert_array_equal(states[0][key], states[1][key])


CHILD = r"""
import os, sys, json
sys.path.insert(0, os.environ["NB_ROOT"])
import numpy as np
import torch.distributed as dist
import ics
import paper_0711_0643_gb300 as pkg
from paper_0711_0643_gb300 import nbody as nb
from paper_0711_0643_gb300.jparallel import GpuOps, JParallel
nb.load()
dist.init_process_group("gloo")
snap = ics.config(1)
c = nb.Context(precision=0, device=0)
c.init(snap)
jp = JParallel(GpuOps(nb, c.ctx, snap.n))
rows = [list(jp.step()) for _ in range(16)]
st = c.state()
print(json.dumps({"rows": rows, "j": [jp.j0, jp.j1], "state": {k: v.tolist() for k, v in st.items()}}))
c.close()
dist.destroy_process_group()
"""


class _TwoSharesOps:
    """One process computing both ranks' shares and adding them in rank order."""

    def __init__(self, base, world):
        self.base = base
        self.world = world

    def __getattr__(self, name):
        return getattr(self.base, name)

    def j_range(self, rank, world):
        return 0, self.base.n

    def partial_forces(self, s, j0, j1):
        parts = [self.base.partial_forces(s, *self.base.j_range(r, self.world)) for r in range(self.world)]
        total = parts[0].copy()
        for p in parts[1:]:
            total += p
        return total


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_processes_on_one_gpu_match_emulation(nb):
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
        out, err = p.communicate(timeout=600)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    from paper_0711_0643_gb300.jparallel import GpuOps, JParallel
    snap = ics.config(1)
    with nb.Context(precision=0) as c:
        c.init(snap)
        jp = JParallel(_TwoSharesOps(GpuOps(nb, c.ctx, snap.n), 2))
        rows = [list(jp.step()) for _ in range(16)]
        st = c.state()
    assert outs[0]["j"] == [0, 512] and outs[1]["j"] == [512, 1024]
    assert outs[0]["rows"] == outs[1]["rows"] == rows
    for key in ("x", "v", "a", "k", "t", "dt"):
        assert outs[0]["state"][key] == outs[1]["state"][key], key
        np.testing.assert_array_equal(np.array(outs[0]["state"][key]), st[key])
