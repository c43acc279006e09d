"""The oracle reproduces its stored block schedule for the Plummer N=1024 workload."""
import os
import zlib

import numpy as np

import ics

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c1_block_schedule.txt")


def load_schedule():
    rows = []
    with open(GOLDEN) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, tn, s, crc = ln.split()
                rows.append((int(k), float.fromhex(tn), int(s), int(crc, 16)))
    return rows


def test_oracle_block_schedule(orc):
    snap = ics.config(1)
    s = orc.System(snap.m, snap.x, snap.v, snap.eps2, eta=0.01, nthreads=orc.default_threads())
    for k, tn, ns, crc in load_schedule():
        st, t_next, idx = s.step()
        assert st == 0
        assert (t_next, idx.size, zlib.crc32(np.ascontiguousarray(idx, dtype=np.int32).tobytes())) == (tn, ns, crc), k
