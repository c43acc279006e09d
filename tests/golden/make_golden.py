"""Write the oracle-derived golden fixtures in this folder.

Calls only ``oracle/`` (the FP64 CPU oracle) and ``ics/`` (seeded inputs):
  python tests/golden/make_golden.py
"""
import os
import sys
import zlib

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import ics  # noqa: E402
import oracle  # noqa: E402


def block_schedule(cfg=1, steps=16):
    snap = ics.config(cfg)
    s = oracle.System(snap.m, snap.x, snap.v, snap.eps2, eta=0.01, dt_max=1.0 / 16, dt_min=2.0 ** -40,
                      nthreads=oracle.default_threads())
    assert s.status == 0
    rows = []
    for k in range(steps):
        st, tn, idx = s.step()
        assert st == 0
        rows.append((k, tn, idx.size, zlib.crc32(np.ascontiguousarray(idx, dtype=np.int32).tobytes())))
    return rows


def main():
    rows = block_schedule()
    with open(os.path.join(HERE, "c1_block_schedule.txt"), "w") as f:
        f.write("# Plummer N=1024 (seed 20071107, eps=1/256), FP64 oracle, eta=0.01, dt_max=1/16.\n")
        f.write("# Written by tests/golden/make_golden.py. Columns: step, t_next (hex float), s, crc32(idx int32).\n")
        for k, tn, s, crc in rows:
            f.write(f"{k} {tn.hex()} {s} {crc:08x}\n")


if __name__ == "__main__":
    main()
