"""Write the oracle-derived golden fixtures in this folder.

Calls only ``oracle/`` (the FP64 CPU oracle) and ``ics/`` (seeded inputs):
  python tests/golden/make_golden.py               # c1 block schedule
  python tests/golden/make_golden.py c2 c3         # energy error of the timed integrations

c2: Plummer N = 16384, eps = 1/1024, t = 0 -> 1 (about 1.1e11 interactions).
c3: Plummer N = 65536 with Salpeter masses, eps = 1/4096, t = 0 -> 0.5 (about 1e12
interactions; tens of minutes on a multi-core host).
"""
import os
import sys
import time
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


def snapshot_crc(snap):
    """CRC32 of the input bytes (m, x, v as little-endian doubles): identifies the inputs."""
    crc = 0
    for a in (snap.m, snap.x, snap.v):
        crc = zlib.crc32(np.ascontiguousarray(a, dtype="<f8").tobytes(), crc)
    return crc


def energy_run(cfg, t_end):
    """The oracle's integration of workload ``cfg`` from t = 0 to t_end: energies at both
    ends (softened W, FP64 sums), |dE/E| and the step counters."""
    snap = ics.config(cfg)
    nth = oracle.default_threads()
    t0 = time.time()
    s = oracle.System(snap.m, snap.x, snap.v, snap.eps2, eta=0.01, dt_max=1.0 / 16, dt_min=2.0 ** -40,
                      nthreads=nth)
    assert s.status == 0
    e0 = s.energy()
    assert s.run(t_end) == 0
    assert np.all(s.t == t_end)
    e1 = s.energy()
    c = s.counters
    return {"cfg": cfg, "name": snap.name, "n": snap.n, "t_end": t_end, "E0": e0, "E1": e1,
            "dE": abs(e1 - e0) / abs(e0), "block_steps": c["block_steps"], "particle_steps": c["particle_steps"],
            "interactions": c["interactions"], "crc": snapshot_crc(snap), "seconds": time.time() - t0,
            "threads": nth}


def write_energy(r):
    path = os.path.join(HERE, f"c{r['cfg']}_energy.txt")
    with open(path, "w") as f:
        f.write(f"# {r['name']}: FP64 oracle (eta = 0.01, dt_max = 1/16), t = 0 -> {r['t_end']}.\n")
        f.write("# Written by tests/golden/make_golden.py (oracle/ and ics/ only). Energies are softened\n")
        f.write("# (W = -1/2 sum m_i m_j / (r^2 + eps^2)^(1/2)); floats as hex.\n")
        f.write(f"# oracle run: {r['seconds']:.0f} s on {r['threads']} threads.\n")
        f.write(f"input_crc32 {r['crc']:08x}\n")
        f.write(f"n {r['n']}\n")
        f.write(f"t_end {float(r['t_end']).hex()}\n")
        f.write(f"E0 {r['E0'].hex()}\n")
        f.write(f"E1 {r['E1'].hex()}\n")
        f.write(f"abs_dE_over_E {r['dE'].hex()}  # {r['dE']:.6e}\n")
        f.write(f"block_steps {r['block_steps']}\n")
        f.write(f"particle_steps {r['particle_steps']}\n")
        f.write(f"interactions {r['interactions']:.17g}\n")
    return path


def load_energy(cfg):
    """The stored values of c<cfg>_energy.txt as a dict (floats, ints)."""
    out = {}
    with open(os.path.join(HERE, f"c{cfg}_energy.txt")) as f:
        for ln in f:
            ln = ln.split("#", 1)[0].strip()
            if not ln:
                continue
            key, val = ln.split()[:2]
            if key == "input_crc32":
                out[key] = int(val, 16)
            elif key in ("n", "block_steps", "particle_steps"):
                out[key] = int(val)
            elif key == "interactions":
                out[key] = float(val)
            else:
                out[key] = float.fromhex(val)
    return out


def main(argv):
    todo = argv or ["c1"]
    if "c1" in todo:
        rows = block_schedule()
        with open(os.path.join(HERE, "c1_block_schedule.txt"), "w") as f:
            f.write("# Plummer N=1024 (seed 20071107, eps=1/256), FP64 oracle, eta=0.01, dt_max=1/16.\n")
            f.write("# Written by tests/golden/make_golden.py. Columns: step, t_next (hex float), s, "
                    "crc32(idx int32).\n")
            for k, tn, s, crc in rows:
                f.write(f"{k} {tn.hex()} {s} {crc:08x}\n")
    for cfg, t_end in (("c2", 1.0), ("c3", 0.5)):
        if cfg in todo:
            r = energy_run(int(cfg[1]), t_end)
            print(write_energy(r), f"|dE/E| = {r['dE']:.4e}", f"{r['seconds']:.0f} s")


if __name__ == "__main__":
    main(sys.argv[1:])
