"""Energy conservation of the timed integrations against the oracle's (the bar: |dE/E| at
the end within 2x the oracle's on the same initial conditions).

The oracle's values are stored in tests/golden/c2_energy.txt (Plummer N = 16384,
eps = 1/1024, t = 0 -> 1) and c3_energy.txt (Plummer N = 65536 with Salpeter masses,
eps = 1/4096, t = 0 -> 0.5), written by tests/golden/make_golden.py from oracle/ and ics/
alone (the integrations take minutes to tens of minutes on the CPU). Each file also holds a
CRC32 of the input arrays, checked here, so the GPU integrates the same initial conditions.
The integrations themselves are chaotic, so only |dE/E| and the step counts are compared;
the step counts are printed beside the oracle's.
"""
import os
import zlib

import numpy as np
import pytest

import ics

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FLOOR = 1e-13   # the energy diagnostic's own error is ~1e-15 relative


@pytest.fixture(scope="module")
def nb():
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody
    nbody.load()
    return nbody


def _golden(cfg):
    out = {}
    with open(os.path.join(GOLDEN, f"c{cfg}_energy.txt")) as f:
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


def _crc(snap):
    crc = 0
    for a in (snap.m, snap.x, snap.v):
        crc = zlib.crc32(np.ascontiguousarray(a, dtype="<f8").tobytes(), crc)
    return crc


def _run(nb, snap, prec, t_end):
    with nb.Context(precision=prec) as c:
        c.init(snap)
        nb.nb_autotune(c.ctx)
        c.init(snap)
        E0, _, _ = nb.nb_energy(c.ctx)
        nb.nb_run(c.ctx, t_end)
        E1, _, _ = nb.nb_energy(c.ctx)
        st = c.state()
        cnt = nb.nb_stats(c.ctx)
    assert np.all(st["t"] == t_end)
    return abs(E1 - E0) / abs(E0), cnt


@pytest.mark.parametrize("cfg,prec", [(2, 0), (2, 1), (3, 0)])
def test_energy_error_within_2x_oracle(nb, cfg, prec):
    gold = _golden(cfg)
    snap = ics.config(cfg)
    assert snap.n == gold["n"]
    assert _crc(snap) == gold["input_crc32"], "initial conditions differ from the oracle's run"
    dE, cnt = _run(nb, snap, prec, gold["t_end"])
    print(f"config {cfg}, precision {prec}: |dE/E| gpu {dE:.4e} oracle {gold['abs_dE_over_E']:.4e}; "
          f"block steps gpu {cnt['block_steps']} oracle {gold['block_steps']}; particle steps gpu "
          f"{cnt['particle_steps']} oracle {gold['particle_steps']}")
    assert dE <= 2.0 * gold["abs_dE_over_E"] + FLOOR, (dE, gold["abs_dE_over_E"])
