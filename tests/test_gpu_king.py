"""Centrally concentrated models (King W0 = 6 and 9): the GPU integration against the oracle.

* FP64 path: the first 16 block steps (t_next, s and the active list) are the oracle's;
* both paths: |dE/E| at t = 1/8 within 2x the oracle's plus 1e-9 (the errors here are ~1e-9,
  where FP32 summation noise is of the same order).
N = 2048, eps = 1/1024, seeds 20071106 + 56 and + 59 (the benchmark's King models at a size
the oracle integrates in seconds).
"""
import zlib

import numpy as np
import pytest

import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody
    nbody.load()
    return nbody


def _king(w0):
    return ics.king(2048, seed=ics.BASE_SEED + 50 + int(w0), w0=w0, eps=1.0 / 1024)


@pytest.mark.parametrize("w0", [6.0, 9.0])
def test_king_fp64_schedule_matches_oracle(nb, orc, w0):
    snap = _king(w0)
    sysr = orc.System(snap.m, snap.x, snap.v, snap.eps2, nthreads=orc.default_threads())
    with nb.Context(precision=1) as c:
        c.init(snap)
        for k in range(16):
            tn, s = nb.nb_next_block(c.ctx)
            idx = nb.nb_get_active(c.ctx, s)
            nb.nb_step(c.ctx)
            _, tr, ir = sysr.step()
            assert tn == tr and s == ir.size and zlib.crc32(idx.tobytes()) == \
                zlib.crc32(np.ascontiguousarray(ir, dtype=np.int32).tobytes()), (w0, k)


@pytest.mark.parametrize("w0", [6.0, 9.0])
@pytest.mark.parametrize("prec", [0, 1])
def test_king_energy_conservation(nb, orc, w0, prec):
    snap = _king(w0)
    t_end = 0.125
    sysr = orc.System(snap.m, snap.x, snap.v, snap.eps2, nthreads=orc.default_threads())
    E0r = sysr.energy()
    assert sysr.run(t_end) == 0
    dEr = abs(sysr.energy() - E0r) / abs(E0r)
    with nb.Context(precision=prec) as c:
        c.init(snap)
        E0 = nb.nb_energy(c.ctx)[0]
        nb.nb_run(c.ctx, t_end)
        E1 = nb.nb_energy(c.ctx)[0]
        st = c.state()
        cnt = nb.nb_stats(c.ctx)
    dE = abs(E1 - E0) / abs(E0)
    print(f"King W0={w0:g} prec {prec}: |dE/E| GPU {dE:.3e} oracle {dEr:.3e}; block steps GPU "
          f"{cnt['block_steps']} oracle {sysr.counters['block_steps']}")
    assert np.all(st["t"] == t_end)
    assert dE <= 2 * dEr + 1e-9, (w0, prec, dE, dEr)   # floor: summation noise at this size
