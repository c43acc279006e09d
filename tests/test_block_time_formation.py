"""The identity the device run loop relies on to form the next block time while
a block is processed (no GPU): with the block time T = min_i(t_i + dt_i) and
m2 = the smallest key other than T, the next block time after correcting the
block is min(m2, smallest new key of the block's particles), because the keys
of the particles outside the block do not change (Sect. 2.1 block steps).
Checked step by step on the oracle's own integration, with its selection."""
import numpy as np

import ics


def test_next_block_time_from_second_smallest_key_and_new_keys(orc):
    snap = ics.plummer(512, seed=11, eps=1.0 / 128)
    s = orc.System(snap.m, snap.x, snap.v, snap.eps2, eta=0.01, nthreads=orc.default_threads())
    assert s.status == 0
    T, idx = orc.next_block(s.t, s.dt)
    for _ in range(300):
        keys = s.t + s.dt
        assert keys.min() == T
        others = keys[keys != T]
        m2 = others.min() if others.size else np.inf
        st, t_step, idx_step = s.step()
        assert st == 0 and t_step == T
        np.testing.assert_array_equal(idx_step, idx)
        new = s.t + s.dt
        inactive = np.ones(s.n, dtype=bool)
        inactive[idx] = False
        np.testing.assert_array_equal(new[inactive], keys[inactive])   # untouched keys
        formed = min(m2, new[idx].min())
        T, idx = orc.next_block(s.t, s.dt)
        assert formed == T
        # the selection at a known block time finds the same ascending list
        np.testing.assert_array_equal(np.flatnonzero(new == formed).astype(np.int32), idx)
