"""Mixed path: block assignment and time steps over the first 16 block steps against the
oracle (Sect. 2.1: the block is every particle with the smallest t_i + dt_i; new steps from
the Aarseth criterion, Eq. (timestep), quantised to powers of two).

Same-input lockstep. Before every GPU block step the oracle takes the GPU's state and does
the same block step on it in FP64 (selection, predictor, force, corrector, Aarseth step,
quantisation). Then, at every one of the 16 steps (and for the start steps of nb_init):
  * the block time, the block size and the active list are identical, bit for bit;
  * the GPU's forces on the block are within the mixed tolerances of the oracle's;
  * the corrected x and v differ from the oracle's by no more than the corrector carries
    the measured force error into them (|dx| <= 0.35 ea dt^2 + 2/15 ek dt^3,
    |dv| <= 1.5 ea dt + 7/12 ek dt^2, plus FP64 rounding);
  * every new time step is identical, except where the oracle's Aarseth candidate lies
    within its tie window delta_i of a power of two. delta_i is the largest relative change
    of the candidate that the GPU's measured force error on particle i can cause through the
    corrector's finite differences (tests/nbtools.aarseth_tie_window). Inside it, both
    quantised steps are correct outcomes of the same rule; the test counts such ties and
    keeps going through all 16 steps.
The oracle integrating its own state (free running) is run beside it; the step at which its
block schedule first differs from the GPU's is printed.

Two drivers: "explicit" calls nb_next_block, nb_predict, nb_force_jerk and nb_correct (the
four-kernel step); "step" calls nb_step with the small-block engine taking blocks of up to
32 particles (its new forces are read back from the corrected state, where the corrector
stores them; its potential is not compared).
"""
import numpy as np
import pytest

import ics
from tests.nbtools import (aarseth_tie_window, condition_scales, pow2_distance, rel_scalar, start_tie_window,
                           stats)

pytestmark = pytest.mark.gpu

ETA = 0.01
TOL = 1e-6


@pytest.fixture(scope="module")
def nb():
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody
    nbody.load()
    return nbody


def _force_errors(m, xr, vr, eps2, idx, a_g, k_g, phi_g, ar, kr, pr, where):
    """Mixed tolerances on the same input; returns the absolute error norms (ea, ek)."""
    A, K = condition_scales(m, xr, vr, eps2, idx)
    ea = np.linalg.norm(a_g - ar, axis=1)
    ek = np.linalg.norm(k_g - kr, axis=1)
    assert (ea / A).max() < TOL and (ek / K).max() < TOL, (where, stats(ea / A), stats(ek / K))
    assert rel_scalar(phi_g, pr).max() < TOL, where
    # FP64 rounding of the oracle's own sums (~1e-16 of the scales) widens the bound slightly
    return ea + 1e-14 * A, ek + 1e-14 * K


@pytest.mark.parametrize("cfg,driver", [(1, "explicit"), (2, "explicit"), (1, "step"), (2, "step")])
def test_block_schedule_mixed_lockstep(nb, orc, cfg, driver):
    snap = ics.config(cfg)
    n = snap.n
    nth = orc.default_threads()
    free = orc.System(snap.m, snap.x, snap.v, snap.eps2, eta=ETA, nthreads=nth)
    free_diverged = None
    ties = 0
    in_window = 0
    windows = []
    with nb.Context(precision=0) as c:
        if driver == "step":
            nb.nb_set_engine(c.ctx, 32)
        c.init(snap)
        if driver == "step":
            assert nb.nb_get_engine(c.ctx)[0] == 32
        g = c.state()
        # start steps: dt0 = 2^floor(log2(eta |a| / |k|)) on the forces of the initial state
        ar, kr, pr = orc.force(snap.m, snap.x, snap.v, snap.eps2, None, nthreads=nth)
        ea, ek = _force_errors(snap.m, snap.x, snap.v, snap.eps2, np.arange(n), g["a"], g["k"],
                               np.zeros(n) + pr, ar, kr, pr, "init")
        dt_r = np.array([orc.initial_dt(ar[i], kr[i], ETA) for i in range(n)])
        for i in range(n):
            assert g["dt"][i] == orc.initial_dt(g["a"][i], g["k"][i], ETA), i
        bad = np.nonzero(g["dt"] != dt_r)[0]
        if bad.size:
            cand = ETA * np.linalg.norm(ar[bad], axis=1) / np.linalg.norm(kr[bad], axis=1)
            win = start_tie_window(ar[bad], kr[bad], ea[bad], ek[bad])
            assert np.all(pow2_distance(cand) <= win), (cand, win)
            ties += bad.size
        for step in range(16):
            before = c.state()
            tn, s = nb.nb_next_block(c.ctx)
            idx = nb.nb_get_active(c.ctx, s)
            if driver == "explicit":
                nb.nb_predict(c.ctx, tn)
                a_g, k_g, phi_g = nb.nb_force_jerk(c.ctx, None, s)
                nb.nb_correct(c.ctx, tn)
                after = c.state()
            else:
                nb.nb_step(c.ctx)
                after = c.state()
                a_g, k_g, phi_g = after["a"][idx], after["k"][idx], None
            # the oracle's block step on the same state
            tr, ir = orc.next_block(before["t"], before["dt"])
            assert tr == tn and np.array_equal(ir, idx), (step, tr, tn)
            xr, vr = orc.predict(before["x"], before["v"], before["a"], before["k"], before["t"], tn)
            ar, kr, pr = orc.force(snap.m, xr, vr, snap.eps2, idx, nthreads=nth)
            ea, ek = _force_errors(snap.m, xr, vr, snap.eps2, idx, a_g, k_g, pr if phi_g is None else phi_g,
                                   ar, kr, pr, step)
            for q, i in enumerate(idx):
                dt = before["dt"][i]
                x1, v1, a2, a3 = orc.correct_one(xr[i], vr[i], before["a"][i], before["k"][i], ar[q], kr[q], dt)
                _, _, cand = orc.correct_particle(xr[i], vr[i], before["a"][i], before["k"][i], ar[q], kr[q],
                                                  dt, ETA)
                bx = 0.35 * ea[q] * dt ** 2 + (2.0 / 15.0) * ek[q] * dt ** 3 + 4e-16 * np.abs(x1).max()
                bv = 1.5 * ea[q] * dt + (7.0 / 12.0) * ek[q] * dt ** 2 + 4e-16 * np.abs(v1).max()
                assert np.abs(after["x"][i] - x1).max() <= bx, (step, i)
                assert np.abs(after["v"][i] - v1).max() <= bv, (step, i)
                win = aarseth_tie_window(ar[q:q + 1], kr[q:q + 1], (a2 + a3 * dt)[None, :], a3[None, :],
                                         np.array([dt]), np.array([ea[q]]), np.array([ek[q]]))[0]
                windows.append(win)
                dist = pow2_distance(np.array([cand]))[0]
                in_window += dist <= win
                if after["dt"][i] != orc.quantise(cand, dt, tn):
                    assert dist <= win, (step, i, cand, dist, win)
                    ties += 1
            # the oracle on its own trajectory
            st_f, tf, idx_f = free.step()
            assert st_f == 0
            if free_diverged is None and not (tf == tn and np.array_equal(idx_f, idx)):
                free_diverged = step
    w = np.array(windows)
    print(f"config {cfg}, {driver}: 16 lockstep block steps, {w.size} corrections; tie window delta_i "
          f"median {np.median(w):.2e}, max {w.max():.2e}; candidates inside their window {in_window}; "
          f"time steps differing from the oracle's (all ties) {ties}; free-running oracle schedule "
          f"{'identical for all 16 steps' if free_diverged is None else f'differs from block step {free_diverged}'}")
