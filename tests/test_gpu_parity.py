"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Forces: every kernel variant, several split factors, ragged sizes. FP64 path:
per-particle relative error of a, k and phi within 1e-12. Mixed path: phi within
1e-6 relative; a and the jerk within 1e-6 of their condition scales
A_i = sum_j |a term|, K_i = sum_j |jerk term| (any FP32 pair arithmetic has an
error of a few u times that scale; for sums that cancel heavily, the forward
error grows with the condition numbers kappa_a = A_i/|a_i|, kappa_k = K_i/|k_i|);
the forward relative errors of a and of k within 1e-6 wherever the condition
number is at most KAPPA_A = 16 for a and KAPPA_K = 8 for k (2e-6 for k up to 16),
and that of a within 1e-6 at the 99th percentile. Forward statistics are printed.
Why the jerk's limit is lower: a single FP32 pair term of the jerk carries several
roundings (r^2 to ~1.5u, enlarged by 3/2 in (r^2)^(-3/2), the rsqrt and its Newton
step, the products forming mu and alpha = 3 (r.w)/r^2), and 64 terms are summed in
FP32 before each two-sum fold, so |dk| <= c u K_i and the forward error is at most
c u kappa_k (u = 2^-24). An FP32 emulation on the CPU attributes ~7e-7 at kappa <= 16
to the pair terms and ~4e-7 to the FP32 partial sums (the FP32 velocities add ~1e-7);
on the GPU c u kappa reaches 1.5e-6 at kappa_k = 16 (c ~ 1.6), so 1e-6 holds up to
kappa_k = 8 and 2e-6 up to 16.
Predictor, corrector, time steps and block selection: bit-exact against the
oracle given the same inputs (the mixed predictor within its derived FP32
bounds). Integration: the FP64 path reproduces the oracle's block schedule for
the first 16 steps; both paths keep |dE/E| at t = 1 within 2x the oracle's.
The mixed path's schedule over the first 16 steps is tested in
tests/test_gpu_schedule.py.
"""
import math
import zlib

import numpy as np
import pytest

import ics
from tests.nbtools import condition_scales, rel_errors, rel_scalar, stats

pytestmark = pytest.mark.gpu

TOL = {0: 1e-6, 1: 1e-12}   # precision -> relative force/jerk tolerance
KAPPA_A = 16.0               # mixed path: forward a within TOL where kappa_a <= this
KAPPA_K = 8.0                # mixed path: forward k within TOL where kappa_k <= this, 2 TOL up to 2 KAPPA_K


@pytest.fixture(scope="module")
def nb():
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody
    nbody.load()
    return nbody


def _cond_scaled(x, xr, scale):
    d = np.linalg.norm(x - xr, axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(d == 0.0, 0.0, d / scale)


def _errors(prec, a, k, phi, ar, kr, pr, A, K):
    """Error set of one comparison: e_a, e_k, e_phi (what the tolerance applies to:
    forward for FP64, condition-scaled for the mixed path), the forward e_a and e_k,
    and the condition numbers kappa_a = A_i/|a_i|, kappa_k = K_i/|k_i|."""
    ea_fwd = rel_errors(a, ar, A)
    ek_fwd = rel_errors(k, kr, K)
    if prec == 1:
        ea, ek = ea_fwd, ek_fwd
    else:
        ea, ek = _cond_scaled(a, ar, A), _cond_scaled(k, kr, K)
    ep = rel_scalar(phi, pr)
    with np.errstate(divide="ignore", invalid="ignore"):
        kap_a = A / np.linalg.norm(ar, axis=1)
        kap_k = K / np.linalg.norm(kr, axis=1)
    return {"ea": ea, "ek": ek, "ep": ep, "eaf": ea_fwd, "ekf": ek_fwd, "kap_a": kap_a, "kap_k": kap_k}


def _check(prec, e, where):
    tol = TOL[prec]
    ea, ek, ep = e["ea"], e["ek"], e["ep"]
    assert ea.max() < tol and ek.max() < tol and ep.max() < tol, (where, stats(ea), stats(ek), stats(ep))
    if prec == 0:
        assert np.percentile(e["eaf"], 99) < tol, (where, stats(e["eaf"]))
        well_a = e["kap_a"] <= KAPPA_A
        well_k, fair_k = e["kap_k"] <= KAPPA_K, e["kap_k"] <= 2 * KAPPA_K
        assert np.all(e["eaf"][well_a] < tol), (where, "a forward, kappa <= 16", e["eaf"][well_a].max())
        assert np.all(e["ekf"][well_k] < tol), (where, "k forward, kappa <= 8", e["ekf"][well_k].max())
        assert np.all(e["ekf"][fair_k] < 2 * tol), (where, "k forward, kappa <= 16", e["ekf"][fair_k].max())


def _forces_vs_oracle(nb, orc, c, snap, idx, prec):
    """GPU forces on idx vs the oracle on the same predicted records."""
    xp, vp = nb.nb_get_predicted(c.ctx, snap.n)
    a, k, phi = nb.nb_force_jerk(c.ctx, idx)
    ar, kr, pr = orc.force(snap.m, xp, vp, snap.eps2, idx, nthreads=orc.default_threads())
    A, K = condition_scales(snap.m, xp, vp, snap.eps2, idx)
    return _errors(prec, a, k, phi, ar, kr, pr, A, K)


SIZES = [(1, 0.01), (2, 0.0), (7, 0.05), (300, 0.01), (1000, 1.0 / 64), (2049, 1.0 / 256)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,eps", SIZES)
def test_force_all_variants(nb, orc, prec, n, eps):
    snap = ics.random_state(n, seed=100 + n, eps=eps) if n < 300 else ics.plummer(n, seed=n, eps=eps)
    rng = ics.SplitMix64(n)
    subsets = [np.arange(n), np.array([n - 1]), np.sort(rng.next_u64(min(n, 37)) % n)]
    with nb.Context(precision=prec) as c:
        c.init(snap)
        nb.nb_predict(c.ctx, 0.0)
        for v in range(nb.nb_num_variants(c.ctx)):
            for split in (1, 3, 64):
                for b in range(32):
                    nb.nb_set_tuning(c.ctx, b, v, split)
                for sub in subsets:
                    idx = np.unique(sub).astype(np.int32)
                    e = _forces_vs_oracle(nb, orc, c, snap, idx, prec)
                    _check(prec, e, (nb.nb_variant_name(c.ctx, v), split, idx.size))


def test_force_many_splits_wide_blocks(nb, orc):
    """Split sums with many splits over wide i-blocks (256 and 32 particles): up to 256
    split partials per particle (more than one batch of loads per lane in the final
    sum), a ragged last i-block, against the oracle on the same predicted records."""
    n = 65536
    snap = ics.plummer(n, seed=n, eps=1.0 / 256)
    rng = ics.SplitMix64(n + 1)
    idx = np.unique(rng.next_u64(700) % n).astype(np.int32)[:600]
    with nb.Context(precision=0) as c:
        c.init(snap)
        nb.nb_predict(c.ctx, 0.0)
        names = [nb.nb_variant_name(c.ctx, v) for v in range(nb.nb_num_variants(c.ctx))]
        for name, splits in (("tile R=1 TJ=1", (5, 9, 150, 256)), ("tile R=1 TJ=8", (7, 150))):
            v = names.index(name)
            for split in splits:
                for b in range(32):
                    nb.nb_set_tuning(c.ctx, b, v, split)
                e = _forces_vs_oracle(nb, orc, c, snap, idx, 0)
                _check(0, e, (name, split, idx.size))


@pytest.mark.parametrize("prec", [0, 1])
def test_force_plummer_16k_all_blocks(nb, orc, prec):
    """Plummer N = 16384 (eps = 1/1024): tuned launch configuration, s = 1 .. N."""
    snap = ics.config(2)
    with nb.Context(precision=prec) as c:
        c.init(snap)
        nb.nb_predict(c.ctx, 0.0)
        rng = ics.SplitMix64(77)
        for s in (1, 5, 64, 1000, 4096, snap.n):
            idx = np.sort(rng.next_u64(s * 2) % snap.n)
            idx = np.unique(idx)[:s].astype(np.int32) if s < snap.n else np.arange(snap.n, dtype=np.int32)
            sample = idx if idx.size <= 512 else idx[:: idx.size // 512]
            xp, vp = nb.nb_get_predicted(c.ctx, snap.n)
            a, k, phi = nb.nb_force_jerk(c.ctx, idx)
            pos = np.searchsorted(idx, sample)
            ar, kr, pr = orc.force(snap.m, xp, vp, snap.eps2, sample, nthreads=orc.default_threads())
            A, K = condition_scales(snap.m, xp, vp, snap.eps2, sample)
            e = _errors(prec, a[pos], k[pos], phi[pos], ar, kr, pr, A, K)
            print(f"prec {prec} s {s}: a {stats(e['ea'])} k {stats(e['ek'])} a(forward) {stats(e['eaf'])} "
                  f"k(forward) {stats(e['ekf'])} phi {stats(e['ep'])}")
            _check(prec, e, s)


def test_predictor_bit_exact(nb, orc):
    """FP64 predicted records equal the oracle's predictor bit for bit. The mixed records:
    positions (a double-single Horner evaluation, split into hi + lo) within 2^-45 of each
    particle's |x|; velocities, stored in FP32, within the bound of the FP32 expression
    that forms them, per component c (u = 2^-24, d = t - t_j):
        |v_gpu - v_ref| <= 2u |v_ref| + 4u |d| |a| + 4u d^2 |k| + 2^-46 |v|
    -- the last two roundings (adding the increment to the high part of v, then the low
    part) cost u |v_ref| each; the increment d (a + d k / 2) carries the FP32 rounding of
    d, a and k and three rounded operations (at most 6u of each term); the double-single
    v itself is exact to ~2^-48. A single rounding to FP32 already costs up to u |v_ref|, so
    no FP32 record can meet a 2^-24 bound per component."""
    snap = ics.config(1)
    for prec in (1, 0):
        with nb.Context(precision=prec) as c:
            c.init(snap)
            for _ in range(5):
                nb.nb_step(c.ctx)
            st = c.state()
            t_new = float(np.max(st["t"] + st["dt"]) / 2 + np.min(st["t"]) / 2)
            nb.nb_predict(c.ctx, t_new)
            xp, vp = nb.nb_get_predicted(c.ctx, snap.n)
            xr, vr = orc.predict(st["x"], st["v"], st["a"], st["k"], st["t"], t_new)
            if prec == 1:
                np.testing.assert_array_equal(xp, xr)
                np.testing.assert_array_equal(vp, vr)
            else:
                ex = np.linalg.norm(xp - xr, axis=1) / np.linalg.norm(xr, axis=1)
                assert ex.max() < 2.0 ** -45, ex.max()
                u = 2.0 ** -24
                d = np.abs(t_new - st["t"])[:, None]
                bound = (2 * u * np.abs(vr) + 4 * u * d * np.abs(st["a"]) + 4 * u * d * d * np.abs(st["k"])
                         + 2.0 ** -46 * np.abs(st["v"]))
                dv = np.abs(vp - vr)
                assert np.all(dv <= bound), float((dv / bound).max())
                print(f"mixed predictor: velocity error / bound, max {(dv / bound).max():.3f}")


def test_corrector_and_steps_bit_exact(nb, orc):
    """Given the GPU's own new forces, the corrected x, v and the new quantised steps equal
    the oracle's corrector + Aarseth + quantisation bit for bit (both precisions)."""
    snap = ics.config(1)
    for prec in (1, 0):
        with nb.Context(precision=prec) as c:
            c.init(snap)
            for _ in range(7):
                nb.nb_step(c.ctx)
            before = c.state()
            tn, s = nb.nb_next_block(c.ctx)
            idx = nb.nb_get_active(c.ctx, s)
            nb.nb_predict(c.ctx, tn)
            a_new, k_new, _ = nb.nb_force_jerk(c.ctx, idx)
            nb.nb_correct(c.ctx, tn)
            after = c.state()
            xr, vr = orc.predict(before["x"], before["v"], before["a"], before["k"], before["t"], tn)
            for q, i in enumerate(idx):
                dt = before["dt"][i]
                x1, v1, cand = orc.correct_particle(xr[i], vr[i], before["a"][i], before["k"][i],
                                                    a_new[q], k_new[q], dt, 0.01)
                dtn = orc.quantise(cand, dt, tn)
                np.testing.assert_array_equal(after["x"][i], x1)
                np.testing.assert_array_equal(after["v"][i], v1)
                np.testing.assert_array_equal(after["a"][i], a_new[q])
                assert after["dt"][i] == dtn and after["t"][i] == tn
            others = np.setdiff1d(np.arange(snap.n), idx)
            np.testing.assert_array_equal(after["x"][others], before["x"][others])


def test_corrector_bit_exact_full_blocks(nb, orc):
    """All 16384 particles of the Plummer workload due at once, for three common
    steps, two accuracy parameters and both precisions (about 2e5 corrector
    evaluations): x, v and the new quantised step equal the oracle's bit for bit,
    given the GPU's own forces. The GPU quantiser decides from an FP32 estimate of
    the Aarseth step and evaluates the FP64 expression only when the estimate lies
    within 2^-14 of a power of two; the test counts candidates in that window, so
    both branches are compared."""
    snap = ics.config(2)
    near = 0
    for prec in (1, 0):
        for eta in (0.01, 0.02):
            with nb.Context(precision=prec, eta=eta) as c:
                c.init(snap)
                for dt in (2.0 ** -6, 2.0 ** -9, 2.0 ** -12):
                    st = c.state()
                    st["dt"][:] = dt          # every t is a multiple of these steps
                    nb.nb_set_state(c.ctx, st)
                    tn, s = nb.nb_next_block(c.ctx)
                    assert s == snap.n and tn == st["t"][0] + dt
                    idx = nb.nb_get_active(c.ctx, s)
                    nb.nb_predict(c.ctx, tn)
                    a_new, k_new, _ = nb.nb_force_jerk(c.ctx, idx)
                    nb.nb_correct(c.ctx, tn)
                    after = c.state()
                    xr, vr = orc.predict(st["x"], st["v"], st["a"], st["k"], st["t"], tn)
                    for i in range(snap.n):
                        x1, v1, cand = orc.correct_particle(xr[i], vr[i], st["a"][i], st["k"][i], a_new[i],
                                                            k_new[i], dt, eta)
                        assert np.array_equal(after["x"][i], x1) and np.array_equal(after["v"][i], v1), \
                            (prec, eta, dt, i)
                        assert after["dt"][i] == orc.quantise(cand, dt, tn), (prec, eta, dt, i, cand)
                        m = 2.0 * math.frexp(cand)[0]
                        near += (m - 1.0 < 2.0 ** -14) or (2.0 - m < 2.0 ** -13)
    print(f"candidates within 2^-14 of a power of two: {near}")
    assert near > 0


def test_initial_steps_and_selection_exact(nb, orc):
    """nb_init's first steps equal the oracle's start rule on the GPU forces; selection
    equals the oracle's definition on the GPU state."""
    snap = ics.config(1)
    with nb.Context(precision=1) as c:
        c.init(snap)
        st = c.state()
        for i in range(snap.n):
            assert st["dt"][i] == orc.initial_dt(st["a"][i], st["k"][i])
        for _ in range(20):
            tn, s = nb.nb_next_block(c.ctx)
            idx = nb.nb_get_active(c.ctx, s)
            st = c.state()
            tr, ir = orc.next_block(st["t"], st["dt"])
            assert tn == tr
            np.testing.assert_array_equal(idx, ir)
            nb.nb_step(c.ctx)


def _schedule(nb, c, steps):
    rows = []
    for _ in range(steps):
        tn, s = nb.nb_next_block(c.ctx)
        idx = nb.nb_get_active(c.ctx, s)
        rows.append((tn, s, zlib.crc32(np.ascontiguousarray(idx, dtype=np.int32).tobytes())))
        nb.nb_predict(c.ctx, tn)
        nb.nb_force_jerk(c.ctx, None, s, want=(False, False, False))
        nb.nb_correct(c.ctx, tn)
    return rows


def test_block_schedule_matches_golden_fp64(nb):
    """FP64 path: the first 16 block steps of the Plummer N = 1024 workload
    (t_next, s, active list) are identical to the oracle's stored schedule."""
    from tests.test_golden_schedule import load_schedule
    gold = load_schedule()
    snap = ics.config(1)
    with nb.Context(precision=1) as c:
        c.init(snap)
        rows = _schedule(nb, c, len(gold))
    for (k, tn, s, crc), got in zip(gold, rows):
        assert got == (tn, s, crc), (k, got, (tn, s, crc))


def test_block_schedule_matches_oracle_16k_fp64(nb, orc):
    """FP64 path, Plummer N = 16384: the first 16 block steps are identical to the oracle's."""
    snap = ics.config(2)
    sysr = orc.System(snap.m, snap.x, snap.v, snap.eps2, nthreads=orc.default_threads())
    with nb.Context(precision=1) as c:
        c.init(snap)
        rows = _schedule(nb, c, 16)
    for k, got in enumerate(rows):
        st, tn, idx = sysr.step()
        want = (tn, idx.size, zlib.crc32(np.ascontiguousarray(idx, dtype=np.int32).tobytes()))
        assert got == want, (k, got, want)


def _energy_cases():
    return [("plummer 16384", lambda: ics.config(2)),
            ("plummer 1000 (ragged tiles)", lambda: ics.plummer(1000, seed=77, eps=1.0 / 64)),
            ("plummer 3001 salpeter, eps 1/4096",
             lambda: ics.plummer(3001, seed=78, eps=1.0 / 4096, masses=ics.salpeter_masses(3001, seed=79))),
            ("random 130, eps 0", lambda: ics.random_state(130, seed=80, eps=0.0))]


@pytest.mark.parametrize("case", range(4))
def test_energy_matches_oracle(nb, orc, case):
    """K within 1e-14 and W within 1e-12 (relative) of the oracle's FP64 sums; the
    GPU sums W in double-single on the FP32 pipe (about 2^-44 per term)."""
    name, make = _energy_cases()[case]
    snap = make()
    K, W = orc.energy(snap.m, snap.x, snap.v, snap.eps2, nthreads=orc.default_threads())
    for prec in (0, 1):
        with nb.Context(precision=prec) as c:
            c.init(snap)
            E, Kg, Wg = nb.nb_energy(c.ctx)
        print(f"{name}, precision {prec}: W rel err {abs(Wg - W) / abs(W):.2e}, K rel err {abs(Kg - K) / K:.2e}")
        assert abs(Kg - K) < 1e-14 * max(1.0, K) and abs(Wg - W) < 1e-12 * abs(W), (name, prec)


@pytest.mark.parametrize("prec", [1, 0])
def test_energy_conservation_plummer_1k(nb, orc, prec):
    """Plummer N = 1024 to t = 1: |dE/E| within 2x the oracle's (and all particles at t = 1)."""
    snap = ics.config(1)
    sysr = orc.System(snap.m, snap.x, snap.v, snap.eps2, nthreads=orc.default_threads())
    E0r = sysr.energy()
    assert sysr.run(1.0) == 0
    dEr = abs(sysr.energy() - E0r) / abs(E0r)
    with nb.Context(precision=prec) as c:
        c.init(snap)
        E0, _, _ = nb.nb_energy(c.ctx)
        nb.nb_run(c.ctx, 1.0)
        E1, _, _ = nb.nb_energy(c.ctx)
        st = c.state()
        cnt = nb.nb_stats(c.ctx)
    dE = abs(E1 - E0) / abs(E0)
    print(f"prec {prec}: |dE/E| gpu {dE:.3e} oracle {dEr:.3e}; steps gpu {cnt['block_steps']} "
          f"oracle {sysr.counters['block_steps']}")
    assert np.all(st["t"] == 1.0)
    assert dE <= 2 * dEr + 1e-15, (dE, dEr)


@pytest.mark.parametrize("engine", [None, 0])
def test_run_step_and_timed_paths_agree(nb, engine):
    """The graph loop (nb_run), host-driven nb_step and nb_run_timed (with and without the
    phase breakdown) give the same state bitwise, with the small-block engine at its
    default size (None: small blocks run in the engine, in all four drivers alike) and
    switched off (0)."""
    snap = ics.plummer(3000, seed=5, eps=1.0 / 128)
    states = []
    for mode in ("run", "timed", "phases", "step"):
        with nb.Context(precision=0) as c:
            if engine is not None:
                nb.nb_set_engine(c.ctx, engine)
            c.init(snap)
            smax, cl = nb.nb_get_engine(c.ctx)
            assert (smax > 0) == (engine is None), (smax, cl)
            if mode == "run":
                nb.nb_run(c.ctx, 1.0 / 16)
            elif mode == "timed":
                t = nb.nb_run_timed(c.ctx, 1.0 / 16)
                assert t["force_launches"] > 0 and t["force_ms"] > 0
                assert (t["engine_steps"] > 0) == (engine is None), t
                assert t["force_interactions"] + t["engine_interactions"] == nb.nb_stats(c.ctx)["interactions"]
            elif mode == "phases":
                t = nb.nb_run_timed(c.ctx, 1.0 / 16, phases=True)
                ph = t["phase_ms"]
                assert t["force_launches"] > 0 and ph["force"] == t["force_ms"]
                assert min(ph[k] for k in ("select", "predict", "force", "correct")) > 0
                assert (ph["engine"] > 0) == (t["engine_steps"] > 0)
                print(f"engine {engine}: {t['force_launches']} four-kernel steps, {t['engine_steps']} engine "
                      f"steps; phases (ms) {ph}")
            else:
                while True:
                    tn, s = nb.nb_next_block(c.ctx)
                    if tn > 1.0 / 16:
                        break
                    nb.nb_step(c.ctx)
            states.append((c.state(), nb.nb_stats(c.ctx)))
    for st, cnt in states[1:]:
        for key in ("x", "v", "a", "k", "t", "dt"):
            np.testing.assert_array_equal(st[key], states[0][0][key])
        assert cnt["block_steps"] == states[0][1]["block_steps"]
        assert cnt["size_hist"] == states[0][1]["size_hist"]
    hist = states[0][1]["size_hist"]
    assert sum(hist) == states[0][1]["block_steps"] and hist[0] >= 0


def test_run_loop_multi_chunk_selection_matches_host_steps(nb):
    """At N = 262144 the run loop's selection at a known block time gives every CTA
    of its cluster several 8192-key chunks (ballots recomputed chunk by chunk); a
    short nb_run must end bitwise where host-driven nb_step does."""
    snap = ics.plummer(262144, seed=21, eps=1.0 / 1024)
    with nb.Context(precision=0) as c:
        c.init(snap)
        t1, _ = nb.nb_next_block(c.ctx)
    t_end = 8 * t1
    states = []
    for mode in ("run", "step"):
        with nb.Context(precision=0) as c:
            c.init(snap)
            if mode == "run":
                nb.nb_run(c.ctx, t_end)
            else:
                while True:
                    tn, _ = nb.nb_next_block(c.ctx)
                    if tn > t_end:
                        break
                    nb.nb_step(c.ctx)
            states.append((c.state(), nb.nb_stats(c.ctx)))
    (st_run, cnt_run), (st_step, cnt_step) = states
    assert cnt_run["block_steps"] == cnt_step["block_steps"] > 0
    for key in ("x", "v", "a", "k", "t", "dt"):
        np.testing.assert_array_equal(st_run[key], st_step[key])


def test_deterministic_and_resume_bitwise(nb):
    """Two runs agree bitwise; a run checkpointed at t = 1/16 and resumed in a new context
    ends bitwise equal to an uninterrupted run."""
    snap = ics.plummer(2000, seed=9, eps=1.0 / 128)
    with nb.Context(precision=0) as c:
        c.init(snap)
        nb.nb_run(c.ctx, 1.0 / 16)
        mid = c.state()
        nb.nb_run(c.ctx, 1.0 / 8)
        ref = c.state()
    with nb.Context(precision=0) as c:
        c.init(snap)
        nb.nb_run(c.ctx, 1.0 / 8)
        again = c.state()
    with nb.Context(precision=0) as c:
        c.init(snap)
        nb.nb_set_state(c.ctx, mid)
        nb.nb_run(c.ctx, 1.0 / 8)
        resumed = c.state()
    for key in ("x", "v", "t", "dt"):
        np.testing.assert_array_equal(again[key], ref[key])
        np.testing.assert_array_equal(resumed[key], ref[key])


def test_error_paths(nb):
    """Host-made failures: bad arguments, calls out of order, coincident bodies with eps = 0,
    a step underflow, and a device wait whose spin limit runs out (the context stays usable)."""
    snap = ics.plummer(500, seed=3, eps=0.01)
    with nb.Context() as c:
        c.init(snap)
        with pytest.raises(nb.NbError) as e:
            nb.nb_force_jerk(c.ctx, np.array([3, 2], dtype=np.int32))
        assert e.value.status == nb.NB_ERR_ARG
        with pytest.raises(nb.NbError) as e:
            nb.nb_force_jerk(c.ctx, np.array([0, 500], dtype=np.int32))
        assert e.value.status == nb.NB_ERR_ARG
        with pytest.raises(nb.NbError) as e:
            nb.nb_correct(c.ctx, 0.5)
        assert e.value.status == nb.NB_ERR_STATE
        tn, s = nb.nb_next_block(c.ctx)
        nb.nb_predict(c.ctx, tn)
        nb.nb_force_jerk(c.ctx, None, s, want=(False, False, False))
        with pytest.raises(nb.NbError) as e:
            nb.nb_correct(c.ctx, tn * 3)          # members are not due then
        assert e.value.status == nb.NB_ERR_STATE
    m = np.array([0.5, 0.5]); x = np.zeros((2, 3)); v = np.zeros((2, 3))
    with nb.Context() as c:
        with pytest.raises(nb.NbError) as e:
            nb.nb_init(c.ctx, m, x, v, 0.0)
        assert e.value.status == nb.NB_ERR_NONFINITE
    with nb.Context(dt_min=2.0 ** -5) as c:
        with pytest.raises(nb.NbError) as e:
            c.init(snap)
        assert e.value.status == nb.NB_ERR_DT_UNDERFLOW
    for prec in (0, 1):
        with nb.Context(precision=prec, inject=1, spin_limit=20000) as c:
            with pytest.raises(nb.NbError) as e:
                c.init(snap)
            assert e.value.status == nb.NB_ERR_TIMEOUT
            c.init(snap)                            # the context and the GPU stay usable
            nb.nb_run(c.ctx, 1.0 / 32)
            assert np.isfinite(nb.nb_energy(c.ctx)[0])


def test_dev_entry_points_match_host(nb):
    torch = pytest.importorskip("torch")
    snap = ics.plummer(1500, seed=4, eps=1.0 / 128)
    dev = torch.device("cuda:0")
    m = torch.tensor(snap.m, device=dev); x = torch.tensor(snap.x, device=dev); v = torch.tensor(snap.v, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    with nb.Context(stream=stream) as c:
        nb.nb_init_dev(c.ctx, snap.n, m.data_ptr(), x.data_ptr(), v.data_ptr(), snap.eps2)
        c.n = snap.n
        idx = np.arange(0, snap.n, 7, dtype=np.int32)
        a_h, k_h, p_h = nb.nb_force_jerk(c.ctx, idx)
        idx_d = torch.tensor(idx, device=dev)
        a_d = torch.zeros((idx.size, 3), dtype=torch.float64, device=dev)
        k_d = torch.zeros_like(a_d); p_d = torch.zeros(idx.size, dtype=torch.float64, device=dev)
        nb.nb_force_jerk_dev(c.ctx, idx_d.data_ptr(), idx.size, a_d.data_ptr(), k_d.data_ptr(), p_d.data_ptr())
        nb.nb_sync(c.ctx)
        np.testing.assert_array_equal(a_d.cpu().numpy(), a_h)
        np.testing.assert_array_equal(k_d.cpu().numpy(), k_h)
        np.testing.assert_array_equal(p_d.cpu().numpy(), p_h)
        st_dev = c.state()
    with nb.Context() as c:
        c.init(snap)
        st_host = c.state()
    # nb_init (host buffers) and nb_init_dev (device buffers) load the same state
    for key in ("m", "x", "v", "a", "k", "t", "dt"):
        np.testing.assert_array_equal(st_dev[key], st_host[key])
