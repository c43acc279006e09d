"""Pins of the FP64 oracle against facts it does not itself define.

Each test ties one oracle function to mathematics or physics that is fixed
independently of its code (closed forms, invariants, derivatives taken by
finite differences, exact reproduction of polynomials), so that a dropped
term, a wrong sign or a swapped index in the oracle fails at least one.
Passages: Sect. 2.1 of the paper (Eq. Force, the predictor and corrector
equations, Eq. timestep, the block-step rules).
"""
import math

import numpy as np
import pytest

import ics

ETA = 0.01


def _circular_binary(m1=0.3, m2=0.7, d=1.3):
    """Two bodies on a circular orbit, centre of mass at rest at the origin."""
    M = m1 + m2
    om = math.sqrt(M / d ** 3)
    x = np.array([[-m2 / M * d, 0, 0], [m1 / M * d, 0, 0]], dtype=float)
    v = np.array([[0, -m2 / M * d * om, 0], [0, m1 / M * d * om, 0]], dtype=float)
    return np.array([m1, m2]), x, v, om


# ------------------------------------------------------------------ force

def test_two_body_closed_form(orc):
    """|a_1| = m_2 d/(d^2+eps^2)^{3/2}, pointing at body 2; phi_1 = -m_2/(d^2+eps^2)^{1/2}."""
    m = np.array([0.25, 0.75])
    x = np.array([[0.1, -0.2, 0.3], [0.1 + 0.6, -0.2 - 0.8, 0.3]])   # separation 1.0
    v = np.zeros((2, 3))
    for eps in (0.0, 0.05, 0.5):
        a, k, phi = orc.force(m, x, v, eps * eps)
        d = 1.0
        mag = d / (d * d + eps * eps) ** 1.5
        u = (x[1] - x[0]) / d
        np.testing.assert_allclose(a[0], m[1] * mag * u, rtol=1e-14, atol=1e-16)
        np.testing.assert_allclose(a[1], -m[0] * mag * u, rtol=1e-14, atol=1e-16)
        np.testing.assert_allclose(phi, [-m[1] / math.hypot(d, eps), -m[0] / math.hypot(d, eps)], rtol=1e-14)
        np.testing.assert_array_equal(k, 0.0)


def test_acceleration_is_minus_gradient_of_potential(orc):
    """a_i = -grad_{x_i} phi_i, by 4th-order central differences of the oracle's phi."""
    s = ics.random_state(7, seed=11, eps=0.05)
    a, _, _ = orc.force(s.m, s.x, s.v, s.eps2)
    h = 1e-3
    for i in range(s.n):
        g = np.zeros(3)
        for c in range(3):
            vals = []
            for off in (-2, -1, 1, 2):
                xx = s.x.copy(); xx[i, c] += off * h
                vals.append(orc.force(s.m, xx, s.v, s.eps2, idx=[i])[2][0])
            g[c] = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
        np.testing.assert_allclose(a[i], -g, rtol=1e-8, atol=1e-9)


def test_jerk_is_time_derivative_of_acceleration(orc):
    """k_i = d a_i / dt along x(t) = x + v t, by 4th-order central differences."""
    s = ics.random_state(8, seed=12, eps=0.02)
    _, k, _ = orc.force(s.m, s.x, s.v, s.eps2)
    h = 1e-4
    acc = [orc.force(s.m, s.x + off * h * s.v, s.v, s.eps2)[0] for off in (-2, -1, 1, 2)]
    dadt = (acc[0] - 8 * acc[1] + 8 * acc[2] - acc[3]) / (12 * h)
    np.testing.assert_allclose(k, dadt, rtol=1e-7, atol=1e-8)


def test_newton_third_law(orc):
    """sum_i m_i a_i = 0 and sum_i m_i k_i = 0 (unequal masses)."""
    s = ics.random_state(300, seed=13, eps=0.01)
    a, k, _ = orc.force(s.m, s.x, s.v, s.eps2)
    scale_a = np.sum(s.m[:, None] * np.abs(a))
    scale_k = np.sum(s.m[:, None] * np.abs(k))
    assert np.all(np.abs((s.m[:, None] * a).sum(0)) < 1e-14 * scale_a)
    assert np.all(np.abs((s.m[:, None] * k).sum(0)) < 1e-14 * scale_k)


def test_circular_orbit_jerk(orc):
    """On a circular orbit |k| = omega |a| and k is perpendicular to a."""
    m, x, v, om = _circular_binary()
    a, k, _ = orc.force(m, x, v, 0.0)
    for i in range(2):
        assert abs(np.linalg.norm(k[i]) - om * np.linalg.norm(a[i])) < 1e-14 * np.linalg.norm(k[i])
        assert abs(np.dot(a[i], k[i])) < 1e-14 * np.linalg.norm(a[i]) * np.linalg.norm(k[i])
    # centripetal: a_i = -omega^2 x_i
    np.testing.assert_allclose(a, -om * om * x, rtol=1e-14, atol=1e-16)


def test_brute_force_high_precision(orc):
    """N <= 8: the oracle's FP64 sums agree with 40-digit sums to ~1e-15."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for n, seed in ((2, 1), (5, 2), (8, 3)):
        s = ics.random_state(n, seed=seed, eps=0.03)
        a, k, phi = orc.force(s.m, s.x, s.v, s.eps2)
        for i in range(n):
            A = [mp.mpf(0)] * 3; K = [mp.mpf(0)] * 3; P = mp.mpf(0)
            for j in range(n):
                if j == i:
                    continue
                r = [mp.mpf(s.x[j, c]) - mp.mpf(s.x[i, c]) for c in range(3)]
                w = [mp.mpf(s.v[j, c]) - mp.mpf(s.v[i, c]) for c in range(3)]
                d2 = sum(q * q for q in r) + mp.mpf(s.eps2)
                rw = sum(r[c] * w[c] for c in range(3))
                mj = mp.mpf(s.m[j])
                for c in range(3):
                    A[c] += mj * r[c] / d2 ** mp.mpf(1.5)
                    K[c] += mj * (w[c] / d2 ** mp.mpf(1.5) - 3 * rw * r[c] / d2 ** mp.mpf(2.5))
                P -= mj / mp.sqrt(d2)
            np.testing.assert_allclose(a[i], [float(q) for q in A], rtol=1e-13, atol=1e-15)
            np.testing.assert_allclose(k[i], [float(q) for q in K], rtol=1e-13, atol=1e-15)
            assert abs(phi[i] - float(P)) < 1e-14 * abs(float(P))


def test_self_exclusion_and_coincidence(orc):
    """j = i is excluded by index; distinct coincident bodies count when eps > 0."""
    m = np.array([0.5, 0.5])
    x = np.zeros((2, 3)); v = np.zeros((2, 3))
    a, k, phi = orc.force(m, x, v, 0.01)
    np.testing.assert_array_equal(a, 0.0)
    np.testing.assert_allclose(phi, [-0.5 / 0.1, -0.5 / 0.1], rtol=1e-15)
    a, k, phi = orc.force(m, x, v, 0.0)
    assert not np.all(np.isfinite(a)) or not np.all(np.isfinite(phi))
    # a single body feels nothing
    a, k, phi = orc.force(m[:1], x[:1], v[:1], 0.0)
    np.testing.assert_array_equal(a, 0.0); np.testing.assert_array_equal(phi, 0.0)


def test_energy_regular_tetrahedron(orc):
    """Four equal masses at the corners of a regular tetrahedron: W = -6 m^2 / sqrt(L^2+eps^2)."""
    L = 1.7
    base = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    x = base * L / math.sqrt(8.0)
    v = np.array([[0.1, 0, 0], [0, 0.2, 0], [0, 0, 0.3], [0.4, 0, 0]])
    m = np.full(4, 0.25)
    for eps in (0.0, 0.1):
        K, W = orc.energy(m, x, v, eps * eps)
        assert abs(W - (-6 * 0.25 ** 2 / math.sqrt(L * L + eps * eps))) < 1e-15
        assert abs(K - 0.5 * 0.25 * (0.01 + 0.04 + 0.09 + 0.16)) < 1e-16


# ------------------------------------------------------- predictor/corrector

def _poly(coef, t, der=0):
    """Value of the der-th derivative of sum_n coef[n] t^n (coef: [deg+1, 3])."""
    out = np.zeros(3)
    for nn in range(der, coef.shape[0]):
        out += coef[nn] * math.perm(nn, der) * t ** (nn - der)
    return out


def test_predictor_exact_on_cubic(orc):
    """The predictor reproduces any cubic trajectory exactly (it is its Taylor series)."""
    rng = ics.SplitMix64(5)
    coef = rng.uniform(12).reshape(4, 3) - 0.5
    t0, t1 = 0.25, 0.25 + 0.125
    x = _poly(coef, t0)[None]; v = _poly(coef, t0, 1)[None]
    a = _poly(coef, t0, 2)[None]; k = _poly(coef, t0, 3)[None]
    xp, vp = orc.predict(x, v, a, k, np.array([t0]), t1)
    np.testing.assert_allclose(xp[0], _poly(coef, t1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(vp[0], _poly(coef, t1, 1), rtol=0, atol=1e-15)


def test_corrector_exact_on_quintic(orc):
    """For a quintic x(t) the Hermite corrector is exact: a2, a3 are x'''' and x''''' at t0,
    and the corrected x, v equal x(t1), v(t1)."""
    rng = ics.SplitMix64(6)
    coef = rng.uniform(18).reshape(6, 3) - 0.5
    t0, dt = 0.5, 0.0625
    t1 = t0 + dt
    x = _poly(coef, t0)[None]; v = _poly(coef, t0, 1)[None]
    a0 = _poly(coef, t0, 2); k0 = _poly(coef, t0, 3)
    xp, vp = orc.predict(x, v, a0[None], k0[None], np.array([t0]), t1)
    a1 = _poly(coef, t1, 2); k1 = _poly(coef, t1, 3)
    x1, v1, a2, a3 = orc.correct_one(xp[0], vp[0], a0, k0, a1, k1, dt)
    np.testing.assert_allclose(a2, _poly(coef, t0, 4), rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(a3, _poly(coef, t0, 5), rtol=1e-8, atol=1e-8)
    np.testing.assert_allclose(x1, _poly(coef, t1), rtol=0, atol=1e-14)
    np.testing.assert_allclose(v1, _poly(coef, t1, 1), rtol=0, atol=1e-14)


def test_new_step_uses_end_of_step_derivatives(orc):
    """The step candidate after a correction is Eq. (timestep) evaluated with the exact
    derivatives at the END of the step (a, k, x and x' at t1) on a quintic path."""
    rng = ics.SplitMix64(7)
    coef = rng.uniform(18).reshape(6, 3) - 0.5
    t0, dt = 0.25, 0.03125
    t1 = t0 + dt
    x = _poly(coef, t0)[None]; v = _poly(coef, t0, 1)[None]
    a0 = _poly(coef, t0, 2); k0 = _poly(coef, t0, 3)
    xp, vp = orc.predict(x, v, a0[None], k0[None], np.array([t0]), t1)
    a1 = _poly(coef, t1, 2); k1 = _poly(coef, t1, 3)
    x1, v1, cand = orc.correct_particle(xp[0], vp[0], a0, k0, a1, k1, dt, ETA)
    want = orc.aarseth_dt(a1, k1, _poly(coef, t1, 4), _poly(coef, t1, 5), ETA)
    assert abs(cand - want) < 1e-9 * want
    np.testing.assert_allclose(x1, _poly(coef, t1), rtol=0, atol=1e-14)


# -------------------------------------------------------------- time steps

def test_aarseth_circular_orbit(orc):
    """Circular orbit: |a| = w^2 R, |k| = w^3 R, |a2| = w^4 R, |a3| = w^5 R gives dt = sqrt(nu)/w."""
    for om, R in ((1.0, 1.0), (3.7, 0.2), (0.01, 50.0)):
        a = np.array([-om ** 2 * R, 0, 0]); k = np.array([0, -om ** 3 * R, 0])
        a2 = np.array([om ** 4 * R, 0, 0]); a3 = np.array([0, om ** 5 * R, 0])
        dt = orc.aarseth_dt(a, k, a2, a3, ETA)
        assert abs(dt - math.sqrt(ETA) / om) < 1e-15 * dt * 8


def test_aarseth_uses_each_derivative(orc):
    """Scaling one derivative at a time moves dt the way the formula's structure demands:
    dt is unchanged under a -> c^2 a, k -> c^3 k ... only in the joint time rescaling t -> t/c."""
    a = np.array([1.0, 0.2, -0.3]); k = np.array([0.5, 1.1, 0.0])
    a2 = np.array([-2.0, 0.4, 1.0]); a3 = np.array([0.3, -4.0, 2.0])
    dt = orc.aarseth_dt(a, k, a2, a3, ETA)
    for c in (2.0, 0.125):
        # a time-unit change by c multiplies each derivative of order p by c^p
        dtc = orc.aarseth_dt(a * c ** 2, k * c ** 3, a2 * c ** 4, a3 * c ** 5, ETA)
        assert abs(dtc - dt / c) < 1e-14 * dt / c
        # amplitude change leaves dt invariant
        dtl = orc.aarseth_dt(a * c, k * c, a2 * c, a3 * c, ETA)
        assert abs(dtl - dt) < 1e-14 * dt
    # larger higher derivatives always shorten the step
    assert orc.aarseth_dt(a, k, a2, 2 * a3, ETA) < dt
    assert orc.aarseth_dt(a, 0.5 * k, a2, a3, ETA) != dt


def test_quantise_rules(orc):
    q = orc.quantise
    # largest power of two below the candidate when shrinking, any number of levels
    assert q(0.3, 0.5, 0.5, dt_max=1.0) == 0.25
    assert q(0.0009, 0.5, 0.5, dt_max=1.0) == 2.0 ** -11
    # unchanged when the candidate lies in [dt_old, 2 dt_old)
    assert q(0.126, 0.125, 0.5, dt_max=1.0) == 0.125
    # doubling only at times commensurate with 2 dt_old, at most one level, capped by dt_max
    assert q(10.0, 2.0 ** -8, 3 * 2.0 ** -7) == 2.0 ** -7
    assert q(10.0, 2.0 ** -8, 3 * 2.0 ** -8) == 2.0 ** -8
    assert q(10.0, 1.0 / 16, 1.0) == 1.0 / 16
    assert q(float("inf"), 2.0 ** -8, 2.0 ** -7) == 2.0 ** -7
    # a candidate whose power of two is exactly 2 dt_old doubles as well
    assert q(1.5 * 2.0 ** -7, 2.0 ** -8, 2.0 ** -7) == 2.0 ** -7
    assert q(1.5 * 2.0 ** -7, 2.0 ** -8, 3 * 2.0 ** -8) == 2.0 ** -8
    # errors
    assert q(float("nan"), 0.5, 0.5, dt_max=1.0) == 0.0
    assert q(0.0, 0.5, 0.5, dt_max=1.0) == 0.0
    assert q(2.0 ** -45, 2.0 ** -30, 1.0) == 0.0
    # result is always an exact power of two
    rng = ics.SplitMix64(9)
    for c in rng.uniform(200) * 0.1 + 1e-9:
        r = q(c, 1.0 / 16, 1.0)
        assert r <= c and r > c / 2 and math.frexp(r)[0] == 0.5


def test_initial_step(orc):
    a = np.array([3.0, 0.0, 4.0]); k = np.array([0.0, 2.0, 0.0])   # eta |a|/|k| = 0.025
    assert orc.initial_dt(a, k, ETA) == 2.0 ** -6
    assert orc.initial_dt(a, np.zeros(3), ETA) == 1.0 / 16
    assert orc.initial_dt(a * 100, k, ETA) == 1.0 / 16


def test_next_block_definition(orc):
    rng = ics.SplitMix64(10)
    n = 500
    lev = (rng.uniform(n) * 6).astype(int)
    dt = 2.0 ** -(4 + lev)
    t = np.floor(rng.uniform(n) * 8) * dt      # t_i multiple of dt_i
    tn, idx = orc.next_block(t, dt)
    assert tn == np.min(t + dt)
    np.testing.assert_array_equal(idx, np.nonzero(t + dt == tn)[0])
    tn0, idx0 = orc.next_block(np.zeros(0), np.zeros(0))
    assert idx0.size == 0 and math.isinf(tn0)


# ------------------------------------------------------------- integration

def _kepler(e=0.5, P=1.0, m1=0.5, m2=0.5):
    """Binary at apocentre with period P (G = 1): a^3 = M (P / 2 pi)^2."""
    M = m1 + m2
    sma = (M * (P / (2 * math.pi)) ** 2) ** (1.0 / 3.0)
    r = sma * (1 + e)
    vrel = math.sqrt(M * (1 - e) / (sma * (1 + e)))
    x = np.array([[-m2 / M * r, 0, 0], [m1 / M * r, 0, 0]])
    v = np.array([[0, -m2 / M * vrel, 0], [0, m1 / M * vrel, 0]])
    return np.array([m1, m2]), x, v, sma


def _elements(m, x, v):
    M = m.sum()
    r = x[1] - x[0]; w = v[1] - v[0]
    E = 0.5 * w @ w - M / np.linalg.norm(r)
    h = np.cross(r, w)
    evec = np.cross(w, h) / M - r / np.linalg.norm(r)
    return -M / (2 * E), np.linalg.norm(evec)


def test_kepler_orbit_ten_periods(orc):
    """e = 0.5 binary, eps = 0, block steps: after ten periods the semi-major axis, the
    eccentricity and the phase (return to apocentre at t = 10 P) match the closed-form
    orbit, and the errors converge at least at 4th order in dt (dt ~ sqrt(eta), so
    eta / 4 halves every step and must cut the errors by >~ 2^4)."""
    res = {}
    for eta in (ETA, ETA / 4):
        m, x, v, sma = _kepler()
        s = orc.System(m, x, v, 0.0, eta=eta)
        assert s.status == 0
        assert s.run(10.0) == 0
        assert np.all(s.t == 10.0)
        a_fin, e_fin = _elements(s.m, s.x, s.v)
        r0 = x[1] - x[0]
        res[eta] = (abs(a_fin / sma - 1), abs(e_fin - 0.5),
                    np.linalg.norm((s.x[1] - s.x[0]) - r0) / np.linalg.norm(r0))
        # centre of mass stays at rest at the origin (momentum conservation)
        assert np.linalg.norm((s.m[:, None] * s.v).sum(0)) < 1e-14
        assert s.counters["block_steps"] > 100
    da, de, dph = res[ETA]
    assert da < 1e-5 and de < 1e-5 and dph < 3e-4, res
    for q in range(3):
        assert res[ETA][q] / res[ETA / 4][q] > 12, res


def test_hermite_fourth_order(orc):
    """With a fixed shared step the energy error after one orbit falls at least as dt^4
    (a lower-order slip in the predictor or corrector gives a ratio <= 8 per halving);
    a ratio above 2^5 would mean the error is not truncation error at all."""
    m, x, v, _ = _kepler(e=0.5)
    errs = []
    for h in (2.0 ** -7, 2.0 ** -8, 2.0 ** -9, 2.0 ** -10):
        s = orc.System(m, x, v, 0.0, eta=ETA, dt_fixed=h)
        E0 = s.energy()
        assert s.run(1.0) == 0
        errs.append(abs(s.energy() - E0))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(14 < r < 34 for r in ratios), (errs, ratios)


def test_plummer_energy_and_block_invariants(orc):
    """Plummer N = 1024 (eps = 1/256, eta = 0.01) to t = 1: energy conserved, every particle
    lands on t = 1, every block step time is a multiple of each active particle's step."""
    snap = ics.config(1)
    s = orc.System(snap.m, snap.x, snap.v, snap.eps2, eta=ETA, nthreads=orc.default_threads())
    assert s.status == 0
    E0 = s.energy()
    t_prev = 0.0
    for _ in range(50):
        st, tn, idx = s.step()
        assert st == 0 and tn >= t_prev and idx.size >= 1
        assert np.all(s.t[idx] == tn)
        assert np.all(np.floor(s.t / s.dt) * s.dt == s.t)
        t_prev = tn
    assert s.run(1.0) == 0
    assert np.all(s.t == 1.0)
    dE = abs(s.energy() - E0) / abs(E0)
    assert dE < 1e-6, dE
    # individual steps evaluate the two halves of a pair force at different times, so
    # momentum is conserved only to truncation level, not to round-off
    mom = np.linalg.norm((s.m[:, None] * s.v).sum(0))
    assert mom < 1e-6


def test_error_codes(orc):
    """Coincident bodies with eps = 0 give a non-finite error; dt below dt_min underflows."""
    m = np.array([0.5, 0.5]); x = np.zeros((2, 3)); v = np.zeros((2, 3))
    s = orc.System(m, x, v, 0.0)
    assert s.status == orc.ERR_NONFINITE
    m, x, v, _ = _kepler()
    s = orc.System(m, x, v, 0.0, dt_min=2.0 ** -3)
    assert s.status == orc.ERR_DT_UNDERFLOW


# ------------------------------------------------------------------ perturber lists

def _binary_at_origin(d, m1, m2):
    """Members on the x axis with their centre of mass at the origin."""
    mb = m1 + m2
    return np.array([[-m2 / mb * d, 0.0, 0.0], [m1 / mb * d, 0.0, 0.0]])


def test_perturber_threshold_closed_form(orc):
    """Sect. 3.1, tidal reading: star j perturbs the binary iff 2 m_j d^3 / (m_b r^3) >= gamma,
    i.e. r <= r_c = d (2 m_j / (gamma m_b))^(1/3) from the centre of mass. Stars placed at
    r_c (1 -+ 1e-6) on the y and z axes (and one along -x) fall on the predicted sides, for
    several star masses and gammas."""
    for gamma, d, mj in ((1e-7, 1e-3, 1e-3), (1e-4, 2.5e-2, 0.3), (1e-2, 0.5, 2.0)):
        xb = _binary_at_origin(d, 0.5, 0.5)
        rc = d * (2.0 * mj / gamma) ** (1.0 / 3.0)
        stars = []
        inside = []
        for q, (f, axis) in enumerate(((1 - 1e-6, 1), (1 + 1e-6, 1), (1 - 1e-6, 2), (1 + 1e-6, 2),
                                       (0.5, 2), (2.0, 1), (1 - 1e-6, 0))):
            p = np.zeros(3)
            p[axis] = rc * f * (-1.0 if axis == 0 else 1.0)
            stars.append(p)
            inside.append(f < 1.0)
        x = np.vstack([xb, np.array(stars)])
        m = np.concatenate([[0.5, 0.5], np.full(len(stars), mj)])
        lists, counts = orc.perturbers(m, x, [[0, 1]], gamma=gamma, nmax=16)
        want = [2 + q for q, ins in enumerate(inside) if ins]
        assert counts[0] == len(want), (gamma, counts[0], want)
        assert list(lists[0, :len(want)]) == want and np.all(lists[0, len(want):] == -1)


def test_perturber_distance_from_centre_of_mass(orc):
    """Unequal members (0.8, 0.2): distances count from the centre of mass, not from either
    member. A star at 0.999 r_c on +x is 1.006 r_c from member 1; one at 1.001 r_c on -x is
    0.994 r_c from member 1. Only the centre-of-mass reading lists the first and not the
    second."""
    gamma, d, mj = 1e-7, 1e-3, 1e-3
    m1, m2 = 0.8, 0.2
    xb = _binary_at_origin(d, m1, m2)
    rc = d * (2.0 * mj / (gamma * (m1 + m2))) ** (1.0 / 3.0)
    x = np.vstack([xb, [[0.999 * rc, 0.0, 0.0], [-1.001 * rc, 0.0, 0.0]]])
    m = np.array([m1, m2, mj, mj])
    lists, counts = orc.perturbers(m, x, [[0, 1]], gamma=gamma, nmax=4)
    assert counts[0] == 1 and lists[0, 0] == 2


def test_perturber_members_order_truncation(orc):
    """The members never perturb their own binary; the list holds the first nmax perturbers
    in ascending index (the serial scan's order), and the count all of them."""
    gamma, d = 1e-3, 1e-2
    rng = np.random.default_rng(5)
    n = 40
    x = rng.normal(size=(n, 3)) * 0.01   # everything well inside r_c
    m = np.full(n, 1.0 / n)
    x[7] = [0.0, 0.0, 0.0]
    x[23] = [d, 0.0, 0.0]
    lists, counts = orc.perturbers(m, x, [[23, 7]], gamma=gamma, nmax=5)
    assert counts[0] == n - 2
    assert list(lists[0]) == [0, 1, 2, 3, 4]
    lists, counts = orc.perturbers(m, x, [[23, 7]], gamma=gamma, nmax=64)
    assert list(lists[0, :n - 2]) == [j for j in range(n) if j not in (7, 23)]
    assert np.all(lists[0, n - 2:] == -1)


def test_perturber_ranges_merge_and_exact_scalings(orc):
    """Lists over j-ranges, concatenated in range order and cut at nmax, are the full list
    (the parallel code's merge, Sect. 3.1), with counts summed; scaling all positions or all
    masses by a power of two leaves the lists unchanged (the criterion is scale free and such
    scalings are exact)."""
    snap = ics.plummer_binaries(600, 40, 31, 1e-3, a_lo=1e-3, a_hi=5e-2)
    pairs = snap.meta["pairs"]
    full, cfull = orc.perturbers(snap.m, snap.x, pairs, gamma=1e-7, nmax=32)
    assert np.any(cfull > 32) and np.any((cfull > 0) & (cfull < 32))
    parts = [orc.perturbers(snap.m, snap.x, pairs, gamma=1e-7, nmax=32, j_lo=lo, j_hi=hi)
             for lo, hi in ((0, 137), (137, 400), (400, 600))]
    for b in range(pairs.shape[0]):
        cat = np.concatenate([p[0][b][p[0][b] >= 0] for p in parts])[:32]
        assert list(cat) == list(full[b][full[b] >= 0])
        assert sum(int(p[1][b]) for p in parts) == cfull[b]
    l2, c2 = orc.perturbers(snap.m, snap.x * 4.0, pairs, gamma=1e-7, nmax=32)
    l3, c3 = orc.perturbers(snap.m * 0.5, snap.x, pairs, gamma=1e-7, nmax=32)
    assert np.array_equal(l2, full) and np.array_equal(c2, cfull)
    assert np.array_equal(l3, full) and np.array_equal(c3, cfull)
