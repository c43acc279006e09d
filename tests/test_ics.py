"""Pins of the seeded input generators (no integrator arithmetic involved)."""
import math
import os

import numpy as np
import pytest

import ics

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_splitmix64_reference_value():
    (row,) = _golden_rows("splitmix64_seed0.txt")
    assert int(ics.SplitMix64(0).next_u64(1)[0]) == int(row[0], 16)


def test_splitmix64_stream_is_contiguous():
    a = ics.SplitMix64(42).next_u64(10)
    g = ics.SplitMix64(42)
    b = np.concatenate([g.next_u64(3), g.next_u64(7)])
    np.testing.assert_array_equal(a, b)
    u = ics.SplitMix64(1).uniform(100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005


def test_plummer_nbody_units_and_profile():
    """E = -1/4 with W = -1/2, K = 1/4 (virial), and the radial mass profile follows
    M(r) = r^3/(1+r^2)^{3/2} (KS test in the raw length unit, truncated at 0.999)."""
    from scipy import stats
    s = ics.plummer(16384, seed=3, eps=0.0)
    K = 0.5 * np.sum(s.m * np.sum(s.v ** 2, axis=1))
    W = ics.unsoftened_potential_energy(s.m, s.x)
    assert abs(K - 0.25) < 1e-13 and abs(W + 0.5) < 1e-12
    np.testing.assert_allclose((s.m[:, None] * s.x).sum(0), 0.0, atol=1e-14)
    np.testing.assert_allclose((s.m[:, None] * s.v).sum(0), 0.0, atol=1e-14)
    lam = -2.0 * s.meta["w_raw"]
    r = np.linalg.norm(s.x, axis=1) / lam

    def cdf(rr):
        return np.minimum(rr ** 3 / (1 + rr * rr) ** 1.5 / 0.999, 1.0)

    assert stats.kstest(r, cdf).pvalue > 1e-3
    # the scale factor is close to the continuum value 3 pi / 16
    assert abs(lam / (3 * math.pi / 16) - 1) < 0.02


def test_king_concentration_matches_tables():
    for w0, c in _golden_rows("king_concentration.txt"):
        r, w, dw, rt = ics.king_profile(float(w0))
        assert abs(math.log10(rt) - float(c)) < 0.01, (w0, math.log10(rt), c)


def test_king_sample_profile():
    """Radii follow the ODE's enclosed mass; velocities stay below the local escape speed."""
    from scipy import stats
    s = ics.king(20000, seed=4, w0=6.0, eps=1e-3)
    K = 0.5 * np.sum(s.m * np.sum(s.v ** 2, axis=1))
    assert abs(K - 0.25) < 1e-12
    W = ics.unsoftened_potential_energy(s.m, s.x)
    assert abs(W + 0.5) < 0.02          # continuum scaling: sampling noise only
    r_grid, w_grid, dw_grid, rt = ics.king_profile(6.0)
    mass = -(r_grid ** 2) * dw_grid
    lam = -2.0 * s.meta["w_raw"]
    r = np.linalg.norm(s.x, axis=1) / lam
    assert stats.kstest(r, lambda q: np.interp(q, r_grid, mass / mass[-1])).pvalue > 1e-3
    assert r.max() <= rt * 1.05


def test_salpeter_slope():
    m = ics.salpeter_masses(200000, seed=5)
    assert abs(m.sum() - 1.0) < 1e-12
    ratio = m.max() / m.min()
    assert ratio <= 1000.0 * (1 + 1e-9)
    # dN/dlog m ~ m^(1 - 2.35): fit the log-histogram
    lm = np.log10(m / m.min() * 0.1)
    h, e = np.histogram(lm, bins=24, range=(-1, 2))
    c = 0.5 * (e[1:] + e[:-1])
    ok = h > 50
    slope = np.polyfit(c[ok], np.log10(h[ok]), 1)[0]
    assert abs(slope - (1 - 2.35)) < 0.05, slope


def test_ensemble_sizes():
    rng = ics.SplitMix64(ics.BASE_SEED + 4)
    u = rng.uniform(256)
    n = np.rint(np.exp(math.log(256) + u * (math.log(8192) - math.log(256))))
    assert n.min() >= 256 and n.max() <= 8192
    small = ics.ensemble(3, seed=99, n_lo=64, n_hi=128)
    assert all(64 <= c.n <= 128 for c in small)
    assert all(abs(c.eps2 - (4.0 / c.n) ** 2) < 1e-18 for c in small)


def test_configs_are_seeded():
    a = ics.config(1)
    b = ics.config(1)
    np.testing.assert_array_equal(a.x, b.x)
    assert a.n == 1024 and a.eps2 == (1 / 256) ** 2
    c = ics.config(3, n=2048)
    assert c.m.max() / c.m.min() > 10
