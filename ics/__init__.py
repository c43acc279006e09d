"""Seeded synthetic initial conditions for the direct N-body path.

This module generates inputs only. It is shared by the FP64 oracle tests, the
CUDA parity tests and ``bench.py``; it holds no force, predictor, corrector or
timestep arithmetic of the integrator.

Contents
--------
* ``SplitMix64`` -- the counter-based generator of Steele, Lea & Flood (2014),
  written from its published definition (golden-ratio increment, two
  xor-shift-multiply rounds).
* ``plummer`` -- a Plummer (1911) sphere sampled with the method of Aarseth,
  Henon & Wielen (1974), the density profile used for the paper's timing runs
  (Sect. 4: 1024-65536 equal-mass stars).
* ``king`` -- a King (1966) lowered-isothermal model, from its Poisson ODE
  integrated with classical RK4 (the paper's concentrated models, Sect. 4).
* ``salpeter_masses`` -- dN/dm ~ m^-2.35 on [0.1, 100] by inverse CDF.
* ``ensemble`` -- a batch of independent Plummer clusters with log-uniform N.
* ``config`` -- the five named workloads with their fixed seeds.

Units: N-body units (Heggie & Mathieu 1986), G = M = 1, E = -1/4 with the
*unsoftened* potential energy. For N <= 65536 the scaling uses the exact pair
potential energy of the sample; above that it uses the continuum model's energy
(an exact pair sum over 10^12 pairs is not affordable for an input generator).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "SplitMix64", "Snapshot", "plummer", "king", "king_profile", "salpeter_masses",
    "ensemble", "config", "random_state", "BASE_SEED", "EXACT_SCALING_MAX_N",
]

BASE_SEED = 20071106
EXACT_SCALING_MAX_N = 65536

_MASK64 = (1 << 64) - 1
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """SplitMix64 stream. ``next_u64(n)`` returns the next n outputs in order.

    state_{k+1} = state_k + 0x9E3779B97F4A7C15 (mod 2^64); the output is the
    new state passed through z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
    z *= 0x94D049BB133111EB; z ^= z>>31.
    """

    def __init__(self, seed: int):
        self.state = np.uint64(int(seed) & _MASK64)

    def next_u64(self, n: int) -> np.ndarray:
        n = int(n)
        if n <= 0:
            return np.zeros(0, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = self.state + np.arange(1, n + 1, dtype=np.uint64) * _GAMMA
            self.state = z[-1]
            z = (z ^ (z >> np.uint64(30))) * _MIX1
            z = (z ^ (z >> np.uint64(27))) * _MIX2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform_open(self, n: int) -> np.ndarray:
        """Doubles in (0, 1): the 53-bit grid shifted by half a step."""
        return ((self.next_u64(n) >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


@dataclass
class Snapshot:
    """A particle system: m[n], x[n,3], v[n,3] (float64, C order) and eps2."""
    m: np.ndarray
    x: np.ndarray
    v: np.ndarray
    eps2: float
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.m.shape[0])

    def copy(self) -> "Snapshot":
        return Snapshot(self.m.copy(), self.x.copy(), self.v.copy(), self.eps2, self.name, dict(self.meta))


# ---------------------------------------------------------------- helpers

def _isotropic(rng: SplitMix64, radius: np.ndarray) -> np.ndarray:
    """Points of length ``radius`` with uniformly distributed directions."""
    n = radius.shape[0]
    u = rng.uniform(n)
    w = rng.uniform(n)
    z = (1.0 - 2.0 * u) * radius
    rho = np.sqrt(np.maximum(radius * radius - z * z, 0.0))
    ang = 2.0 * math.pi * w
    return np.stack([rho * np.cos(ang), rho * np.sin(ang), z], axis=1)


def _recentre(m: np.ndarray, x: np.ndarray, v: np.ndarray) -> None:
    mt = m.sum()
    x -= (m[:, None] * x).sum(axis=0) / mt
    v -= (m[:, None] * v).sum(axis=0) / mt


def _kinetic(m: np.ndarray, v: np.ndarray) -> float:
    return float(0.5 * np.sum(m * np.sum(v * v, axis=1)))


def unsoftened_potential_energy(m: np.ndarray, x: np.ndarray, rows: int = 256) -> float:
    """W = -sum_{i<j} m_i m_j / |x_i - x_j| by chunked distance matrices.

    Used only to put a sample into N-body units (the IC definition), never as
    a check of the integrator.
    """
    from scipy.spatial.distance import cdist

    n = m.shape[0]
    total = 0.0
    for a in range(0, n, rows):
        b = min(n, a + rows)
        d = cdist(x[a:b], x)
        d[np.arange(b - a), np.arange(a, b)] = np.inf
        total += float(m[a:b] @ ((1.0 / d) @ m))
    return -0.5 * total


def _to_nbody_units(m, x, v, w_model=None):
    """Scale lengths so that W = -1/2 and velocities so that K = 1/4."""
    _recentre(m, x, v)
    w = unsoftened_potential_energy(m, x) if w_model is None else w_model
    lam = -2.0 * w            # r' = lam r  =>  W' = W / lam = -1/2
    x *= lam
    k = _kinetic(m, v)
    v *= math.sqrt(0.25 / k)
    return w


# ---------------------------------------------------------------- samplers

def salpeter_masses(n: int, seed: int, alpha: float = 2.35, m_lo: float = 0.1,
                    m_hi: float = 100.0) -> np.ndarray:
    """Masses with dN/dm ~ m^-alpha on [m_lo, m_hi] by inverse CDF, then sum(m) = 1."""
    rng = SplitMix64(seed)
    u = rng.uniform(n)
    p = 1.0 - alpha
    lo, hi = m_lo ** p, m_hi ** p
    mass = (lo + u * (hi - lo)) ** (1.0 / p)
    return mass / mass.sum()


def plummer(n: int, seed: int, eps: float, masses: np.ndarray | None = None,
            mfrac: float = 0.999, scale: str = "auto", name: str = "plummer") -> Snapshot:
    """Plummer sphere by Aarseth, Henon & Wielen (1974), in N-body units.

    Radii from the inverted cumulative mass M(r) = r^3/(1+r^2)^{3/2}, truncated
    at mass fraction ``mfrac``; speeds q*v_esc with q drawn by rejection from
    g(q) = q^2 (1-q^2)^{7/2} (bounded by 0.1); isotropic directions.
    """
    rng = SplitMix64(seed)
    m = np.full(n, 1.0 / n) if masses is None else np.asarray(masses, dtype=np.float64).copy()
    assert m.shape == (n,)
    xm = rng.uniform_open(n) * mfrac
    r = 1.0 / np.sqrt(xm ** (-2.0 / 3.0) - 1.0)
    x = _isotropic(rng, r)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x4 = rng.uniform(todo.size)
        x5 = rng.uniform(todo.size)
        ok = 0.1 * x5 < x4 * x4 * (1.0 - x4 * x4) ** 3.5
        q[todo[ok]] = x4[ok]
        todo = todo[~ok]
    vesc = math.sqrt(2.0) * (1.0 + r * r) ** -0.25
    v = _isotropic(rng, q * vesc)
    exact = (scale == "exact") or (scale == "auto" and n <= EXACT_SCALING_MAX_N)
    # continuum Plummer model with a = 1, M = 1: W = -3 pi / 32
    w = _to_nbody_units(m, x, v, None if exact else -3.0 * math.pi / 32.0)
    meta = {"seed": seed, "model": "plummer", "scaling": "exact" if exact else "continuum", "w_raw": w}
    return Snapshot(m, np.ascontiguousarray(x), np.ascontiguousarray(v), float(eps) ** 2, name, meta)


def _king_density(w: np.ndarray | float):
    """rho(W)/rho_1 = e^W erf(sqrt W) - sqrt(4W/pi) (1 + 2W/3) (King 1966); 0 for W <= 0."""
    from scipy.special import erf

    w = np.maximum(np.asarray(w, dtype=np.float64), 0.0)
    return np.exp(w) * erf(np.sqrt(w)) - np.sqrt(4.0 * w / math.pi) * (1.0 + 2.0 * w / 3.0)


def king_profile(w0: float, h: float = 1e-3, r_max: float = 1e4):
    """Integrate W'' + (2/r) W' = -9 rho(W)/rho(W0) with RK4 out to W = 0.

    Radii are in units of the King radius r0 = sqrt(9 sigma^2 / (4 pi G rho0)).
    Returns (r, W, dW/dr, r_t); the enclosed mass is M(r) = -r^2 dW/dr in units
    G = sigma = r0 = 1.
    """
    rho0 = float(_king_density(w0))

    def rhs(r, y):
        w, dw = y
        return np.array([dw, -9.0 * float(_king_density(w)) / rho0 - 2.0 * dw / r])

    # start off-centre with the series W = W0 - (3/2) r^2 (since lap W = -9 at r = 0)
    r = h
    y = np.array([w0 - 1.5 * h * h, -3.0 * h])
    rs, ws, dws = [0.0, r], [w0, y[0]], [0.0, y[1]]
    step = h
    while y[0] > 0.0 and r < r_max:
        k1 = rhs(r, y)
        k2 = rhs(r + 0.5 * step, y + 0.5 * step * k1)
        k3 = rhs(r + 0.5 * step, y + 0.5 * step * k2)
        k4 = rhs(r + step, y + step * k3)
        y_new = y + (step / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        r_new = r + step
        if y_new[0] <= 0.0:
            # linear root of W between r and r_new
            frac = y[0] / (y[0] - y_new[0])
            r_t = r + frac * step
            dw_t = y[1] + frac * (y_new[1] - y[1])
            rs.append(r_t); ws.append(0.0); dws.append(dw_t)
            return np.array(rs), np.array(ws), np.array(dws), r_t
        r, y = r_new, y_new
        rs.append(r); ws.append(y[0]); dws.append(y[1])
        step = min(step * 1.01, 0.02 * max(r, 1.0))   # grow the step in the halo
    raise RuntimeError("King profile did not reach W = 0")


def king(n: int, seed: int, w0: float, eps: float, name: str = "king") -> Snapshot:
    """Equal-mass King (1966) model of depth W0, in N-body units.

    Radii by inverting the enclosed-mass fraction of the ODE solution; speeds by
    rejection from f(v) ~ v^2 (exp(W - v^2/2) - 1), v < sqrt(2W) (sigma = 1);
    isotropic directions. Lengths are scaled with the continuum model's
    potential energy -int M dM / r, velocities with the sample's K.
    """
    rng = SplitMix64(seed)
    r_grid, w_grid, dw_grid, r_t = king_profile(w0)
    mass = -(r_grid ** 2) * dw_grid
    mass[0] = 0.0
    mt = mass[-1]
    frac = mass / mt
    r = np.interp(rng.uniform_open(n), frac, r_grid)
    x = _isotropic(rng, r)
    w_at = np.maximum(np.interp(r, r_grid, w_grid), 0.0)
    vesc = np.sqrt(2.0 * w_at)
    # bound of g(v) = v^2 (e^{W - v^2/2} - 1) on [0, sqrt(2W)]: g <= 2 e^{W-1} (W >= 1) or 2W,
    # and g <= e^W max_y y (W - y/2) = e^W W^2 / 2 (from e^x - 1 <= x e^x); take the smaller
    b1 = np.where(w_at >= 1.0, 2.0 * np.exp(w_at - 1.0), 2.0 * w_at)
    bound = np.minimum(b1, np.exp(w_at) * w_at * w_at / 2.0)
    speed = np.zeros(n)
    todo = np.nonzero(vesc > 0.0)[0]
    while todo.size:
        kk = int(min(64, max(1, (1 << 18) // todo.size)))       # candidates per particle this round
        vv = vesc[todo, None] * rng.uniform(todo.size * kk).reshape(todo.size, kk)
        g = vv * vv * (np.exp(w_at[todo, None] - 0.5 * vv * vv) - 1.0)
        ok = rng.uniform(todo.size * kk).reshape(todo.size, kk) * bound[todo, None] < g
        hit = ok.any(axis=1)
        first = np.argmax(ok, axis=1)
        speed[todo[hit]] = vv[np.nonzero(hit)[0], first[hit]]
        todo = todo[~hit]
    v = _isotropic(rng, speed)
    m = np.full(n, 1.0 / n)
    # continuum energy of the unit-mass model: W = -int F dF / r
    fm = 0.5 * (frac[1:] + frac[:-1])
    rm = 0.5 * (r_grid[1:] + r_grid[:-1])
    w_cont = -float(np.sum(fm * np.diff(frac) / rm))
    _to_nbody_units(m, x, v, w_cont)
    meta = {"seed": seed, "model": "king", "w0": w0, "r_t": r_t,
            "c": math.log10(r_t), "scaling": "continuum", "w_raw": w_cont}
    return Snapshot(m, np.ascontiguousarray(x), np.ascontiguousarray(v), float(eps) ** 2, name, meta)


def ensemble(n_clusters: int, seed: int, n_lo: int = 256, n_hi: int = 8192,
             eps_num: float = 4.0) -> list[Snapshot]:
    """Independent Plummer clusters, N_c = round(exp(U[ln n_lo, ln n_hi])), eps = eps_num / N_c.

    The cluster sizes come from the stream ``seed``; cluster c is drawn from
    the stream ``seed + 1000 (c + 1)``.
    """
    rng = SplitMix64(seed)
    u = rng.uniform(n_clusters)
    sizes = np.rint(np.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))).astype(np.int64)
    out = []
    for c, nc in enumerate(sizes):
        s = plummer(int(nc), seed + 1000 * (c + 1), eps=eps_num / float(nc), name=f"cluster{c}")
        out.append(s)
    return out


def plummer_binaries(n: int, n_bin: int, seed: int, eps: float, a_lo: float = 1e-4,
                     a_hi: float = 1e-2) -> Snapshot:
    """A Plummer model of n stars of which 2 n_bin are in primordial binaries (equal masses
    1/n): a Plummer model of n - n_bin centres of mass (each binary centre twice the mass),
    then the first n_bin centres (in the stream's order) split into two stars at a
    separation d drawn log-uniformly in [a_lo, a_hi], isotropic orientation, on a circular
    relative orbit (|v_rel|^2 = m_b / d) in a random plane. Member 1 of binary b keeps index
    b, member 2 takes index n - n_bin + b. ``meta["pairs"]`` holds the [n_bin, 2] index pairs.
    """
    n_c = n - n_bin
    assert 0 <= n_bin <= n_c
    mc = np.full(n_c, 1.0 / n)
    mc[:n_bin] *= 2.0
    base = plummer(n_c, seed, eps=eps, masses=mc, name="plummer-binaries")
    rng = SplitMix64(seed + 700_000)
    d = np.exp(math.log(a_lo) + rng.uniform(n_bin) * (math.log(a_hi) - math.log(a_lo)))
    nhat = _isotropic(rng, np.ones(n_bin))
    # a unit vector perpendicular to nhat: nhat x w, w isotropic, normalised
    w = _isotropic(rng, np.ones(n_bin))
    perp = np.cross(nhat, w)
    perp /= np.linalg.norm(perp, axis=1)[:, None]
    m = np.full(n, 1.0 / n)
    x = np.empty((n, 3))
    v = np.empty((n, 3))
    x[:n_c] = base.x
    v[:n_c] = base.v
    mb = 2.0 / n
    vrel = np.sqrt(mb / d)
    # equal members: each at +-d/2 from the centre, velocities +-v_rel/2
    x[n_c:] = base.x[:n_bin] - 0.5 * d[:, None] * nhat
    v[n_c:] = base.v[:n_bin] - 0.5 * vrel[:, None] * perp
    x[:n_bin] = base.x[:n_bin] + 0.5 * d[:, None] * nhat
    v[:n_bin] = base.v[:n_bin] + 0.5 * vrel[:, None] * perp
    pairs = np.stack([np.arange(n_bin), n_c + np.arange(n_bin)], axis=1).astype(np.int32)
    meta = dict(base.meta)
    meta.update({"model": "plummer+binaries", "n_bin": n_bin, "pairs": pairs, "sep": d})
    return Snapshot(m, np.ascontiguousarray(x), np.ascontiguousarray(v), float(eps) ** 2,
                    f"plummer N={n} with {n_bin} binaries", meta)


def random_state(n: int, seed: int, eps: float, spread: float = 1.0) -> Snapshot:
    """Small uniform-cube systems with unequal masses (for tiny parity cases)."""
    rng = SplitMix64(seed)
    x = (rng.uniform(3 * n).reshape(n, 3) - 0.5) * 2.0 * spread
    v = (rng.uniform(3 * n).reshape(n, 3) - 0.5)
    m = 0.5 + rng.uniform(n)
    m /= m.sum()
    return Snapshot(m, x, v, float(eps) ** 2, f"random{n}", {"seed": seed})


# ---------------------------------------------------------------- named workloads

def config(k: int, n: int | None = None) -> Snapshot:
    """The five named workloads (seed = 20071106 + k).

    1: Plummer N=1024, equal masses, eps = 1/256
    2: Plummer N=16384, equal masses, eps = 1/1024
    3: Plummer N=65536, Salpeter masses (0.1-100, slope -2.35, sum 1), eps = 1/4096
    4: use ``ensemble(256, 20071110)`` (256 clusters, eps = 4/N_c)
    5: King W0 = 6, N = 1,048,576, equal masses, eps = 1e-3
    ``n`` overrides the particle count (same recipe, for scaled-down cases).
    """
    seed = BASE_SEED + k
    if k == 1:
        return plummer(n or 1024, seed, eps=1.0 / 256, name="C1 plummer N=1024")
    if k == 2:
        return plummer(n or 16384, seed, eps=1.0 / 1024, name="C2 plummer N=16384")
    if k == 3:
        nn = n or 65536
        return plummer(nn, seed, eps=1.0 / 4096, masses=salpeter_masses(nn, seed + 500_000),
                       name="C3 plummer-salpeter N=65536")
    if k == 5:
        return king(n or 1_048_576, seed, w0=6.0, eps=1e-3, name="C5 king W0=6 N=1048576")
    raise ValueError("config 4 is an ensemble: use ensemble(256, BASE_SEED + 4)")
