"""Host checks of the corrector's integer-pipe exact arithmetic (no GPU).

The corrector replaces the FP64 divisions by 6, 24 and 120 and the products with
3, 6 and 12 by integer code that must give the bits of the IEEE operation
(Granlund-Montgomery division by an invariant integer, round to nearest), splits
doubles into double-single pairs on the integer pipe, and quantises steps on bit
patterns. The same header compiled for the host is checked here against the
host's IEEE arithmetic on random and edge values over every exponent, and the
quantiser against the oracle's."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(d):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = os.path.join(d, "exact_int_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_0711_0643_gb300", "csrc"),
                    "-o", exe, os.path.join(ROOT, "tests", "exact_int_check.cu")], check=True)
    return exe


def test_integer_division_product_and_split_match_ieee():
    with tempfile.TemporaryDirectory() as d:
        exe = _build(d)
        out = subprocess.run([exe, "8000000"], capture_output=True, text=True)
        assert out.returncode == 0, out.stdout + out.stderr
        assert "mismatches 0" in out.stdout


def test_bit_pattern_quantiser_matches_oracle(orc):
    """The corrector's quantiser works on bit patterns (largest power of two below the
    candidate from the exponent field, the doubling test from the lowest set bit of
    t_new); it must give the oracle's step (frexp-based, Sect. 2.1 powers of two) for
    every candidate, including zero, negative, subnormal, infinite and NaN ones."""
    import numpy as np
    rng = np.random.default_rng(20071106)
    rows = []
    specials = [0.0, -0.0, -1.0, np.inf, np.nan, 5e-324, 2.0 ** -1030, 2.0 ** -1022, 1.0, 2.0 ** -40, 2.0 ** -41]
    for q in range(20000):
        lvl = int(rng.integers(4, 41))            # dt_old = 2^-lvl in [2^-40, 2^-4]
        dt_old = 2.0 ** -lvl
        t_new = float(rng.integers(0, 2 ** min(lvl, 30))) * dt_old
        if q % 5 == 0:
            cand = specials[int(rng.integers(0, len(specials)))]
        elif q % 5 == 1:
            cand = dt_old * float(rng.choice([0.5, 1.0, 2.0, 4.0, 0.999999, 1.000001, 2.000001, 1.999999]))
        else:
            cand = float(2.0 ** rng.uniform(-60, 4))
        rows.append((cand, dt_old, t_new, 1.0 / 16, 2.0 ** -40))
    with tempfile.TemporaryDirectory() as d:
        exe = _build(d)
        payload = np.array([len(rows)], dtype=np.int64).tobytes() + np.array(rows, dtype=np.float64).tobytes()
        out = subprocess.run([exe, "quantise"], input=payload, capture_output=True, check=True)
    got = np.frombuffer(out.stdout, dtype=np.float64)
    assert got.size == len(rows)
    for (cand, dt_old, t_new, dt_max, dt_min), g in zip(rows, got):
        ref = orc.quantise(cand, dt_old, t_new, dt_max, dt_min)
        assert np.float64(g).tobytes() == np.float64(ref).tobytes(), (cand, dt_old, t_new, g, ref)


def test_fp32_aarseth_estimate_decides_like_the_fp64_step(orc):
    """The corrector takes the new step's power of two from an FP32 estimate of the
    Aarseth step (Eq. timestep) when the estimate is at least 2^-14 (relative) away
    from a power of two, and from the FP64 expression otherwise. Wherever it decides,
    its power of two must be the one below the oracle's FP64 step, also for steps
    placed within 10^-4 or 10^-6 of a power of two (without the window, FP32 rounding
    puts some of those on the wrong side: 54 of 4000 at 10^-6)."""
    import math

    import numpy as np
    rng = np.random.default_rng(20071107)

    def vec(scale):
        u = rng.normal(size=3)
        return u / np.linalg.norm(u) * scale

    def n2(u):
        return (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]   # the oracle's dot3 order

    cases = []
    for q in range(20000):
        a, k, a2p, a3 = (vec(10.0 ** rng.uniform(-6, 6)) for _ in range(4))
        eta = 0.01
        if q % 2:   # move the step to within 1e-4 (or 1e-6) of a power of two through eta
            c0 = orc.aarseth_dt(a, k, a2p, a3, eta)
            spread = 1e-4 if q % 4 == 1 else 1e-6
            target = 2.0 ** round(math.log2(c0)) * (1.0 + rng.uniform(-spread, spread))
            eta = eta * (target / c0) ** 2
        cases.append((a, k, a2p, a3, eta))
    rows = np.array([(n2(a), n2(k), n2(a2p), n2(a3), eta) for a, k, a2p, a3, eta in cases], dtype=np.float64)
    with tempfile.TemporaryDirectory() as d:
        exe = _build(d)
        payload = np.array([len(rows)], dtype=np.int64).tobytes() + rows.tobytes()
        out = subprocess.run([exe, "aarseth"], input=payload, capture_output=True, check=True)
    res = np.frombuffer(out.stdout, dtype=np.float64).reshape(-1, 2)
    decided = [0, 0]   # random steps, steps near a power of two
    for q, ((a, k, a2p, a3, eta), (dec, qb)) in enumerate(zip(cases, res)):
        if dec == 0.0:
            continue
        decided[q % 2] += 1
        cand = orc.aarseth_dt(a, k, a2p, a3, eta)
        m, e = math.frexp(cand)
        assert qb == math.ldexp(0.5, e), (cand, qb)
    # away from powers of two the estimate decides almost always (the window is
    # 2^-14 above and 2^-13 below a power of two); near them it must also decide
    # some (the exact path is not taken for all of them)
    assert decided[0] > 0.99 * len(cases) / 2 and decided[1] > 0.05 * len(cases) / 2, decided


def test_fp32_norm_estimate_decides_like_the_fp64_step(orc):
    """The corrector forms the squared norms of the step estimate in FP32 from RN32 copies
    of the FP64 components (integer pipe), each square flushed below 2^-126, summed in
    the oracle's order, and decides only when every norm lies in [2^-100, 2^120]. Wherever
    it decides, the power of two must be the one below the oracle's FP64 step, also for
    steps within 10^-4 or 10^-6 of a power of two, vectors with components of very
    different sizes and cancelling a2p."""
    import math

    import numpy as np
    rng = np.random.default_rng(20071108)

    def vec(scale):
        u = rng.normal(size=3)
        if rng.uniform() < 0.2:   # one component much smaller than the others
            u[int(rng.integers(0, 3))] *= 10.0 ** rng.uniform(-12, -3)
        return u / np.linalg.norm(u) * scale

    cases = []
    for q in range(20000):
        a, k, a2p, a3 = (vec(10.0 ** rng.uniform(-8, 8)) for _ in range(4))
        eta = 0.01
        if q % 2:
            c0 = orc.aarseth_dt(a, k, a2p, a3, eta)
            spread = 1e-4 if q % 4 == 1 else 1e-6
            target = 2.0 ** round(math.log2(c0)) * (1.0 + rng.uniform(-spread, spread))
            eta = eta * (target / c0) ** 2
        cases.append((a, k, a2p, a3, eta))
    rows = np.array([np.concatenate([a, k, a2p, a3, [eta]]) for a, k, a2p, a3, eta in cases], dtype=np.float64)
    with tempfile.TemporaryDirectory() as d:
        exe = _build(d)
        payload = np.array([len(rows)], dtype=np.int64).tobytes() + rows.tobytes()
        out = subprocess.run([exe, "aarseth32"], input=payload, capture_output=True, check=True)
    res = np.frombuffer(out.stdout, dtype=np.float64).reshape(-1, 2)
    decided = [0, 0]
    for q, ((a, k, a2p, a3, eta), (dec, qb)) in enumerate(zip(cases, res)):
        if dec == 0.0:
            continue
        decided[q % 2] += 1
        cand = orc.aarseth_dt(a, k, a2p, a3, eta)
        m, e = math.frexp(cand)
        assert qb == math.ldexp(0.5, e), (q, cand, qb)
    assert decided[0] > 0.99 * len(cases) / 2 and decided[1] > 0.05 * len(cases) / 2, decided
