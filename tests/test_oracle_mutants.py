"""The oracle's pins catch plausible mistakes.

Each mutant below plants one typical slip in a copy of ``oracle/oracle.c`` (a
sign, a dropped term, a swapped index or operand, a wrong coefficient or
power) and the pin suite ``test_oracle_pins.py`` must fail against it. The
mutants are compiled on the CPU into a temporary directory; nothing here
touches the CUDA library.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = [
    # Eq. Force
    ("force: r_i - r_j (repulsive)", "double rx = x[3 * j + 0] - x[3 * i + 0];", "double rx = x[3 * i + 0] - x[3 * j + 0];"),
    ("force: softening dropped", "rz * rz + eps2;", "rz * rz;"),
    ("force: d^5 as d^4", "double d5 = d3 * d2;", "double d5 = d3 * d;"),
    ("force: jerk factor 3 -> 2", "kx += m[j] * (wx / d3 - 3.0", "kx += m[j] * (wx / d3 - 2.0"),
    ("force: jerk sign", "ky += m[j] * (wy / d3 - 3.0", "ky += m[j] * (wy / d3 + 3.0"),
    ("force: m_i for m_j", "ax += m[j] * rx / d3;", "ax += m[i] * rx / d3;"),
    ("force: potential 1/d^2", "p -= m[j] / d;", "p -= m[j] / d2;"),
    ("force: self term kept", "if (j == i) continue;", "if (j == i && eps2 == 0.0) continue;"),
    ("force: r.w drops z", "double rw = rx * wx + ry * wy + rz * wz;", "double rw = rx * wx + ry * wy;"),
    # predictor
    ("predict: a d^2/6", "a[q] * d2 / 2.0 + k[q] * d3 / 6.0;", "a[q] * d2 / 6.0 + k[q] * d3 / 6.0;"),
    ("predict: k d^3/2", "a[q] * d2 / 2.0 + k[q] * d3 / 6.0;", "a[q] * d2 / 2.0 + k[q] * d3 / 2.0;"),
    ("predict: jerk dropped from v", "vp[q] = v[q] + a[q] * d + k[q] * d2 / 2.0;", "vp[q] = v[q] + a[q] * d;"),
    ("predict: v d dropped from x", "xp[q] = x[q] + v[q] * d + a[q]", "xp[q] = x[q] + a[q]"),
    ("predict: a d^2 in v", "vp[q] = v[q] + a[q] * d + k[q] * d2 / 2.0;", "vp[q] = v[q] + a[q] * d2 + k[q] * d2 / 2.0;"),
    # corrector
    ("correct: sign of 6 da", "a2[c] = -6.0 * da / dt2", "a2[c] = 6.0 * da / dt2"),
    ("correct: k_old/k_new swapped", "(4.0 * k_old[c] + 2.0 * k_new[c])", "(2.0 * k_old[c] + 4.0 * k_new[c])"),
    ("correct: 12 da / dt^2", "a3[c] = 12.0 * da / dt3", "a3[c] = 12.0 * da / dt2"),
    ("correct: da = a_new - a_old", "double da = a_old[c] - a_new[c];", "double da = a_new[c] - a_old[c];"),
    ("correct: a3 from k_old - k_new", "6.0 * (k_old[c] + k_new[c]) / dt2", "6.0 * (k_old[c] - k_new[c]) / dt2"),
    ("correct: x a2 dt^4/6", "x1[c] = xp[c] + a2[c] * dt4 / 24.0", "x1[c] = xp[c] + a2[c] * dt4 / 6.0"),
    ("correct: v a3 dt^4/6", "a3[c] * dt4 / 24.0;", "a3[c] * dt4 / 6.0;"),
    ("correct: a3 dt^5/24", "a3[c] * dt5 / 120.0", "a3[c] * dt5 / 24.0"),
    ("correct: a2 dt^3/2", "v1[c] = vp[c] + a2[c] * dt3 / 6.0", "v1[c] = vp[c] + a2[c] * dt3 / 2.0"),
    ("step: a2p without a3 dt", "a2p[c] = a2[c] + a3[c] * dt;", "a2p[c] = a2[c];"),
    ("step: old a in the criterion", "*dt_cand = orc_aarseth_dt(a_new, k_new,", "*dt_cand = orc_aarseth_dt(a_old, k_new,"),
    # Eq. timestep
    ("aarseth: |a||a3|", "double num = amag * a2mag + dot3(k_new, k_new);", "double num = amag * a3mag + dot3(k_new, k_new);"),
    ("aarseth: |k||a2|", "double den = kmag * a3mag + dot3(a2p, a2p);", "double den = kmag * a2mag + dot3(a2p, a2p);"),
    ("aarseth: no square root", "return sqrt(eta * num / den);", "return eta * num / den;"),
    ("aarseth: |a2|^2 dropped", "double den = kmag * a3mag + dot3(a2p, a2p);", "double den = kmag * a3mag;"),
    # block steps
    ("quantise: 2^ceil", "return ldexp(1.0, e - 1);", "return ldexp(1.0, e);"),
    ("quantise: doubles anywhere", "dt = (u == floor(u)) ? dt2 : dt_old;", "dt = dt2;"),
    ("quantise: doubles only above 2 dt_old", "} else if (q >= dt2 && dt2 <= dt_max) {", "} else if (q > dt2 && dt2 <= dt_max) {"),
    ("quantise: no dt_min floor", "    if (dt > dt_max) dt = dt_max;\n    if (dt < dt_min) return 0.0;\n    return dt;\n}\n\ndouble orc_initial_dt",
     "    if (dt > dt_max) dt = dt_max;\n    return dt;\n}\n\ndouble orc_initial_dt"),
    ("initial dt: |k|/|a|", "eta * amag / kmag", "eta * kmag / amag"),
    ("initial dt: eta dropped", "eta * amag / kmag", "amag / kmag"),
    ("initial dt: no power-of-two floor", "double dt = isinf(cand) ? dt_max : pow2_floor(cand);", "double dt = isinf(cand) ? dt_max : cand;"),
    ("next_block: max for min", "if (ti < tmin) tmin = ti;\n    }\n    int64_t s", "if (ti > tmin) tmin = ti;\n    }\n    int64_t s"),
    ("next_block: first hit only", "if (t[i] + dt[i] == tmin) {", "if (t[i] + dt[i] == tmin && s == 0) {"),
    ("next_block: t_i for t_i + dt_i", "double ti = t[i] + dt[i];", "double ti = t[i];"),
    # energy
    ("energy: W double-counted", "pot += 0.5 * m[i] * phi[i];", "pot += m[i] * phi[i];"),
    ("energy: sign of W", "pot += 0.5 * m[i] * phi[i];", "pot -= 0.5 * m[i] * phi[i];"),
    ("energy: K without the 1/2", "kin += 0.5 * m[i] * v2;", "kin += m[i] * v2;"),
    ("energy: v^2 drops z", " + v[3 * i + 2] * v[3 * i + 2];", ";"),
    # perturber lists (Sect. 3.1)
    ("perturbers: factor 2 dropped", "double tm = 2.0 * m[j];", "double tm = m[j];"),
    ("perturbers: d^4 for d^6", "double d6 = d2 * d2 * d2;", "double d6 = d2 * d2;"),
    ("perturbers: distance from member 1", "double r2 = dist2(x + 3 * j, cm);", "double r2 = dist2(x + 3 * j, x + 3 * i);"),
    ("perturbers: members not excluded", "if (j == i || j == k) continue;", "if (j == i) continue;"),
    ("perturbers: last nmax kept", "if (found < nmax) lists[(int64_t)b * nmax + found] = (int32_t)j;", "lists[(int64_t)b * nmax + found % nmax] = (int32_t)j;"),
    ("perturbers: m_b for gamma m_b", "double gm = gamma * mb;", "double gm = gamma;"),
]


def _run_mutant(tmp, k, name, old, new):
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert src.count(old) == 1, f"mutant '{name}' does not match exactly one site"
    d = os.path.join(tmp, f"m{k}")
    os.makedirs(d, exist_ok=True)
    path = os.path.join(d, "oracle.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    sys.path.insert(0, ROOT)
    import oracle
    lib = oracle.build(force=True, src=path, out=os.path.join(d, "liboracle.so"))
    env = dict(os.environ, NB_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=240)
        return name, r.returncode
    except subprocess.TimeoutExpired:
        return name, "timeout"


def test_pins_catch_every_mutant(tmp_path):
    jobs = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(jobs) as ex:
        futs = [ex.submit(_run_mutant, str(tmp_path), k, *m) for k, m in enumerate(MUTANTS)]
        results = [f.result() for f in futs]
    survivors = [name for name, rc in results if rc == 0]
    assert not survivors, f"pins did not catch: {survivors}"


def test_unmutated_copy_passes(tmp_path):
    """The harness itself: an unchanged copy of the source passes the pins."""
    name, rc = _run_mutant(str(tmp_path), 0, "identity", "#include <math.h>", "#include <math.h>")
    assert rc == 0
