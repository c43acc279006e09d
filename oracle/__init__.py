"""ctypes wrapper around the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. The CUDA library never imports it.
``build()`` compiles ``oracle.c`` with ``gcc -O2 -ffp-contract=off -fopenmp``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERR_NONFINITE = -3
ERR_DT_UNDERFLOW = -4


def build(force: bool = False, src: str | None = None, out: str | None = None) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (no-op if up to date).

    ``src``/``out`` compile another copy of the source (the mutation tests)."""
    src = src or _SRC
    out = out or _LIB
    with _lock:
        newest = max(os.path.getmtime(src), os.path.getmtime(_HDR))
        if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
            return out
        tmp = out + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                "-I", _HERE, src, "-o", tmp, "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True)   # no OpenMP: sequential oracle
        os.replace(tmp, out)
        return out


def use_library(path: str) -> None:
    """Bind this module to another compiled copy of the oracle (mutation tests)."""
    global _lib
    _lib = _bind(C.CDLL(path))


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(C.CDLL(_LIB))
    return _lib


def _bind(lib):
    d, i64, p = C.c_double, C.c_int64, C.c_void_p
    lib.orc_force.argtypes = [i64, p, p, p, d, i64, p, p, p, p, C.c_int]
    lib.orc_predict.argtypes = [i64, p, p, p, p, p, d, p, p]
    lib.orc_correct_one.argtypes = [p, p, p, p, p, p, d, p, p, p, p]
    lib.orc_correct_particle.argtypes = [p, p, p, p, p, p, d, d, p, p, p]
    lib.orc_aarseth_dt.argtypes = [p, p, p, p, d]
    lib.orc_aarseth_dt.restype = d
    lib.orc_quantise.argtypes = [d, d, d, d, d]
    lib.orc_quantise.restype = d
    lib.orc_initial_dt.argtypes = [p, p, d, d, d]
    lib.orc_initial_dt.restype = d
    lib.orc_next_block.argtypes = [i64, p, p, p, p]
    lib.orc_next_block.restype = i64
    lib.orc_energy.argtypes = [i64, p, p, p, d, p, p, C.c_int]
    lib.orc_perturbers.argtypes = [i64, p, p, C.c_int32, p, d, C.c_int32, i64, i64, p, p]
    lib.orc_init.argtypes = [p]
    lib.orc_init.restype = C.c_int
    lib.orc_step.argtypes = [p, p, p, p]
    lib.orc_step.restype = C.c_int
    lib.orc_run.argtypes = [p, d, i64]
    lib.orc_run.restype = C.c_int
    return lib


def _f64(a, shape=None):
    out = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        out = out.reshape(shape)
    return out


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def force(m, x, v, eps2, idx=None, nthreads: int = 1):
    """(a[s,3], k[s,3], phi[s]) on the active list ``idx`` (all particles if None)."""
    lib = _load()
    m = _f64(m); n = m.shape[0]
    x = _f64(x, (n, 3)); v = _f64(v, (n, 3))
    idx = np.arange(n, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, dtype=np.int32)
    s = idx.shape[0]
    a = np.zeros((s, 3)); k = np.zeros((s, 3)); phi = np.zeros(s)
    lib.orc_force(n, _ptr(m), _ptr(x), _ptr(v), float(eps2), s, _ptr(idx), _ptr(a), _ptr(k), _ptr(phi),
                  int(nthreads))
    return a, k, phi


def predict(x, v, a, k, t, t_new):
    lib = _load()
    t = _f64(t); n = t.shape[0]
    x, v, a, k = (_f64(u, (n, 3)) for u in (x, v, a, k))
    xp = np.zeros((n, 3)); vp = np.zeros((n, 3))
    lib.orc_predict(n, _ptr(x), _ptr(v), _ptr(a), _ptr(k), _ptr(t), float(t_new), _ptr(xp), _ptr(vp))
    return xp, vp


def correct_one(xp, vp, a_old, k_old, a_new, k_new, dt):
    """(x1, v1, a2, a3) for one particle."""
    lib = _load()
    ins = [_f64(u, (3,)) for u in (xp, vp, a_old, k_old, a_new, k_new)]
    outs = [np.zeros(3) for _ in range(4)]
    lib.orc_correct_one(*[_ptr(u) for u in ins], float(dt), *[_ptr(u) for u in outs])
    return tuple(outs)


def correct_particle(xp, vp, a_old, k_old, a_new, k_new, dt, eta=0.01):
    """(x1, v1, dt_cand) for one particle: corrector plus the unquantised new step."""
    lib = _load()
    ins = [_f64(u, (3,)) for u in (xp, vp, a_old, k_old, a_new, k_new)]
    x1 = np.zeros(3); v1 = np.zeros(3); cand = C.c_double()
    lib.orc_correct_particle(*[_ptr(u) for u in ins], float(dt), float(eta), _ptr(x1), _ptr(v1), C.byref(cand))
    return x1, v1, cand.value


def aarseth_dt(a_new, k_new, a2p, a3, eta=0.01):
    lib = _load()
    ins = [_f64(u, (3,)) for u in (a_new, k_new, a2p, a3)]
    return lib.orc_aarseth_dt(*[_ptr(u) for u in ins], float(eta))


def quantise(dt_cand, dt_old, t_new, dt_max=1.0 / 16, dt_min=2.0 ** -40):
    return _load().orc_quantise(float(dt_cand), float(dt_old), float(t_new), float(dt_max), float(dt_min))


def initial_dt(a, k, eta=0.01, dt_max=1.0 / 16, dt_min=2.0 ** -40):
    lib = _load()
    a = _f64(a, (3,)); k = _f64(k, (3,))
    return lib.orc_initial_dt(_ptr(a), _ptr(k), float(eta), float(dt_max), float(dt_min))


def next_block(t, dt):
    lib = _load()
    t = _f64(t); dt = _f64(dt); n = t.shape[0]
    idx = np.zeros(max(n, 1), dtype=np.int32)
    tn = C.c_double(0.0)
    s = lib.orc_next_block(n, _ptr(t), _ptr(dt), C.byref(tn), _ptr(idx))
    return tn.value, idx[:s].copy()


def perturbers(m, x, pairs, gamma=1e-7, nmax=256, j_lo=0, j_hi=None):
    """Perturber lists of the binaries pairs[b] = (i, k) over stars [j_lo, j_hi) (Sect. 3.1):
    (lists [nbin][nmax] with -1 padding, counts [nbin]); see orc_perturbers."""
    m = _f64(m); n = m.shape[0]
    x = _f64(x, (n, 3))
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    nb = pairs.shape[0]
    lists = np.full((nb, int(nmax)), -1, dtype=np.int32)
    counts = np.zeros(nb, dtype=np.int32)
    _load().orc_perturbers(n, _ptr(m), _ptr(x), nb, _ptr(pairs), float(gamma), int(nmax), int(j_lo),
                           int(n if j_hi is None else j_hi), _ptr(lists), _ptr(counts))
    return lists, counts


def energy(m, x, v, eps2, nthreads: int = 1):
    """(K, W) with W the softened potential energy."""
    lib = _load()
    m = _f64(m); n = m.shape[0]
    x = _f64(x, (n, 3)); v = _f64(v, (n, 3))
    K = C.c_double(); W = C.c_double()
    lib.orc_energy(n, _ptr(m), _ptr(x), _ptr(v), float(eps2), C.byref(K), C.byref(W), int(nthreads))
    return K.value, W.value


class _OrcSystem(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(nm, C.c_void_p) for nm in ("m", "x", "v", "a", "k", "t", "dt")] + [
        ("eps2", C.c_double), ("eta", C.c_double), ("dt_max", C.c_double), ("dt_min", C.c_double),
        ("dt_fixed", C.c_double), ("nthreads", C.c_int),
        ("block_steps", C.c_int64), ("particle_steps", C.c_int64), ("interactions", C.c_double)]


class System:
    """The oracle's integrator state (numpy-owned arrays)."""

    def __init__(self, m, x, v, eps2, eta=0.01, dt_max=1.0 / 16, dt_min=2.0 ** -40, dt_fixed=0.0,
                 nthreads: int = 1):
        self.m = _f64(m).copy(); n = self.m.shape[0]
        self.x = _f64(x, (n, 3)).copy(); self.v = _f64(v, (n, 3)).copy()
        self.a = np.zeros((n, 3)); self.k = np.zeros((n, 3))
        self.t = np.zeros(n); self.dt = np.zeros(n)
        self.eps2 = float(eps2)
        self._s = _OrcSystem(n, *[_ptr(u) for u in (self.m, self.x, self.v, self.a, self.k, self.t, self.dt)],
                             float(eps2), float(eta), float(dt_max), float(dt_min), float(dt_fixed),
                             int(nthreads), 0, 0, 0.0)
        self.status = _load().orc_init(C.byref(self._s))

    @property
    def n(self):
        return int(self._s.n)

    @property
    def counters(self):
        return {"block_steps": self._s.block_steps, "particle_steps": self._s.particle_steps,
                "interactions": self._s.interactions}

    def step(self):
        """One block step: returns (status, t_next, idx)."""
        lib = _load()
        idx = np.zeros(max(self.n, 1), dtype=np.int32)
        tn = C.c_double(); s = C.c_int64()
        st = lib.orc_step(C.byref(self._s), C.byref(tn), C.byref(s), _ptr(idx))
        return st, tn.value, idx[: s.value].copy()

    def run(self, t_end, max_steps: int = 0) -> int:
        return _load().orc_run(C.byref(self._s), float(t_end), int(max_steps))

    def energy(self, nthreads: int | None = None):
        K, W = energy(self.m, self.x, self.v, self.eps2, nthreads or int(self._s.nthreads))
        return K + W
