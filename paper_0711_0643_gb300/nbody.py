"""ctypes binding of libnbody.so (include/nbody.h), same names as the C ABI.

Argument marshalling only: numpy arrays for the host-pointer entry points,
raw device pointers (e.g. ``torch.Tensor.data_ptr()``) for the ``_dev`` ones.
Every computation runs in the library's CUDA kernels; if the library is
missing or cannot be loaded, ``load()`` raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnbody.so")

NB_OK = 0
NB_ERR_ARG = -1
NB_ERR_CUDA = -2
NB_ERR_NONFINITE = -3
NB_ERR_DT_UNDERFLOW = -4
NB_ERR_TIMEOUT = -5
NB_ERR_STATE = -6
STATUS_NAMES = {0: "NB_OK", -1: "NB_ERR_ARG", -2: "NB_ERR_CUDA", -3: "NB_ERR_NONFINITE",
                -4: "NB_ERR_DT_UNDERFLOW", -5: "NB_ERR_TIMEOUT", -6: "NB_ERR_STATE"}

NB_PREC_MIXED = 0
NB_PREC_FP64 = 1


class NbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class nb_config(C.Structure):
    _fields_ = [("eta", C.c_double), ("dt_max", C.c_double), ("dt_min", C.c_double),
                ("precision", C.c_int32), ("autotune", C.c_int32), ("spin_limit", C.c_int64),
                ("device", C.c_int32), ("inject", C.c_int32)]


class nb_counters(C.Structure):
    _fields_ = [("block_steps", C.c_int64), ("particle_steps", C.c_int64), ("interactions", C.c_double),
                ("t_now", C.c_double), ("size_hist", C.c_int64 * 32), ("loop_slots", C.c_int64)]


class nb_timing(C.Structure):
    _fields_ = [("force_ms", C.c_double), ("phase_ms", C.c_double * 5), ("force_launches", C.c_int64),
                ("engine_steps", C.c_int64), ("force_interactions", C.c_double),
                ("engine_interactions", C.c_double)]


class nb_state_view(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, C.c_void_p) for k in ("m", "x", "v", "a", "k", "t", "dt")]


_lib = None

# (name, restype, argtypes)
_P, _I64, _I32, _D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
_SIGS = [
    ("nb_config_default", None, [_P]),
    ("nb_create", C.c_int, [_P, _P, _P]),
    ("nb_destroy", None, [_P]),
    ("nb_last_error", C.c_char_p, [_P]),
    ("nb_init", C.c_int, [_P, _I64, _P, _P, _P, _D]),
    ("nb_init_dev", C.c_int, [_P, _I64, _P, _P, _P, _D]),
    ("nb_next_block", C.c_int, [_P, _P, _P]),
    ("nb_get_active", C.c_int, [_P, _P]),
    ("nb_predict", C.c_int, [_P, _D]),
    ("nb_get_predicted", C.c_int, [_P, _P, _P]),
    ("nb_force_jerk", C.c_int, [_P, _P, _I64, _P, _P, _P]),
    ("nb_force_jerk_dev", C.c_int, [_P, _P, _I64, _P, _P, _P]),
    ("nb_correct", C.c_int, [_P, _D]),
    ("nb_j_range", C.c_int, [_P, _I32, _I32, _P, _P]),
    ("nb_force_jerk_range", C.c_int, [_P, _P, _I64, _I64, _I64, _P, _P, _P]),
    ("nb_force_jerk_range_dev", C.c_int, [_P, _P, _I64, _I64, _I64, _P, _P, _P]),
    ("nb_correct_forces", C.c_int, [_P, _D, _P, _P]),
    ("nb_correct_forces_dev", C.c_int, [_P, _D, _P, _P]),
    ("nb_step", C.c_int, [_P]),
    ("nb_run", C.c_int, [_P, _D]),
    ("nb_run_timed", C.c_int, [_P, _D, _I32, _P]),
    ("nb_set_engine", C.c_int, [_P, _I32]),
    ("nb_get_engine", C.c_int, [_P, _P, _P]),
    ("nb_energy", C.c_int, [_P, _P, _P, _P]),
    ("nb_get_state", C.c_int, [_P, _P]),
    ("nb_set_state", C.c_int, [_P, _P]),
    ("nb_stats", C.c_int, [_P, _P]),
    ("nb_sync", C.c_int, [_P]),
    ("nb_autotune", C.c_int, [_P]),
    ("nb_set_tuning", C.c_int, [_P, _I32, _I32, _I32]),
    ("nb_get_tuning", C.c_int, [_P, _P, _P]),
    ("nb_num_variants", C.c_int32, [_P]),
    ("nb_variant_name", C.c_char_p, [_P, _I32]),
    ("nb_force_jerk_static", C.c_int, [_I64, _P, _P, _P, _D, _P, _I64, _P, _P, _P, _P]),
    ("nb_ensemble_init", C.c_int, [_P, _I32, _P, _P, _P, _P, _P]),
    ("nb_ensemble_run", C.c_int, [_P, _D]),
    ("nb_ensemble_energy", C.c_int, [_P, _P]),
    ("nb_ensemble_stats", C.c_int, [_P, _P, _P, _P]),
    ("nb_ensemble_get_state", C.c_int, [_P, _P]),
    ("nb_perturbers", C.c_int, [_P, _I32, _P, _D, _I32, _I64, _I64, _P, _P]),
    ("nb_perturbers_dev", C.c_int, [_P, _I32, _P, _D, _I32, _I64, _I64, _P, _P]),
    ("nb_ensemble_set_shape", C.c_int, [_P, _I32, _I32]),
    ("nb_ensemble_get_shape", C.c_int, [_P, _P, _P, _P]),
    ("nb_ensemble_autotune", C.c_int, [_P, _D, _P]),
]
EXPORTED = [s[0] for s in _SIGS]


def load(path: str | None = None):
    """Loads libnbody.so (raises if it is missing; build it with ``build()``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libnbody.so not found at {p}; run paper_0711_0643_gb300.build() "
                           "(needs nvcc) -- there is no CPU fallback")
    lib = C.CDLL(p)
    for name, res, args in _SIGS:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _f64(a, shape=None):
    out = np.ascontiguousarray(a, dtype=np.float64)
    return out.reshape(shape) if shape is not None else out


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(ctx, st):
    if st != NB_OK:
        msg = load().nb_last_error(ctx).decode() if ctx else ""
        raise NbError(st, msg)
    return st


# ------------------------------------------------------------ same-name wrappers

def nb_config_default() -> nb_config:
    cfg = nb_config()
    load().nb_config_default(C.byref(cfg))
    return cfg


def nb_create(cfg: nb_config | None = None, stream: int | None = None):
    ctx = C.c_void_p()
    st = load().nb_create(C.byref(ctx), C.byref(cfg) if cfg is not None else None,
                          C.c_void_p(stream) if stream else None)
    if st != NB_OK:
        raise NbError(st, "nb_create failed")
    return ctx


def nb_destroy(ctx):
    load().nb_destroy(ctx)


def nb_last_error(ctx) -> str:
    return load().nb_last_error(ctx).decode()


def nb_init(ctx, m, x, v, eps2):
    m = _f64(m); n = m.shape[0]
    x = _f64(x, (n, 3)); v = _f64(v, (n, 3))
    return _check(ctx, load().nb_init(ctx, n, _ptr(m), _ptr(x), _ptr(v), float(eps2)))


def nb_init_dev(ctx, n, m_dev, x_dev, v_dev, eps2):
    return _check(ctx, load().nb_init_dev(ctx, int(n), C.c_void_p(m_dev), C.c_void_p(x_dev),
                                          C.c_void_p(v_dev), float(eps2)))


def nb_next_block(ctx):
    tn = C.c_double(); s = C.c_int64()
    _check(ctx, load().nb_next_block(ctx, C.byref(tn), C.byref(s)))
    return tn.value, s.value


def nb_get_active(ctx, s):
    idx = np.zeros(max(int(s), 1), dtype=np.int32)
    _check(ctx, load().nb_get_active(ctx, _ptr(idx)))
    return idx[: int(s)]


def nb_predict(ctx, t):
    return _check(ctx, load().nb_predict(ctx, float(t)))


def nb_get_predicted(ctx, n):
    """Returns (xp[n,3], vp[n,3]) as the force kernel sees them."""
    xp = np.zeros((int(n), 3)); vp = np.zeros((int(n), 3))
    _check(ctx, load().nb_get_predicted(ctx, _ptr(xp), _ptr(vp)))
    return xp, vp


def nb_force_jerk(ctx, idx=None, s=None, want=(True, True, True)):
    """Returns (a[s,3], k[s,3], phi[s]); idx None uses the last selected block (then s is required)."""
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        s = idx.shape[0]
    s = int(s)
    a = np.zeros((s, 3)) if want[0] else None
    k = np.zeros((s, 3)) if want[1] else None
    phi = np.zeros(s) if want[2] else None
    _check(ctx, load().nb_force_jerk(ctx, _ptr(idx), s, _ptr(a), _ptr(k), _ptr(phi)))
    return a, k, phi


def nb_force_jerk_dev(ctx, idx_dev, s, a_dev=0, k_dev=0, phi_dev=0):
    return _check(ctx, load().nb_force_jerk_dev(ctx, C.c_void_p(idx_dev), int(s), C.c_void_p(a_dev or None),
                                                C.c_void_p(k_dev or None), C.c_void_p(phi_dev or None)))


def nb_correct(ctx, t_block):
    return _check(ctx, load().nb_correct(ctx, float(t_block)))


def nb_j_range(ctx, rank, world):
    """(j_begin, j_end): the share of j of rank `rank` of `world` in the j-parallel step."""
    b = C.c_int64(); e = C.c_int64()
    _check(ctx, load().nb_j_range(ctx, int(rank), int(world), C.byref(b), C.byref(e)))
    return b.value, e.value


def nb_force_jerk_range(ctx, idx, s, j_begin, j_end, want=(True, True, True)):
    """Partial (a[s,3], k[s,3], phi[s]) over j in [j_begin, j_end); idx None = the last block."""
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        s = idx.shape[0]
    s = int(s)
    a = np.zeros((s, 3)) if want[0] else None
    k = np.zeros((s, 3)) if want[1] else None
    phi = np.zeros(s) if want[2] else None
    _check(ctx, load().nb_force_jerk_range(ctx, _ptr(idx), s, int(j_begin), int(j_end), _ptr(a), _ptr(k),
                                           _ptr(phi)))
    return a, k, phi


def nb_force_jerk_range_dev(ctx, idx_dev, s, j_begin, j_end, a_dev=0, k_dev=0, phi_dev=0):
    return _check(ctx, load().nb_force_jerk_range_dev(ctx, C.c_void_p(idx_dev or None), int(s), int(j_begin),
                                                      int(j_end), C.c_void_p(a_dev or None),
                                                      C.c_void_p(k_dev or None), C.c_void_p(phi_dev or None)))


def nb_correct_forces(ctx, t_block, a, k):
    a = _f64(a, (-1, 3)); k = _f64(k, (-1, 3))
    return _check(ctx, load().nb_correct_forces(ctx, float(t_block), _ptr(a), _ptr(k)))


def nb_correct_forces_dev(ctx, t_block, a_dev, k_dev):
    return _check(ctx, load().nb_correct_forces_dev(ctx, float(t_block), C.c_void_p(a_dev), C.c_void_p(k_dev)))


def nb_step(ctx):
    return _check(ctx, load().nb_step(ctx))


def nb_run(ctx, t_end):
    return _check(ctx, load().nb_run(ctx, float(t_end)))


PHASES = ("select", "predict", "force", "correct", "engine")


def nb_run_timed(ctx, t_end, phases=False):
    """Runs like nb_run, host-driven with CUDA events; returns a dict: force_ms, force_launches,
    engine_steps, force_interactions, engine_interactions and phase_ms (select, predict, force,
    correct, engine; the first, second and fourth only with phases=True)."""
    t = nb_timing()
    _check(ctx, load().nb_run_timed(ctx, float(t_end), 1 if phases else 0, C.byref(t)))
    return {"force_ms": t.force_ms, "force_launches": t.force_launches, "engine_steps": t.engine_steps,
            "force_interactions": t.force_interactions, "engine_interactions": t.engine_interactions,
            "phase_ms": dict(zip(PHASES, list(t.phase_ms)))}


def nb_set_engine(ctx, s_max):
    return _check(ctx, load().nb_set_engine(ctx, int(s_max)))


def nb_get_engine(ctx):
    """Returns (s_max, cluster): the largest block the small-block engine takes (0 = none)."""
    sm = C.c_int32(); cl = C.c_int32()
    _check(ctx, load().nb_get_engine(ctx, C.byref(sm), C.byref(cl)))
    return sm.value, cl.value


def nb_energy(ctx):
    """Returns (E, K, W)."""
    E, K, W = C.c_double(), C.c_double(), C.c_double()
    _check(ctx, load().nb_energy(ctx, C.byref(E), C.byref(K), C.byref(W)))
    return E.value, K.value, W.value


def nb_get_state(ctx, n):
    n = int(n)
    arr = {"m": np.zeros(n), "x": np.zeros((n, 3)), "v": np.zeros((n, 3)), "a": np.zeros((n, 3)),
           "k": np.zeros((n, 3)), "t": np.zeros(n), "dt": np.zeros(n)}
    view = nb_state_view(n, *[_ptr(arr[key]) for key in ("m", "x", "v", "a", "k", "t", "dt")])
    _check(ctx, load().nb_get_state(ctx, C.byref(view)))
    return arr


def nb_set_state(ctx, state):
    n = state["m"].shape[0]
    arr = {key: _f64(state[key], (n, 3) if key in ("x", "v", "a", "k") else (n,))
           for key in ("m", "x", "v", "a", "k", "t", "dt")}
    view = nb_state_view(n, *[_ptr(arr[key]) for key in ("m", "x", "v", "a", "k", "t", "dt")])
    return _check(ctx, load().nb_set_state(ctx, C.byref(view)))


def nb_stats(ctx) -> dict:
    c = nb_counters()
    _check(ctx, load().nb_stats(ctx, C.byref(c)))
    return {"block_steps": c.block_steps, "particle_steps": c.particle_steps,
            "interactions": c.interactions, "t_now": c.t_now, "size_hist": list(c.size_hist),
            "loop_slots": c.loop_slots}


def nb_sync(ctx):
    return _check(ctx, load().nb_sync(ctx))


def nb_autotune(ctx):
    return _check(ctx, load().nb_autotune(ctx))


def nb_set_tuning(ctx, bucket, variant, split):
    return _check(ctx, load().nb_set_tuning(ctx, int(bucket), int(variant), int(split)))


def nb_get_tuning(ctx):
    v = np.zeros(32, dtype=np.int32); s = np.zeros(32, dtype=np.int32)
    _check(ctx, load().nb_get_tuning(ctx, _ptr(v), _ptr(s)))
    return v, s


def nb_num_variants(ctx) -> int:
    return int(load().nb_num_variants(ctx))


def nb_variant_name(ctx, v) -> str:
    return load().nb_variant_name(ctx, int(v)).decode()


NB_STATIC_MAX_N = 65536


def nb_force_jerk_static(n, m_dev, x_dev, v_dev, eps2, idx_dev, s, a_dev=0, k_dev=0, phi_dev=0, stream=0):
    """Force evaluation that allocates nothing (device pointers in and out); returns the
    nb_status code (0 = NB_OK) instead of raising, since there is no context to describe it."""
    return int(load().nb_force_jerk_static(int(n), C.c_void_p(m_dev), C.c_void_p(x_dev), C.c_void_p(v_dev),
                                           float(eps2), C.c_void_p(idx_dev or None), int(s),
                                           C.c_void_p(a_dev or None), C.c_void_p(k_dev or None),
                                           C.c_void_p(phi_dev or None), C.c_void_p(stream or None)))


def nb_ensemble_init(ctx, offsets, m, x, v, eps2):
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    nc = offsets.shape[0] - 1
    m = _f64(m); N = m.shape[0]
    x = _f64(x, (N, 3)); v = _f64(v, (N, 3)); eps2 = _f64(eps2)
    return _check(ctx, load().nb_ensemble_init(ctx, nc, _ptr(offsets), _ptr(m), _ptr(x), _ptr(v), _ptr(eps2)))


def nb_ensemble_run(ctx, t_end):
    return _check(ctx, load().nb_ensemble_run(ctx, float(t_end)))


def nb_ensemble_energy(ctx, nc):
    E = np.zeros(int(nc))
    _check(ctx, load().nb_ensemble_energy(ctx, _ptr(E)))
    return E


def nb_ensemble_stats(ctx, nc):
    """Per-system (block_steps, particle_steps, interactions) arrays."""
    b = np.zeros(int(nc), dtype=np.int64); p = np.zeros(int(nc), dtype=np.int64); i = np.zeros(int(nc))
    _check(ctx, load().nb_ensemble_stats(ctx, _ptr(b), _ptr(p), _ptr(i)))
    return b, p, i


def nb_ensemble_get_state(ctx, N):
    N = int(N)
    arr = {"m": np.zeros(N), "x": np.zeros((N, 3)), "v": np.zeros((N, 3)), "a": np.zeros((N, 3)),
           "k": np.zeros((N, 3)), "t": np.zeros(N), "dt": np.zeros(N)}
    view = nb_state_view(N, *[_ptr(arr[key]) for key in ("m", "x", "v", "a", "k", "t", "dt")])
    _check(ctx, load().nb_ensemble_get_state(ctx, C.byref(view)))
    return arr


NB_PERT_MAX = 4096


def nb_perturbers(ctx, pairs, gamma=1e-7, nmax=256, j_lo=0, j_hi=-1):
    """Perturber lists of the binaries pairs[b] = (i, k) from the context's positions
    (Sect. 3.1): (lists [nbin][nmax] with -1 padding, counts [nbin])."""
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    nb = pairs.shape[0]
    lists = np.full((nb, int(nmax)), -1, dtype=np.int32)
    counts = np.zeros(nb, dtype=np.int32)
    _check(ctx, load().nb_perturbers(ctx, nb, _ptr(pairs), float(gamma), int(nmax), int(j_lo), int(j_hi),
                                     _ptr(lists), _ptr(counts)))
    return lists, counts


def nb_perturbers_dev(ctx, nbin, pairs_dev, gamma, nmax, j_lo, j_hi, lists_dev, counts_dev):
    return _check(ctx, load().nb_perturbers_dev(ctx, int(nbin), C.c_void_p(pairs_dev), float(gamma), int(nmax),
                                                int(j_lo), int(j_hi), C.c_void_p(lists_dev),
                                                C.c_void_p(counts_dev)))


def nb_ensemble_set_shape(ctx, cluster=0, split_cap=0):
    return _check(ctx, load().nb_ensemble_set_shape(ctx, int(cluster), int(split_cap)))


def nb_ensemble_get_shape(ctx):
    """(cluster, nclusters, split_cap) of the loaded ensemble's launch."""
    c = C.c_int32(0); n = C.c_int32(0); s = C.c_int32(0)
    _check(ctx, load().nb_ensemble_get_shape(ctx, C.byref(c), C.byref(n), C.byref(s)))
    return c.value, n.value, s.value


def nb_ensemble_autotune(ctx, t_probe=0.0):
    """Probes the launch shapes on the loaded ensemble, keeps the fastest; returns its time in ms."""
    ms = C.c_float(0.0)
    _check(ctx, load().nb_ensemble_autotune(ctx, float(t_probe), C.byref(ms)))
    return ms.value


# ----------------------------------------------------------------- convenience

class Context:
    """Owns an nb_ctx; ``with Context(precision=...) as c: c.init(snap)``."""

    def __init__(self, precision: int = NB_PREC_MIXED, eta: float = 0.01, dt_max: float = 1.0 / 16,
                 dt_min: float = 2.0 ** -40, autotune: bool = False, spin_limit: int | None = None,
                 device: int = -1, inject: int = 0, stream: int | None = None):
        cfg = nb_config_default()
        cfg.precision = precision
        cfg.eta = eta
        cfg.dt_max = dt_max
        cfg.dt_min = dt_min
        cfg.autotune = 1 if autotune else 0
        if spin_limit is not None:
            cfg.spin_limit = spin_limit
        cfg.device = device
        cfg.inject = inject
        self.cfg = cfg
        self.ctx = nb_create(cfg, stream)
        self.n = 0

    def close(self):
        if self.ctx:
            nb_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, snap):
        nb_init(self.ctx, snap.m, snap.x, snap.v, snap.eps2)
        self.n = snap.n

    def state(self):
        return nb_get_state(self.ctx, self.n)
