"""Batched ensemble (one persistent cluster launch over many independent systems)
against the FP64 CPU oracle and against itself.

* initial forces of every member within the mixed-precision tolerance of the
  parity tests, first steps exactly the oracle's rule on those forces, energies
  within 1e-12 of the oracle's;
* every member lands on t_end, conserves energy within 2x the oracle's error
  plus a round-off floor of 1e-9 (at t = 0.25 both errors sit near the level of
  summation noise, where a factor of 2 is not resolved);
* results are bitwise reproducible and do not depend on which other systems
  share the launch.
"""
import numpy as np
import pytest

import ics
from tests.nbtools import condition_scales, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody
    nbody.load()
    return nbody


def _pack(members):
    off = np.zeros(len(members) + 1, dtype=np.int64)
    off[1:] = np.cumsum([s.n for s in members])
    m = np.concatenate([s.m for s in members])
    x = np.concatenate([s.x for s in members])
    v = np.concatenate([s.v for s in members])
    e2 = np.array([s.eps2 for s in members])
    return off, m, x, v, e2


def _members():
    return ics.ensemble(10, seed=4242, n_lo=40, n_hi=700)


def test_ensemble_initial_state(nb, orc):
    mem = _members()
    off, m, x, v, e2 = _pack(mem)
    with nb.Context() as c:
        nb.nb_ensemble_init(c.ctx, off, m, x, v, e2)
        st = nb.nb_ensemble_get_state(c.ctx, off[-1])
        E = nb.nb_ensemble_energy(c.ctx, len(mem))
    for q, s in enumerate(mem):
        sl = slice(off[q], off[q + 1])
        np.testing.assert_array_equal(st["t"][sl], 0.0)
        ar, kr, _ = orc.force(s.m, s.x, s.v, s.eps2)
        A, K = condition_scales(s.m, s.x, s.v, s.eps2, np.arange(s.n))
        assert (np.linalg.norm(st["a"][sl] - ar, axis=1) / A).max() < 1e-6, q
        assert np.percentile(rel_errors(st["a"][sl], ar, A), 99) < 1e-6, q
        assert (np.linalg.norm(st["k"][sl] - kr, axis=1) / K).max() < 1e-6, q
        for i in range(s.n):
            assert st["dt"][sl][i] == orc.initial_dt(st["a"][sl][i], st["k"][sl][i])
        Kr, Wr = orc.energy(s.m, s.x, s.v, s.eps2)
        assert abs(E[q] - (Kr + Wr)) < 1e-12 * abs(Kr + Wr), q


_ORACLE = {}


def _oracle_run(orc, s, t_end):
    """The oracle's |dE/E| and block steps for member s to t_end (cached)."""
    key = (s.n, float(s.eps2), float(s.x[0, 0]), t_end)
    if key not in _ORACLE:
        sysr = orc.System(s.m, s.x, s.v, s.eps2, nthreads=orc.default_threads())
        Er0 = sysr.energy()
        assert sysr.run(t_end) == 0
        _ORACLE[key] = (abs(sysr.energy() - Er0) / abs(Er0), sysr.counters["block_steps"])
    return _ORACLE[key]


def _run_and_check(nb, orc, mem, t_end, cluster=0, split_cap=0):
    off, m, x, v, e2 = _pack(mem)
    with nb.Context() as c:
        nb.nb_ensemble_init(c.ctx, off, m, x, v, e2)
        if cluster or split_cap:
            nb.nb_ensemble_set_shape(c.ctx, cluster, split_cap)
        shape = nb.nb_ensemble_get_shape(c.ctx)
        E0 = nb.nb_ensemble_energy(c.ctx, len(mem))
        nb.nb_ensemble_run(c.ctx, t_end)
        E1 = nb.nb_ensemble_energy(c.ctx, len(mem))
        st = nb.nb_ensemble_get_state(c.ctx, off[-1])
        bs, ps, inter = nb.nb_ensemble_stats(c.ctx, len(mem))
    np.testing.assert_array_equal(st["t"], t_end)
    assert np.all(bs > 0) and np.all(ps >= bs)
    np.testing.assert_allclose(inter, ps * np.diff(off), rtol=0)
    for q, s in enumerate(mem):
        dEr, steps_r = _oracle_run(orc, s, t_end)
        dE = abs(E1[q] - E0[q]) / abs(E0[q])
        print(f"shape {shape} member {q} N={s.n}: |dE/E| {dE:.3e} oracle {dEr:.3e}; steps {bs[q]} oracle {steps_r}")
        assert dE <= 2 * dEr + 1e-9, (q, dE, dEr)
    return st, shape


def test_ensemble_run_conserves_energy_and_lands(nb, orc):
    _run_and_check(nb, orc, _members(), 0.25)


def test_ensemble_i_split_and_cluster_shapes(nb, orc):
    """A split cap of 16 sends every block of more than 16 active particles through the
    i-split (each CTA a share of the active particles against all j); clusters of 4 and
    16 CTAs change the j-shares. Each shape conserves energy like the oracle and gives
    the same bits on a rerun."""
    mem = _members()
    for cluster, cap in ((0, 16), (4, 0), (16, 64)):
        st, shape = _run_and_check(nb, orc, mem, 0.25, cluster, cap)
        if cluster:
            assert shape[0] == cluster
        if cap:
            assert shape[2] == cap
        st2, _ = _run_and_check(nb, orc, mem, 0.25, cluster, cap)
        for key in ("x", "v", "a", "k", "dt"):
            np.testing.assert_array_equal(st[key], st2[key])


def test_ensemble_autotune_keeps_state(nb, orc):
    """The tuner's probes leave the state bitwise as it was; the chosen shape is one of
    the candidates, and the run continues from the restored state."""
    mem = _members()
    off, m, x, v, e2 = _pack(mem)
    nmax = int(np.diff(off).max())
    with nb.Context() as c:
        nb.nb_ensemble_init(c.ctx, off, m, x, v, e2)
        nb.nb_ensemble_run(c.ctx, 0.0625)
        before = nb.nb_ensemble_get_state(c.ctx, off[-1])
        E_before = nb.nb_ensemble_energy(c.ctx, len(mem))
        bs_before = nb.nb_ensemble_stats(c.ctx, len(mem))[0]
        ms = nb.nb_ensemble_autotune(c.ctx, 1.0 / 64)
        after = nb.nb_ensemble_get_state(c.ctx, off[-1])
        cluster, ncl, cap = nb.nb_ensemble_get_shape(c.ctx)
        np.testing.assert_array_equal(nb.nb_ensemble_energy(c.ctx, len(mem)), E_before)
        np.testing.assert_array_equal(nb.nb_ensemble_stats(c.ctx, len(mem))[0], bs_before)
        nb.nb_ensemble_run(c.ctx, 0.125)
        st = nb.nb_ensemble_get_state(c.ctx, off[-1])
    print(f"tuned shape: cluster {cluster} x {ncl}, split cap {cap}, probe {ms:.2f} ms")
    for key in ("x", "v", "a", "k", "t", "dt"):
        np.testing.assert_array_equal(before[key], after[key])
    assert cluster in (4, 8, 16) and ncl >= 1 and ms > 0
    assert cap in [min(nmax, 8192)] + [q for q in (4096, 2048, 1024) if q < min(nmax, 8192)]
    np.testing.assert_array_equal(st["t"], 0.125)


def test_ensemble_shape_arguments(nb):
    mem = _members()
    off, m, x, v, e2 = _pack(mem)
    with nb.Context() as c:
        with pytest.raises(nb.NbError) as e:
            nb.nb_ensemble_set_shape(c.ctx, 8, 0)
        assert e.value.status == nb.NB_ERR_STATE
        nb.nb_ensemble_init(c.ctx, off, m, x, v, e2)
        for bad in ((3, 0), (32, 0), (8, -1)):
            with pytest.raises(nb.NbError) as e:
                nb.nb_ensemble_set_shape(c.ctx, *bad)
            assert e.value.status == nb.NB_ERR_ARG
        nb.nb_ensemble_set_shape(c.ctx, 0, 100000)
        assert nb.nb_ensemble_get_shape(c.ctx)[2] == int(np.diff(off).max())


def test_ensemble_deterministic_and_independent(nb):
    mem = _members()
    off, m, x, v, e2 = _pack(mem)
    states = []
    for _ in range(2):
        with nb.Context() as c:
            nb.nb_ensemble_init(c.ctx, off, m, x, v, e2)
            nb.nb_ensemble_run(c.ctx, 0.125)
            states.append(nb.nb_ensemble_get_state(c.ctx, off[-1]))
    for key in ("x", "v", "a", "k", "t", "dt"):
        np.testing.assert_array_equal(states[0][key], states[1][key])
    # member 3 alone gives the same bits as member 3 inside the batch
    q = 3
    s = mem[q]
    with nb.Context() as c:
        o1, m1, x1, v1, e1 = _pack([s])
        nb.nb_ensemble_init(c.ctx, o1, m1, x1, v1, e1)
        nb.nb_ensemble_run(c.ctx, 0.125)
        alone = nb.nb_ensemble_get_state(c.ctx, s.n)
    sl = slice(off[q], off[q + 1])
    for key in ("x", "v", "t", "dt"):
        np.testing.assert_array_equal(alone[key], states[0][key][sl])


def test_ensemble_largest_energy_error_member_matches_oracle(nb, orc):
    """Member 46 (N = 4633, eps = 4/N) of the 256-cluster workload (N log-uniform in
    [256, 8192], seed 20071110) has that workload's largest |dE/E| at t = 1 on the GPU.
    The oracle integrating the same member gives the same energy error (a close
    encounter at this softening), so the GPU run must agree within 2x plus a floor."""
    members = ics.ensemble(256, ics.BASE_SEED + 4, n_lo=256, n_hi=8192)
    s = members[46]
    assert s.n == 4633
    off, m, x, v, e2 = _pack([s])
    with nb.Context() as c:
        nb.nb_ensemble_init(c.ctx, off, m, x, v, e2)
        E0 = nb.nb_ensemble_energy(c.ctx, 1)[0]
        nb.nb_ensemble_run(c.ctx, 1.0)
        E1 = nb.nb_ensemble_energy(c.ctx, 1)[0]
    sysr = orc.System(s.m, s.x, s.v, s.eps2, nthreads=orc.default_threads())
    Er0 = sysr.energy()
    assert sysr.run(1.0) == 0
    dEr = abs(sysr.energy() - Er0) / abs(Er0)
    dE = abs(E1 - E0) / abs(E0)
    print(f"member 46: |dE/E| GPU {dE:.6e}, oracle {dEr:.6e}")
    assert dEr > 1e-6                       # the encounter is there in the oracle too
    assert dE <= 2 * dEr + 1e-9 and dEr <= 2 * dE + 1e-9


def test_ensemble_argument_errors(nb):
    with nb.Context() as c:
        with pytest.raises(nb.NbError) as e:
            nb.nb_ensemble_run(c.ctx, 1.0)
        assert e.value.status == nb.NB_ERR_STATE
        with pytest.raises(nb.NbError) as e:
            nb.nb_ensemble_init(c.ctx, np.array([0, 5, 5], dtype=np.int64), np.ones(5), np.zeros((5, 3)),
                                np.zeros((5, 3)), np.array([0.01, 0.01]))
        assert e.value.status == nb.NB_ERR_ARG
