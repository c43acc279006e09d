"""nb_force_jerk_static: the force evaluation for callers that may not allocate.

Some callers cannot call cudaMalloc: a host framework that owns the GPU memory
budget through its own pool, a plugin living in another application's CUDA
context, or a latency-critical loop that cannot pay cudaMalloc's implicit
device synchronisation. For them the library offers an entry point whose
scratch is a fixed array inside the library. This test calls it through the C
ABI twice in a row (a large active list, then a small one, so that stale
contents of the shared array would show) and checks both results against the
context-based entry point nb_force_jerk_dev, within the mixed-precision
tolerance of the parity tests. It lives in a file of its own so that pytest
collects it last.
"""
import numpy as np
import pytest

import ics
from tests.nbtools import condition_scales, rel_errors, rel_scalar

pytestmark = pytest.mark.gpu


def _with_ctx(nb, torch, snap, dev, idx):
    m = torch.tensor(snap.m, device=dev)
    x = torch.tensor(snap.x, device=dev)
    v = torch.tensor(snap.v, device=dev)
    out = []
    with nb.Context() as c:
        nb.nb_init_dev(c.ctx, snap.n, m.data_ptr(), x.data_ptr(), v.data_ptr(), snap.eps2)
        c.n = snap.n
        for ix in idx:
            idx_d = torch.tensor(ix, device=dev)
            a = torch.zeros((ix.size, 3), dtype=torch.float64, device=dev)
            k = torch.zeros_like(a)
            p = torch.zeros(ix.size, dtype=torch.float64, device=dev)
            nb.nb_force_jerk_dev(c.ctx, idx_d.data_ptr(), ix.size, a.data_ptr(), k.data_ptr(), p.data_ptr())
            nb.nb_sync(c.ctx)
            out.append((a.cpu().numpy(), k.cpu().numpy(), p.cpu().numpy()))
    return out


@pytest.mark.parametrize("n", [5000, 65536])
def test_static_entry_matches_context_entry_twice(n):
    """n = 5000: the whole system, then about 40 particles. n = NB_STATIC_MAX_N: the whole
    system (one split: s x 8 words fill the partial area exactly) and 21845 particles (the
    split factor lowered to what the partial area holds), which also uses the array's top
    offsets."""
    torch = pytest.importorskip("torch")
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody as nb
    nb.load()
    dev = torch.device("cuda:0")
    snap = ics.plummer(n, seed=21, eps=1.0 / 512)
    rng = ics.SplitMix64(22)
    if n == nb.NB_STATIC_MAX_N:
        idx = [np.arange(snap.n, dtype=np.int32),
               np.sort(np.argsort(rng.uniform(n))[:21845]).astype(np.int32)]
    else:
        idx = [np.arange(snap.n, dtype=np.int32),
               np.unique(rng.next_u64(40) % snap.n).astype(np.int32)]
    ref = _with_ctx(nb, torch, snap, dev, idx)
    m = torch.tensor(snap.m, device=dev)
    x = torch.tensor(snap.x, device=dev)
    v = torch.tensor(snap.v, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for ix, (ar, kr, pr) in zip(idx, ref):
        idx_d = torch.tensor(ix, device=dev)
        a = torch.full((ix.size, 3), float("nan"), dtype=torch.float64, device=dev)
        k = torch.full_like(a, float("nan"))
        p = torch.full((ix.size,), float("nan"), dtype=torch.float64, device=dev)
        st = nb.nb_force_jerk_static(snap.n, m.data_ptr(), x.data_ptr(), v.data_ptr(), snap.eps2, idx_d.data_ptr(),
                                     ix.size, a.data_ptr(), k.data_ptr(), p.data_ptr(), stream)
        assert st == nb.NB_OK
        a, k, p = a.cpu().numpy(), k.cpu().numpy(), p.cpu().numpy()
        if ix.size > 4096:   # compare a seeded sample against the context entry point's sums
            sel = np.unique(np.linspace(0, ix.size - 1, 4096).astype(np.int64))
            a, k, p, ar, kr, pr, ix = a[sel], k[sel], p[sel], ar[sel], kr[sel], pr[sel], ix[sel]
        A, K = condition_scales(snap.m, snap.x, snap.v, snap.eps2, ix)
        assert (np.linalg.norm(a - ar, axis=1) / A).max() < 1e-6
        assert np.percentile(rel_errors(a, ar, A), 99) < 1e-6
        assert (np.linalg.norm(k - kr, axis=1) / K).max() < 1e-6
        assert rel_scalar(p, pr).max() < 1e-6


def test_static_entry_rejects_oversize():
    from paper_0711_0643_gb300 import nbody as nb
    nb.load()
    st = nb.nb_force_jerk_static(nb.NB_STATIC_MAX_N + 1, 1, 1, 1, 0.01, 1, 1, 0, 0, 0, 0)
    assert st == nb.NB_ERR_ARG
