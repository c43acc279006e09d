"""Perturber lists of binaries (Sect. 3.1) against the FP64 oracle: the lists decide which
stars are perturbers (an integer result), so they must agree bit for bit — the same stars,
in the same (ascending, serial-scan) order, truncated at the same place, with the same
counts — on Plummer models with primordial binaries, over the whole star range and over the
shares of a j-parallel step, before and after an integration."""
import numpy as np
import pytest

import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody
    nbody.load()
    return nbody


def _check(nb, orc, c, m, x, pairs, gamma, nmax, j_lo=0, j_hi=None):
    gl, gc = nb.nb_perturbers(c.ctx, pairs, gamma=gamma, nmax=nmax, j_lo=j_lo, j_hi=-1 if j_hi is None else j_hi)
    ol, oc = orc.perturbers(m, x, pairs, gamma=gamma, nmax=nmax, j_lo=j_lo, j_hi=j_hi)
    np.testing.assert_array_equal(gc, oc)
    np.testing.assert_array_equal(gl, ol)
    return gl, gc


@pytest.mark.parametrize("n,nbin", [(4096, 400), (16384, 1638)])
def test_perturber_lists_match_oracle(nb, orc, n, nbin):
    snap = ics.plummer_binaries(n, nbin, ics.BASE_SEED + 40 + n.bit_length(), 1.0 / 1024)
    pairs = snap.meta["pairs"]
    with nb.Context() as c:
        c.init(snap)
        for gamma, nmax in ((1e-7, 256), (1e-5, 256), (1e-7, 17)):
            gl, gc = _check(nb, orc, c, snap.m, snap.x, pairs, gamma, nmax)
            print(f"n={n} gamma={gamma} nmax={nmax}: counts min/median/max {gc.min()}/{int(np.median(gc))}/"
                  f"{gc.max()}, {int((gc > nmax).sum())} lists full")
        # the shares of a three-rank j-parallel step, and their merge
        shares = [nb.nb_j_range(c.ctx, g, 3) for g in range(3)]
        parts = [_check(nb, orc, c, snap.m, snap.x, pairs, 1e-7, 256, lo, hi) for lo, hi in shares]
        full, cfull = nb.nb_perturbers(c.ctx, pairs, gamma=1e-7, nmax=256)
        for b in range(pairs.shape[0]):
            cat = np.concatenate([p[0][b][p[0][b] >= 0] for p in parts])[:256]
            assert list(cat) == list(full[b][full[b] >= 0])
        np.testing.assert_array_equal(sum(p[1] for p in parts), cfull)


def test_perturber_lists_after_a_run_and_device_entry(nb, orc):
    """The lists come from the context's current positions (after an integration), and the
    device entry gives the same lists."""
    import torch
    snap = ics.plummer_binaries(2048, 200, ics.BASE_SEED + 47, 1.0 / 512)
    pairs = snap.meta["pairs"]
    with nb.Context() as c:
        c.init(snap)
        nb.nb_run(c.ctx, 1.0 / 64)
        st = c.state()
        gl, gc = _check(nb, orc, c, st["m"], st["x"], pairs, 1e-7, 256)
        dev = torch.device("cuda", 0)
        p_d = torch.tensor(pairs, device=dev)
        l_d = torch.empty((pairs.shape[0], 256), dtype=torch.int32, device=dev)
        c_d = torch.empty(pairs.shape[0], dtype=torch.int32, device=dev)
        nb.nb_perturbers_dev(c.ctx, pairs.shape[0], p_d.data_ptr(), 1e-7, 256, 0, -1, l_d.data_ptr(), c_d.data_ptr())
        nb.nb_sync(c.ctx)
        np.testing.assert_array_equal(l_d.cpu().numpy(), gl)
        np.testing.assert_array_equal(c_d.cpu().numpy(), gc)


def test_perturber_argument_errors(nb):
    import torch
    snap = ics.plummer_binaries(512, 20, 5, 1e-2)
    with nb.Context() as c:
        c.init(snap)
        for bad in ([[3, 3]], [[0, 512]], [[-1, 2]]):
            with pytest.raises(nb.NbError) as e:
                nb.nb_perturbers(c.ctx, bad)
            assert e.value.status == nb.NB_ERR_ARG
        for kw in ({"nmax": 0}, {"nmax": nb.NB_PERT_MAX + 1}, {"gamma": 0.0}):
            with pytest.raises(nb.NbError) as e:
                nb.nb_perturbers(c.ctx, [[0, 1]], **kw)
            assert e.value.status == nb.NB_ERR_ARG
        # device entry: an invalid pair gives an empty row and a count of -1
        dev = torch.device("cuda", 0)
        p_d = torch.tensor([[0, 492], [7, 7]], dtype=torch.int32, device=dev)
        l_d = torch.zeros((2, 8), dtype=torch.int32, device=dev)
        c_d = torch.zeros(2, dtype=torch.int32, device=dev)
        nb.nb_perturbers_dev(c.ctx, 2, p_d.data_ptr(), 1e-7, 8, 0, -1, l_d.data_ptr(), c_d.data_ptr())
        nb.nb_sync(c.ctx)
        assert int(c_d[1]) == -1 and bool((l_d[1] == -1).all())
        assert int(c_d[0]) >= 0
