"""A stand-in for the GPU block-step operations of paper_0711_0643_gb300/jparallel.py,
written on the FP64 CPU oracle, so that the j-parallel driver can run on CPU ranks
(tests only; the library never uses it).

Partial forces over a share [j0, j1) of j are the oracle's sums with the masses outside
the share set to zero (those terms then add exact zeros); the corrector is the oracle's,
particle by particle. The shares follow the library's rule (nb_j_range): whole tiles of
256 particles, tile t to rank floor(t p / T)."""
import numpy as np

TILE = 256


class OracleOps:
    def __init__(self, orc, snap, eta=0.01, nthreads=1):
        self.orc = orc
        self.eps2 = snap.eps2
        self.eta = eta
        self.nthreads = nthreads
        sysr = orc.System(snap.m, snap.x, snap.v, snap.eps2, eta=eta, nthreads=nthreads)
        assert sysr.status == 0
        self.st = {k: getattr(sysr, k).copy() for k in ("m", "x", "v", "a", "k", "t", "dt")}
        self.n = snap.n
        self.idx = None
        self.last_forces = None

    def j_range(self, rank, world):
        T = (self.n + TILE - 1) // TILE
        lo, hi = T * rank // world, T * (rank + 1) // world
        return min(lo * TILE, self.n), min(hi * TILE, self.n)

    def next_block(self):
        tn, self.idx = self.orc.next_block(self.st["t"], self.st["dt"])
        return tn, int(self.idx.size)

    def predict(self, t):
        st = self.st
        self.xp, self.vp = self.orc.predict(st["x"], st["v"], st["a"], st["k"], st["t"], t)

    def partial_forces(self, s, j0, j1):
        assert s == self.idx.size
        mm = np.zeros_like(self.st["m"])
        mm[j0:j1] = self.st["m"][j0:j1]
        a, k, phi = self.orc.force(mm, self.xp, self.vp, self.eps2, self.idx, nthreads=self.nthreads)
        return np.concatenate([a, k, phi[:, None]], axis=1)

    def perturbers(self, pairs, gamma, nmax, j0, j1):
        return self.orc.perturbers(self.st["m"], self.st["x"], pairs, gamma=gamma, nmax=nmax, j_lo=j0, j_hi=j1)

    def correct(self, t, total):
        st = self.st
        self.last_forces = np.array(total, copy=True)
        for q, i in enumerate(self.idx):
            dt = st["dt"][i]
            x1, v1, cand = self.orc.correct_particle(self.xp[i], self.vp[i], st["a"][i], st["k"][i], total[q, 0:3],
                                                     total[q, 3:6], dt, self.eta)
            st["x"][i], st["v"][i] = x1, v1
            st["a"][i], st["k"][i] = total[q, 0:3], total[q, 3:6]
            st["dt"][i] = self.orc.quantise(cand, dt, t)
            st["t"][i] = t
