"""The paper's j-parallel block step (Sect. 3 and its Flowchart) across torch.distributed ranks.

Every rank holds the whole system, as in the paper. For each block step every rank
selects the same block and predicts all particles (the state is replicated bit for bit),
rank g sums the forces on the block over its own share of j only (whole 256-particle
tiles, ``nb_j_range``), the partial forces are added over the ranks (the paper's
MPI_Allreduce), and every rank corrects the block with the same totals, so the replicas
stay identical. The paper's Allgatherv of the corrected particles is not needed: every
rank corrects every active particle itself.

The partial sums are added in rank order after an all-gather, not by an all-reduce whose
order the collective library chooses: the totals, and therefore the trajectory, do not
depend on the collective's algorithm and are the same on every rank, run after run.

The block-step operations come from an ``ops`` object (``GpuOps`` drives one GPU through
the C ABI; anything with the same methods can stand in). The exchange goes through host
tensors with the gloo backend and through device tensors with NCCL.
"""
from __future__ import annotations

import numpy as np


class GpuOps:
    """One rank's block-step operations on its GPU, through libnbody.so.

    ``device``: exchange partial forces as CUDA tensors (NCCL); otherwise host arrays."""

    def __init__(self, nb, ctx, n, device=None):
        self.nb = nb
        self.ctx = ctx
        self.n = int(n)
        self.device = device

    def j_range(self, rank, world):
        return self.nb.nb_j_range(self.ctx, rank, world)

    def next_block(self):
        return self.nb.nb_next_block(self.ctx)

    def active(self, s):
        return self.nb.nb_get_active(self.ctx, s)

    def predict(self, t):
        self.nb.nb_predict(self.ctx, t)

    def partial_forces(self, s, j0, j1):
        """(s, 7) partial sums a, k, phi over j in [j0, j1) for the active list of the last block."""
        if self.device is None:
            a, k, phi = self.nb.nb_force_jerk_range(self.ctx, None, s, j0, j1)
            return np.concatenate([a, k, phi[:, None]], axis=1)
        import torch
        a = torch.empty((s, 3), dtype=torch.float64, device=self.device)
        k = torch.empty_like(a)
        phi = torch.empty((s, 1), dtype=torch.float64, device=self.device)
        self.nb.nb_force_jerk_range_dev(self.ctx, 0, s, j0, j1, a.data_ptr(), k.data_ptr(), phi.data_ptr())
        self.nb.nb_sync(self.ctx)
        return torch.cat([a, k, phi], dim=1)

    def perturbers(self, pairs, gamma, nmax, j0, j1):
        """This rank's perturber lists over its share [j0, j1) (Sect. 3.1): (lists, counts)."""
        return self.nb.nb_perturbers(self.ctx, pairs, gamma=gamma, nmax=nmax, j_lo=j0, j_hi=j1)

    def correct(self, t, total):
        if self.device is None:
            self.nb.nb_correct_forces(self.ctx, t, np.ascontiguousarray(total[:, 0:3]),
                                      np.ascontiguousarray(total[:, 3:6]))
        else:
            a = total[:, 0:3].contiguous()
            k = total[:, 3:6].contiguous()
            self.nb.nb_correct_forces_dev(self.ctx, t, a.data_ptr(), k.data_ptr())


class JParallel:
    """Block steps of one system replicated on every rank of a process group, with the force
    sum split over j (rank g owns ``j_range``) and the partial forces added in rank order.
    Without an initialised process group it runs as a single rank."""

    def __init__(self, ops, group=None, check=True):
        self.ops = ops
        self.group = group
        self.check = check
        try:
            import torch.distributed as dist
            self.dist = dist if dist.is_available() and dist.is_initialized() else None
        except ImportError:
            self.dist = None
        self.world = self.dist.get_world_size(group) if self.dist else 1
        self.rank = self.dist.get_rank(group) if self.dist else 0
        self.j0, self.j1 = ops.j_range(self.rank, self.world)

    def _gather(self, x):
        """All ranks' copies of x (a numpy array or a tensor), in rank order."""
        import torch
        host = isinstance(x, np.ndarray)
        t = torch.from_numpy(np.ascontiguousarray(x)) if host else x.contiguous()
        parts = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(parts, t, group=self.group)
        return [p.numpy() for p in parts] if host else parts

    def sum_over_ranks(self, part):
        """The partial forces of all ranks added in rank order (the same totals on every rank)."""
        if self.world == 1:
            return part
        parts = self._gather(part)
        total = parts[0].copy() if isinstance(part, np.ndarray) else parts[0].clone()
        for p in parts[1:]:
            total += p
        return total

    def perturbers(self, pairs, gamma=1e-7, nmax=256):
        """Perturber lists of the binaries ``pairs`` (Sect. 3.1), found in parallel and put back
        in the serial order: each rank scans its own share of the stars (ascending), the
        ranks' lists are gathered and concatenated in rank order (the shares ascend, so
        this is the order of a serial scan) and cut at nmax, and the counts are added. The
        paper broadcasts the lists and sorts them; here the shares' order makes the merge
        a concatenation. Returns (lists [nbin][nmax] with -1 padding, counts), the same on
        every rank."""
        lists, counts = self.ops.perturbers(pairs, gamma, nmax, self.j0, self.j1)
        if self.world == 1:
            return lists, counts
        all_l = self._gather(np.ascontiguousarray(lists, dtype=np.int32))
        all_c = self._gather(np.ascontiguousarray(counts, dtype=np.int32))
        nbin = lists.shape[0]
        out = np.full((nbin, nmax), -1, dtype=np.int32)
        for b in range(nbin):
            cat = np.concatenate([lr[b][lr[b] >= 0] for lr in all_l])[:nmax]
            out[b, :cat.size] = cat
        return out, np.sum(np.stack(all_c), axis=0).astype(np.int32)

    def _agree(self, tn, s):
        """Every rank must be at the same block (the replicas are identical)."""
        if self.world == 1 or not self.check:
            return
        rows = self._gather(np.array([tn, float(s)]))
        for r, row in enumerate(rows):
            if row[0] != tn or row[1] != s:
                raise RuntimeError(f"rank {r} is at block (t = {row[0]}, s = {row[1]}), rank {self.rank} at "
                                   f"(t = {tn}, s = {s}): the replicas have diverged")

    def step(self, block=None):
        """One block step; ``block`` = (t_next, s) of a selection already made. Returns (t_next, s)."""
        tn, s = block if block is not None else self.ops.next_block()
        self._agree(tn, s)
        self.ops.predict(tn)
        part = self.ops.partial_forces(s, self.j0, self.j1)
        self.ops.correct(tn, self.sum_over_ranks(part))
        return tn, s

    def run(self, t_end, max_steps=None):
        """Block steps while the next block time is at most t_end; returns the steps done."""
        done = 0
        while max_steps is None or done < max_steps:
            tn, s = self.ops.next_block()
            if not tn <= t_end:
                break
            self.step((tn, s))
            done += 1
        return done
