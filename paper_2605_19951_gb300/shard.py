"""Pole partition of the shifted systems over ranks (Algorithm 1, Fig. 1).

The poles are independent: each rank factors A_i = K - xi_i M and solves
only for its own poles i, and every output of the path is a sum over poles
(the residue sums of the data and of J v, Section 2.3 and Section 3.1; the
cell sums of J^T w, Section 3.1).  So a rank builds its model with its poles
and their residue columns alpha_i^[j], and one all-reduce (sum) per product
assembles the full result:
  forward, J v:  partial data [n_tx][n_rx][K] summed over ranks;
  J^T w:         partial model vector [P] summed over ranks (w replicated).
The local operator is anything with forward(), jvp(v), jtvp(w): a tem.Model
on this rank's GPU (NCCL) or, for tests without a GPU, the oracle (gloo).
"""
from __future__ import annotations

import numpy as np


def pole_partition(m, world):
    """Contiguous blocks of poles, sizes differing by at most one (every pole
    costs the same: one factorisation and the same sweeps)."""
    if world < 1 or m < world:
        raise ValueError(f"{m} poles cannot be split over {world} ranks")
    bounds = np.linspace(0, m, world + 1).round().astype(int)
    return [list(range(bounds[r], bounds[r + 1])) for r in range(world)]


def local_poles(xi, alpha, rank, world):
    """This rank's poles xi_i and residue rows alpha_i^[j]."""
    part = pole_partition(len(xi), world)[rank]
    return np.asarray(xi)[part], np.asarray(alpha)[part]


class ShardedOperator:
    """Forward / J v / J^T w of the full pole set from a rank-local operator
    over this rank's poles: each product is the local partial sum followed by
    one all-reduce (sum) over the process group."""

    def __init__(self, local, dist, group=None, device="cpu"):
        self.local = local
        self.dist = dist
        self.group = group
        self.device = device

    def _allreduce(self, x):
        import torch
        t = x if isinstance(x, torch.Tensor) else torch.as_tensor(np.ascontiguousarray(x))
        t = t.to(self.device, dtype=torch.float64).contiguous()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t

    def forward(self):
        return self._allreduce(self.local.forward())

    def jvp(self, v):
        return self._allreduce(self.local.jvp(v))

    def jtvp(self, w):
        return self._allreduce(self.local.jtvp(w))
