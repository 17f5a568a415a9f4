"""Velocity-space split of one steady primal solve.

Every part (a rank with its own GPU, or a state on a shared device) holds all cells for a slice of the
velocity grid.  The point-implicit sweep of Eq. (numerpr_gov) couples velocities only through velocity
sums (the cell moments of Eq. macint_reduce, the wall density of Eq. formula_bgk_fdw, the normaliser of
Eq. barg, the drag of Eq. numer_J and the residual), so one exchange per sweep suffices: each part writes
the partial sums of its slice, the parts add them (an all-reduce), and each installs the total before
its next sweep.  The library does the sweeps and the installation (dvm_state_set_shard,
dvm_state_shard_partials, dvm_state_shard_combine); this module only sequences them around an
all-reduce it is given, so the orchestration runs unchanged on gloo ranks over host buffers, on NCCL
ranks over device buffers, or on one device.
"""
from __future__ import annotations

import numpy as np


def split_grid(vx, vy, w, parts: int):
    """Interleaved, balanced slices of a velocity list: slice p holds the velocities p, p + parts,
    p + 2 parts, ...  Every slice then spans all directions, so each wall face keeps velocities
    toward the wall and away from it (its normaliser D_l stays positive), and the slices carry
    similar work.  Returns [(vx, vy, w, index), ...]."""
    n = len(w)
    if not 1 <= parts <= n:
        raise ValueError("parts must be between 1 and the number of velocities")
    vx, vy, w = np.asarray(vx), np.asarray(vy), np.asarray(w)
    out = []
    for p in range(parts):
        idx = np.arange(p, n, parts)
        out.append((vx[idx].copy(), vy[idx].copy(), w[idx].copy(), idx))
    return out


class ShardRank:
    """One part of a split solve.  `state` offers set_shard / shard_partials / shard_combine / iterate
    (dvm.State does); `allreduce(buf)` adds `buf` across the parts in place."""

    def __init__(self, state, allreduce):
        self.state = state
        self.allreduce = allreduce
        self.buf = None

    def _exchange(self):
        self.buf = self.state.shard_partials(self.buf)
        self.allreduce(self.buf)
        return self.state.shard_combine(self.buf)

    def start(self):
        """Enter shard mode and install the whole grid's moments and wall constants of the current f."""
        self.state.set_shard(True)
        return self._exchange()

    def sweep(self):
        """One sweep of every part, then the exchange: (residual sum of squares of the sweep's input,
        drag of the new state)."""
        self.state.iterate(1)
        return self._exchange()


def torch_allreduce(group=None):
    """An allreduce(buf) over torch.distributed for host numpy buffers (gloo)."""
    import torch
    import torch.distributed as dist

    def reduce(buf):
        t = torch.from_numpy(buf)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)

    return reduce


class LocalShards:
    """Several parts on one process (one device): the all-reduce is a sum of their host buffers."""

    def __init__(self, states):
        self.states = states

    def _exchange(self):
        parts = [s.shard_partials() for s in self.states]
        total = np.sum(parts, axis=0)
        return [s.shard_combine(total) for s in self.states][0]

    def start(self):
        for s in self.states:
            s.set_shard(True)
        return self._exchange()

    def sweep(self):
        for s in self.states:
            s.iterate(1)
        return self._exchange()
