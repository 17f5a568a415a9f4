"""Host orchestration of the velocity-space split (paper_2501_00923_gb300.shard) on two gloo ranks,
no GPU.  Each rank drives a stand-in state with the library's shard protocol over its half of a
velocity list; the stand-in's sweep couples the velocities only through velocity sums, as the DVM sweep
does (a relaxation toward a Gaussian scaled by the cell's total density, plus upwind transport from the
previous cell).  After the all-reduce of partials every rank must hold the same totals, and the split
iterates must equal those of one process holding the whole list."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2501_00923_gb300 import shard

NC, SWEEPS = 6, 5


class StandIn:
    """The shard protocol of dvm.State on a toy problem: f[c, k] over cells c and the velocities k of a
    slice.  Partial buffer: [NC] sums w f, [NC] residual sums w (f_new - f)^2."""

    def __init__(self, v, w):
        self.v, self.w = np.asarray(v, float), np.asarray(w, float)
        self.f = np.exp(-0.5 * (self.v[None, :] - 0.3) ** 2) * (1.0 + 0.1 * np.arange(NC)[:, None])
        self.rho = None
        self.res = np.zeros(NC)
        self.on = False

    def set_shard(self, on):
        self.on = bool(on)
        self.res[:] = 0.0

    def shard_partials(self, out=None):
        buf = np.concatenate([(self.w[None, :] * self.f).sum(1), self.res])
        if out is None:
            return buf
        out[:] = buf
        return out

    def shard_combine(self, total):
        self.rho = total[:NC].copy()
        return float(total[NC:].sum()), float(self.rho.sum())

    def iterate(self, n):
        assert n == 1 and self.rho is not None
        g = np.exp(-0.5 * self.v ** 2) / np.sqrt(2 * np.pi)
        up = np.vstack([self.f[-1:], self.f[:-1]])                 # periodic upwind neighbour
        new = 0.5 * (self.rho[:, None] * g[None, :]) + 0.5 * up
        self.res = (self.w[None, :] * (new - self.f) ** 2).sum(1)
        self.f = new


def _velocities():
    x, wx = np.polynomial.legendre.leggauss(12)
    return 4 * x, 4 * wx


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v, w = _velocities()
    vx, _, wk, _ = shard.split_grid(v, np.zeros_like(v), w, world)[rank]
    part = shard.ShardRank(StandIn(vx, wk), shard.torch_allreduce())
    hist = [part.start()]
    for _ in range(SWEEPS):
        hist.append(part.sweep())
    q.put((rank, part.state.f, hist))
    dist.destroy_process_group()


def test_two_gloo_ranks_follow_the_unsplit_iteration():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 2000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, (f, h)) for r, f, h in (q.get(timeout=120) for _ in range(2)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # one process with the whole velocity list
    v, w = _velocities()
    whole = shard.ShardRank(StandIn(v, w), lambda buf: None)
    ref = [whole.start()] + [whole.sweep() for _ in range(SWEEPS)]
    f_split = np.empty_like(whole.state.f)
    for r, (_, _, _, idx) in enumerate(shard.split_grid(v, v, w, 2)):
        f_split[:, idx] = out[r][0]
    assert np.abs(f_split - whole.state.f).max() < 1e-13
    for r in range(2):                                   # both ranks saw the same totals as one process
        assert np.allclose(out[r][1], ref, rtol=1e-13, atol=1e-15)
    assert ref[-1][0] > 0 and ref[1][0] > ref[-1][0]     # the stand-in iteration converges


def test_split_grid_is_balanced_and_complete():
    v, w = _velocities()
    parts = shard.split_grid(v, v, w, 5)
    assert sum(len(p[2]) for p in parts) == len(w)
    assert max(len(p[2]) for p in parts) - min(len(p[2]) for p in parts) <= 1
    idx = np.concatenate([p[3] for p in parts])
    assert np.array_equal(np.sort(idx), np.arange(len(w)))
    for p in parts:
        assert np.array_equal(p[0], v[p[3]])
    with pytest.raises(ValueError):
        shard.split_grid(v, v, w, 0)
