"""Velocity-space split of one primal solve on one GPU: the two halves of a velocity grid as two
states (velocity shards) whose partial sums are added between sweeps, against the unsplit state.  The
sweeps couple velocities only through the summed moments, wall density, wall normaliser, drag and
residual, so the split iterates must follow the unsplit ones to round-off."""
import numpy as np
import pytest

from paper_2501_00923_gb300 import build, dvm, shard
from paper_2501_00923_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = dvm.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("parts", [2, 3])
def test_split_sweeps_follow_the_unsplit_sweeps(ctx, storage, tol, parts):
    rng = np.random.default_rng(90 + parts)
    mesh = W.omesh(40, 12, rng.uniform(-0.01, 0.01, 4))
    grid = W.velocity_grid(14, 4.0)                    # 196 velocities: slices of 98 / 65-66, ragged chunks
    Kn, Ma = 0.3, 0.9
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    whole = dvm.State(ctx, m, g, Kn, Ma, storage=storage)
    slices = shard.split_grid(grid.vx, grid.vy, grid.w, parts)
    grids = [dvm.VGrid(ctx, *sl[:3]) for sl in slices]
    states = [dvm.State(ctx, m, gg, Kn, Ma, storage=storage) for gg in grids]
    f0 = W.random_state(mesh.ncell, grid, rng)
    whole.set(f0)
    for s, sl in zip(states, slices):
        s.set(np.ascontiguousarray(f0[:, sl[3]]))
    split = shard.LocalShards(states)
    split.start()
    for _ in range(12):
        r_whole = whole.iterate(1)[0] * _r0(whole)
        J_whole = whole.functional("drag")
        res_sq, J = split.sweep()
        assert abs(np.sqrt(res_sq) - r_whole) <= tol * r_whole
        assert abs(J - J_whole) <= tol * max(abs(J_whole), 1e-2)   # the drag of a random state can be near 0
    fw = whole.get()
    fs = np.empty_like(fw)
    for s, sl in zip(states, slices):
        fs[:, sl[3]] = s.get()
    scale = np.abs(fw).max(axis=(1, 2))[:, None, None]
    assert (np.abs(fs - fw) / scale).max() < tol
    # the split is refused where it does not apply
    with pytest.raises(dvm.DVMError):
        dvm.Adjoint(states[0])
    with pytest.raises(dvm.DVMError):
        states[0].iterate(2)
    states[0].set_shard(False)                         # back to a grid of its own
    states[0].iterate(1)
    for h in states + grids + [whole, g, m]:
        h.close()


def _r0(st):
    """|R| of the free-stream state of `st` (the normaliser of the residuals iterate() reports)."""
    _, res = dvm.primal_solve(st.ctx, st.mesh, st.grid, st.flow.Kn, st.flow.Ma, tol=0.0, max_iter=0,
                              storage=st.storage, state=st)
    return res.r0
