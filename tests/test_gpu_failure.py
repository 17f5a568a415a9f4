"""Failure detection without a GPU fault: a device wait that nothing completes gives up at its bound,
the host reads DVM_ERR_TIMEOUT, and the context goes on working."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_00923_gb300 import build, dvm
from paper_2501_00923_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_the_context_stays_usable():
    build.build()
    ctx = dvm.Context(0)
    t = time.perf_counter()
    st = dvm.lib().dvm_selftest_wait_timeout(ctx.h)
    dt = time.perf_counter() - t
    assert st == dvm.DVM_ERR_TIMEOUT, dvm.status_string(st)
    assert 1.5 < dt < 60.0
    # the same context still sweeps correctly afterwards
    rng = np.random.default_rng(4)
    mesh = W.omesh(16, 6, rng.uniform(-0.01, 0.01, 4))
    grid = W.velocity_grid(8, 4.0)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    s = dvm.State(ctx, m, g, 0.5, 0.7, storage="fp64")
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, 0.5, 0.7)
    s.set(W.random_state(pr.ncell, grid, rng))
    f_in = s.get()
    ref, _ = pr.jacobi(f_in)
    s.iterate(1)
    assert np.abs(s.get() - ref).max() < 1e-12 * np.abs(ref).max()
    s.close(); g.close(); m.close(); ctx.close()
