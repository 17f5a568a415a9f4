"""dvm_sensitivity_noalloc: the sensitivity for callers that must not allocate device memory during
the call (its scratch is a static device array owned by the library).

It must return what the allocating dvm_sensitivity returns, call after call, although every call
reuses the scratch the previous one left behind, and it must refuse, with a clear message, a mesh
whose intermediates do not fit the static array.  Kept in its own file so that it runs last.
"""
import numpy as np
import pytest

from paper_2501_00923_gb300 import build, dvm
from paper_2501_00923_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12     # same kernels, same inputs: the two entry points agree to round-off


def _solved(ctx, mesh, grid, Kn, Ma):
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st, _ = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-6, max_iter=400, storage="fp32")
    ad, _ = dvm.adjoint_solve(ctx, st, tol=1e-6, max_iter=400)
    return m, g, st, ad


def test_noalloc_sensitivity_matches_allocating_entry_point():
    build.build()
    ctx = dvm.Context(0)
    rng = np.random.default_rng(31)
    cases = [(W.omesh(48, 16, rng.uniform(-0.01, 0.01, 6)), W.velocity_grid(12, 4.0), 0.5, 0.8),
             (W.omesh(32, 10, rng.uniform(-0.01, 0.01, 4)), W.velocity_grid(10, 6.0), 1.0, 1.5)]
    for mesh, grid, Kn, Ma in cases:          # the second case reuses the scratch of the first
        m, g, st, ad = _solved(ctx, mesh, grid, Kn, Ma)
        # on an adjoint that has never run the allocating entry point (so has no scratch of its own),
        # the scratch-free calls take no device memory: no allocation, no bytes held
        allocs, held = ctx.allocations, ctx.bytes
        first = {mode: dvm.sensitivity(ctx, st, ad, mesh.dwall, sj, mode=mode, node_grad=True, noalloc=True)
                 for mode, sj in (("full", mesh.s), ("paper", None))}
        assert ctx.allocations == allocs and ctx.bytes == held
        for mode, sj in (("full", mesh.s), ("paper", None)):
            ref, ref_nodes = dvm.sensitivity(ctx, st, ad, mesh.dwall, sj, mode=mode, node_grad=True)
            got, nodes = first[mode]
            assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()
            assert np.abs(nodes - ref_nodes).max() <= TOL * np.abs(ref_nodes).max()
            for _ in range(2):                # two calls in a row
                allocs = ctx.allocations
                got, nodes = dvm.sensitivity(ctx, st, ad, mesh.dwall, sj, mode=mode, node_grad=True,
                                             noalloc=True)
                assert ctx.allocations == allocs
                assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()
                assert np.abs(nodes - ref_nodes).max() <= TOL * np.abs(ref_nodes).max()
    ctx.close()


def test_allocating_sensitivity_moves_the_counter():
    """Control for the test above: the allocation counter does see the allocating entry point's
    first call on a fresh adjoint, so an unchanged counter means no allocation."""
    build.build()
    ctx = dvm.Context(0)
    mesh, grid = W.omesh(24, 8, np.zeros(2)), W.velocity_grid(8, 4.0)
    m, g, st, ad = _solved(ctx, mesh, grid, 1.0, 0.5)
    allocs = ctx.allocations
    dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full")
    assert ctx.allocations > allocs
    ctx.close()


def test_noalloc_sensitivity_rejects_oversized_mesh():
    build.build()
    ctx = dvm.Context(0)
    mesh = W.omesh(512, 400, np.zeros(2))     # 204 800 cells: intermediates exceed the static array
    grid = W.velocity_grid(2, 4.0)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st = dvm.State(ctx, m, g, 1.0, 0.5)
    ad = dvm.Adjoint(st)
    with pytest.raises(dvm.DVMError) as e:
        dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full", noalloc=True)
    assert e.value.status == dvm.DVM_ERR_INVALID_ARG
    assert "static limit" in str(e.value)
    ctx.close()
