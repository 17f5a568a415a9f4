"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances
* FP64 storage: one sweep agrees to 1e-12 relative (same arithmetic, different summation order;
  the exp and division of the GPU are correctly rounded or within 1-2 ulp);
* FP32 storage: one sweep to 2e-6 relative to the largest value of the cell (storage rounding
  2^-24, the update is a convex combination of stored values);
* BF16 storage: one sweep to 1.6e-2 relative (8-bit mantissa);
* converged FP32 solves: drag within 1e-5 and each sensitivity within 1e-4 relative of the FP64
  oracle (the stated targets for FP32).
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_00923_gb300 import dvm
from paper_2501_00923_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c1_oracle.json")


@pytest.fixture(scope="module")
def ctx():
    from paper_2501_00923_gb300 import build
    build.build()
    c = dvm.Context(0)
    yield c
    c.close()


def _gpu_problem(ctx, mesh, grid, Kn, Ma, storage, Tw=1.0, aoa=0.0):
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st = dvm.State(ctx, m, g, Kn, Ma, Tw, aoa, storage=storage)
    return m, g, st


def _rel(a, b, scale=None):
    scale = np.abs(b).max() if scale is None else scale
    return np.abs(a - b).max() / scale


# ------------------------------------------------------------------------------- one sweep
@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp32", 2e-6), ("bf16", 1.6e-2)])
@pytest.mark.parametrize("shape", [(40, 12, 12, 12), (24, 6, 11, 9), (3, 1, 8, 8), (16, 6, 33, 31)])
def test_one_primal_sweep_matches_oracle(ctx, storage, tol, shape):
    """Several warps' worth of cells, a ragged velocity count (99 -> padded to 100), the degenerate
    one-layer mesh whose cells touch both the wall and the far field, and a velocity count whose
    chunks fill more stage rows than the pipeline has stages in every storage (so stages are
    refilled), with a ragged last row (1023 -> 1024)."""
    ni, nj, nvx, nvy = shape
    rng = np.random.default_rng(100 + ni)
    mesh = W.omesh(ni, nj, rng.uniform(-0.01, 0.01, 4)) if ni > 3 else W.omesh(ni, nj, np.zeros(0))
    grid = W.velocity_grid(nvx, 4.0, ny=nvy)
    Kn, Ma = 0.3, 0.9
    m, g, st = _gpu_problem(ctx, mesh, grid, Kn, Ma, storage)
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma)
    f = W.random_state(pr.ncell, grid, rng)
    st.set(f)
    f_in = st.get()                      # the stored (rounded) input is what both sides use
    fn_ref, nrm = pr.jacobi(f_in)
    _, r0 = pr.residual(pr.freestream())
    res = st.iterate(1)
    fn = st.get()
    cell_scale = np.abs(fn_ref).max(axis=(1, 2))[:, None, None]
    assert (np.abs(fn - fn_ref) / cell_scale).max() < tol
    # the residual D (f_old - f_new) cancels in the storage precision: its norm is a convergence
    # monitor, checked to 1e-9 in FP64 and to 1e-3 (FP32) / 0.1 (BF16) relative
    rtol = {"fp64": 1e-9, "fp32": 1e-3, "bf16": 0.1}[storage]
    assert abs(res[0] - nrm / r0) < rtol * (nrm / r0)
    # the moments carried to the next sweep are those of the new state
    prim = st.moments()
    W_ref = pr.moments(fn if storage != "fp64" else fn_ref)
    assert np.abs(prim[:, 0] - W_ref[:, 0]).max() < max(tol, 1e-13) * 10


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-11), ("fp32", 5e-6), ("bf16", 2e-2)])
@pytest.mark.parametrize("nv", [(12, 10), (33, 31)])
def test_one_adjoint_sweep_matches_oracle(ctx, storage, tol, nv):
    rng = np.random.default_rng(7)
    mesh = W.omesh(36, 10, rng.uniform(-0.01, 0.01, 4))
    grid = W.velocity_grid(nv[0], 4.0, ny=nv[1])
    Kn, Ma = 0.5, 0.7
    m, g, st = _gpu_problem(ctx, mesh, grid, Kn, Ma, storage)
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma)
    f = W.random_state(pr.ncell, grid, rng)
    st.set(f)
    f_in = st.get()
    ad = dvm.Adjoint(st)
    phi = W.random_adjoint(pr.ncell, grid.nv, rng)
    ad.set(phi)
    phi_in = ad.get()
    ref, nrm = pr.adjoint_jacobi(f_in, phi_in)
    ad.iterate(1)
    out = ad.get()
    assert _rel(out, ref) < tol
    # and from phi = 0 the first sweep is -D^{-1} dJ/df / w (the drag source alone)
    ad0 = dvm.Adjoint(st)
    ad0.iterate(1)
    ref0, _ = pr.adjoint_jacobi(f_in, np.zeros_like(phi_in))
    assert _rel(ad0.get(), ref0) < tol


# ------------------------------------------------------------------------------- sensitivities
@pytest.mark.parametrize("storage,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_sensitivities_match_oracle_on_given_states(ctx, storage, tol):
    """K4 alone: the same (f, phi) on both sides, both sensitivity modes."""
    rng = np.random.default_rng(11)
    mesh = W.omesh(32, 12, rng.uniform(-0.01, 0.01, 6))
    grid = W.velocity_grid(12, 4.0)
    Kn, Ma = 1.0, 0.6
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma)
    f, _ = pr.primal_solve(tol=1e-10, max_sweeps=3000)
    phi, _ = pr.adjoint_solve(f, tol=1e-10, max_sweeps=3000)
    m, g, st = _gpu_problem(ctx, mesh, grid, Kn, Ma, storage)
    st.set(f)
    ad = dvm.Adjoint(st)
    ad.set(phi)
    f_in, phi_in = st.get(), ad.get()
    full_ref = pr.sens_full(f_in, phi_in, mesh.dnodes())
    paper_ref, node_ref, _ = pr.sens_paper(f_in, phi_in, mesh.dwall)
    full, _ = dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full", node_grad=True)
    paper, node = dvm.sensitivity(ctx, st, ad, mesh.dwall, mode="paper", node_grad=True)
    assert _rel(full, full_ref) < tol
    assert _rel(paper, paper_ref) < tol
    assert _rel(node, node_ref) < tol


# ------------------------------------------------------------------------------- converged solves
@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_c1_fp64_converged_drag_and_sensitivities(ctx, golden):
    wl = W.config(0)
    m, g, _ = _gpu_problem(ctx, wl.mesh, wl.grid, wl.flow.Kn, wl.flow.Ma, "fp64")
    st, res = dvm.primal_solve(ctx, m, g, wl.flow.Kn, wl.flow.Ma, tol=1e-12, max_iter=200000, storage="fp64")
    assert res.status == dvm.DVM_OK
    assert abs(res.J - golden["J"]) < 1e-9 * abs(golden["J"])
    assert abs(res.Cd - golden["Cd"]) < 1e-9 * abs(golden["Cd"])
    assert abs(st.functional("lift")) < 1e-11 * abs(golden["J"])
    ad, ares = dvm.adjoint_solve(ctx, st, tol=1e-12, max_iter=200000)
    assert ares.status == dvm.DVM_OK
    full = dvm.sensitivity(ctx, st, ad, wl.mesh.dwall, wl.mesh.s, mode="full")
    paper = dvm.sensitivity(ctx, st, ad, wl.mesh.dwall, mode="paper")
    assert _rel(full, np.array(golden["grad_full"])) < 1e-8
    assert _rel(paper, np.array(golden["grad_paper"])) < 1e-8


def test_c1_fp32_meets_stated_tolerances(ctx, golden):
    """FP32 storage and updates with FP64 reductions: drag within 1e-5, sensitivities within 1e-4."""
    wl = W.config(0)
    m = dvm.Mesh(ctx, wl.mesh.nodes)
    g = dvm.VGrid(ctx, wl.grid.vx, wl.grid.vy, wl.grid.w)
    st, res = dvm.primal_solve(ctx, m, g, wl.flow.Kn, wl.flow.Ma, tol=1e-7, max_iter=200000, storage="fp32",
                               stall_window=4000)
    assert abs(res.J - golden["J"]) < 1e-5 * abs(golden["J"])
    ad, ares = dvm.adjoint_solve(ctx, st, tol=1e-7, max_iter=200000, stall_window=4000)
    full = dvm.sensitivity(ctx, st, ad, wl.mesh.dwall, wl.mesh.s, mode="full")
    paper = dvm.sensitivity(ctx, st, ad, wl.mesh.dwall, mode="paper")
    gf, gp = np.array(golden["grad_full"]), np.array(golden["grad_paper"])
    assert np.all(np.abs(full - gf) < 1e-4 * np.abs(gf).max())
    assert np.all(np.abs(paper - gp) < 1e-4 * np.abs(gp).max())


# ------------------------------------------------------------------------------- full size, sampled
@pytest.mark.parametrize("index,storage,ptol,atol", [(1, "fp32", 2e-6, 5e-6), (2, "fp32", 2e-6, 5e-6),
                                                     (4, "bf16", 1.6e-2, 2e-2)],
                         ids=["256x128-gl48-fp32", "384x192-v64-Kn0.001-Ma2-fp32", "256x128-gl48-bf16"])
def test_full_size_sweep_sampled_cells(ctx, index, storage, ptol, atol):
    """The full-size workloads (256x128 cells with the 48x48 Gauss-Legendre grid; the largest,
    384x192 cells with 64x64 velocities at Kn 0.001 and Ma 2; the BF16 design workload) in the
    benchmark's launch configuration: one primal and one adjoint sweep from a seeded random state,
    checked on sampled cells (wall row, far-field row, interior, the periodic seam) against the
    oracle's per-cell update."""
    wl = W.config(index)
    rng = np.random.default_rng(21)
    m, g, st = _gpu_problem(ctx, wl.mesh, wl.grid, wl.flow.Kn, wl.flow.Ma, storage)
    pr = O.Problem.from_workload(wl)
    f = W.random_state(pr.ncell, wl.grid, rng)
    st.set(f)
    f_in = st.get()
    ni, nj = wl.mesh.ni, wl.mesh.nj
    cells = np.unique(np.concatenate([[0, ni - 1, ni, (nj - 1) * ni, nj * ni - 1, (nj // 2) * ni + ni // 2],
                                      rng.integers(0, ni, 6), rng.integers(0, ni * nj, 10)]))
    ref = pr.jacobi_cells(f_in, cells)
    ad = dvm.Adjoint(st)
    phi = W.random_adjoint(pr.ncell, wl.grid.nv, rng)
    ad.set(phi)
    phi_in = ad.get()
    aref = pr.adjoint_jacobi_cells(f_in, phi_in, cells)
    ad.iterate(1)                    # the adjoint is linearised at f_in: sweep it before f moves
    aout = ad.get()[cells]
    ascale = np.abs(aref).max(axis=(1, 2))[:, None, None]
    assert (np.abs(aout - aref) / ascale).max() < atol
    st.iterate(1)
    out = st.get()[cells]
    scale = np.abs(ref).max(axis=(1, 2))[:, None, None]
    assert (np.abs(out - ref) / scale).max() < ptol
    for h in (ad, st, g, m):
        h.close()


# ------------------------------------------------------------------------------- properties / errors
def test_uniform_maxwellian_stays_put_on_gpu(ctx):
    mesh = W.omesh(32, 10, np.array([0.004, -0.002]))
    grid = W.velocity_grid(16, 4.0)
    m, g, st = _gpu_problem(ctx, mesh, grid, 1e12, 0.0, "fp64")
    f0 = st.get()
    st.iterate(3)
    assert _rel(st.get(), f0) < 1e-13


def test_status_codes(ctx):
    mesh = W.omesh(16, 6, np.zeros(2))
    grid = W.velocity_grid(8, 4.0)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st, res = dvm.primal_solve(ctx, m, g, 1.0, 0.5, tol=1e-30, max_iter=40, storage="fp32")
    assert res.status == dvm.DVM_NOT_CONVERGED and res.iters == 40
    bad = st.get()
    bad[3, 2, 0] = np.nan
    st.set(bad)
    with pytest.raises(dvm.DVMError) as e:
        st.iterate(2)
    assert e.value.status == dvm.DVM_ERR_NONFINITE
    small = dvm.Context(0, hbm_budget=1024)
    m2 = dvm.Mesh(small, mesh.nodes)
    g2 = dvm.VGrid(small, grid.vx, grid.vy, grid.w)
    with pytest.raises(dvm.DVMError) as e:
        dvm.State(small, m2, g2, 1.0, 0.5)
    assert e.value.status == dvm.DVM_ERR_ADMISSION
    tangled = mesh.nodes.copy()
    tangled[1, 3] = tangled[0, 3] - 5.0 * (tangled[1, 3] - tangled[0, 3])     # first layer folded inside
    with pytest.raises(dvm.DVMError) as e:
        dvm.Mesh(ctx, tangled)
    assert e.value.status == dvm.DVM_ERR_INVALID_ARG


def test_deterministic(ctx):
    mesh = W.omesh(32, 10, np.array([0.004, -0.002]))
    grid = W.velocity_grid(12, 4.0)
    outs = []
    for _ in range(2):
        m, g, st = _gpu_problem(ctx, mesh, grid, 0.5, 0.8, "fp32")
        st.iterate(25)
        outs.append(st.get())
    assert np.array_equal(outs[0], outs[1])
