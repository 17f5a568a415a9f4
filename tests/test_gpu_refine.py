"""Mixed-precision refinement of FP32 primal solves (dvm_solve_opts.refine_tol): FP64 residuals of
fbar + delta from one FP64 sweep, FP32 linearised correction sweeps, two-sum renormalisation.

The linearised sweep is checked element by element against the oracle: from a correction of zero, two
sweeps give e2 = 2 s - (dR/df) s / D, with s the increment of one FP64 point-implicit sweep and dR/df
the Jacobian of the steady residual (the oracle's forward-mode duals).  The refined solution is checked
against the oracle's own converged solve on a small case."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_00923_gb300 import build, dvm
from paper_2501_00923_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = dvm.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("shape", [(24, 10, 18, 18), (16, 1, 10, 9), (40, 12, 8, 8)])
def test_two_linearised_sweeps_match_oracle_jacobian(ctx, shape):
    """Shapes: three stage rows of 64 chunks (a ragged last one) with wall- and far-field rows; a
    one-layer mesh whose cells touch both boundaries, with a ragged velocity count; several blocks of
    cells.  One correction step of two linearised sweeps leaves fl(fbar + e2) in the state."""
    ni, nj, nvx, nvy = shape
    rng = np.random.default_rng(300 + ni)
    mesh = W.omesh(ni, nj, rng.uniform(-0.01, 0.01, 4))
    grid = W.velocity_grid(nvx, 4.0, ny=nvy)
    Kn, Ma = 0.2, 0.9
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st = dvm.State(ctx, m, g, Kn, Ma, storage="fp32")
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma)
    st.set(W.random_state(pr.ncell, grid, rng))
    fbar = st.get()
    _, res = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=0.0, max_iter=0, storage="fp32", state=st,
                              refine_tol=1e-30, refine_max=1, refine_sweeps=2)
    assert res.refine_steps == 1 and res.refine_sweeps == 2
    s = pr.jacobi(fbar)[0] - fbar
    _, Js = pr.residual_dir(fbar, s)
    D = pr.diagonal(fbar)[..., None]
    ref = fbar + 2.0 * s - Js / D
    out = st.get()
    scale = np.abs(ref).max(axis=(1, 2))[:, None, None]
    assert (np.abs(out - ref) / scale).max() < 3e-6
    # the correction is not small here: a wrong coupling term would show
    assert np.abs(2.0 * s - Js / D).max() > 0.05 * np.abs(fbar).max()
    for h in (st, g, m):
        h.close()


def test_refined_fp32_solution_matches_the_oracle_solve(ctx):
    """Small case the oracle solves to round-off: plain FP32 sweeps stop at their rounding floor, the
    refinement continues to an FP64 residual of 1e-11, and the refined state and drag then agree with
    the oracle's FP64 solution to FP32 rounding of the state."""
    rng = np.random.default_rng(77)
    mesh = W.omesh(24, 8, rng.uniform(-0.01, 0.01, 4))
    grid = W.velocity_grid(10, 4.0)
    Kn, Ma = 0.05, 0.8
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma)
    f_ref, info = pr.primal_solve(tol=1e-13, max_sweeps=60000)
    assert info["status"] == 0
    J_ref = pr.functional(f_ref)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    _, plain = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-12, max_iter=200000, storage="fp32", stall_window=2000)
    st, res = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-12, max_iter=200000, storage="fp32", stall_window=2000,
                               refine_tol=1e-11)
    assert res.status == dvm.DVM_OK and res.residual <= 1e-11
    assert res.residual_fp32 > 1e-9                       # the FP32 sweeps alone stalled far above it
    f = st.get()
    assert np.abs(f - f_ref).max() < 2e-7 * np.abs(f_ref).max()
    assert abs(res.J - J_ref) < 1e-9 * abs(J_ref)
    assert abs(plain.J - J_ref) > 10 * abs(res.J - J_ref)
    print(f"drag error: plain FP32 {abs(plain.J - J_ref) / abs(J_ref):.2e}, refined {abs(res.J - J_ref) / abs(J_ref):.2e}"
          f" ({res.refine_steps} steps, {res.refine_sweeps} sweeps)")
    for h in (st, g, m):
        h.close()


def test_refinement_arguments(ctx):
    mesh = W.omesh(8, 3, np.zeros(2))
    grid = W.velocity_grid(8, 4.0)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    for storage in ("fp64", "bf16"):
        with pytest.raises(dvm.DVMError) as e:
            dvm.primal_solve(ctx, m, g, 1.0, 0.5, tol=1e-6, max_iter=4, storage=storage, refine_tol=1e-10)
        assert e.value.status == dvm.DVM_ERR_INVALID_ARG
    with pytest.raises(dvm.DVMError) as e:
        dvm.primal_solve(ctx, m, g, 1.0, 0.5, tol=1e-6, max_iter=4, storage="fp32", refine_tol=-1.0)
    assert e.value.status == dvm.DVM_ERR_INVALID_ARG
    for h in (g, m):
        h.close()
