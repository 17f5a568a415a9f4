"""Mixed-precision refinement of FP32 primal solves (dvm_solve_opts.refine_tol): FP64 residuals of
fbar + delta from one FP64 sweep, FP32 linearised correction sweeps, two-sum renormalisation.

The linearised sweep is checked element by element against the oracle: from a correction of zero, two
sweeps give e2 = 2 s - (dR/df) s / D, with s the increment of one FP64 point-implicit sweep and dR/df
the Jacobian of the steady residual (the oracle's forward-mode duals).  The refined solution is checked
against the oracle's own converged solve on a small case, and against an FP64 solve on a mid-size
near-continuum case, where plain FP32 sweeps stall short of the stated drag tolerance's margin."""
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


@pytest.mark.parametrize("noise", [0.0, 0.02])
def test_linearised_sweeps_on_maxwellian_cells_match_oracle(ctx, noise):
    """The same check where the moment couplings dominate: every cell holds a Maxwellian of its own
    (random density, velocity and temperature), so the increment s comes from transport and carries
    large moment changes, and Kn = 0.01 makes the linearised Maxwellian V/tau dg the largest term of
    the second sweep; with noise the relaxation-rate term V d(1/tau) (g - f) is active too."""
    rng = np.random.default_rng(400 + int(100 * noise))
    mesh = W.omesh(24, 10, rng.uniform(-0.01, 0.01, 4))
    grid = W.velocity_grid(16, 5.0)
    Kn, Ma = 0.01, 0.8
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st = dvm.State(ctx, m, g, Kn, Ma, storage="fp32")
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma)
    nc = pr.ncell
    rho, T = rng.uniform(0.8, 1.2, nc), rng.uniform(0.8, 1.2, nc)
    u = rng.uniform(-0.3, 0.3, (nc, 2)) + np.array([Ma * W.A_INF, 0.0])
    c2 = (grid.vx[None, :] - u[:, :1]) ** 2 + (grid.vy[None, :] - u[:, 1:]) ** 2
    g1 = rho[:, None] / (2 * np.pi * T[:, None]) * np.exp(-c2 / (2 * T[:, None]))
    f = np.stack([g1, 0.5 * T[:, None] * g1], axis=-1) * (1.0 + noise * rng.uniform(-1, 1, (nc, grid.nv, 2)))
    st.set(np.ascontiguousarray(f))
    fbar = st.get()
    _, res = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=0.0, max_iter=0, storage="fp32", state=st,
                              refine_tol=1e-30, refine_max=1, refine_sweeps=2)
    s = pr.jacobi(fbar)[0] - fbar
    _, Js = pr.residual_dir(fbar, s)
    D = pr.diagonal(fbar)[..., None]
    corr = 2.0 * s - Js / D
    out = st.get() - fbar                  # fl(fbar + e2) - fbar: e2 up to the rounding of the state
    scale = np.maximum(np.abs(corr).max(axis=(1, 2)), 1e-3 * np.abs(fbar).max(axis=(1, 2)))[:, None, None]
    assert (np.abs(out - corr) / scale).max() < 1e-3
    # the linearised Maxwellian carries most of the second sweep in most cells (not in the thin wall
    # cells, where transport dominates)
    Vt = (pr.geometry()[0] * rho * np.sqrt(T) / (5.0 / 16.0 * Kn * np.sqrt(2 * np.pi)))[:, None, None]
    assert np.median(Vt / D) > 0.5
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


def test_refinement_meets_stated_fp32_tolerances_near_continuum(ctx):
    """Mid-size near-continuum case (128x64 O-mesh, 24x24 velocities, Kn 0.01, Ma 0.8): the refined FP32
    solve's drag within 1e-5 of an FP64 solve to 1e-11 (the FP64 sweeps are the oracle-checked ones),
    and the FP32 adjoint and full sensitivity on the refined state within 1e-4 of the FP64 ones per
    component."""
    rng = np.random.default_rng(2025)
    mesh = W.omesh(128, 64, rng.uniform(-0.005, 0.005, 8))
    grid = W.velocity_grid(24, 6.0)
    Kn, Ma = 0.01, 0.8
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    s64, r64 = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-11, max_iter=400000, storage="fp64", accel=(5, 10, "moments"))
    assert r64.status == dvm.DVM_OK
    a64, ar64 = dvm.adjoint_solve(ctx, s64, tol=1e-11, max_iter=400000)
    g64 = dvm.sensitivity(ctx, s64, a64, mesh.dwall, mesh.s, mode="full")
    s32, r32 = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-7, max_iter=400000, storage="fp32", stall_window=3000,
                                refine_tol=1e-9)
    assert r32.status == dvm.DVM_OK and r32.residual <= 1e-9
    a32, ar32 = dvm.adjoint_solve(ctx, s32, tol=1e-7, max_iter=400000, stall_window=3000)
    g32 = dvm.sensitivity(ctx, s32, a32, mesh.dwall, mesh.s, mode="full")
    drag_err = abs(r32.J - r64.J) / abs(r64.J)
    s_plain, r_plain = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-7, max_iter=400000, storage="fp32", stall_window=3000)
    plain_err = abs(r_plain.J - r64.J) / abs(r64.J)
    sens_err = np.abs(g32 - g64) / np.abs(g64)
    print(f"Kn 0.01: drag error plain FP32 {plain_err:.2e}, refined {drag_err:.2e} ({r32.refine_steps} steps, "
          f"{r32.refine_sweeps} sweeps from the FP32 floor {r32.residual_fp32:.1e}); sensitivities per component "
          f"{sens_err.max():.2e}")
    assert drag_err < 1e-5 and drag_err < 0.1 * plain_err
    assert sens_err.max() < 1e-4
    for h in (s_plain, a32, s32, a64, s64, g, m):
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
