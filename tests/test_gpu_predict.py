"""Macroscopic prediction of the primal sweeps (dvm_solve_opts.predict_iters): after every block of
sweeps the moments of the steady residual are cancelled by a moment correction from the linearised
moment equations (block-Jacobi on the device), imposed on f by a Maxwellian shift.

The prediction changes the path to the steady state, not the state: the shift g(W + dW) - g(W)
vanishes with the residual.  So a predicted solve must reach the oracle's converged solution to the
same tolerance as plain sweeps, in far fewer sweeps where the sweeps are slow (small Kn)."""
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


@pytest.mark.parametrize("Kn", [0.02, 0.5])
def test_predicted_solve_reaches_the_oracle_solution(ctx, Kn):
    """Small case the oracle solves to round-off: the FP64 predicted solve agrees with it to the
    solve tolerance, in fewer sweeps than plain FP64 sweeps to the same tolerance."""
    rng = np.random.default_rng(91)
    mesh = W.omesh(24, 8, rng.uniform(-0.01, 0.01, 4))
    grid = W.velocity_grid(10, 4.0)
    Ma = 0.8
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma)
    f_ref, info = pr.primal_solve(tol=1e-13, max_sweeps=100000)
    assert info["status"] == 0
    J_ref = pr.functional(f_ref)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    sp, plain = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-12, max_iter=200000, storage="fp64")
    st, res = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-12, max_iter=200000, storage="fp64", predict=20)
    assert plain.status == dvm.DVM_OK and res.status == dvm.DVM_OK
    assert res.predictions == res.iters // 20 - 1 or res.predictions == res.iters // 20
    f = st.get()
    assert np.abs(f - f_ref).max() < 1e-9 * np.abs(f_ref).max()
    assert abs(res.J - J_ref) < 1e-10 * abs(J_ref)
    print(f"Kn {Kn}: sweeps plain {plain.iters}, predicted {res.iters} ({res.predictions} predictions)")
    if Kn < 0.1:
        assert res.iters * 5 < plain.iters
    for h in (sp, st, g, m):
        h.close()


@pytest.mark.parametrize("Kn", [0.02, 0.5])
def test_predicted_adjoint_reaches_the_oracle_adjoint(ctx, Kn):
    """The transposed prediction: on the oracle-converged primal state, the FP64 predicted adjoint solve
    agrees with the oracle's adjoint to the solve tolerance, in fewer sweeps than plain adjoint sweeps."""
    rng = np.random.default_rng(92)
    mesh = W.omesh(24, 8, rng.uniform(-0.01, 0.01, 4))
    grid = W.velocity_grid(10, 4.0)
    Ma = 0.8
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma)
    f_ref, info = pr.primal_solve(tol=1e-13, max_sweeps=100000)
    assert info["status"] == 0
    phi_ref, ainfo = pr.adjoint_solve(f_ref, tol=1e-13, max_sweeps=100000)
    assert ainfo["status"] == 0
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st = dvm.State(ctx, m, g, Kn, Ma, storage="fp64")
    st.set(f_ref)
    ap, plain = dvm.adjoint_solve(ctx, st, tol=1e-12, max_iter=200000)
    ad, res = dvm.adjoint_solve(ctx, st, tol=1e-12, max_iter=200000, predict=40)
    assert plain.status == dvm.DVM_OK and res.status == dvm.DVM_OK
    phi = ad.get()
    err = np.abs(phi - phi_ref).max() / np.abs(phi_ref).max()
    print(f"Kn {Kn}: adjoint sweeps plain {plain.iters}, predicted {res.iters} ({res.predictions} predictions); "
          f"phi error {err:.1e}")
    assert err < 1e-9
    if Kn < 0.1:
        assert res.iters * 5 < plain.iters
    for h in (ap, ad, st, g, m):
        h.close()


def test_prediction_near_continuum_mid_size(ctx):
    """128x64 O-mesh, 24x24 velocities, Kn 0.001, Ma 0.8 (transport dominates the point-implicit sweeps'
    slow modes): the FP64 predicted solve to 1e-12 and the FP64 Anderson-mixed solve to 1e-11 agree in
    drag to 1e-8 and in f to 1e-7 (at this Kn the error of a state is up to ~1e4 times its relative
    residual: the slowest sweep mode contracts by ~1e-4 per sweep).  FP32: predicted sweeps to 1e-5,
    then the refinement with predicted correction sweeps to an FP64 residual of 1e-9, match the FP64
    drag to 1e-6 in at least four times fewer sweeps (both kinds counted) than plain FP32 sweeps take to
    their own floor, where their drag is off by far more."""
    rng = np.random.default_rng(2026)
    mesh = W.omesh(128, 64, rng.uniform(-0.005, 0.005, 8))
    grid = W.velocity_grid(24, 6.0)
    Kn, Ma = 0.001, 0.8
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    s64, r64 = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-11, max_iter=600000, storage="fp64",
                                accel=(5, 10, "moments"))
    assert r64.status == dvm.DVM_OK
    p64, q64 = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-12, max_iter=600000, storage="fp64", predict=40)
    assert q64.status == dvm.DVM_OK
    f_a, f_p = s64.get(), p64.get()
    print(f"FP64 drag {abs(q64.J - r64.J) / abs(r64.J):.2e}, f {np.abs(f_a - f_p).max() / np.abs(f_a).max():.2e}")
    assert abs(q64.J - r64.J) < 1e-8 * abs(r64.J)
    assert np.abs(f_a - f_p).max() < 1e-7 * np.abs(f_a).max()
    s32, r32 = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-7, max_iter=600000, storage="fp32", stall_window=3000)
    p32, q32 = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-5, max_iter=600000, storage="fp32", predict=40,
                                refine_tol=1e-9)
    err = abs(q32.J - q64.J) / abs(q64.J)
    err_plain = abs(r32.J - q64.J) / abs(q64.J)
    print(f"Kn 0.001 128x64: sweeps FP64 Anderson {r64.iters}, FP64 predicted {q64.iters}; FP32 plain {r32.iters} "
          f"(drag error {err_plain:.1e}), FP32 predicted {q32.iters} + {q32.refine_sweeps} refinement sweeps in "
          f"{q32.refine_steps} steps, {q32.predictions} predictions (status {q32.status}, FP64 residual "
          f"{q32.residual:.1e}); drag error {err:.2e}")
    assert q32.status == dvm.DVM_OK and q32.residual <= 1e-9
    assert err < 1e-6 and err_plain > 100 * err
    assert (q32.iters + q32.refine_sweeps) * 4 < r32.iters
    # adjoints on the predicted states: FP64 to 1e-11, FP32 to its floor, both predicted; the FP32 full
    # sensitivity within 1e-4 of the FP64 one per component (largest component scale)
    a64, b64 = dvm.adjoint_solve(ctx, p64, tol=1e-11, max_iter=600000, predict=40)
    assert b64.status == dvm.DVM_OK
    g64 = dvm.sensitivity(ctx, p64, a64, mesh.dwall, mesh.s, mode="full")
    a32p, b32p = dvm.adjoint_solve(ctx, p32, tol=1e-7, max_iter=600000, stall_window=1000, predict=40)
    a32, b32 = dvm.adjoint_solve(ctx, p32, tol=1e-7, max_iter=600000, stall_window=3000)
    g32 = dvm.sensitivity(ctx, p32, a32p, mesh.dwall, mesh.s, mode="full")
    gerr = np.abs(g32 - g64).max() / np.abs(g64).max()
    print(f"adjoint sweeps: FP64 predicted {b64.iters}; FP32 predicted {b32p.iters} (residual {b32p.residual:.1e}), "
          f"plain {b32.iters} (residual {b32.residual:.1e}); FP32 sensitivity error {gerr:.1e}")
    assert gerr < 1e-4
    assert b32p.iters * 4 < b32.iters
    for h in (a32, a32p, a64, p32, s32, p64, s64, g, m):
        h.close()


def test_fp32_prediction_switches_off_at_its_noise_floor(ctx):
    """From a converged FP64 state rounded to FP32, predicted FP32 sweeps see residual moments made of the
    rounding of the relaxation term only; the solve switches the prediction off within a few blocks,
    so the drag stays within 1e-3 of the converged one (without that rule, the amplified noise walks
    the state away block after block)."""
    rng = np.random.default_rng(2026)
    mesh = W.omesh(128, 64, rng.uniform(-0.005, 0.005, 8))
    grid = W.velocity_grid(24, 6.0)
    Kn, Ma = 0.001, 0.8
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    s64, r64 = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-12, max_iter=600000, storage="fp64", predict=40)
    assert r64.status == dvm.DVM_OK
    st = dvm.State(ctx, m, g, Kn, Ma, storage="fp32")
    st.set(s64.get())
    _, r = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=0.0, max_iter=2000, storage="fp32", state=st, predict=40)
    print(f"predictions {r.predictions} of {r.iters // 20 - 1} blocks, drag error {abs(r.J - r64.J) / abs(r64.J):.2e}")
    assert r.predictions < 20
    assert abs(r.J - r64.J) < 1e-3 * abs(r64.J)
    for h in (st, s64, g, m):
        h.close()


def test_prediction_arguments(ctx):
    mesh = W.omesh(8, 3, np.zeros(2))
    grid = W.velocity_grid(8, 4.0)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    bad = [dict(predict=5, accel=(3, 10)), dict(predict=-1), dict(predict=5, predict_omega=1.5),
           dict(predict=5, predict_reuse=-2), dict(predict=5, storage="bf16")]
    for kw in bad:
        kw = {"storage": "fp32", **kw}
        with pytest.raises(dvm.DVMError) as e:
            dvm.primal_solve(ctx, m, g, 1.0, 0.5, tol=1e-6, max_iter=4, **kw)
        assert e.value.status == dvm.DVM_ERR_INVALID_ARG
    for setup in (lambda s: s.set_order(2), lambda s: setattr(s, "maxwellian", "conservative")):
        st = dvm.State(ctx, m, g, 1.0, 0.5, storage="fp32")
        setup(st)
        with pytest.raises(dvm.DVMError) as e:
            dvm.primal_solve(ctx, m, g, 1.0, 0.5, tol=1e-6, max_iter=4, storage="fp32", state=st, predict=5)
        assert e.value.status == dvm.DVM_ERR_INVALID_ARG
        with pytest.raises(dvm.DVMError) as e:
            dvm.adjoint_solve(ctx, st, tol=1e-6, max_iter=4, predict=5)
        assert e.value.status == dvm.DVM_ERR_INVALID_ARG
        st.close()
    st = dvm.State(ctx, m, g, 1.0, 0.5, storage="bf16")
    with pytest.raises(dvm.DVMError) as e:
        dvm.adjoint_solve(ctx, st, tol=1e-6, max_iter=4, predict=5)
    assert e.value.status == dvm.DVM_ERR_INVALID_ARG
    st.close()
    for h in (g, m):
        h.close()


def test_multigrid_preconditioned_prediction(ctx):
    """predict_precond = 1: a multigrid V-cycle of the moment system (Galerkin levels of the O-mesh,
    damped block-Jacobi smoothing) preconditions each GMRES step in place of the diagonal blocks.  The
    predicted FP64 solve and adjoint still reach the oracle's on the small case, and on a 128x64 mesh
    at Kn 0.01 two multigrid steps reach the solution of 40 diagonal ones (sweep counts printed)."""
    rng = np.random.default_rng(91)
    mesh = W.omesh(24, 8, rng.uniform(-0.01, 0.01, 4))
    grid = W.velocity_grid(10, 4.0)
    Kn, Ma = 0.02, 0.8
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma)
    f_ref, info = pr.primal_solve(tol=1e-13, max_sweeps=100000)
    phi_ref, ainfo = pr.adjoint_solve(f_ref, tol=1e-13, max_sweeps=100000)
    assert info["status"] == 0 and ainfo["status"] == 0
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st, res = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=1e-12, max_iter=200000, storage="fp64", predict=4,
                               predict_precond=1)
    assert res.status == dvm.DVM_OK
    assert np.abs(st.get() - f_ref).max() < 1e-9 * np.abs(f_ref).max()
    st.set(f_ref)
    ad, ares = dvm.adjoint_solve(ctx, st, tol=1e-12, max_iter=200000, predict=4, predict_precond=1)
    assert ares.status == dvm.DVM_OK
    assert np.abs(ad.get() - phi_ref).max() < 1e-9 * np.abs(phi_ref).max()
    print(f"small case, multigrid: primal {res.iters}, adjoint {ares.iters} sweeps")
    for h in (ad, st, g, m):
        h.close()
    mesh = W.omesh(128, 64, rng.uniform(-0.005, 0.005, 8))
    grid = W.velocity_grid(24, 6.0)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    sb, rb = dvm.primal_solve(ctx, m, g, 0.01, 0.8, tol=1e-11, max_iter=200000, storage="fp64", predict=40)
    sm, rm = dvm.primal_solve(ctx, m, g, 0.01, 0.8, tol=1e-11, max_iter=200000, storage="fp64", predict=2,
                              predict_precond=1)
    print(f"128x64 Kn 0.01 FP64 to 1e-11: block-Jacobi GMRES-40 {rb.iters} sweeps, multigrid GMRES-2 {rm.iters} "
          f"sweeps; drag difference {abs(rm.J - rb.J) / abs(rb.J):.1e}")
    assert rb.status == dvm.DVM_OK and rm.status == dvm.DVM_OK
    assert abs(rm.J - rb.J) < 1e-8 * abs(rb.J)
    for h in (sm, sb, g, m):
        h.close()
