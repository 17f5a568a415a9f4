"""Volume constraint (Eq. formula_opt, Eq. sens_con_nod) through the library against the oracle, and
the design loop (L-BFGS steps with the stopping rule of Eq. criterion_opt) on a small problem, both
with blocking solves and with several loops sharing one served batch."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_00923_gb300 import build, design, dvm
from paper_2501_00923_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = dvm.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("ni,nj,P", [(64, 32, 8), (130, 7, 24), (16, 1, 2)])
def test_volume_constraint_matches_the_oracle(ctx, ni, nj, P):
    rng = np.random.default_rng(ni + P)
    raw = rng.uniform(-0.01, 0.01, P)
    mesh = W.omesh(ni, nj, raw * W.valid_amplitude_scale(ni, raw))
    g = W.velocity_grid(4, 4.0)
    pr = O.Problem(mesh.nodes, g.vx, g.vy, g.w, 1.0, 0.5)
    vmin = 0.0817
    Qo, _, dQo = pr.volume_constraint(vmin, mesh.dwall)
    m = dvm.Mesh(ctx, mesh.nodes)
    Q, dQ = dvm.volume_constraint(ctx, m, vmin, mesh.dwall)
    m.close()
    assert abs(Q - Qo) < 1e-13
    np.testing.assert_allclose(dQ, dQo, rtol=1e-11, atol=1e-14)


def _loop(Kn, n_params=6, max_iter=4):
    return design.DesignLoop(48, 16, W.velocity_grid(12, 4.0), W.Flow(Kn, 0.6), n_params=n_params,
                             max_iter=max_iter, first_step=1e-3, bound=0.008)


def _accepted(loop):
    acc = [loop.history[0]]
    for e in loop.history[1:]:
        if e.ok and e.Cd < acc[-1].Cd:
            acc.append(e)
    return acc


def test_design_loop_reduces_drag_under_the_volume_constraint(ctx):
    loop = design.run(ctx, _loop(1.0), storage="fp32", tol=1e-7, adjoint_tol=1e-7, stall_window=20000)
    assert loop.stopped in ("criterion_opt", "max_iter")
    acc = _accepted(loop)
    assert len(acc) >= 3
    assert acc[-1].Cd < acc[0].Cd
    # every evaluated design keeps the area >= V_min (Q is affine in alpha; projection is exact)
    assert all(e.Q <= 1e-12 for e in loop.history if e.ok)
    if loop.stopped == "criterion_opt":
        assert design.criterion_opt(acc[-2].Cd, acc[-1].Cd)


def test_concurrent_loops_share_one_served_batch(ctx):
    """Two loops at different Kn through one dvm_batch: each one's first evaluation (the symmetric
    section) equals the blocking solve within the FP32 tolerance, and each loop makes progress."""
    loops = design.run_concurrent(ctx, [_loop(1.0, max_iter=3), _loop(0.3, max_iter=3)], tol=1e-7)
    for loop in loops:
        assert loop.done
        acc = _accepted(loop)
        assert len(acc) >= 2 and acc[-1].Cd < acc[0].Cd
        assert all(e.Q <= 1e-12 for e in loop.history if e.ok)
    ref = design.DesignLoop(48, 16, W.velocity_grid(12, 4.0), W.Flow(1.0, 0.6), n_params=6, max_iter=0)
    from paper_2501_00923_gb300.autograd import DragProblem
    prob = DragProblem(ctx, 48, 16, ref.grid, ref.flow, storage="fp32", tol=1e-7, stall_window=20000)
    cd0 = prob.solve(np.zeros(6))
    prob.release()
    assert abs(loops[0].history[0].Cd - cd0) < 1e-5 * abs(cd0)


def test_cst_sensitivities_match_the_oracle(ctx):
    """The 18 CST variables of Sec. 3.3 through the same sensitivity path: parity with the oracle's
    full-discrete gradient on the same converged state."""
    params = W.cst_naca(48)
    mesh = W.omesh_cst(48, 12, params)
    grid = W.velocity_grid(12, 4.0)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st, _ = dvm.primal_solve(ctx, m, g, 1.0, 0.6, tol=1e-12, max_iter=100000, storage="fp64")
    ad, _ = dvm.adjoint_solve(ctx, st, tol=1e-12, max_iter=100000)
    grad = dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full")
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, 1.0, 0.6)
    ref = pr.sens_full(st.get(), ad.get(), mesh.dnodes())
    assert np.abs(grad - ref).max() < 1e-9 * np.abs(ref).max()
    for h in (ad, st, g, m):
        h.close()


def test_cst_design_loop_keeps_the_constraints(ctx):
    loop = design.DesignLoop(48, 12, W.velocity_grid(12, 4.0), W.Flow(1.0, 0.6), n_params=W.cst_count(),
                             shape="cst", max_iter=3, first_step=2e-3)
    design.run(ctx, loop, storage="fp32", tol=1e-7, adjoint_tol=1e-7, stall_window=20000)
    acc = _accepted(loop)
    assert len(acc) >= 2 and acc[-1].Cd < acc[0].Cd
    nb = loop.nb
    for e in loop.history:
        a = e.alpha
        assert a[0] >= 0.01 and a[1] >= 0.01 and np.all(a[2:3 + nb] >= 0) and np.all(a[3 + nb:4 + 2 * nb] <= 0)
        assert np.all(a[4 + 2 * nb:] == 0)
        if e.ok:    # Q is not affine in N1, N2: the re-linearised half-space keeps it to second order
            assert e.Q <= 1e-4 * loop.v_min


def test_second_order_paper_sensitivity_design_loop(ctx):
    """The paper's pipeline: second-order reconstruction in the primal and adjoint solves, the paper's
    boundary sensitivity (Eq. sens_J_itf, sens_B_itf) as the gradient, L-BFGS with the volume
    constraint.  The loop makes progress and keeps the constraint."""
    loop = _loop(1.0, max_iter=3)
    design.run(ctx, loop, storage="fp32", tol=1e-7, adjoint_tol=1e-7, stall_window=20000, order=2)
    acc = _accepted(loop)
    assert len(acc) >= 2 and acc[-1].Cd < acc[0].Cd
    assert all(e.Q <= 1e-12 for e in loop.history if e.ok)
