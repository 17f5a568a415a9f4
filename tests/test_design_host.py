"""Host logic of the design loop: the L-BFGS step, its line search, the projection onto the box and
the volume-constraint half-space, and the stopping rule of Eq. (criterion_opt), on analytic
objectives (no GPU)."""
import numpy as np
import pytest

from paper_2501_00923_gb300 import design as D
from paper_2501_00923_gb300 import workloads as W


def _minimise(opt, fun, max_evals=500):
    while opt.phase != "done" and opt.evaluations < max_evals:
        x = opt.ask()
        f, g = fun(x)
        opt.tell(f, g)
        if opt.phase != "done" and opt.g is not None and np.linalg.norm(opt.g) < 1e-11:
            break
    return opt


def test_criterion_opt_is_relative_change_below_3e5():
    assert D.criterion_opt(1.0, 1.0 - 2.9e-5)
    assert not D.criterion_opt(1.0, 1.0 - 3.1e-5)
    assert D.criterion_opt(-2.0, -2.0 + 5.9e-5)
    assert not D.criterion_opt(0.5, 0.6)


def test_two_loop_direction_equals_the_explicit_bfgs_inverse_update():
    """With memory >= number of pairs, -H g from the two-loop recursion equals the product of the
    textbook BFGS inverse-Hessian updates H <- (I - r s y^T) H (I - r y s^T) + r s s^T from
    H0 = (s.y / y.y) I of the newest pair (Nocedal and Wright, Eq. 6.17 and 7.20)."""
    rng = np.random.default_rng(5)
    n = 7
    Mx = rng.normal(size=(n, n))
    A = Mx @ Mx.T + n * np.eye(n)
    opt = D.LBFGS(np.zeros(n), m=10)
    for _ in range(5):
        s = rng.normal(size=n)
        opt.S.append(s)
        opt.Y.append(A @ s)
    g = rng.normal(size=n)
    s_new, y_new = opt.S[-1], opt.Y[-1]
    H = (s_new @ y_new) / (y_new @ y_new) * np.eye(n)
    for s, y in zip(opt.S, opt.Y):
        r = 1.0 / (y @ s)
        V = np.eye(n) - r * np.outer(y, s)
        H = V.T @ H @ V + r * np.outer(s, s)
    np.testing.assert_allclose(opt.direction(g), -H @ g, rtol=1e-12, atol=1e-13)


def test_lbfgs_reaches_the_minimum_of_a_convex_quadratic():
    rng = np.random.default_rng(6)
    n = 12
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    A = Q @ np.diag(np.geomspace(1.0, 100.0, n)) @ Q.T
    b = rng.normal(size=n)
    x_star = np.linalg.solve(A, b)
    opt = _minimise(D.LBFGS(np.zeros(n), first_step=0.1), lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b))
    assert np.abs(opt.x - x_star).max() < 1e-7 * np.abs(x_star).max()
    assert opt.evaluations < 150


def test_lbfgs_on_rosenbrock():
    def rosen(x):
        f = 100 * (x[1] - x[0] ** 2) ** 2 + (1 - x[0]) ** 2
        g = np.array([-400 * x[0] * (x[1] - x[0] ** 2) - 2 * (1 - x[0]), 200 * (x[1] - x[0] ** 2)])
        return f, g
    opt = _minimise(D.LBFGS(np.array([-1.2, 1.0]), first_step=0.1), rosen, max_evals=2000)
    np.testing.assert_allclose(opt.x, [1.0, 1.0], atol=1e-6)


def test_bounds_hold_and_the_projected_minimum_is_found():
    """Separable quadratic with its minimum outside the box: the iterate ends on the clipped point."""
    c = np.array([0.3, -0.02, 0.004, 0.05])
    opt = _minimise(D.LBFGS(np.zeros(4), lower=-0.01, upper=0.01, first_step=1e-3),
                    lambda x: (float(((x - c) ** 2).sum()), 2 * (x - c)))
    np.testing.assert_allclose(opt.x, np.clip(c, -0.01, 0.01), atol=1e-9)
    assert all(np.all(np.abs(e) <= 0.01 + 1e-15) for e in [opt.x])


def test_unevaluable_trials_are_backtracked():
    """An infinite objective (a design that could not be solved) cuts the step, it is never accepted."""
    bad = []

    def fun(x):
        if x[0] > 0.5:
            bad.append(x.copy())
            return np.inf, np.zeros_like(x)
        return float((x[0] - 1.0) ** 2 + x[1] ** 2), np.array([2 * (x[0] - 1.0), 2 * x[1]])
    opt = _minimise(D.LBFGS(np.array([0.0, 0.3]), first_step=0.8), fun, max_evals=200)
    assert bad and opt.x[0] <= 0.5


def test_projection_onto_box_and_halfspace_is_the_nearest_feasible_point():
    rng = np.random.default_rng(9)
    n = 8
    lo, hi = -0.01, 0.01
    for _ in range(20):
        c = rng.normal(size=n)
        b = rng.uniform(-0.01, 0.01)
        x = rng.normal(size=n) * 0.02
        y = D.project_box_halfspace(x, lo, hi, c, b)
        assert np.all(y >= lo - 1e-15) and np.all(y <= hi + 1e-15) and c @ y <= b + 1e-12
        d = np.linalg.norm(x - y)
        for _ in range(200):                   # no sampled feasible point is nearer
            z = rng.uniform(lo, hi, n)
            if c @ z <= b:
                assert np.linalg.norm(x - z) >= d - 1e-12
        z = np.clip(x, lo, hi)                  # feasible clip => the projection is the clip
        if c @ z <= b:
            np.testing.assert_allclose(y, z, atol=1e-15)


def test_volume_constraint_is_affine_in_the_bump_amplitudes():
    """The bumps move the wall nodes in y only, so the shoelace area, and Q, is affine in alpha:
    Q(alpha) = Q(0) + dQ . alpha exactly.  The projected L-BFGS relies on it."""
    from oracle import oracle as O
    g = W.velocity_grid(4, 4.0)
    rng = np.random.default_rng(10)
    m0 = W.omesh(64, 4, np.zeros(8))
    Q0, _, dQ = O.Problem(m0.nodes, g.vx, g.vy, g.w, 1.0, 0.5).volume_constraint(0.08, m0.dwall)
    for _ in range(5):
        a = rng.uniform(-0.01, 0.01, 8) * 0.5
        m = W.omesh(64, 4, a)
        Qa, _, dQa = O.Problem(m.nodes, g.vx, g.vy, g.w, 1.0, 0.5).volume_constraint(0.08, m.dwall)
        assert abs(Qa - (Q0 + dQ @ a)) < 1e-15
        np.testing.assert_allclose(dQa, dQ, rtol=1e-12, atol=1e-17)


def test_design_loop_stops_by_criterion_opt_on_an_analytic_problem():
    """Drag-like convex objective with the volume constraint: the loop decreases the merit
    monotonically over accepted steps and stops by Eq. (criterion_opt) before max_iter."""
    n = 6
    rng = np.random.default_rng(8)
    A = np.diag(np.linspace(20.0, 60.0, n))
    c = rng.uniform(-0.004, 0.004, n)
    q = -np.abs(rng.normal(size=n)) * 0.05      # area grows with positive amplitudes
    loop = D.DesignLoop(64, 8, W.velocity_grid(4, 4.0), W.Flow(1.0, 0.5), n_params=n, v_min=0.08,
                        max_iter=50, bound=0.01)
    loop.feasible_mesh = lambda a: True
    loop.constrain(0.0, q)                      # Q(alpha) = q . alpha <= 0

    def evaluate(a):
        Cd = 0.5 + 0.5 * (a - c) @ A @ (a - c)
        return D.Evaluation(a, Cd, A @ (a - c), q @ a, q.copy())
    D.drive(loop, evaluate)
    assert loop.stopped == "criterion_opt"
    assert all(e.Q <= 1e-15 for e in loop.history)          # every evaluated design is feasible
    acc = [loop.history[0]]
    for e in loop.history[1:]:
        if e.Cd < acc[-1].Cd:
            acc.append(e)
    assert len(acc) >= 3 and loop.best.Cd < loop.history[0].Cd
    # the constrained minimiser: min 1/2 (a-c)^T A (a-c) s.t. q.a <= 0, |a| <= 0.01 (inactive box)
    lam = max(0.0, (q @ c) / (q @ np.linalg.solve(A, q)))
    a_star = c - lam * np.linalg.solve(A, q)
    assert np.abs(loop.best.alpha - a_star).max() < 2e-4


# ----------------------------------------------------------------------------- CST (Sec. 3.3)
def test_cst_tangents_match_central_differences():
    rng = np.random.default_rng(12)
    q = W.cst_naca(48, 4)
    q[2:] += rng.uniform(-0.01, 0.01, q.size - 2) * np.r_[np.ones(10), 0, 0]
    q[-2:] = [0.002, -0.001]
    _, d = W.cst_wall_nodes(48, q, 4)
    h = 1e-6
    for p in range(q.size):
        e = np.zeros(q.size)
        e[p] = h
        fd = (W.cst_wall_nodes(48, q + e, 4)[0] - W.cst_wall_nodes(48, q - e, 4)[0]) / (2 * h)
        np.testing.assert_allclose(d[p], fd, atol=1e-8)


def test_cst_closed_form_and_least_squares_recovery():
    """N_B = 0 with N1 = 1/2, N2 = 1: eta_u = A sqrt(xi) (1 - xi) + xi eta_T; and the fit of
    Eq. (cstini) recovers the nodes of a CST section to round-off."""
    ni = 40
    xw, _ = W.cst_wall_nodes(ni, [0.5, 1.0, 0.2, -0.1, 0.003, -0.002], 0)
    xi = xw[:, 0]
    up = np.sign(np.round(np.sin(2 * np.pi * np.arange(ni) / ni), 14)) > 0
    np.testing.assert_allclose(xw[up, 1], 0.2 * np.sqrt(xi[up]) * (1 - xi[up]) + 0.003 * xi[up], atol=1e-15)
    q = W.cst_naca(64, 6)
    q[0], q[1] = 0.52, 0.95
    q[2:9] *= 1.05
    target = W.cst_wall_nodes(64, q, 6)[0][:, 1]
    fit = W.cst_fit(64, target, 6)
    assert np.abs(W.cst_wall_nodes(64, fit, 6)[0][:, 1] - target).max() < 1e-10


def test_cst_fits_the_base_section():
    for ni in (64, 256):
        xw, _ = W.cst_wall_nodes(ni, W.cst_naca(ni))
        assert np.abs(xw[:, 1] - W.wall_nodes(ni, np.zeros(0))[0][:, 1]).max() < 1e-4
