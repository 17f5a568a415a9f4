"""Host logic of the design loop: the L-BFGS step, its line search and bounds, the stopping rule of
Eq. (criterion_opt) and the constraint penalty, all on analytic objectives (no GPU)."""
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


def test_penalty_gradient_matches_finite_differences():
    loop = D.DesignLoop(16, 4, W.velocity_grid(4, 4.0), W.Flow(1.0, 0.5), n_params=3, v_min=0.08, mu=50.0)
    rng = np.random.default_rng(7)
    dCd, dQ = rng.normal(size=3), rng.normal(size=3)
    a0 = rng.normal(size=3) * 0.01

    def phi(a):
        Cd = 0.3 + dCd @ a
        Q = 0.001 + dQ @ a                  # violated: the penalty is active
        return loop.penalty(Cd, dCd, Q, dQ)
    _, g = phi(a0)
    h = 1e-6
    fd = np.array([(phi(a0 + h * e)[0] - phi(a0 - h * e)[0]) / (2 * h) for e in np.eye(3)])
    np.testing.assert_allclose(g, fd, rtol=1e-7)
    assert phi(a0 - 10 * dQ)[0] == pytest.approx(0.3 + dCd @ (a0 - 10 * dQ))   # satisfied: no penalty


def test_design_loop_stops_by_criterion_opt_on_an_analytic_problem():
    """Drag-like convex objective with the volume constraint: the loop decreases the merit
    monotonically over accepted steps and stops by Eq. (criterion_opt) before max_iter."""
    n = 6
    rng = np.random.default_rng(8)
    A = np.diag(np.linspace(20.0, 60.0, n))
    c = rng.uniform(-0.004, 0.004, n)
    q = -np.abs(rng.normal(size=n)) * 0.05      # area grows with positive amplitudes
    loop = D.DesignLoop(64, 8, W.velocity_grid(4, 4.0), W.Flow(1.0, 0.5), n_params=n, v_min=0.08,
                        mu=1e4, max_iter=50, bound=0.01)
    loop.feasible_mesh = lambda a: True

    def evaluate(a):
        Cd = 0.5 + 0.5 * (a - c) @ A @ (a - c)
        dCd = A @ (a - c)
        Q = q @ a
        return D.Evaluation(a, Cd, dCd, Q, q.copy(), *loop.penalty(Cd, dCd, Q, q))
    D.drive(loop, evaluate)
    assert loop.stopped == "criterion_opt"
    acc = [loop.history[0]]
    for e in loop.history[1:]:
        if e.phi < acc[-1].phi:
            acc.append(e)
    assert all(b.phi < a.phi for a, b in zip(acc, acc[1:]))
    assert loop.best.Cd < loop.history[0].Cd
