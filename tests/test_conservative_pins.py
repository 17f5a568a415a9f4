"""Pins of the oracle's conservative discrete Maxwellian (no GPU): the cell Maxwellian whose discrete
moments equal the cell's, found by Newton's method (the conservative schemes the paper builds on,
Sec. 2.3).  Conservation on any velocity grid, agreement with the plain Maxwellian where the
quadrature is exact, stationarity of a sampled Maxwellian, and the adjoint identities of the
resulting residual (the implicit derivative of the fit carried by dual numbers)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_00923_gb300 import workloads as W


def _problem(mesh, grid, conservative, Kn=1.0, Ma=0.5):
    return O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma, conservative=conservative)


def _moment_defect(grid, Q):
    """sum_k w_k Psi_k Q_k per cell, Psi = (1, vx, vy, |v|^2/2) on f1 and (0, 0, 0, 1) on f2."""
    psi1 = np.stack([np.ones(grid.nv), grid.vx, grid.vy, 0.5 * (grid.vx ** 2 + grid.vy ** 2)])
    return (np.einsum("k,ck,mk->cm", grid.w, Q[:, :, 0], psi1)
            + np.einsum("k,ck->c", grid.w, Q[:, :, 1])[:, None] * np.array([0, 0, 0, 1.0]))


def test_conservative_maxwellian_conserves_on_a_coarse_grid():
    """On a coarse, narrow grid the plain Maxwellian's discrete moments miss the cell's (the guard
    shows the defect); the fitted one matches them to round-off."""
    grid = W.velocity_grid(8, 4.0)
    mesh = W.omesh(8, 4)
    rng = np.random.default_rng(11)
    f = W.random_state(mesh.ni * mesh.nj, grid, rng, noise=0.2)
    scale = np.abs(_problem(mesh, grid, False).moments(f)).max()
    d_plain = _moment_defect(grid, _problem(mesh, grid, False).collision(f))
    d_cons = _moment_defect(grid, _problem(mesh, grid, True).collision(f))
    assert np.abs(d_plain).max() > 1e-6 * scale
    assert np.abs(d_cons).max() < 1e-13 * scale


def test_conservative_equals_plain_where_the_quadrature_is_exact():
    grid = W.velocity_grid(64, 10.0 / W.A_INF)
    mesh = W.omesh(8, 4)
    rng = np.random.default_rng(12)
    f = W.random_state(mesh.ni * mesh.nj, grid, rng, noise=0.2)
    Qp = _problem(mesh, grid, False).collision(f)
    Qc = _problem(mesh, grid, True).collision(f)
    assert np.abs(Qp - Qc).max() < 1e-11 * np.abs(Qp).max()


def test_sampled_maxwellian_is_stationary_only_with_the_fit():
    """f = the Maxwellian (rho, u, T) sampled on a coarse grid: its discrete moments are not
    (rho, rho u, ...), so the plain collision term does not vanish, while the fit recovers the
    sampled parameters and the collision term is zero."""
    grid = W.velocity_grid(8, 4.0)
    mesh = W.omesh(8, 4)
    rho, u1, u2, T = 1.3, 0.4, -0.2, 0.8
    c2 = (grid.vx - u1) ** 2 + (grid.vy - u2) ** 2
    g1 = rho / (2 * np.pi * T) * np.exp(-c2 / (2 * T))
    f = np.broadcast_to(np.stack([g1, 0.5 * T * g1], 1), (mesh.ni * mesh.nj, grid.nv, 2)).copy()
    assert np.abs(_problem(mesh, grid, False).collision(f)).max() > 1e-6 * g1.max()
    assert np.abs(_problem(mesh, grid, True).collision(f)).max() < 1e-13 * g1.max()


@pytest.fixture(scope="module")
def tiny_c():
    rng = np.random.default_rng(6)
    mesh = W.omesh(16, 8, rng.uniform(-0.01, 0.01, 4))
    grid = W.velocity_grid(8, 4.0)
    pr = _problem(mesh, grid, True, Kn=1.0, Ma=0.5)
    f, info = pr.primal_solve(tol=1e-30, max_sweeps=2400)
    phi, ainfo = pr.adjoint_solve(f, tol=1e-30, max_sweeps=2400)
    return mesh, grid, pr, f, phi


def test_conservative_transpose_matches_forward_mode(tiny_c):
    """<lam, (dR/df) df> = <(dR/df)^T lam, df> with the fitted Maxwellian: the transpose built
    from the collision partials against dual numbers of the residual."""
    mesh, grid, pr, f, phi = tiny_c
    rng = np.random.default_rng(7)
    fr = W.random_state(pr.ncell, grid, rng)
    for _ in range(3):
        df = rng.standard_normal(fr.shape)
        lam = rng.standard_normal(fr.shape)
        _, dR = pr.residual_dir(fr, df)
        assert abs(np.sum(lam * dR) - np.sum(pr.apply_RT(fr, lam) * df)) < 1e-12 * np.sum(np.abs(lam * dR))


def test_fit_derivative_matches_finite_differences(tiny_c):
    """The implicit derivative of the fit, carried by the duals of the residual, against central
    differences of the residual itself (step 1e-6)."""
    mesh, grid, pr, f, phi = tiny_c
    rng = np.random.default_rng(9)
    df = rng.standard_normal(f.shape) * np.abs(f)
    _, dR = pr.residual_dir(f, df)
    h = 1e-6
    fd = (pr.residual(f + h * df)[0] - pr.residual(f - h * df)[0]) / (2 * h)
    assert np.abs(fd - dR).max() < 1e-7 * np.abs(dR).max()


def test_conservative_dual_consistency_and_gradient(tiny_c):
    """<w phi, (dR/df) df> = -(dJ/df) df for the converged conservative adjoint, and dJ/dalpha
    against central differences of two conservative solves (step 1e-5)."""
    mesh, grid, pr, f, phi = tiny_c
    rng = np.random.default_rng(8)
    for _ in range(2):
        df = rng.standard_normal(f.shape)
        _, dR = pr.residual_dir(f, df)
        _, dJ = pr.functional_dir(f, df)
        assert abs(np.sum(grid.w[None, :, None] * phi * dR) + dJ) < 1e-12 * abs(dJ)
    g_adj = pr.sens_full(f, phi, mesh.dnodes())
    h = 1e-5
    for p in range(mesh.alpha.size):
        vals = []
        for s in (1, -1):
            a = mesh.alpha.copy()
            a[p] += s * h
            pp = _problem(W.omesh(16, 8, a), grid, True, Kn=1.0, Ma=0.5)
            ff, info = pp.primal_solve(tol=1e-30, max_sweeps=1200, f0=f)
            vals.append(pp.functional(ff))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g_adj[p]) <= 1e-6 * abs(g_adj[p])
    # the fit changes the answer on this coarse grid
    pl = _problem(mesh, grid, False, Kn=1.0, Ma=0.5)
    f1, _ = pl.primal_solve(tol=1e-30, max_sweeps=2400)
    assert abs(pl.functional(f1) - pr.functional(f)) > 1e-8 * abs(pr.functional(f))
