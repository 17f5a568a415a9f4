"""Pins of the oracle's second-order reconstruction (oracle/second_order.py): its first-order face
logic against the C++ oracle's residual, second-order accuracy of the reconstructed face values on
refined meshes, the affine structure of dR, and the exact discrete adjoint of the second-order
residual through a source perturbation."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.second_order import SecondOrder
from paper_2501_00923_gb300 import workloads as W


def _so(ni, nj, nv, Kn=1.0, Ma=0.5, alpha=None, **mesh_kw):
    alpha = np.array([0.004, -0.003, 0.002, 0.001]) if alpha is None else alpha
    mesh = W.omesh(ni, nj, alpha, **mesh_kw)
    g = W.velocity_grid(nv, 4.0)
    pr = O.Problem(mesh.nodes, g.vx, g.vy, g.w, Kn, Ma)
    return mesh, g, pr, SecondOrder(pr)


def test_first_order_face_values_reproduce_the_oracle_residual():
    """sum_e a_e F1_e + V/tau (f - g) from the numpy face logic equals the C++ first-order residual:
    the second-order terms are added to the same interface values the pinned oracle uses."""
    mesh, g, pr, so = _so(12, 5, 8)
    f = W.random_state(pr.ncell, g, np.random.default_rng(1))
    R1, _ = pr.residual(f)
    Wm = pr.moments(f)
    rho = Wm[:, 0]
    u = Wm[:, 1:3] / rho[:, None]
    T = (2.0 / 3.0) * (Wm[:, 3] / rho - 0.5 * (u ** 2).sum(1))
    tau = (5.0 / 16.0) * pr.Kn * np.sqrt(2 * np.pi) / (rho * np.sqrt(T))
    far, wall = so._boundary_values(f)
    tr = np.zeros_like(f)
    for e in range(4):
        F1, _ = so.face_values(f, e)
        inside = (so.nb[:, e] >= 0)[:, None, None]
        if e == 1:
            F1 = np.where(inside, F1, far)
        if e == 3:
            F1 = np.where(inside, F1, wall)
        tr += so.a[:, e, :, None] * F1
    assert np.abs(tr - (so.V / tau)[:, None, None] * pr.collision(f) - R1).max() < 1e-13 * np.abs(R1).max()


def test_reconstruction_is_second_order_on_refined_meshes():
    """A smooth field sampled at the cell centres: the reconstructed interior face values converge to
    the field at the face midpoints at second order (error ratio approaching 4 per halving of the
    spacing: 3.1, 3.5, ... on these meshes), the first-order (upwind cell) values at first order
    (~2).  Cells of the two boundary rows and their neighbours are left out: their gradients see the
    boundary values."""
    def field(x):
        return np.sin(1.3 * x[..., 0]) * np.cos(0.9 * x[..., 1]) + 0.4 * x[..., 0]

    e1, e2 = [], []
    for ni, nj in [(32, 8), (64, 16), (128, 32), (256, 64)]:
        mesh, g, pr, so = _so(ni, nj, 4, alpha=np.zeros(4), first=1.0, radius=1.5)
        fc = field(so.xc)
        f = np.repeat(fc[:, None, None], pr.nv * 2, 1).reshape(pr.fshape())
        keep = ((np.arange(pr.ncell) // ni) >= 2) & ((np.arange(pr.ncell) // ni) <= nj - 3)
        m1 = m2 = 0.0
        for e in range(4):
            F1, F2 = so.face_values(f, e)
            exact = field(so.xe[:, e])[:, None, None]
            m1 = max(m1, np.abs(F1 - exact)[keep].max())
            m2 = max(m2, np.abs(F2 - exact)[keep].max())
        e1.append(m1)
        e2.append(m2)
    r1 = [e1[k] / e1[k + 1] for k in range(3)]
    r2 = [e2[k] / e2[k + 1] for k in range(3)]
    assert all(1.6 < r < 2.6 for r in r1), r1
    assert all(r > 2.9 for r in r2) and r2[-1] > 3.6, r2
    assert e2[-1] < 0.1 * e1[-1]


def test_delta_r_is_affine_in_f():
    mesh, g, pr, so = _so(8, 4, 6)
    rng = np.random.default_rng(2)
    L, b = so.matrix()
    f = W.random_state(pr.ncell, g, rng)
    h = rng.normal(size=f.shape)
    ref = so.delta_r(f).ravel() + 0.7 * (L @ h.ravel())
    assert np.abs(so.delta_r(f + 0.7 * h).ravel() - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs((L @ f.ravel() + b) - so.delta_r(f).ravel()).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.slow
def test_second_order_adjoint_is_exact_through_a_source():
    """With R2(f) + eps s = 0, dJ/deps = sum w phi . s for the second-order adjoint phi
    ((dR2/df)^T (w phi) = -dJ/df): central differences in eps of the second-order steady drag, both
    solves to round-off, against the adjoint prediction."""
    mesh, g, pr, so = _so(8, 4, 8)
    f, it = so.solve(tol=1e-15, max_sweeps=8000)
    assert it < 8000
    phi, ait = so.adjoint_solve(f, tol=1e-15, max_sweeps=8000)
    assert ait < 8000
    rng = np.random.default_rng(3)
    s = rng.normal(size=f.shape) * 1e-2 * np.abs(f).max()
    pred = float(np.sum(g.w[None, :, None] * phi * s))
    eps = 1e-4
    Jp = pr.functional(so.solve(f0=f, source=eps * s, tol=1e-15, max_sweeps=8000)[0])
    Jm = pr.functional(so.solve(f0=f, source=-eps * s, tol=1e-15, max_sweeps=8000)[0])
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - pred) < 1e-7 * abs(pred)


def test_frozen_defect_groups_reach_the_same_fixed_point():
    """Sweeps with dR recomputed every sweep (where that converges) and with dR frozen over groups of
    4 sweeps end at the same second-order steady state, R1 + dR = 0."""
    mesh, g, pr, so = _so(8, 4, 6)
    f1, it1 = so.solve(tol=1e-14, max_sweeps=8000, period=1)
    f4, it4 = so.solve(tol=1e-14, max_sweeps=8000, period=4)
    assert it1 < 8000 and it4 < 8000
    assert np.abs(f1 - f4).max() < 1e-11 * np.abs(f1).max()
    R = so.residual(f4)
    assert np.abs(R).max() < 1e-10 * np.abs(so.a).max() * np.abs(f4).max()


def test_probed_transpose_at_interior_cells_equals_the_assembled_one():
    """The large-problem form of the transposed defect (one probe per component of each listed cell,
    valid three or more rows from the wall) against the transpose assembled column by column."""
    mesh, g, pr, so = _so(10, 9, 4, Kn=0.3, Ma=0.9)
    rng = np.random.default_rng(4)
    phi = W.random_adjoint(pr.ncell, g.nv, rng)
    L, _ = so.matrix()
    E = so.adjoint_defect(phi, L)
    cells = np.array([30, 35, 44, 51, 59, 79])
    assert np.abs(so.adjoint_defect_cells(phi, cells) - E[cells]).max() < 1e-13 * np.abs(E).max()
    with pytest.raises(ValueError):
        so.adjoint_defect_cells(phi, np.array([5]))


def test_geometry_of_reproduces_the_oracle_geometry():
    mesh, g, pr, so = _so(10, 5, 4)
    S, V, xc, xe = so.geometry_of(mesh.nodes)
    assert np.abs(S - so.S).max() < 1e-15 * np.abs(so.S).max()
    assert np.abs(V - so.V).max() < 1e-15 * np.abs(so.V).max()
    assert np.abs(xc - so.xc).max() == 0.0 and np.abs(xe - so.xe).max() == 0.0


@pytest.mark.slow
def test_second_order_full_gradient_matches_central_differences():
    """dJ/dalpha of the second-order discrete problem (the first-order full sensitivity with the
    second-order adjoint, plus sum w phi . d(dR)/dalpha by a complex step in the nodes) against central
    differences of two second-order solves per bump amplitude (step 1e-5), all solves to round-off."""
    alpha = np.array([0.004, -0.003, 0.002, 0.001])
    mesh, g, pr, so = _so(8, 4, 6, alpha=alpha)
    f, it = so.solve(tol=1e-15, max_sweeps=20000)
    assert it < 20000
    phi, ait = so.adjoint_solve(f, tol=1e-15, max_sweeps=20000)
    assert ait < 20000
    grad = so.sens_full(f, phi, mesh.dnodes())
    h = 1e-5
    for p in range(alpha.size):
        J = []
        for s in (1, -1):
            a = alpha.copy()
            a[p] += s * h
            _, _, pp, sp = _so(8, 4, 6, alpha=a)
            fp, _ = sp.solve(f0=f, tol=1e-15, max_sweeps=20000)
            J.append(pp.functional(fp))
        fd = (J[0] - J[1]) / (2 * h)
        assert abs(fd - grad[p]) <= 1e-6 * np.abs(grad).max(), (p, fd, grad[p])
    # the second-order term matters: the first-order formula with the same phi differs
    g1 = pr.sens_full(f, phi, mesh.dnodes())
    assert np.abs(g1 - grad).max() > 1e-4 * np.abs(grad).max()
