"""The conservative discrete Maxwellian (dvm_state_set_maxwellian) through the library against the
oracle with the same fit: one primal and one adjoint sweep, converged drag and full-discrete
sensitivities, the combination with the second-order reconstruction, and the argument checks."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.second_order import SecondOrder
from paper_2501_00923_gb300 import build, dvm
from paper_2501_00923_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = dvm.Context(0)
    yield c
    c.close()


def _case(ctx, ni, nj, nvx, nvy, Kn, Ma, storage, seed, bumps=True):
    rng = np.random.default_rng(seed)
    mesh = W.omesh(ni, nj, rng.uniform(-0.01, 0.01, 4) if bumps else np.zeros(0))
    grid = W.velocity_grid(nvx, 4.0, ny=nvy)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st = dvm.State(ctx, m, g, Kn, Ma, storage=storage)
    st.maxwellian = "conservative"
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma, conservative=True)
    return rng, mesh, grid, m, g, st, pr


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("bf16", 2e-2)])
@pytest.mark.parametrize("shape", [(24, 6, 11, 9), (16, 6, 33, 31), (3, 1, 8, 8)])
def test_one_conservative_primal_sweep_matches_oracle(ctx, storage, tol, shape):
    """A ragged velocity count, a count that refills the pipeline stages, and the one-layer mesh;
    the 8-point grids are coarse enough that the fit differs visibly from the plain Maxwellian."""
    ni, nj, nvx, nvy = shape
    rng, mesh, grid, m, g, st, pr = _case(ctx, ni, nj, nvx, nvy, 0.3, 0.9, storage, 600 + ni, bumps=ni > 3)
    assert st.maxwellian == "conservative"
    st.set(W.random_state(pr.ncell, grid, rng))
    f_in = st.get()
    ref, _ = pr.jacobi(f_in)
    st.iterate(1)
    out = st.get()
    scale = np.abs(ref).max(axis=(1, 2))[:, None, None]
    assert (np.abs(out - ref) / scale).max() < tol
    plain = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, 0.3, 0.9).jacobi(f_in)[0]
    if storage == "fp64":
        assert np.abs(plain - ref).max() > 1e3 * tol * np.abs(ref).max()


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-11), ("fp32", 1e-5), ("bf16", 2e-2)])
def test_one_conservative_adjoint_sweep_matches_oracle(ctx, storage, tol):
    rng, mesh, grid, m, g, st, pr = _case(ctx, 36, 10, 12, 10, 0.5, 0.7, storage, 7)
    st.set(W.random_state(pr.ncell, grid, rng))
    f_in = st.get()
    ad = dvm.Adjoint(st)
    phi = W.random_adjoint(pr.ncell, grid.nv, rng)
    ad.set(phi)
    phi_in = ad.get()
    ref, _ = pr.adjoint_jacobi(f_in, phi_in)
    ad.iterate(1)
    assert np.abs(ad.get() - ref).max() < tol * np.abs(ref).max()
    ad.close()


def test_conservative_converged_drag_and_sensitivities(ctx):
    """FP64 solves to round-off on a coarse velocity grid: drag and both sensitivity modes against
    the oracle with the fitted Maxwellian on the same states; the plain drag differs."""
    rng, mesh, grid, m, g, st, pr = _case(ctx, 32, 12, 8, 8, 1.0, 0.6, "fp64", 3)
    _, res = dvm.primal_solve(ctx, m, g, 1.0, 0.6, tol=1e-13, max_iter=200000, storage="fp64", state=st)
    assert res.status == dvm.DVM_OK
    f_ref, _ = pr.primal_solve(tol=1e-14, max_sweeps=20000)
    J_ref = pr.functional(f_ref)
    assert abs(res.J - J_ref) < 1e-10 * abs(J_ref)
    plain = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, 1.0, 0.6)
    f_pl, _ = plain.primal_solve(tol=1e-14, max_sweeps=20000)
    assert abs(plain.functional(f_pl) - J_ref) > 1e-7 * abs(J_ref)
    ad, ares = dvm.adjoint_solve(ctx, st, tol=1e-13, max_iter=200000)
    assert ares.status == dvm.DVM_OK
    f, phi = st.get(), ad.get()
    full = dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full")
    ref = pr.sens_full(f, phi, mesh.dnodes())
    assert np.abs(full - ref).max() < 1e-9 * np.abs(ref).max()
    paper = dvm.sensitivity(ctx, st, ad, mesh.dwall, mode="paper")
    pref, _, _ = pr.sens_paper(f, phi, mesh.dwall)
    assert np.abs(paper - pref).max() < 1e-9 * np.abs(pref).max()
    ad.close()


def test_conservative_with_second_order(ctx):
    """Both options on one state: one FP64 sweep against the oracle's second-order sweep built on the
    conservative residual."""
    rng, mesh, grid, m, g, st, pr = _case(ctx, 24, 6, 11, 9, 0.3, 0.9, "fp64", 8)
    st.order = 2
    st.set(W.random_state(pr.ncell, grid, rng))
    f_in = st.get()
    ref = SecondOrder(pr).jacobi(f_in)
    st.iterate(1)
    assert np.abs(st.get() - ref).max() < 1e-12 * np.abs(ref).max()


def test_maxwellian_arguments(ctx):
    rng, mesh, grid, m, g, st, pr = _case(ctx, 8, 3, 4, 4, 1.0, 0.5, "fp32", 1)
    with pytest.raises(KeyError):
        st.maxwellian = "other"
    assert dvm.lib().dvm_state_set_maxwellian(st.h, 2) == dvm.DVM_ERR_INVALID_ARG
    st.maxwellian = "plain"
    assert st.maxwellian == "plain"
    st.set(W.random_state(pr.ncell, grid, rng))
    f_in = st.get()
    ref, _ = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, 1.0, 0.5).jacobi(f_in)
    st.iterate(1)
    scale = np.abs(ref).max(axis=(1, 2))[:, None, None]
    assert (np.abs(st.get() - ref) / scale).max() < 2e-6
