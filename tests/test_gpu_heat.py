"""The heat functional (Eq. formula_opt with m_J = |v|^2/2) through the library: its value, its
discrete adjoint and both boundary sensitivities against the oracle on the same converged state
(the oracle's heat functional is pinned by the free-molecular closed form and by central
differences)."""
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


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-9), ("fp32", 2e-4)])
def test_heat_adjoint_and_sensitivities_match_the_oracle(ctx, storage, tol):
    rng = np.random.default_rng(31)
    mesh = W.omesh(24, 8, rng.uniform(-0.01, 0.01, 4))
    grid = W.velocity_grid(10, 4.0)
    Kn, Ma, Tw = 1.0, 0.5, 1.5              # a wall hotter than the gas: the heat is not zero
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st, _ = dvm.primal_solve(ctx, m, g, Kn, Ma, Tw=Tw, tol=1e-13 if storage == "fp64" else 1e-7,
                             max_iter=200000, storage=storage, stall_window=0 if storage == "fp64" else 5000)
    f = st.get()
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma, Tw=Tw, direction=(0.0, 0.0, 1.0))
    Jh = st.functional("heat")
    # the library integrates with the wall density F_rhow of the last sweep (FP32-accumulated in
    # FP32 storage); the oracle recomputes it from f in FP64
    jtol = 1e-12 if storage == "fp64" else 1e-6
    assert abs(Jh - pr.functional(f)) < jtol * abs(Jh)
    assert abs(Jh) > 1e-3
    ad, _ = dvm.adjoint_solve(ctx, st, functional="heat", tol=1e-13 if storage == "fp64" else 1e-7,
                              max_iter=200000, stall_window=0 if storage == "fp64" else 5000)
    phi = ad.get()
    phi_ref, _ = pr.adjoint_solve(f, tol=1e-30, max_sweeps=6000)
    assert np.abs(phi - phi_ref).max() < tol * np.abs(phi_ref).max()
    gf = dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full")
    gp = dvm.sensitivity(ctx, st, ad, mesh.dwall, mode="paper")
    ref_f = pr.sens_full(f, phi_ref, mesh.dnodes())
    ref_p = pr.sens_paper(f, phi_ref, mesh.dwall)[0]
    assert np.abs(gf - ref_f).max() < tol * np.abs(ref_f).max()
    assert np.abs(gp - ref_p).max() < tol * np.abs(ref_p).max()
    for h in (ad, st, g, m):
        h.close()
