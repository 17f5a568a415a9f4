"""Second-order reconstruction (Eq. gaussgrad) through the library against the oracle's
SecondOrder: one primal sweep (deferred correction with the first-order diagonal), one adjoint
sweep with the exact transpose of dR (element by element on small cases where the oracle assembles
the transpose, by the duality sum lambda . dR(h) = sum h . dR^T(lambda) on larger ones), converged
second-order solves, and the argument checks of dvm_state_set_order."""
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


def _case(ctx, ni, nj, nvx, nvy, Kn, Ma, storage, seed):
    rng = np.random.default_rng(seed)
    mesh = W.omesh(ni, nj, rng.uniform(-0.01, 0.01, 4)) if ni > 3 else W.omesh(ni, nj, np.zeros(0))
    grid = W.velocity_grid(nvx, 4.0, ny=nvy)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st = dvm.State(ctx, m, g, Kn, Ma, storage=storage)
    st.order = 2
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma)
    return rng, mesh, grid, m, g, st, pr, SecondOrder(pr)


def _norm(pr, R):
    """|R| = sqrt(sum_{c,k,comp} w_k (R / V_c)^2), the sweeps' residual norm."""
    V, _ = pr.geometry()
    return float(np.sqrt(np.sum(pr.w[None, :, None] * (R / V[:, None, None]) ** 2)))


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp32", 3e-6), ("bf16", 2e-2)])
@pytest.mark.parametrize("shape", [(40, 12, 12, 12), (24, 6, 11, 9), (3, 1, 8, 8), (16, 6, 33, 31)])
def test_one_second_order_primal_sweep_matches_oracle(ctx, storage, tol, shape):
    """The same shapes as the first-order sweep test: several warps of cells, a ragged velocity
    count, the one-layer mesh whose cells touch the wall and the far field, and a velocity count
    that refills the pipeline stages."""
    ni, nj, nvx, nvy = shape
    rng, mesh, grid, m, g, st, pr, so = _case(ctx, ni, nj, nvx, nvy, 0.3, 0.9, storage, 200 + ni)
    assert st.order == 2
    f = W.random_state(pr.ncell, grid, rng)
    st.set(f)
    f_in = st.get()
    ref = so.jacobi(f_in)
    res = st.iterate(1)
    fn = st.get()
    cell_scale = np.abs(ref).max(axis=(1, 2))[:, None, None]
    assert (np.abs(fn - ref) / cell_scale).max() < tol
    # the defect moved the update (by 1.4% of the largest value on the one-layer mesh, 24-37% on the
    # others): where that exceeds the storage tolerance, check that it is not zero
    fn1, _ = pr.jacobi(f_in)
    if storage != "bf16":
        assert np.abs(fn1 - ref).max() > 5 * tol * np.abs(ref).max()
    # residual monitor of the second-order residual R1 + dR
    R1, n1 = pr.residual(f_in)
    assert abs(_norm(pr, R1) - n1) < 1e-12 * n1
    _, r0 = pr.residual(pr.freestream())
    nrm = _norm(pr, so.residual(f_in))
    rtol = {"fp64": 1e-9, "fp32": 1e-3, "bf16": 0.1}[storage]
    assert abs(res[0] - nrm / r0) < rtol * (nrm / r0)
    # the moments carried to the next sweep are those of the new state
    prim = st.moments()
    W_ref = pr.moments(fn if storage != "fp64" else ref)
    assert np.abs(prim[:, 0] - W_ref[:, 0]).max() < max(tol, 1e-13) * 10


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-11), ("fp32", 5e-6), ("bf16", 2e-2)])
@pytest.mark.parametrize("shape", [(8, 3, 4, 4), (5, 2, 6, 5), (3, 1, 4, 4)])
def test_one_second_order_adjoint_sweep_matches_oracle(ctx, storage, tol, shape):
    """Element by element against the oracle's assembled transpose (small cases: the oracle builds
    dR's matrix column by column)."""
    ni, nj, nvx, nvy = shape
    rng, mesh, grid, m, g, st, pr, so = _case(ctx, ni, nj, nvx, nvy, 0.5, 0.7, storage, 300 + ni)
    f = W.random_state(pr.ncell, grid, rng)
    st.set(f)
    f_in = st.get()
    L, _ = so.matrix()
    ad = dvm.Adjoint(st)
    phi = W.random_adjoint(pr.ncell, grid.nv, rng)
    ad.set(phi)
    phi_in = ad.get()
    ref = so.adjoint_jacobi(f_in, phi_in, L)
    ad.iterate(1)
    out = ad.get()
    assert np.abs(out - ref).max() < tol * np.abs(ref).max()
    ref1, _ = pr.adjoint_jacobi(f_in, phi_in)
    if storage != "bf16":
        assert np.abs(ref1 - ref).max() > 5 * tol * np.abs(ref).max()
    ad.close()


@pytest.mark.parametrize("period", [4, 3])
def test_defect_is_frozen_over_groups_of_sweeps(ctx, period):
    """Nine FP64 sweeps from an uploaded state: the defect is taken at sweeps 1, 1 + period, ...
    and held in between, primal and adjoint alike, as the oracle's frozen-defect iteration."""
    rng, mesh, grid, m, g, st, pr, so = _case(ctx, 8, 4, 6, 6, 1.0, 0.5, "fp64", 500 + period)
    st.set_order(2, period)
    # a perturbed free stream: from a far-from-equilibrium random state the unlimited reconstruction
    # drives f negative within a few sweeps (in the oracle too)
    f0 = pr.freestream()
    st.set(f0 * (1 + 0.2 * rng.uniform(-1, 1, f0.shape)))
    fr = st.get()
    st.iterate(9)
    for it in range(9):
        if it % period == 0:
            dR = so.delta_r(fr)
        fr = so.jacobi(fr, defect=dR)
    out = st.get()
    assert np.abs(out - fr).max() < 1e-11 * np.abs(fr).max()
    L, _ = so.matrix()
    ad = dvm.Adjoint(st)
    phi = W.random_adjoint(pr.ncell, grid.nv, rng)
    ad.set(phi)
    pr_ = ad.get()
    ad.iterate(9)
    for it in range(9):
        if it % period == 0:
            E = so.adjoint_defect(pr_, L)
        pr_ = so.adjoint_jacobi(out, pr_, defect=E)
    assert np.abs(ad.get() - pr_).max() < 1e-10 * np.abs(pr_).max()
    ad.close()


@pytest.mark.parametrize("shape", [(40, 12, 12, 12), (16, 6, 33, 31)])
def test_second_order_adjoint_defect_is_the_transpose(ctx, shape):
    """Larger cases, FP64: the adjoint sweep's defect E = dR^T(w phi) / w, read back from the sweep as
    E = D (phi1 - phi2) (phi1 the oracle's first-order sweep, phi2 the library's second-order one),
    satisfies sum_{c,k} w E . h = sum (w phi) . (dR(h) - dR(0)) for random h: the duality that
    defines the transpose, with dR from the oracle."""
    ni, nj, nvx, nvy = shape
    rng, mesh, grid, m, g, st, pr, so = _case(ctx, ni, nj, nvx, nvy, 0.5, 0.7, "fp64", 400 + ni)
    f = W.random_state(pr.ncell, grid, rng)
    st.set(f)
    f_in = st.get()
    ad = dvm.Adjoint(st)
    phi = W.random_adjoint(pr.ncell, grid.nv, rng)
    ad.set(phi)
    phi_in = ad.get()
    ad.iterate(1)
    phi2 = ad.get()
    phi1, _ = pr.adjoint_jacobi(f_in, phi_in)
    D = pr.diagonal(f_in)[..., None]
    E = D * (phi1 - phi2)
    w = pr.w[None, :, None]
    b0 = so.delta_r(np.zeros_like(f_in))
    for _ in range(3):
        h = rng.normal(size=f_in.shape)
        lhs = float(np.sum(w * E * h))
        rhs = float(np.sum(w * phi_in * (so.delta_r(h) - b0)))
        assert abs(lhs - rhs) < 1e-10 * np.sum(np.abs(w * phi_in * (so.delta_r(h) - b0)))
    ad.close()


def test_second_order_steady_state_and_adjoint_match_oracle(ctx):
    """Converged FP64 solves on a small case: the second-order steady state and drag, and the
    second-order adjoint, against the oracle's deferred-correction iterations."""
    rng, mesh, grid, m, g, st, pr, so = _case(ctx, 8, 4, 8, 8, 1.0, 0.5, "fp64", 7)
    st2, res = dvm.primal_solve(ctx, m, g, 1.0, 0.5, tol=1e-13, max_iter=200000, storage="fp64", state=st)
    assert res.status == dvm.DVM_OK
    f_ref, it = so.solve(tol=1e-15, max_sweeps=20000)
    assert it < 20000
    f_gpu = st.get()
    # the library stops on the residual of a group's last sweep, whose defect is up to 19 sweeps old:
    # a looser bound than the residual tolerance alone would give
    assert np.abs(f_gpu - f_ref).max() < 1e-9 * np.abs(f_ref).max()
    J_ref = pr.functional(f_ref)
    assert abs(res.J - J_ref) < 1e-9 * abs(J_ref)
    # the first-order drag differs: the reconstruction changes the answer
    f1, _ = pr.primal_solve(tol=1e-13, max_sweeps=20000)
    assert abs(pr.functional(f1) - J_ref) > 1e-6 * abs(J_ref)
    ad, ares = dvm.adjoint_solve(ctx, st, tol=1e-13, max_iter=200000)
    assert ares.status == dvm.DVM_OK
    phi_ref, ait = so.adjoint_solve(f_gpu, tol=1e-15, max_sweeps=20000)
    assert ait < 20000
    assert np.abs(ad.get() - phi_ref).max() < 1e-9 * np.abs(phi_ref).max()
    # both sensitivity modes: the paper's boundary formula, and the full discrete gradient of the
    # second-order problem (its oracle is pinned by central differences of second-order solves)
    phi_gpu = ad.get()
    grad = dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="paper")
    pref, _, _ = pr.sens_paper(f_gpu, phi_gpu, mesh.dwall)
    assert np.abs(grad - pref).max() < 1e-9 * np.abs(pref).max()
    full = dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full")
    fref = so.sens_full(f_gpu, phi_gpu, mesh.dnodes())
    assert np.abs(full - fref).max() < 1e-9 * np.abs(fref).max()
    with pytest.raises(dvm.DVMError) as e:        # the scratch-free entry point stays first order in FULL
        dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full", noalloc=True)
    assert e.value.status == dvm.DVM_ERR_INVALID_ARG
    ad.close()


def test_fp32_second_order_solve_is_close_to_fp64(ctx):
    rng, mesh, grid, m, g, st64, pr, so = _case(ctx, 32, 12, 12, 12, 0.3, 0.6, "fp64", 9)
    _, r64 = dvm.primal_solve(ctx, m, g, 0.3, 0.6, tol=1e-11, max_iter=200000, storage="fp64", state=st64)
    st32 = dvm.State(ctx, m, g, 0.3, 0.6, storage="fp32")
    st32.order = 2
    _, r32 = dvm.primal_solve(ctx, m, g, 0.3, 0.6, tol=1e-9, max_iter=200000, storage="fp32", state=st32,
                              stall_window=3000)
    assert r64.status == dvm.DVM_OK and r32.status in (dvm.DVM_OK, dvm.DVM_ERR_STAGNATED)
    assert abs(r32.J - r64.J) < 1e-5 * abs(r64.J)


def test_order_arguments(ctx):
    rng, mesh, grid, m, g, st, pr, so = _case(ctx, 8, 3, 4, 4, 1.0, 0.5, "fp32", 1)
    for bad in (0, 3, -1):
        with pytest.raises(dvm.DVMError) as e:
            st.order = bad
        assert e.value.status == dvm.DVM_ERR_INVALID_ARG
    with pytest.raises(dvm.DVMError) as e:
        st.set_order(2, -1)
    assert e.value.status == dvm.DVM_ERR_INVALID_ARG
    assert st.order == 2
    st.order = 1
    assert st.order == 1
    # back at order 1 the sweep is the first-order one again
    st.set(W.random_state(pr.ncell, grid, rng))
    f_in = st.get()
    fn1, _ = pr.jacobi(f_in)
    st.iterate(1)
    assert np.abs(st.get() - fn1).max() < 3e-6 * np.abs(fn1).max()


@pytest.mark.parametrize("index,storage,ptol,atol", [(1, "fp32", 3e-6, 6e-6), (2, "fp32", 3e-6, 6e-6)],
                         ids=["256x128-gl48-fp32", "384x192-v64-Kn0.001-Ma2-fp32"])
def test_full_size_second_order_sweeps_sampled_cells(ctx, index, storage, ptol, atol):
    """The full-size workloads in the benchmark's launch configuration at order 2: one primal sweep
    from a seeded random state on sampled cells (wall row, far-field row, the periodic seam,
    interior) against the oracle's first-order update less dR / D; one adjoint sweep on sampled
    cells three or more rows from the wall against the oracle's first-order adjoint update less the
    probed transposed defect over D."""
    wl = W.config(index)
    rng = np.random.default_rng(22)
    m = dvm.Mesh(ctx, wl.mesh.nodes)
    g = dvm.VGrid(ctx, wl.grid.vx, wl.grid.vy, wl.grid.w)
    st = dvm.State(ctx, m, g, wl.flow.Kn, wl.flow.Ma, storage=storage)
    st.order = 2
    pr = O.Problem.from_workload(wl)
    so = SecondOrder(pr)
    f = W.random_state(pr.ncell, wl.grid, rng)
    st.set(f)
    f_in = st.get()
    ni, nj = wl.mesh.ni, wl.mesh.nj
    cells = np.unique(np.concatenate([[0, ni - 1, ni, (nj - 1) * ni, nj * ni - 1, (nj // 2) * ni + ni // 2],
                                      rng.integers(0, ni, 4), rng.integers(0, ni * nj, 8)]))
    D = pr.diagonal(f_in)
    ref = pr.jacobi_cells(f_in, cells) - so.delta_r(f_in, cells) / D[cells][..., None]
    acells = np.unique(np.concatenate([[3 * ni, 3 * ni + ni - 1, (nj - 1) * ni + 7],
                                       rng.integers(3 * ni, ni * nj, 6)]))
    ad = dvm.Adjoint(st)
    phi = W.random_adjoint(pr.ncell, wl.grid.nv, rng)
    ad.set(phi)
    phi_in = ad.get()
    aref = pr.adjoint_jacobi_cells(f_in, phi_in, acells) - so.adjoint_defect_cells(phi_in, acells) / D[acells][..., None]
    ad.iterate(1)                    # the adjoint is linearised at f_in: sweep it before f moves
    aout = ad.get()[acells]
    ascale = np.abs(aref).max(axis=(1, 2))[:, None, None]
    assert (np.abs(aout - aref) / ascale).max() < atol
    st.iterate(1)
    out = st.get()[cells]
    scale = np.abs(ref).max(axis=(1, 2))[:, None, None]
    assert (np.abs(out - ref) / scale).max() < ptol
    for h in (ad, st, g, m):
        h.close()


@pytest.mark.parametrize("storage,maxwellian,tol", [("fp32", "plain", 1e-4), ("fp32", "conservative", 1e-4),
                                                    ("bf16", "plain", 1e-2)])
def test_second_order_full_sensitivity_in_reduced_storage(ctx, storage, maxwellian, tol):
    """Mode FULL at second order (k_so_sens_cells, k_so_sens_nodes on top of the first-order face and
    volume terms) in FP32 and BF16 storage against the oracle's full discrete gradient of the
    second-order problem, evaluated on the very state and adjoint the GPU holds (their stored values
    read back), after second-order solves in that storage.  16x16 velocities: 128 FP32 chunks (64 BF16)
    per cell, so every lane of a cell's warp sums several chunks.  FP32 must meet the stated 1e-4
    relative per component; BF16 storage changes only the inputs, which the oracle sees too, so it is
    bounded loosely and its error printed.  (On random states and adjoints, instead of solved ones, the
    gradient is a small remainder of large terms of both signs, and FP32 rounding of the terms alone
    moves it by about 1%.)"""
    rng = np.random.default_rng(61)
    mesh = W.omesh(16, 8, rng.uniform(-0.01, 0.01, 4))
    grid = W.velocity_grid(16, 4.0)
    Kn, Ma = 0.4, 0.7
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    st = dvm.State(ctx, m, g, Kn, Ma, storage=storage)
    if maxwellian != "plain":
        st.maxwellian = maxwellian
    opts = dict(tol=1e-7, max_iter=200000, storage=storage, state=st, stall_window=2000)
    dvm.primal_solve(ctx, m, g, Kn, Ma, **opts)          # second order starts from the first-order state
    st.order = 2
    dvm.primal_solve(ctx, m, g, Kn, Ma, **opts)
    ad, _ = dvm.adjoint_solve(ctx, st, tol=1e-7, max_iter=200000, stall_window=2000)
    pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma, conservative=(maxwellian != "plain"))
    so = SecondOrder(pr)
    f_in, phi_in = st.get(), ad.get()
    got = dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full")
    ref = so.sens_full(f_in, phi_in, mesh.dnodes())
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max())
    print(f"order-2 FULL sensitivity, {storage} {maxwellian}: max relative error per component {rel.max():.2e}")
    assert rel.max() < tol
    for h in (ad, st, g, m):
        h.close()
