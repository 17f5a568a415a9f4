"""torch.autograd wrapping of the steady solve: backward = implicit-function adjoint.

The gradient of Cd with respect to the bump amplitudes must match the oracle's full-discrete
sensitivity evaluated on the same converged state, and central finite differences of the forward.
The discrete drag is only piecewise smooth in the shape: the upwind choice of a face flips when
v_k . n_f changes sign as the face turns, so a difference step that straddles such a flip carries
an error of its own.  On this case one of the six components does at step 1e-4 (5.7e-5 of the
largest component) and none does at 1e-5, where the differences agree with the adjoint to 1e-6."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2501_00923_gb300 import build, dvm
from paper_2501_00923_gb300 import workloads as W
from paper_2501_00923_gb300.autograd import DragProblem, drag

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = dvm.Context(0)
    yield c
    c.close()


def _problem(ctx, storage, tol):
    return DragProblem(ctx, 48, 16, W.velocity_grid(12, 4.0), W.Flow(1.0, 0.6), storage=storage, tol=tol,
                       adjoint_tol=tol, max_iter=400000, stall_window=20000 if storage != "fp64" else 0)


def _fd(prob, a0, h=1e-4):
    g = np.zeros_like(a0)
    for p in range(a0.size):
        e = np.zeros_like(a0)
        e[p] = h
        g[p] = (prob.solve(a0 + e) - prob.solve(a0 - e)) / (2 * h)
    return g


def test_drag_gradient_matches_central_differences_and_the_oracle(ctx):
    rng = np.random.default_rng(41)
    a0 = rng.uniform(-0.005, 0.005, 6)
    prob = _problem(ctx, "fp64", 1e-12)
    alpha = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    cd = drag(alpha, prob)
    cd.backward()
    g_adj = alpha.grad.numpy().copy()
    # oracle full-discrete sensitivity on the very same state and adjoint
    mesh = prob.last["mesh"]
    pr = O.Problem(mesh.nodes, prob.grid.vx, prob.grid.vy, prob.grid.w, prob.flow.Kn, prob.flow.Ma)
    f = prob._warm[1].get()
    phi = prob._warm[2].get()
    g_orc = pr.sens_full(f, phi, mesh.dnodes()) / prob.q_ref
    assert np.abs(g_adj - g_orc).max() < 1e-9 * np.abs(g_orc).max()
    g_fd = _fd(prob, a0, h=1e-5)
    assert np.abs(g_adj - g_fd).max() < 1e-6 * np.abs(g_fd).max()
    g_fd4 = _fd(prob, a0, h=1e-4)
    assert np.abs(g_adj - g_fd4).max() < 1e-4 * np.abs(g_fd4).max()
    prob.close()


def test_fp32_drag_gradient_within_stated_tolerance(ctx):
    rng = np.random.default_rng(42)
    a0 = rng.uniform(-0.005, 0.005, 6)
    ref = _problem(ctx, "fp64", 1e-12)
    alpha = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    cd64 = drag(alpha, ref)
    cd64.backward()
    g64 = alpha.grad.numpy().copy()
    p32 = _problem(ctx, "fp32", 1e-7)
    alpha32 = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    cd32 = drag(alpha32, p32)
    cd32.backward()
    assert abs(cd32.item() - cd64.item()) < 1e-5 * abs(cd64.item())
    assert np.abs(alpha32.grad.numpy() - g64).max() < 1e-4 * np.abs(g64).max()
    ref.close()
    p32.close()


def test_device_warm_start_equals_host_round_trip(ctx):
    """The next design of a DragProblem starts from the last design's f and phi by device-to-device
    copies (dvm_state_copy_from, dvm_adjoint_copy_from).  Its drag and gradient are bitwise those of
    the same next design warm-started through the host (download f and phi, upload them into the new
    state and adjoint): FP32 values survive the round trip through FP64 exactly, and both routes
    recompute the moments, the wall density and the adjoint couplings with the same kernels."""
    rng = np.random.default_rng(43)
    a0 = rng.uniform(-0.005, 0.005, 6)
    a1 = a0 + rng.uniform(-1e-3, 1e-3, 6)
    prob = _problem(ctx, "fp32", 1e-6)
    prob.solve(a0)
    cold = prob.last["primal"].iters
    prob.gradient()
    f_w, phi_w = prob._warm[1].get(), prob._warm[2].get()
    cd1 = prob.solve(a1)
    g1 = prob.gradient()
    assert prob.last["primal"].iters < cold                 # the warm start took
    fl = prob.flow
    mesh = W.omesh(48, 16, a1)
    m = dvm.Mesh(ctx, mesh.nodes)
    st = dvm.State(ctx, m, prob._grid, fl.Kn, fl.Ma, fl.Tw, fl.aoa, storage="fp32")
    st.set(f_w)
    st, res = dvm.primal_solve(ctx, m, prob._grid, fl.Kn, fl.Ma, fl.Tw, fl.aoa, tol=prob.tol,
                               max_iter=prob.max_iter, storage="fp32", state=st, stall_window=prob.stall_window)
    ad = dvm.Adjoint(st)
    ad.set(phi_w)
    ad, ares = dvm.adjoint_solve(ctx, st, tol=prob.adjoint_tol, max_iter=prob.max_iter, adjoint=ad,
                                 stall_window=prob.stall_window)
    g = dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full")
    assert res.iters == prob.last["primal"].iters and ares.iters == prob.last["adjoint"].iters
    assert res.J / prob.q_ref == cd1
    assert np.array_equal(g / prob.q_ref, g1)
    ad.close(); st.close(); m.close()
    prob.close()


def test_order2_drag_gradient_matches_central_differences(ctx):
    """Second-order reconstruction: DragProblem(order=2) backs the drag with the full discrete gradient
    (its default mode; design.run takes the paper's boundary sensitivity at order 2 unless told), which
    must match central differences of second-order forward solves."""
    rng = np.random.default_rng(44)
    a0 = rng.uniform(-0.005, 0.005, 6)
    prob = DragProblem(ctx, 48, 16, W.velocity_grid(12, 4.0), W.Flow(1.0, 0.6), storage="fp64", tol=1e-11,
                       adjoint_tol=1e-11, max_iter=400000, order=2)
    alpha = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    cd = drag(alpha, prob)
    cd.backward()
    g = alpha.grad.numpy().copy()
    g_fd = _fd(prob, a0, h=1e-5)
    print(f"order 2: max |adjoint - FD| / max |FD| = {np.abs(g - g_fd).max() / np.abs(g_fd).max():.2e}")
    assert np.abs(g - g_fd).max() < 1e-5 * np.abs(g_fd).max()
    prob.close()
