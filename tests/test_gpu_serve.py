"""Served solves on the GPU: continuous batching through dvm_batch_*.

A request's result must not depend on the rest of the batch: alone, in a mix of other sizes and
flows, and through the one-request API (same sweeps per tick as graph size) the drag and the
gradient agree bit for bit.  Admission by HBM budget, warm starts and the iteration cap are
checked too."""
import dataclasses

import numpy as np
import pytest

from paper_2501_00923_gb300 import build, dvm, serve
from paper_2501_00923_gb300 import workloads as W

pytestmark = pytest.mark.gpu
M = 20


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = dvm.Context(0, graph_iters=M)
    yield c
    c.close()


def _specs():
    rng = np.random.default_rng(5)
    out = []
    for (ni, nj, nv, Kn, Ma) in [(48, 16, 12, 1.0, 0.6), (64, 24, 16, 0.5, 1.2), (32, 12, 10, 2.0, 0.4)]:
        out.append(serve.SolveSpec(W.omesh(ni, nj, rng.uniform(-0.01, 0.01, 6)), W.velocity_grid(nv, 4.0),
                                   W.Flow(Kn, Ma), tol=1e-5, adjoint_tol=1e-5, max_iter=4000))
    return out


def _run(ctx, specs, **kw):
    srv = serve.BatchServer(ctx, sweeps_per_tick=M, **kw)
    tickets = [srv.submit(s) for s in specs]
    for _ in range(10000):
        a, q = srv.tick()
        if a == 0 and q == 0:
            break
    res = [srv.poll(t) for t in tickets]
    srv.close()
    return res


def test_result_is_the_same_alone_in_a_mix_and_through_the_plain_api(ctx):
    specs = _specs()
    mixed = _run(ctx, specs)
    for k, s in enumerate(specs):
        alone = _run(ctx, [s])[0]
        for key in ("J", "residual", "adjoint_residual", "primal_iters", "adjoint_iters", "status"):
            assert alone[key] == mixed[k][key], key
        assert np.array_equal(alone["grad"], mixed[k]["grad"])
        m = dvm.Mesh(ctx, s.mesh.nodes)
        g = dvm.VGrid(ctx, s.grid.vx, s.grid.vy, s.grid.w)
        st, res = dvm.primal_solve(ctx, m, g, s.flow.Kn, s.flow.Ma, tol=s.tol, max_iter=s.max_iter)
        ad, ares = dvm.adjoint_solve(ctx, st, tol=s.adjoint_tol, max_iter=s.max_iter)
        grad = dvm.sensitivity(ctx, st, ad, s.mesh.dwall, s.mesh.s, mode="full")
        assert res.J == mixed[k]["J"] and res.iters == mixed[k]["primal_iters"]
        assert ares.iters == mixed[k]["adjoint_iters"]
        assert np.array_equal(grad, mixed[k]["grad"])
        assert mixed[k]["status"] == dvm.DVM_OK


def test_admission_by_hbm_budget_queues_then_serves(ctx):
    specs = _specs()
    srv = serve.BatchServer(ctx, sweeps_per_tick=M, hbm_budget=int(14e6))   # room for one request at a time
    tickets = [srv.submit(s) for s in specs]
    a, q = srv.tick()
    assert a == 1 and q == 2
    for _ in range(10000):
        a, q = srv.tick()
        assert a <= 1
        if a == 0 and q == 0:
            break
    assert all(srv.poll(t)["done"] for t in tickets)
    with pytest.raises(dvm.DVMError) as e:
        serve.BatchServer(ctx, sweeps_per_tick=M, hbm_budget=1000).submit(specs[0])
    assert e.value.status == dvm.DVM_ERR_ADMISSION
    srv.close()


def test_warm_start_reuses_the_previous_state(ctx):
    rng = np.random.default_rng(9)
    alpha = rng.uniform(-0.01, 0.01, 6)
    base = serve.SolveSpec(W.omesh(48, 16, alpha), W.velocity_grid(12, 4.0), W.Flow(1.0, 0.6), tol=1e-5,
                           adjoint_tol=1e-5, max_iter=4000, warm_key=7)
    nudged = serve.SolveSpec(W.omesh(48, 16, alpha + 1e-4), W.velocity_grid(12, 4.0), W.Flow(1.0, 0.6), tol=1e-5,
                             adjoint_tol=1e-5, max_iter=4000, warm_key=7)
    srv = serve.BatchServer(ctx, sweeps_per_tick=M)
    t0 = srv.submit(base)
    while srv.tick() != (0, 0):
        pass
    t1 = srv.submit(nudged)
    while srv.tick() != (0, 0):
        pass
    r0, r1 = srv.poll(t0), srv.poll(t1)
    assert r1["warm_started"] == 1 and r0["warm_started"] == 0
    assert r1["primal_iters"] < r0["primal_iters"] and r1["adjoint_iters"] < r0["adjoint_iters"]
    assert abs(r1["J"] - r0["J"]) < 1e-2 * abs(r0["J"])
    srv.close()


def test_iteration_cap_reports_not_converged(ctx):
    s = _specs()[0]
    s.max_iter = 40
    s.tol = s.adjoint_tol = 1e-12
    r = _run(ctx, [s])[0]
    assert r["done"] and r["status"] == dvm.DVM_NOT_CONVERGED
    assert r["primal_iters"] == 40 and r["adjoint_iters"] == 40


def test_ticks_run_as_one_graph_and_reuse_device_tables(ctx):
    """Every tick of a graph-capable context is one CUDA-graph launch (sweeps, reductions, read-back);
    the graph is captured again only when a table outgrows its capacity, and the tables are uploaded
    again only when the admitted set or a request's phase changes.  A context without graphs runs the
    same launches directly and gives bit-for-bit the same results."""
    specs = _specs()
    srv = serve.BatchServer(ctx, sweeps_per_tick=M)
    tickets = [srv.submit(s) for s in specs]
    for _ in range(10000):
        if srv.tick() == (0, 0):
            break
    st = srv.stats()
    res = [srv.poll(t) for t in tickets]
    srv.close()
    assert st["ticks"] > 20 and st["graph_launches"] == st["ticks"]
    assert 1 <= st["graph_builds"] <= 4
    assert st["table_uploads"] <= 3 * len(specs)           # admission, adjoint start and retirement at most
    assert st["peak_active"] == len(specs) and st["peak_bytes"] > 0
    plain = dvm.Context(0, graph_iters=M, graphs=False)
    srv2 = serve.BatchServer(plain, sweeps_per_tick=M)
    t2 = [srv2.submit(s) for s in specs]
    for _ in range(10000):
        if srv2.tick() == (0, 0):
            break
    assert srv2.stats()["graph_launches"] == 0
    for a, t in zip(res, t2):
        b = srv2.poll(t)
        assert a["J"] == b["J"] and a["primal_iters"] == b["primal_iters"]
        assert np.array_equal(a["grad"], b["grad"])
    srv2.close()
    plain.close()


def test_predicted_requests_converge_and_do_not_depend_on_the_batch(ctx):
    """Requests with the macroscopic prediction (FP64, Kn 0.02 and 0.05): the result is the same alone
    and in a mix (bit for bit: the prediction runs per request on its own buffers), the solve converges
    where the same request without prediction stops at the cap, and drag and gradient match the
    predicted one-request API (whose residual moments come from inside its last sweep rather than from
    the tick's last input and output) to the solve tolerance."""
    rng = np.random.default_rng(6)
    specs = []
    for (ni, nj, nv, Kn, Ma) in [(32, 12, 10, 0.02, 0.8), (48, 16, 12, 0.05, 0.6)]:
        specs.append(serve.SolveSpec(W.omesh(ni, nj, rng.uniform(-0.01, 0.01, 6)), W.velocity_grid(nv, 4.0),
                                     W.Flow(Kn, Ma), storage="fp64", tol=1e-11, adjoint_tol=1e-11, max_iter=2000,
                                     predict=20))
    mixed = _run(ctx, specs)
    for k, s in enumerate(specs):
        alone = _run(ctx, [s])[0]
        for key in ("J", "residual", "adjoint_residual", "primal_iters", "adjoint_iters", "status", "predictions"):
            assert alone[key] == mixed[k][key], key
        assert np.array_equal(alone["grad"], mixed[k]["grad"])
        assert mixed[k]["status"] == dvm.DVM_OK and mixed[k]["predictions"] > 0
        unpredicted = _run(ctx, [dataclasses.replace(s, predict=0)])[0]
        assert unpredicted["status"] == dvm.DVM_NOT_CONVERGED
        m = dvm.Mesh(ctx, s.mesh.nodes)
        g = dvm.VGrid(ctx, s.grid.vx, s.grid.vy, s.grid.w)
        st, res = dvm.primal_solve(ctx, m, g, s.flow.Kn, s.flow.Ma, tol=s.tol, max_iter=s.max_iter, storage="fp64",
                                   predict=20)
        ad, ares = dvm.adjoint_solve(ctx, st, tol=s.adjoint_tol, max_iter=s.max_iter, predict=20)
        grad = dvm.sensitivity(ctx, st, ad, s.mesh.dwall, s.mesh.s, mode="full")
        print(f"Kn {s.flow.Kn}: served {mixed[k]['primal_iters']} + {mixed[k]['adjoint_iters']} sweeps "
              f"({mixed[k]['predictions']} predictions), API {res.iters} + {ares.iters}; drag difference "
              f"{abs(res.J - mixed[k]['J']) / abs(res.J):.1e}, gradient {np.abs(grad - mixed[k]['grad']).max() / np.abs(grad).max():.1e}")
        assert abs(res.J - mixed[k]["J"]) < 1e-7 * abs(res.J)
        assert np.abs(grad - mixed[k]["grad"]).max() < 1e-6 * np.abs(grad).max()
        for h in (ad, st, g, m):
            h.close()
