"""Served solves: continuous batching through the library's dvm_batch_* calls.

`BatchServer` wraps one dvm_batch: submit whole requests (primal solve, adjoint solve, sensitivity),
tick, poll.  `replay` drives a request trace against wall-clock arrival times, submitting each
request when it arrives and ticking while work is in flight; it returns per-request latencies
(arrival to retirement).  `replay_serial` is the one-at-a-time baseline: each request alone, in
arrival order, with plain FP32 solves and no batching or graph capture.

The clock and the submit/tick/poll callables are injectable so the scheduling logic can be
exercised without a GPU.
"""
from __future__ import annotations

import ctypes as C
import time
from dataclasses import dataclass, field

import numpy as np

from . import dvm
from . import workloads as W

_dp = C.POINTER(C.c_double)


class BatchOptions(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("sweeps_per_tick", C.c_int), ("max_active", C.c_int)]


class Request(C.Structure):
    _fields_ = [("ni", C.c_int), ("nj", C.c_int), ("nodes_xy", _dp), ("nv", C.c_int),
                ("vx", _dp), ("vy", _dp), ("w", _dp), ("flow", dvm.Flow), ("storage", C.c_int),
                ("tol", C.c_double), ("adjoint_tol", C.c_double), ("max_iter", C.c_int),
                ("functional", C.c_int), ("n_params", C.c_int), ("dwall_dalpha", _dp), ("s_j", _dp),
                ("sens_mode", C.c_int), ("warm_key", C.c_uint64), ("stall_window", C.c_int),
                ("predict_iters", C.c_int), ("predict_omega", C.c_double)]


class BatchStats(C.Structure):
    _fields_ = [("ticks", C.c_uint64), ("graph_launches", C.c_uint64), ("graph_builds", C.c_uint64),
                ("table_uploads", C.c_uint64), ("peak_active", C.c_int), ("peak_bytes", C.c_size_t)]


class RequestResult(C.Structure):
    _fields_ = [("done", C.c_int), ("status", C.c_int), ("phase", C.c_int), ("primal_iters", C.c_int),
                ("adjoint_iters", C.c_int), ("J", C.c_double), ("Cd", C.c_double), ("residual", C.c_double),
                ("adjoint_residual", C.c_double), ("warm_started", C.c_int), ("predictions", C.c_int)]


def _bind():
    L = dvm.lib()
    if getattr(L, "_batch_bound", False):
        return L
    vp, i = C.c_void_p, C.c_int
    sig = {
        "dvm_batch_create": (i, [vp, C.POINTER(BatchOptions), C.POINTER(vp)]),
        "dvm_batch_destroy": (None, [vp]),
        "dvm_batch_submit": (i, [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
        "dvm_batch_tick": (i, [vp, C.POINTER(i), C.POINTER(i)]),
        "dvm_batch_poll": (i, [vp, C.c_uint64, C.POINTER(RequestResult), _dp, i]),
        "dvm_batch_get_stats": (i, [vp, C.POINTER(BatchStats)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    L._batch_bound = True
    return L


@dataclass
class SolveSpec:
    """One request: geometry, velocity grid, flow and what to compute."""
    mesh: W.OMesh
    grid: W.VGrid
    flow: W.Flow
    storage: str = "fp32"
    tol: float = 1e-5
    adjoint_tol: float = 1e-5
    max_iter: int = 2000
    sens: bool = True
    sens_mode: str = "full"
    functional: str = "drag"
    warm_key: int = 0
    stall_window: int = 0
    predict: int = 0                 # > 0: macroscopic prediction of both phases (GMRES steps)
    predict_omega: float = 0.0
    _keep: list = field(default_factory=list, repr=False)

    def to_c(self) -> Request:
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in
                (self.mesh.nodes, self.grid.vx, self.grid.vy, self.grid.w, self.mesh.dwall, self.mesh.s)]
        self._keep = arrs
        nodes, vx, vy, w, dwall, s = arrs
        P = dwall.shape[0] if self.sens else 0
        p = lambda a: a.ctypes.data_as(_dp)  # noqa: E731
        return Request(self.mesh.ni, self.mesh.nj, p(nodes), self.grid.nv, p(vx), p(vy), p(w),
                       dvm.Flow(self.flow.Kn, self.flow.Ma, self.flow.Tw, self.flow.aoa),
                       dvm.STORAGE[self.storage], self.tol, self.adjoint_tol, self.max_iter,
                       dvm.FUNCTIONAL[self.functional], P, p(dwall) if P else None, p(s) if P else None,
                       dvm.SENS[self.sens_mode], self.warm_key, self.stall_window, self.predict,
                       self.predict_omega)


class BatchServer:
    """One dvm_batch.  Owned by its Context: Context.close() releases it first."""

    _rank = 4

    def __init__(self, ctx: dvm.Context, sweeps_per_tick: int = 20, hbm_budget: int = 0, max_active: int = 0):
        self.L = _bind()
        self.ctx = ctx
        self.h = None
        h = C.c_void_p()
        dvm._check(self.L.dvm_batch_create(ctx.h, C.byref(BatchOptions(hbm_budget, sweeps_per_tick, max_active)),
                                           C.byref(h)))
        self.h = h
        self.nparams = {}
        ctx._adopt(self)

    def submit(self, spec: SolveSpec) -> int:
        req = spec.to_c()
        t = C.c_uint64()
        dvm._check(self.L.dvm_batch_submit(self.h, C.byref(req), C.byref(t)))
        self.nparams[t.value] = req.n_params
        return t.value

    def tick(self):
        a, q = C.c_int(), C.c_int()
        dvm._check(self.L.dvm_batch_tick(self.h, C.byref(a), C.byref(q)))
        return a.value, q.value

    def poll(self, ticket: int, forget: bool = False):
        r = RequestResult()
        n = self.nparams.get(ticket, 0)
        g = np.zeros(max(n, 1))
        dvm._check(self.L.dvm_batch_poll(self.h, ticket, C.byref(r), g.ctypes.data_as(_dp), int(forget)))
        out = {k: getattr(r, k) for k, _ in RequestResult._fields_}
        out["grad"] = g[:n].copy()
        if forget and r.done:
            self.nparams.pop(ticket, None)
        return out

    def stats(self) -> dict:
        st = BatchStats()
        dvm._check(self.L.dvm_batch_get_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in BatchStats._fields_}

    def close(self):
        if self.h:
            self.L.dvm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------------- traces
def trace_specs(trace, storage="fp32", max_iter=2000, tol=1e-5, warm=False, predict=0):
    """SolveSpecs of a request trace (see workloads.request_trace); predict > 0 asks every request for
    the macroscopic prediction with that many GMRES steps."""
    specs = []
    for r in trace:
        mesh = W.omesh(r["ni"], r["nj"], r["alpha"])
        grid = W.velocity_grid(r["nv"], r["range"])
        specs.append(SolveSpec(mesh, grid, W.Flow(r["Kn"], r["Ma"]), storage=storage, tol=tol, adjoint_tol=tol,
                               max_iter=max_iter, warm_key=(hash((r["ni"], r["nj"], r["nv"])) & 0xffff) + 1
                               if warm else 0, predict=predict))
    return specs


def replay(arrivals, submit, tick, poll_done, clock=time.perf_counter, sleep=time.sleep, idle_wait=1e-3):
    """Drive a trace: submit request k once clock() - t0 >= arrivals[k], tick while anything is in
    flight, collect retirement times.  poll_done(handle) -> bool.  Returns (latencies, makespan)."""
    n = len(arrivals)
    order = np.argsort(arrivals)
    t0 = clock()
    handles, t_arr, t_done = {}, {}, {}
    nxt = 0
    inflight = set()
    while len(t_done) < n:
        now = clock() - t0
        while nxt < n and arrivals[order[nxt]] <= now:
            k = int(order[nxt])
            handles[k] = submit(k)
            t_arr[k] = arrivals[k]
            inflight.add(k)
            nxt += 1
        if inflight:
            tick()
            now = clock() - t0
            for k in list(inflight):
                if poll_done(handles[k]):
                    t_done[k] = now
                    inflight.discard(k)
        elif nxt < n:
            sleep(min(idle_wait, max(0.0, arrivals[order[nxt]] - now)))
    lat = np.array([t_done[k] - t_arr[k] for k in range(n)])
    return lat, max(t_done.values())


def latency_stats(lat, makespan):
    return {"solves": int(len(lat)), "solves_per_s": len(lat) / makespan, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_ms": 1e3 * float(np.mean(lat)),
            "makespan_s": float(makespan)}


def replay_batched(ctx, specs, arrivals, sweeps_per_tick=20, hbm_budget=0):
    """Returns (latencies, makespan, {ticket: result}, batch counters)."""
    server = BatchServer(ctx, sweeps_per_tick, hbm_budget)
    results = {}

    def poll_done(t):
        r = server.poll(t)
        if r["done"]:
            results[t] = r
        return bool(r["done"])

    lat, span = replay(arrivals, lambda k: server.submit(specs[k]), server.tick, poll_done)
    stats = server.stats()
    server.close()
    return lat, span, results, stats


def replay_serial(ctx, specs, arrivals):
    """One request at a time in arrival order, no batching and no graph capture: ctx should be
    created with graphs=False.  Returns (latencies, makespan, {k: error status or None},
    {k: solve status})."""
    queue = []
    done_flags = {}
    failures = {}
    statuses = {}

    def submit(k):
        queue.append(k)
        return k

    def tick():
        if not queue:
            return
        k = queue.pop(0)
        s = specs[k]
        objs = []
        try:
            m = dvm.Mesh(ctx, s.mesh.nodes)
            objs.append(m)
            g = dvm.VGrid(ctx, s.grid.vx, s.grid.vy, s.grid.w)
            objs.append(g)
            st, pres = dvm.primal_solve(ctx, m, g, s.flow.Kn, s.flow.Ma, s.flow.Tw, s.flow.aoa, tol=s.tol,
                                        max_iter=s.max_iter, storage=s.storage, predict=s.predict,
                                        predict_omega=s.predict_omega)
            objs.append(st)
            status = pres.status
            if s.sens:
                ad, ares = dvm.adjoint_solve(ctx, st, tol=s.adjoint_tol, max_iter=s.max_iter, predict=s.predict,
                                             predict_omega=s.predict_omega)
                objs.append(ad)
                dvm.sensitivity(ctx, st, ad, s.mesh.dwall, s.mesh.s, mode=s.sens_mode)
                status = status if status != dvm.DVM_OK else ares.status
            failures[k] = None
            statuses[k] = status
        except dvm.DVMError as e:          # the request fails; the replay goes on
            failures[k] = e.status
        for o in reversed(objs):
            o.close()
        done_flags[k] = True

    lat, span = replay(arrivals, submit, tick, lambda k: done_flags.get(k, False))
    return lat, span, failures, statuses
