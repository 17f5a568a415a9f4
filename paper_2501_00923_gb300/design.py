"""Design loop: drag minimisation over the bump amplitudes under the volume constraint.

One optimisation step follows the paper's procedure: move the wall nodes for the new design
variables and the interior nodes with them (Step 2; the blend (1 - s_j) dwall replaces the paper's
RBF deformation), solve the primal and the adjoint problem and evaluate J and Q (Step 3), form
dJ/dalpha and dQ/dalpha (Step 4, Eq. sens_nod and Eq. sens_con_nod), update the design variables
with a quasi-Newton step (Step 5) and stop once the relative change of J between two accepted
steps is below 3e-5 (Step 6, Eq. criterion_opt).

The paper's optimiser is an SQP method with BFGS updates from a third-party library.  Here Step 5
is a limited-memory BFGS (the two-loop recursion of Nocedal and Wright, Algorithm 7.4) with a
projected Armijo backtracking line search.  The bumps move the wall nodes in y only, so the
polygon area, and with it Q, is an affine function of alpha: Q(alpha) = Q0 + dQ . (alpha - alpha0)
exactly.  The feasible set {|alpha_p| <= bound, Q <= 0} is then a box cut by one half-space, and
every trial design is its Euclidean projection onto that set: the constraint holds at every
evaluated design instead of being penalised.  The optimiser is an ask/tell object: `ask` returns
the next design to evaluate, `tell` takes (Cd, dCd/dalpha) of that design, so several loops can
share one served batch of GPU solves (`run_concurrent`).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import dvm
from . import workloads as W

CRITERION_OPT = 3e-5


def criterion_opt(J_old: float, J_new: float, tol: float = CRITERION_OPT) -> bool:
    """Eq. (criterion_opt): |J_new - J_old| / |J_old| < tol."""
    return abs(J_new - J_old) < tol * abs(J_old)


def project_box_halfspace(x, lower, upper, c=None, b=0.0, iters=200):
    """Euclidean projection of x onto {lower <= y <= upper, c . y <= b}.  The minimiser is
    y(nu) = clip(x - nu c) for the smallest nu >= 0 with c . y(nu) <= b; c . y(nu) does not increase
    with nu, so nu is found by bisection."""
    y = np.minimum(np.maximum(x, lower), upper)
    if c is None or float(c @ y) <= b:
        return y
    lo, hi = 0.0, 1.0
    while float(c @ np.minimum(np.maximum(x - hi * c, lower), upper)) > b:
        hi *= 2.0
        if hi > 1e30:
            raise ValueError("the half-space does not meet the box")
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if float(c @ np.minimum(np.maximum(x - mid * c, lower), upper)) > b:
            lo = mid
        else:
            hi = mid
    return np.minimum(np.maximum(x - hi * c, lower), upper)


class LBFGS:
    """Ask/tell L-BFGS with projected Armijo backtracking on the box [lower, upper].

    Phases: 'init' (x0 asked), 'trial' (a line-search point asked), 'done'.  `tell` returns
    'accepted' when the trial point became the new iterate, 'rejected' when the step was cut,
    'failed' when the line search gave up after a steepest-descent restart, or 'init'.
    halfspace = (c, b) adds the linear constraint c . x <= b to the box."""

    def __init__(self, x0, m: int = 8, lower=None, upper=None, first_step: float = 1e-3,
                 c1: float = 1e-4, shrink: float = 0.5, max_backtracks: int = 8, halfspace=None):
        self.x = np.array(x0, dtype=np.float64)
        n = self.x.size
        self.lower = np.full(n, -np.inf) if lower is None else np.broadcast_to(np.asarray(lower, float), (n,)).copy()
        self.upper = np.full(n, np.inf) if upper is None else np.broadcast_to(np.asarray(upper, float), (n,)).copy()
        self.halfspace = None if halfspace is None else (np.asarray(halfspace[0], float), float(halfspace[1]))
        self.x = self.project(self.x)
        self.m, self.first_step, self.c1, self.shrink, self.max_backtracks = m, first_step, c1, shrink, max_backtracks
        self.S: list[np.ndarray] = []
        self.Y: list[np.ndarray] = []
        self.f = None
        self.g = None
        self.phase = "init"
        self.iterations = 0
        self.evaluations = 0
        self._trial = None
        self._t = 1.0
        self._d = None
        self._backtracks = 0

    def project(self, x):
        if self.halfspace is None:
            return np.minimum(np.maximum(x, self.lower), self.upper)
        return project_box_halfspace(x, self.lower, self.upper, *self.halfspace)

    def direction(self, g):
        """-H g by the two-loop recursion, H0 = (s.y / y.y) I from the newest pair."""
        q = np.array(g, dtype=np.float64)
        rho = [1.0 / float(y @ s) for s, y in zip(self.S, self.Y)]
        a = []
        for s, y, r in zip(reversed(self.S), reversed(self.Y), reversed(rho)):
            ai = r * float(s @ q)
            a.append(ai)
            q -= ai * y
        if self.S:
            s, y = self.S[-1], self.Y[-1]
            q *= float(s @ y) / float(y @ y)
        for (s, y, r), ai in zip(zip(self.S, self.Y, rho), reversed(a)):
            b = r * float(y @ q)
            q += (ai - b) * s
        return -q

    def _new_direction(self):
        d = self.direction(self.g)
        if not self.S:                     # no curvature yet: the largest component moves by first_step
            nrm = np.abs(d).max()
            d = d * (self.first_step / nrm) if nrm > 0 else d
        self._d = d
        self._t = 1.0
        self._backtracks = 0
        self._trial = self.project(self.x + d)

    def ask(self):
        if self.phase == "init":
            return self.x.copy()
        if self.phase == "trial":
            return self._trial.copy()
        raise RuntimeError("optimiser finished")

    def tell(self, f: float, g) -> str:
        self.evaluations += 1
        g = np.asarray(g, dtype=np.float64)
        if self.phase == "init":
            if not np.isfinite(f):
                raise ValueError("initial design is not evaluable")
            self.f, self.g = float(f), g.copy()
            self.phase = "trial"
            self._new_direction()
            return "init"
        step = self._trial - self.x
        slope = float(self.g @ step)
        if np.isfinite(f) and slope < 0 and f <= self.f + self.c1 * slope:
            y = g - self.g
            sy = float(step @ y)
            if sy > 1e-12 * np.linalg.norm(step) * np.linalg.norm(y):
                self.S.append(step.copy())
                self.Y.append(y)
                if len(self.S) > self.m:
                    self.S.pop(0)
                    self.Y.pop(0)
            self.x, self.f, self.g = self._trial.copy(), float(f), g.copy()
            self.iterations += 1
            self._new_direction()
            return "accepted"
        self._backtracks += 1
        if slope >= 0 or self._backtracks > self.max_backtracks:
            if not self.S:                 # already on steepest descent: give up
                self.phase = "done"
                return "failed"
            self.S.clear()                 # curvature pairs misled the step: restart from -g
            self.Y.clear()
            self._new_direction()
            return "rejected"
        self._t *= self.shrink
        self._trial = self.project(self.x + self._t * self._d)
        return "rejected"


@dataclass
class Evaluation:
    alpha: np.ndarray
    Cd: float
    dCd: np.ndarray
    Q: float
    dQ: np.ndarray
    ok: bool = True


@dataclass
class DesignLoop:
    """One drag-minimisation loop at fixed flow conditions.

    ni, nj, grid, flow: the O-mesh size, velocity grid and flow; n_params bumps start at alpha0
    (zeros: the symmetric section).  v_min is the section area of alpha0 unless given; bound
    limits each amplitude; max_iter counts accepted steps.  `constrain(Q0, dQ)` with the volume
    constraint and its gradient at alpha0 must be called before the first `ask`."""
    ni: int
    nj: int
    grid: W.VGrid
    flow: W.Flow
    n_params: int = 24
    alpha0: np.ndarray | None = None
    v_min: float | None = None
    bound: float = 0.01
    max_iter: int = 12
    first_step: float = 1e-3
    tol: float = CRITERION_OPT
    shape: str = "bumps"
    history: list = field(default_factory=list)

    def __post_init__(self):
        if self.shape == "cst":
            # Sec. 3.3: CST variables of the base section by Eq. (cstini); bounds of Eq. (cst_constraint)
            nb = (self.n_params - 6) // 2
            if self.n_params != W.cst_count(nb):
                raise ValueError("a CST section has 2 N_B + 6 design variables")
            self.nb = nb
            self.a0 = W.cst_naca(self.ni, nb) if self.alpha0 is None else np.asarray(self.alpha0, float)
            lo = np.full(self.n_params, -np.inf)
            hi = np.full(self.n_params, np.inf)
            lo[0] = lo[1] = 0.01                              # N1, N2 >= 0.01
            lo[2:3 + nb] = 0.0                                # A_u >= 0
            hi[3 + nb:4 + 2 * nb] = 0.0                       # A_l <= 0
            lo[4 + 2 * nb:] = hi[4 + 2 * nb:] = 0.0           # sharp trailing edge
            self.lower, self.upper = lo, hi
        elif self.shape == "bumps":
            self.a0 = np.zeros(self.n_params) if self.alpha0 is None else np.asarray(self.alpha0, float)
            self.lower, self.upper = -self.bound, self.bound
        else:
            raise ValueError(f"unknown shape parameterisation {self.shape!r}")
        self.opt = None
        self.J_old = None
        self.converged = False
        self.stopped = None

    def mesh(self, alpha) -> W.OMesh:
        if self.shape == "cst":
            return W.omesh_cst(self.ni, self.nj, alpha, self.nb)
        return W.omesh(self.ni, self.nj, alpha)

    def constrain(self, Q0: float, dQ):
        """Q(alpha) ~ Q0 + dQ . (alpha - alpha0) <= 0, i.e. dQ . alpha <= dQ . alpha0 - Q0 (exact for
        the bumps, re-linearised at every accepted design otherwise)."""
        dQ = np.asarray(dQ, float)
        self.opt = LBFGS(self.a0, lower=self.lower, upper=self.upper, first_step=self.first_step,
                         halfspace=(dQ, float(dQ @ self.a0) - Q0))

    @property
    def q_ref(self) -> float:
        U = self.flow.Ma * W.A_INF
        return 0.5 * U * U

    def feasible_mesh(self, alpha) -> bool:
        if self.shape == "cst":        # A_u >= 0 >= A_l: the surfaces cannot cross
            return True
        return W.valid_amplitude_scale(self.ni, alpha, margin=1.0) >= 1.0

    def finish(self, ev: Evaluation) -> str:
        """Hand one evaluation to the optimiser; apply Eq. (criterion_opt) on accepted steps."""
        self.history.append(ev)
        phase = self.opt.phase
        out = self.opt.tell(ev.Cd if ev.ok else np.inf, ev.dCd if ev.ok else np.zeros_like(ev.alpha))
        if ev.ok and out in ("init", "accepted") and self.opt.phase != "done":
            # the volume half-space through the accepted design (unchanged when Q is affine)
            self.opt.halfspace = (np.asarray(ev.dQ, float), float(ev.dQ @ ev.alpha) - ev.Q)
        if phase == "init":
            self.J_old = ev.Cd
        elif out == "accepted":
            if criterion_opt(self.J_old, ev.Cd, self.tol):
                self.converged, self.stopped = True, "criterion_opt"
            self.J_old = ev.Cd
            if not self.converged and self.opt.iterations >= self.max_iter:
                self.stopped = "max_iter"
        elif out == "failed":
            self.stopped = "line_search"
        return out

    @property
    def done(self) -> bool:
        return self.stopped is not None

    @property
    def best(self) -> Evaluation:
        return min((e for e in self.history if e.ok), key=lambda e: e.Cd)


def _volume(ctx, nodes, v_min, dwall):
    m = dvm.Mesh(ctx, nodes)
    try:
        return dvm.volume_constraint(ctx, m, v_min, dwall)
    finally:
        m.close()


# a solve that met its tolerance, stopped at its rounding floor or ran out of sweeps still returns
# its final iterate; only non-finite or failed solves reject a design
_USABLE = (dvm.DVM_OK, dvm.DVM_NOT_CONVERGED, dvm.DVM_ERR_STAGNATED)


def _failed(alpha):
    z = np.zeros_like(alpha)
    return Evaluation(alpha, np.nan, z, np.nan, z, ok=False)


def drive(loop: DesignLoop, evaluate):
    """Run `loop` to its stop with blocking evaluations: evaluate(alpha) -> Evaluation (ok=False
    when the design could not be solved).  Designs whose mesh would fold are not evaluated."""
    while not loop.done:
        a = loop.opt.ask()
        loop.finish(evaluate(a) if loop.feasible_mesh(a) else _failed(a))
    return loop


def run(ctx: dvm.Context, loop: DesignLoop, storage: str = "fp32", tol: float = 1e-6,
        adjoint_tol: float = 1e-6, max_sweeps: int = 200000, stall_window: int = 0, order: int = 1,
        maxwellian: str = "plain", mode: str | None = None):
    """Drive one loop with blocking GPU solves (autograd.DragProblem keeps f and phi of the last
    design as warm starts for the next).  order 2 (second-order reconstruction) takes the paper's
    boundary sensitivity (mode "paper") unless mode says otherwise; order 1 the full discrete gradient."""
    from .autograd import DragProblem
    mode = mode or ("paper" if order == 2 else "full")
    prob = DragProblem(ctx, loop.ni, loop.nj, loop.grid, loop.flow, storage=storage, tol=tol,
                       adjoint_tol=adjoint_tol, max_iter=max_sweeps, stall_window=stall_window,
                       mesh_fn=loop.mesh, order=order, maxwellian=maxwellian, mode=mode)
    _start(ctx, loop)

    def evaluate(a):
        try:
            Cd = prob.solve(a)
            dCd = prob.gradient()
        except dvm.DVMError:
            prob.release()
            return _failed(a)
        mesh = prob.last["mesh"]
        Q, dQ = _volume(ctx, mesh.nodes, loop.v_min, mesh.dwall)
        prob.release()
        return Evaluation(a, Cd, dCd, Q, dQ)

    try:
        return drive(loop, evaluate)
    finally:
        prob.close()


def section_area(ctx: dvm.Context, ni: int, nj: int, alpha) -> float:
    """Area of the section for `alpha` (Q with V_min = 0 is minus the area)."""
    return -_volume(ctx, W.omesh(ni, nj, alpha).nodes, 0.0, np.zeros((1, ni, 2)))[0]


def _start(ctx, loop: DesignLoop):
    """V_min (the initial area unless given) and the linear volume constraint of the loop."""
    if loop.opt is not None:
        return
    mesh = loop.mesh(loop.a0)
    if loop.v_min is None:
        loop.v_min = -_volume(ctx, mesh.nodes, 0.0, np.zeros((1, loop.ni, 2)))[0]
    Q0, dQ = _volume(ctx, mesh.nodes, loop.v_min, mesh.dwall)
    loop.constrain(Q0, dQ)


def run_concurrent(ctx: dvm.Context, loops: list[DesignLoop], storage: str = "fp32", tol: float = 1e-6,
                   max_sweeps: int = 200000, sweeps_per_tick: int = 20, stall_window: int = 3000):
    """Drive several loops at once through one served batch: every loop's pending evaluation is a
    request in flight; a loop's next design is submitted as soon as its previous one retires, with
    its own warm-start key so f and phi carry over from that loop's last solve."""
    from .serve import BatchServer, SolveSpec
    server = BatchServer(ctx, sweeps_per_tick)
    pending = {}

    def submit(k):
        loop = loops[k]
        while not loop.done:
            a = loop.opt.ask()
            if loop.feasible_mesh(a):
                mesh = loop.mesh(a)
                spec = SolveSpec(mesh, loop.grid, loop.flow, storage=storage, tol=tol, adjoint_tol=tol,
                                 max_iter=max_sweeps, warm_key=1000 + k, stall_window=stall_window)
                pending[server.submit(spec)] = (k, a, mesh)
                return
            loop.finish(_failed(a))

    try:
        for k, loop in enumerate(loops):
            _start(ctx, loop)
            submit(k)
        while pending:
            server.tick()
            for t in list(pending):
                r = server.poll(t, forget=False)
                if not r["done"]:
                    continue
                server.poll(t, forget=True)
                k, a, mesh = pending.pop(t)
                loop = loops[k]
                if r["status"] not in _USABLE:
                    loop.finish(_failed(a))
                else:
                    Cd, dCd = r["J"] / loop.q_ref, r["grad"] / loop.q_ref
                    Q, dQ = _volume(ctx, mesh.nodes, loop.v_min, mesh.dwall)
                    loop.finish(Evaluation(a, Cd, dCd, Q, dQ))
                submit(k)
    finally:
        server.close()
    return loops


def main(argv=None):
    """Drag minimisation on the design workload (O-mesh 256x128, 48x48 Gauss-Legendre grid on
    [-6, 6]^2, Ma 0.8, 24 bumps from the symmetric section), one loop per Kn; prints one JSON line per
    loop with the accepted history and the wall time."""
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(prog="python -m paper_2501_00923_gb300.design")
    ap.add_argument("--kn", default="1,0.1,0.01")
    ap.add_argument("--iters", type=int, default=12)
    ap.add_argument("--mesh", default="256x128")
    ap.add_argument("--nv", type=int, default=48)
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--concurrent", action="store_true", help="all Kn loops through one served batch")
    ap.add_argument("--shape", default="bumps", choices=["bumps", "cst"],
                    help="24 Hicks-Henne bumps, or the 18 CST variables (N_B = 6) of Sec. 3.3")
    ap.add_argument("--order", type=int, default=1, choices=[1, 2],
                    help="2: second-order reconstruction with the paper's boundary sensitivity")
    ap.add_argument("--maxwellian", default="plain", choices=["plain", "conservative"])
    args = ap.parse_args(argv)
    if args.concurrent and (args.order != 1 or args.maxwellian != "plain"):
        ap.error("served batches are first order with the plain Maxwellian")
    from . import build
    build.build()
    ni, nj = (int(x) for x in args.mesh.lower().split("x"))
    wl = W.config(4)
    grid = W.velocity_grid(args.nv, 6.0, "gauss")
    ctx = dvm.Context(0)
    P = 24 if args.shape == "bumps" else W.cst_count()
    loops = [DesignLoop(ni, nj, grid, W.Flow(float(k), wl.flow.Ma), n_params=P, max_iter=args.iters,
                        shape=args.shape) for k in args.kn.split(",")]
    t0 = time.perf_counter()
    if args.concurrent:
        run_concurrent(ctx, loops, storage=args.storage, tol=args.tol)
        spans = [time.perf_counter() - t0] * len(loops)
    else:
        spans = []
        for loop in loops:
            t = time.perf_counter()
            run(ctx, loop, storage=args.storage, tol=args.tol, adjoint_tol=args.tol, stall_window=3000,
                order=args.order, maxwellian=args.maxwellian)
            spans.append(time.perf_counter() - t)
    for loop, span in zip(loops, spans):
        acc, best = [], None
        for e in loop.history:
            if e.ok and (best is None or e.Cd < best):
                best = e.Cd
                acc.append({"Cd": e.Cd, "Q_over_Vmin": e.Q / loop.v_min})
        print(json.dumps({"Kn": loop.flow.Kn, "Ma": loop.flow.Ma, "mesh": args.mesh, "nv": args.nv, "shape": args.shape,
                          "order": args.order, "maxwellian": args.maxwellian,
                          "storage": args.storage, "stopped": loop.stopped, "iterations": loop.opt.iterations,
                          "evaluations": loop.opt.evaluations, "Cd0": loop.history[0].Cd, "Cd_best": best,
                          "seconds": span, "concurrent": args.concurrent, "accepted": acc}))
    ctx.close()


if __name__ == "__main__":
    main()
