"""Drag of an airfoil as a differentiable function of its shape parameters (torch.autograd).

forward(alpha) builds the O-mesh for the bump amplitudes alpha, solves the steady primal problem
(Eq. numerpr_gov) on the GPU and returns Cd = J / (rho |u|^2 / 2 * chord) (Eq. numer_J).  backward is the
implicit-function adjoint: the discrete adjoint solve (Eq. numerad_gov, transposed) at the converged
state followed by the full-discrete sensitivity, so grad = grad_out * dCd/dalpha.  The device state
and adjoint are kept by the problem object and reused as warm starts by the next evaluation of the
same problem (a line search or a design sweep moves alpha only a little): the next design's state
and adjoint start from them by device-to-device copies (dvm_state_copy_from, dvm_adjoint_copy_from),
so no f or phi crosses to the host between evaluations.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import dvm
from . import workloads as W


@dataclass
class DragProblem:
    ctx: dvm.Context
    ni: int
    nj: int
    grid: W.VGrid
    flow: W.Flow
    storage: str = "fp32"
    tol: float = 1e-6
    adjoint_tol: float = 1e-6
    max_iter: int = 200000
    stall_window: int = 0
    mode: str = "full"              # gradient: the full discrete one (at order 2 too); "paper": the paper's
                                    # boundary sensitivity (design.run takes it by default at order 2)
    mesh_fn: object = None          # alpha -> OMesh; default: the Hicks-Henne bump section
    order: int = 1                  # 2: second-order reconstruction
    maxwellian: str = "plain"       # or "conservative"
    refine_tol: float = 0.0         # > 0 (FP32, order 1, plain): mixed-precision refinement of the primal to this
                                    # FP64 residual after the sweeps (dvm_solve_opts.refine_tol)
    predict: int = 0                # > 0 (FP64/FP32, order 1, plain): macroscopic prediction after every block of
                                    # primal and adjoint sweeps, this many GMRES steps (dvm_solve_opts.predict_iters)
    predict_precond: int = 0        # 1: those steps preconditioned by a multigrid V-cycle
    last: dict = field(default_factory=dict, repr=False)

    def __post_init__(self):
        self._grid = dvm.VGrid(self.ctx, self.grid.vx, self.grid.vy, self.grid.w)
        self._warm = None           # (mesh, state, adjoint) of the last design whose gradient was taken

    @property
    def q_ref(self) -> float:
        U = self.flow.Ma * W.A_INF
        return 0.5 * U * U if U > 0 else 1.0

    def solve(self, alpha: np.ndarray):
        mesh = self.mesh_fn(alpha) if self.mesh_fn is not None else W.omesh(self.ni, self.nj, alpha)
        m = dvm.Mesh(self.ctx, mesh.nodes)
        st = dvm.State(self.ctx, m, self._grid, self.flow.Kn, self.flow.Ma, self.flow.Tw, self.flow.aoa,
                       storage=self.storage)
        if self.maxwellian != "plain":
            st.maxwellian = self.maxwellian
        if self._warm is not None:
            st.copy_from(self._warm[1])
        elif self.order == 2:               # second order starts from the converged first-order state
            dvm.primal_solve(self.ctx, m, self._grid, self.flow.Kn, self.flow.Ma, self.flow.Tw, self.flow.aoa,
                             tol=self.tol, max_iter=self.max_iter, storage=self.storage, state=st,
                             stall_window=self.stall_window,
                             predict=self.predict if self.maxwellian == "plain" and self.storage != "bf16" else 0)
        st.order = self.order
        plain1 = self.order == 1 and self.maxwellian == "plain" and self.storage != "bf16"
        st, res = dvm.primal_solve(self.ctx, m, self._grid, self.flow.Kn, self.flow.Ma, self.flow.Tw,
                                   self.flow.aoa, tol=self.tol, max_iter=self.max_iter, storage=self.storage,
                                   state=st, stall_window=self.stall_window, refine_tol=self.refine_tol,
                                   predict=self.predict if plain1 else 0, predict_precond=self.predict_precond)
        self.last = {"mesh": mesh, "m": m, "state": st, "primal": res}
        return res.J / self.q_ref

    def gradient(self):
        st, mesh = self.last["state"], self.last["mesh"]
        ad = dvm.Adjoint(st)
        if self._warm is not None:
            ad.copy_from(self._warm[2])
        plain1 = self.order == 1 and self.maxwellian == "plain" and self.storage != "bf16"
        ad, ares = dvm.adjoint_solve(self.ctx, st, tol=self.adjoint_tol, max_iter=self.max_iter, adjoint=ad,
                                     stall_window=self.stall_window, predict=self.predict if plain1 else 0,
                                     predict_precond=self.predict_precond)
        g = dvm.sensitivity(self.ctx, st, ad, mesh.dwall, mesh.s, mode=self.mode)
        self._drop_warm()
        self._warm = (self.last["m"], st, ad)     # stays on the device as the next design's warm start
        self.last["adjoint"] = ares
        return g / self.q_ref

    def _is_warm(self, obj) -> bool:
        return self._warm is not None and any(obj is w for w in self._warm)

    def _drop_warm(self):
        if self._warm is not None:
            m, st, ad = self._warm
            self._warm = None
            for obj in (ad, st, m):
                if not any(obj is self.last.get(k) for k in ("state", "m")):
                    obj.close()

    def release(self):
        """Free the last design's state and mesh unless they are kept as the warm start."""
        for k in ("state", "m"):
            if k in self.last and not self._is_warm(self.last[k]):
                self.last[k].close()
        self.last = {}

    def close(self):
        """Free everything, the warm start included."""
        self.release()
        self._drop_warm()
        self._grid.close()


class DragFn(torch.autograd.Function):
    """Cd(alpha): forward = primal solve, backward = adjoint solve + sensitivity."""

    @staticmethod
    def forward(ctx, alpha: torch.Tensor, problem: DragProblem):
        a = alpha.detach().to("cpu", torch.float64).numpy()
        cd = problem.solve(a)
        ctx.problem = problem
        ctx.alpha_meta = (alpha.dtype, alpha.device)
        return torch.tensor(cd, dtype=alpha.dtype, device=alpha.device)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.problem.gradient()
        dtype, device = ctx.alpha_meta
        return grad_out * torch.as_tensor(g, dtype=dtype, device=device), None


def drag(alpha: torch.Tensor, problem: DragProblem) -> torch.Tensor:
    return DragFn.apply(alpha, problem)


def main(argv=None):
    """Cd and dCd/dalpha through DragFn on a workload at full size, with central differences of the
    forward on the first `--fd` amplitudes.  One JSON line: times, sweep counts and statuses of the
    forward and backward solves, the gradient, and the largest difference from the differences."""
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(prog="python -m paper_2501_00923_gb300.autograd")
    ap.add_argument("--workload", type=int, default=2, help="recipe index (2: 384x192, 64x64, Kn 0.001, Ma 2)")
    ap.add_argument("--kn", type=float, default=None, help="override the recipe's Kn")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-sweeps", type=int, default=200000)
    ap.add_argument("--stall", type=int, default=3000)
    ap.add_argument("--fd", type=int, default=0, help="amplitudes checked by central differences")
    ap.add_argument("--h", type=float, default=1e-4, help="difference step")
    ap.add_argument("--refine-tol", type=float, default=0.0,
                    help="> 0: mixed-precision refinement of every primal solve to this FP64 residual")
    ap.add_argument("--predict", type=int, default=0,
                    help="> 0: macroscopic prediction of the primal sweeps (block-Jacobi iterations)")
    ap.add_argument("--adjoint-tol", type=float, default=None, help="adjoint tolerance (default: --tol)")
    ap.add_argument("--predict-precond", type=int, default=0, choices=[0, 1],
                    help="1: multigrid-preconditioned prediction steps")
    args = ap.parse_args(argv)
    from . import build
    build.build()
    wl = W.config(args.workload)
    flow = W.Flow(args.kn if args.kn is not None else wl.flow.Kn, wl.flow.Ma, wl.flow.Tw, wl.flow.aoa)
    ctx = dvm.Context(0)
    a0 = wl.mesh.alpha
    prob = DragProblem(ctx, wl.mesh.ni, wl.mesh.nj, wl.grid, flow, storage=args.storage, tol=args.tol,
                       adjoint_tol=args.adjoint_tol if args.adjoint_tol is not None else args.tol,
                       max_iter=args.max_sweeps, stall_window=args.stall, refine_tol=args.refine_tol,
                       predict=args.predict, predict_precond=args.predict_precond)
    alpha = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    t0 = time.perf_counter()
    cd = drag(alpha, prob)
    t1 = time.perf_counter()
    cd.backward()
    t2 = time.perf_counter()
    g = alpha.grad.numpy().copy()
    pres, ares = prob.last["primal"], prob.last["adjoint"]
    out = {"workload": wl.name, "Kn": flow.Kn, "storage": args.storage, "cells": wl.mesh.ncell, "velocities": wl.grid.nv,
           "Cd": float(cd.item()), "forward_s": t1 - t0, "backward_s": t2 - t1,
           "primal_sweeps": pres.iters, "primal_status": dvm.status_string(pres.status), "primal_residual": pres.residual,
           "refine_steps": pres.refine_steps, "refine_sweeps": pres.refine_sweeps, "predictions": pres.predictions,
           "adjoint_sweeps": ares.iters, "adjoint_predictions": ares.predictions,
           "adjoint_status": dvm.status_string(ares.status),
           "adjoint_residual": ares.residual, "grad": g.tolist()}
    prob.release()
    if args.fd > 0:
        fd = []
        t3 = time.perf_counter()
        for p in range(args.fd):
            e = np.zeros_like(a0)
            e[p] = args.h
            up = prob.solve(a0 + e)
            prob.release()
            dn = prob.solve(a0 - e)
            prob.release()
            fd.append((up - dn) / (2 * args.h))
        fd = np.array(fd)
        out.update({"fd_params": args.fd, "fd_step": args.h, "fd": fd.tolist(), "fd_s": time.perf_counter() - t3,
                    "fd_max_diff_rel_to_max_grad": float(np.abs(fd - g[:args.fd]).max() / np.abs(g).max())})
    print(json.dumps(out))
    ctx.close()


if __name__ == "__main__":
    main()
