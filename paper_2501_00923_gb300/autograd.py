"""Drag of an airfoil as a differentiable function of its shape parameters (torch.autograd).

forward(alpha) builds the O-mesh for the bump amplitudes alpha, solves the steady primal problem
(Eq. numerpr_gov) on the GPU and returns Cd = J / (rho |u|^2 / 2 * chord) (Eq. numer_J).  backward is the
implicit-function adjoint: the discrete adjoint solve (Eq. numerad_gov, transposed) at the converged
state followed by the full-discrete sensitivity, so grad = grad_out * dCd/dalpha.  The device state
and adjoint are kept by the problem object and reused as warm starts by the next evaluation of the
same problem (a line search or a design sweep moves alpha only a little).
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
    mode: str = "full"
    mesh_fn: object = None          # alpha -> OMesh; default: the Hicks-Henne bump section
    last: dict = field(default_factory=dict, repr=False)

    def __post_init__(self):
        self._grid = dvm.VGrid(self.ctx, self.grid.vx, self.grid.vy, self.grid.w)
        self._warm_f = None
        self._warm_phi = None

    @property
    def q_ref(self) -> float:
        U = self.flow.Ma * W.A_INF
        return 0.5 * U * U if U > 0 else 1.0

    def solve(self, alpha: np.ndarray):
        mesh = self.mesh_fn(alpha) if self.mesh_fn is not None else W.omesh(self.ni, self.nj, alpha)
        m = dvm.Mesh(self.ctx, mesh.nodes)
        st = dvm.State(self.ctx, m, self._grid, self.flow.Kn, self.flow.Ma, self.flow.Tw, self.flow.aoa,
                       storage=self.storage)
        if self._warm_f is not None:
            st.set(self._warm_f)
        st, res = dvm.primal_solve(self.ctx, m, self._grid, self.flow.Kn, self.flow.Ma, self.flow.Tw,
                                   self.flow.aoa, tol=self.tol, max_iter=self.max_iter, storage=self.storage,
                                   state=st, stall_window=self.stall_window)
        self.last = {"mesh": mesh, "m": m, "state": st, "primal": res}
        return res.J / self.q_ref

    def gradient(self):
        st, mesh = self.last["state"], self.last["mesh"]
        ad = dvm.Adjoint(st)
        if self._warm_phi is not None:
            ad.set(self._warm_phi)
        ad, ares = dvm.adjoint_solve(self.ctx, st, tol=self.adjoint_tol, max_iter=self.max_iter, adjoint=ad,
                                     stall_window=self.stall_window)
        g = dvm.sensitivity(self.ctx, st, ad, mesh.dwall, mesh.s, mode=self.mode)
        self._warm_f = st.get()
        self._warm_phi = ad.get()
        self.last["adjoint"] = ares
        ad.close()
        return g / self.q_ref

    def release(self):
        for k in ("state", "m"):
            if k in self.last:
                self.last[k].close()
        self.last = {}


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
