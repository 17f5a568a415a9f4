"""ctypes wrapper of the FP64 CPU oracle (oracle/dvm_oracle.cpp).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg import
this module.  The CUDA library never calls it.  Every function here follows the paper section named
in the C++ source; this file only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dvm_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

_dp = C.POINTER(C.c_double)


class _Problem(C.Structure):
    _fields_ = [("ni", C.c_int), ("nj", C.c_int), ("nv", C.c_int),
                ("nodes", _dp), ("vx", _dp), ("vy", _dp), ("w", _dp),
                ("Kn", C.c_double), ("Ma", C.c_double), ("Tw", C.c_double), ("aoa", C.c_double),
                ("dir", C.c_double * 3), ("conservative", C.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, OpenMP).  Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i = C.c_double, C.c_int
        P = C.POINTER(_Problem)
        sig = {
            "orc_threads": (i, [i]),
            "orc_geometry": (i, [P, _dp, _dp]),
            "orc_freestream": (i, [P, _dp]),
            "orc_moments": (i, [P, _dp, _dp]),
            "orc_collision": (i, [P, _dp, _dp]),
            "orc_residual": (i, [P, _dp, _dp, _dp]),
            "orc_residual_dir": (i, [P, _dp, _dp, _dp, _dp]),
            "orc_functional_dir": (i, [P, _dp, _dp, _dp, _dp]),
            "orc_functional": (d, [P, _dp]),
            "orc_functional_grad": (i, [P, _dp, _dp]),
            "orc_apply_RT": (i, [P, _dp, _dp, _dp]),
            "orc_jacobi": (i, [P, _dp, _dp, _dp]),
            "orc_adjoint_jacobi": (i, [P, _dp, _dp, _dp, _dp]),
            "orc_primal_solve": (i, [P, _dp, d, i, _dp, C.POINTER(i)]),
            "orc_adjoint_solve": (i, [P, _dp, _dp, d, i, _dp, C.POINTER(i)]),
            "orc_sens_full": (i, [P, _dp, _dp, i, _dp, _dp]),
            "orc_sens_nod": (i, [_dp, _dp, _dp, _dp, _dp]),
            "orc_sens_paper": (i, [P, _dp, _dp, i, _dp, _dp, _dp, _dp]),
            "orc_wall_face_functional": (d, [_dp, i, _dp, _dp, _dp, _dp, d, _dp]),
            "orc_diagonal": (i, [P, _dp, _dp]),
            "orc_jacobi_cells": (i, [P, _dp, i, C.POINTER(C.c_int), _dp]),
            "orc_volume_constraint": (d, [P, d, i, _dp, _dp, _dp]),
            "orc_adjoint_jacobi_cells": (i, [P, _dp, _dp, i, C.POINTER(C.c_int), _dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """One discrete problem: O-mesh nodes, velocity grid, flow, and the moment of J (Eq. formula_opt):
    m_J(v) = d . v + h |v|^2 / 2 for direction = (dx, dy) (h = 0: a force, drag = (1, 0)) or
    (dx, dy, h) (heat: (0, 0, 1))."""

    def __init__(self, nodes, vx, vy, w, Kn, Ma, Tw=1.0, aoa=0.0, direction=(1.0, 0.0), conservative=False):
        self.nodes = _c(nodes)
        self.nj = self.nodes.shape[0] - 1
        self.ni = self.nodes.shape[1]
        self.vx, self.vy, self.w = _c(vx), _c(vy), _c(w)
        self.nv = self.vx.size
        self.Kn, self.Ma, self.Tw, self.aoa = float(Kn), float(Ma), float(Tw), float(aoa)
        self.direction = _moment(direction)
        self.conservative = bool(conservative)
        self._s = _Problem(self.ni, self.nj, self.nv, _ptr(self.nodes), _ptr(self.vx),
                           _ptr(self.vy), _ptr(self.w), self.Kn, self.Ma, self.Tw, self.aoa,
                           (C.c_double * 3)(*self.direction), int(self.conservative))

    @classmethod
    def from_workload(cls, wl, direction=(1.0, 0.0), conservative=False):
        return cls(wl.mesh.nodes, wl.grid.vx, wl.grid.vy, wl.grid.w, wl.flow.Kn, wl.flow.Ma,
                   wl.flow.Tw, wl.flow.aoa, direction, conservative)

    @property
    def ncell(self):
        return self.ni * self.nj

    @property
    def ref(self):
        return C.byref(self._s)

    def fshape(self):
        return (self.ncell, self.nv, 2)

    # ---------------------------------------------------------------- geometry / state
    def geometry(self):
        V = np.zeros(self.ncell)
        S = np.zeros((self.ncell, 4, 2))
        lib().orc_geometry(self.ref, _ptr(V), _ptr(S))
        return V, S

    def freestream(self):
        f = np.zeros(self.fshape())
        lib().orc_freestream(self.ref, _ptr(f))
        return f

    def moments(self, f):
        f = _c(f)
        W = np.zeros((self.ncell, 4))
        lib().orc_moments(self.ref, _ptr(f), _ptr(W))
        return W

    def collision(self, f):
        f = _c(f)
        Q = np.zeros(self.fshape())
        lib().orc_collision(self.ref, _ptr(f), _ptr(Q))
        return Q

    # ---------------------------------------------------------------- residual / functional
    def residual(self, f):
        f = _c(f)
        R = np.zeros(self.fshape())
        nrm = C.c_double()
        lib().orc_residual(self.ref, _ptr(f), _ptr(R), C.byref(nrm))
        return R, nrm.value

    def residual_dir(self, f, df):
        f, df = _c(f), _c(df)
        R = np.zeros(self.fshape())
        dR = np.zeros(self.fshape())
        lib().orc_residual_dir(self.ref, _ptr(f), _ptr(df), _ptr(R), _ptr(dR))
        return R, dR

    def functional(self, f):
        return lib().orc_functional(self.ref, _ptr(_c(f)))

    def functional_dir(self, f, df):
        J, dJ = C.c_double(), C.c_double()
        lib().orc_functional_dir(self.ref, _ptr(_c(f)), _ptr(_c(df)), C.byref(J), C.byref(dJ))
        return J.value, dJ.value

    def functional_grad(self, f):
        g = np.zeros(self.fshape())
        lib().orc_functional_grad(self.ref, _ptr(_c(f)), _ptr(g))
        return g

    def apply_RT(self, f, lam):
        out = np.zeros(self.fshape())
        lib().orc_apply_RT(self.ref, _ptr(_c(f)), _ptr(_c(lam)), _ptr(out))
        return out

    # ---------------------------------------------------------------- iterations and solves
    def diagonal(self, f):
        """Point-implicit diagonal D = V/tau + sum_e max(a_e, 0), [ncell, nv]."""
        D = np.zeros((self.ncell, self.nv))
        lib().orc_diagonal(self.ref, _ptr(_c(f)), _ptr(D))
        return D

    def jacobi(self, f):
        f = _c(f)
        fn = np.zeros(self.fshape())
        nrm = C.c_double()
        lib().orc_jacobi(self.ref, _ptr(f), _ptr(fn), C.byref(nrm))
        return fn, nrm.value

    def adjoint_jacobi(self, f, phi):
        out = np.zeros(self.fshape())
        nrm = C.c_double()
        lib().orc_adjoint_jacobi(self.ref, _ptr(_c(f)), _ptr(_c(phi)), _ptr(out), C.byref(nrm))
        return out, nrm.value

    def jacobi_cells(self, f, cells):
        """Point-implicit update of the listed cells only: [len(cells), nv, 2]."""
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        out = np.zeros((cells.size, self.nv, 2))
        lib().orc_jacobi_cells(self.ref, _ptr(_c(f)), cells.size, cells.ctypes.data_as(C.POINTER(C.c_int)),
                               _ptr(out))
        return out

    def adjoint_jacobi_cells(self, f, phi, cells):
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        out = np.zeros((cells.size, self.nv, 2))
        lib().orc_adjoint_jacobi_cells(self.ref, _ptr(_c(f)), _ptr(_c(phi)), cells.size,
                                       cells.ctypes.data_as(C.POINTER(C.c_int)), _ptr(out))
        return out

    def primal_solve(self, tol=1e-12, max_sweeps=20000, f0=None):
        f = self.freestream() if f0 is None else _c(f0).copy()
        rel, sw = C.c_double(), C.c_int()
        st = lib().orc_primal_solve(self.ref, _ptr(f), tol, max_sweeps, C.byref(rel), C.byref(sw))
        return f, {"status": st, "rel": rel.value, "sweeps": sw.value}

    def adjoint_solve(self, f, tol=1e-12, max_sweeps=20000, phi0=None):
        phi = np.zeros(self.fshape()) if phi0 is None else _c(phi0).copy()
        rel, sw = C.c_double(), C.c_int()
        st = lib().orc_adjoint_solve(self.ref, _ptr(_c(f)), _ptr(phi), tol, max_sweeps,
                                     C.byref(rel), C.byref(sw))
        return phi, {"status": st, "rel": rel.value, "sweeps": sw.value}

    # ---------------------------------------------------------------- sensitivities
    def sens_full(self, f, phi, dnodes):
        dnodes = _c(dnodes)
        P = dnodes.shape[0]
        g = np.zeros(P)
        lib().orc_sens_full(self.ref, _ptr(_c(f)), _ptr(_c(phi)), P, _ptr(dnodes), _ptr(g))
        return g

    def volume_constraint(self, vmin, dwall):
        """Q = (1/2) sum_l x_l . n_l A_l + V_min and dQ/dx (wall nodes), dQ/dalpha."""
        dwall = _c(dwall)
        P = dwall.shape[0]
        dQ = np.zeros((self.ni, 2))
        dQda = np.zeros(max(P, 1))
        Q = lib().orc_volume_constraint(self.ref, float(vmin), P, _ptr(dwall), _ptr(dQ), _ptr(dQda))
        return Q, dQ, dQda[:P]

    def sens_paper(self, f, phi, dwall):
        dwall = _c(dwall)
        P = dwall.shape[0]
        g = np.zeros(P)
        ng = np.zeros((self.ni, 2))
        el = np.zeros((self.ni, 5))
        lib().orc_sens_paper(self.ref, _ptr(_c(f)), _ptr(_c(phi)), P, _ptr(dwall), _ptr(g),
                             _ptr(ng), _ptr(el))
        return g, ng, el


def threads(n: int = 0) -> int:
    return lib().orc_threads(n)


def sens_nod(xa, xb, n):
    dA = np.zeros(2)
    dn = np.zeros((2, 2))
    lib().orc_sens_nod(_ptr(_c(xa)), _ptr(_c(xb)), _ptr(_c(n)), _ptr(dA), _ptr(dn))
    return dA, dn


def wall_face_functional(S, vx, vy, w, f1, Tw=1.0, direction=(1.0, 0.0)):
    vx, vy, w, f1 = _c(vx), _c(vy), _c(w), _c(f1)
    return lib().orc_wall_face_functional(_ptr(_c(S)), vx.size, _ptr(vx), _ptr(vy), _ptr(w),
                                          _ptr(f1), Tw, _ptr(_c(_moment(direction))))


def _moment(direction):
    d = tuple(float(x) for x in direction)
    if len(d) not in (2, 3):
        raise ValueError("direction is (dx, dy) or (dx, dy, h)")
    return d + (0.0,) * (3 - len(d))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
