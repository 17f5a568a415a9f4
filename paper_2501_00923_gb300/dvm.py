"""Thin Python binding of the C ABI in include/dvm.h (ctypes; argument marshalling only).

Every step of the DVM path runs in the CUDA library libdvm.so.  If the library is missing this
module raises at import time of the library (no CPU fallback exists).
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdvm.so")

DVM_OK, DVM_ERR_INVALID_ARG, DVM_ERR_OOM, DVM_ERR_ADMISSION = 0, 1, 2, 3
DVM_NOT_CONVERGED, DVM_ERR_NONFINITE, DVM_ERR_CUDA, DVM_ERR_TIMEOUT, DVM_ERR_STAGNATED = 4, 5, 6, 7, 8
STORAGE = {"fp64": 0, "fp32": 1, "bf16": 2}
FUNCTIONAL = {"drag": 0, "lift": 1, "heat": 2}
SENS = {"paper": 0, "full": 1}

_dp = C.POINTER(C.c_double)
_vp = C.c_void_p


class Options(C.Structure):
    _fields_ = [("graph_iters", C.c_int), ("hbm_budget", C.c_size_t), ("stream", C.c_void_p), ("flags", C.c_int)]


DVM_OPT_NO_GRAPHS = 1


class Flow(C.Structure):
    _fields_ = [("Kn", C.c_double), ("Ma", C.c_double), ("Tw", C.c_double), ("aoa", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("stall_window", C.c_int), ("accel_depth", C.c_int),
                ("accel_period", C.c_int), ("accel_space", C.c_int), ("refine_tol", C.c_double),
                ("refine_max", C.c_int), ("refine_sweeps", C.c_int), ("predict_omega", C.c_double),
                ("predict_iters", C.c_int), ("predict_reuse", C.c_int), ("predict_precond", C.c_int)]


def _accel(accel):
    """accel: None (plain sweeps), (depth m, period K) of the Anderson mixing of the state, or
    (m, K, "moments") to mix the primal's cell moments instead."""
    if accel is None:
        return 0, 0, 0
    m, k = accel[0], accel[1]
    space = accel[2] if len(accel) > 2 else "state"
    return int(m), int(k), {"state": 0, "moments": 1}[space]


class PrimalResult(C.Structure):
    _fields_ = [("J", C.c_double), ("Cd", C.c_double), ("residual", C.c_double), ("r0", C.c_double),
                ("iters", C.c_int), ("status", C.c_int), ("refine_steps", C.c_int), ("refine_sweeps", C.c_int),
                ("residual_fp32", C.c_double), ("residual_fp64", C.c_double), ("predictions", C.c_int)]


class AdjointResult(C.Structure):
    _fields_ = [("residual", C.c_double), ("r0", C.c_double), ("iters", C.c_int), ("status", C.c_int),
                ("predictions", C.c_int)]


class DVMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libdvm.so (built by paper_2501_00923_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2501_00923_gb300.build.build() "
                              "(the DVM path has no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        i, d, s, u64 = C.c_int, C.c_double, C.c_size_t, C.c_uint64
        pp = C.POINTER(C.c_void_p)
        sig = {
            "dvm_context_create": (i, [pp, i, C.POINTER(Options)]),
            "dvm_context_destroy": (None, [_vp]),
            "dvm_context_bytes": (s, [_vp]),
            "dvm_context_launches": (u64, [_vp]),
            "dvm_context_allocations": (u64, [_vp]),
            "dvm_selftest_wait_timeout": (i, [_vp]),
            "dvm_status_string": (C.c_char_p, [i]),
            "dvm_last_error": (C.c_char_p, []),
            "dvm_mesh_create": (i, [_vp, i, i, _dp, pp]),
            "dvm_mesh_destroy": (None, [_vp]),
            "dvm_vgrid_create": (i, [_vp, i, _dp, _dp, _dp, pp]),
            "dvm_vgrid_destroy": (None, [_vp]),
            "dvm_state_create": (i, [_vp, _vp, _vp, C.POINTER(Flow), i, pp]),
            "dvm_state_destroy": (None, [_vp]),
            "dvm_state_set": (i, [_vp, _dp]),
            "dvm_state_get": (i, [_vp, _dp]),
            "dvm_state_copy_from": (i, [_vp, _vp]),
            "dvm_state_set_shard": (i, [_vp, i]),
            "dvm_state_shard_count": (s, [_vp]),
            "dvm_state_shard_partials": (i, [_vp, _dp, s]),
            "dvm_state_shard_combine": (i, [_vp, _dp, s, _dp, _dp]),
            "dvm_state_moments": (i, [_vp, _dp]),
            "dvm_state_set_order": (i, [_vp, i, i]),
            "dvm_state_get_order": (i, [_vp, C.POINTER(i)]),
            "dvm_state_set_maxwellian": (i, [_vp, i]),
            "dvm_state_get_maxwellian": (i, [_vp, C.POINTER(i)]),
            "dvm_primal_iterate": (i, [_vp, i, _dp]),
            "dvm_state_functional": (i, [_vp, i, _dp]),
            "dvm_primal_solve": (i, [_vp, _vp, _vp, C.POINTER(Flow), C.POINTER(SolveOpts), i, pp,
                                     C.POINTER(PrimalResult)]),
            "dvm_adjoint_create": (i, [_vp, i, pp]),
            "dvm_adjoint_destroy": (None, [_vp]),
            "dvm_adjoint_set": (i, [_vp, _dp]),
            "dvm_adjoint_get": (i, [_vp, _dp]),
            "dvm_adjoint_copy_from": (i, [_vp, _vp]),
            "dvm_adjoint_iterate": (i, [_vp, i, _dp]),
            "dvm_adjoint_solve": (i, [_vp, _vp, i, C.POINTER(SolveOpts), pp, C.POINTER(AdjointResult)]),
            "dvm_sensitivity": (i, [_vp, _vp, _vp, i, _dp, _dp, i, _dp, _dp]),
            "dvm_sensitivity_noalloc": (i, [_vp, _vp, _vp, i, _dp, _dp, i, _dp, _dp]),
            "dvm_volume_constraint": (i, [_vp, _vp, d, i, _dp, _dp, _dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(st: int) -> str:
    return lib().dvm_status_string(st).decode()


def last_error() -> str:
    return lib().dvm_last_error().decode()


def _check(st: int, ok=(DVM_OK,)):
    if st not in ok:
        raise DVMError(st, last_error())
    return st


def _arr(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


# ----------------------------------------------------------------------------------- handles
class Context:
    def __init__(self, device: int = 0, graph_iters: int = 20, hbm_budget: int = 0, stream=None,
                 graphs: bool = True):
        h = C.c_void_p()
        opt = Options(graph_iters, hbm_budget, stream, 0 if graphs else DVM_OPT_NO_GRAPHS)
        _check(lib().dvm_context_create(C.byref(h), device, C.byref(opt)))
        self.h = h
        self.device = device
        self._children = weakref.WeakSet()

    def _adopt(self, obj):
        self._children.add(obj)

    def close(self):
        """Release every live handle of this context (batch servers, adjoints, states, then meshes
        and grids), then the context itself."""
        if self.h:
            for rank in (4, 3, 2, 1):
                for ch in list(self._children):
                    if getattr(ch, "_rank", 0) == rank:
                        ch.close()
            lib().dvm_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def bytes(self) -> int:
        return lib().dvm_context_bytes(self.h)

    @property
    def launches(self) -> int:
        return lib().dvm_context_launches(self.h)

    @property
    def allocations(self) -> int:
        """Device allocations made for this context so far (pool blocks, transient ones included)."""
        return lib().dvm_context_allocations(self.h)


class Mesh:
    _rank = 1

    def __init__(self, ctx: Context, nodes: np.ndarray):
        nodes = _arr(nodes)
        self.nj, self.ni = nodes.shape[0] - 1, nodes.shape[1]
        self.ctx = ctx
        h = C.c_void_p()
        _check(lib().dvm_mesh_create(ctx.h, self.ni, self.nj, _p(nodes), C.byref(h)))
        self.h = h
        ctx._adopt(self)

    @property
    def ncell(self):
        return self.ni * self.nj

    def close(self):
        if self.h:
            lib().dvm_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class VGrid:
    _rank = 1

    def __init__(self, ctx: Context, vx, vy, w):
        vx, vy, w = _arr(vx), _arr(vy), _arr(w)
        self.nv = vx.size
        self.ctx = ctx
        h = C.c_void_p()
        _check(lib().dvm_vgrid_create(ctx.h, self.nv, _p(vx), _p(vy), _p(w), C.byref(h)))
        self.h = h
        ctx._adopt(self)

    def close(self):
        if self.h:
            lib().dvm_vgrid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """Primal distribution f of one (mesh, velocity grid, flow) on the device."""

    _rank = 2

    def __init__(self, ctx: Context, mesh: Mesh, grid: VGrid, Kn, Ma, Tw=1.0, aoa=0.0, storage="fp32",
                 _handle=None):
        self.ctx, self.mesh, self.grid = ctx, mesh, grid
        self.flow = Flow(Kn, Ma, Tw, aoa)
        self.storage = storage
        if _handle is not None:
            self.h = _handle
        else:
            h = C.c_void_p()
            _check(lib().dvm_state_create(ctx.h, mesh.h, grid.h, C.byref(self.flow), STORAGE[storage], C.byref(h)))
            self.h = h
        ctx._adopt(self)

    def shape(self):
        return (self.mesh.ncell, self.grid.nv, 2)

    def set(self, f):
        f = _arr(f, self.shape())
        _check(lib().dvm_state_set(self.h, _p(f)))

    def get(self):
        f = np.empty(self.shape())
        _check(lib().dvm_state_get(self.h, _p(f)))
        return f

    # ---------------------------------------------------------------- velocity shards
    def set_shard(self, on: bool = True):
        """Make this state a velocity shard (its grid is a slice of the velocity grid): its sweeps
        write partial sums, combined across shards with shard_combine."""
        _check(lib().dvm_state_set_shard(self.h, int(bool(on))))

    def shard_partials(self, out=None):
        """This shard's partial sums: into a new host array, or into `out` (a host array or the data
        pointer, an int, of device memory holding shard_count doubles)."""
        n = lib().dvm_state_shard_count(self.h)
        if out is None:
            out = np.empty(n)
        if isinstance(out, int):
            _check(lib().dvm_state_shard_partials(self.h, C.cast(out, _dp), n))
            return None
        _check(lib().dvm_state_shard_partials(self.h, _p(out), n))
        return out

    def shard_combine(self, total):
        """Install the summed partials of all shards (host array, or device data pointer as an int);
        returns (residual sum of squares of the last sweep's input, drag of the current f)."""
        n = lib().dvm_state_shard_count(self.h)
        r, J = C.c_double(), C.c_double()
        host = None if isinstance(total, int) else _arr(total, (n,))     # kept alive over the call
        ptr = C.cast(total, _dp) if host is None else _p(host)
        _check(lib().dvm_state_shard_combine(self.h, ptr, n, C.byref(r), C.byref(J)))
        return r.value, J.value

    def copy_from(self, other: "State"):
        """Device-to-device warm start: f of `other` (same shape and storage) becomes this state's f."""
        _check(lib().dvm_state_copy_from(self.h, other.h))

    def moments(self):
        m = np.empty((self.mesh.ncell, 4))
        _check(lib().dvm_state_moments(self.h, _p(m)))
        return m

    def iterate(self, n: int):
        r = np.empty(max(n, 1))
        _check(lib().dvm_primal_iterate(self.h, n, _p(r)))
        return r[:n]

    @property
    def order(self) -> int:
        """Spatial order of the face values (1 upwind, 2 linear reconstruction)."""
        o = C.c_int()
        _check(lib().dvm_state_get_order(self.h, C.byref(o)))
        return o.value

    @order.setter
    def order(self, order: int):
        self.set_order(order)

    @property
    def maxwellian(self) -> str:
        """Cell Maxwellian of the collision term: "plain" or "conservative" (fitted moments)."""
        k = C.c_int()
        _check(lib().dvm_state_get_maxwellian(self.h, C.byref(k)))
        return ("plain", "conservative")[k.value]

    @maxwellian.setter
    def maxwellian(self, kind: str):
        _check(lib().dvm_state_set_maxwellian(self.h, {"plain": 0, "conservative": 1}[kind]))

    def set_order(self, order: int, defect_period: int = 0):
        """order 2: linear reconstruction with the defect frozen over groups of defect_period sweeps
        (0 -> 20); order 1: first-order upwind."""
        _check(lib().dvm_state_set_order(self.h, int(order), int(defect_period)))

    def functional(self, which="drag"):
        J = C.c_double()
        _check(lib().dvm_state_functional(self.h, FUNCTIONAL[which], C.byref(J)))
        return J.value

    def close(self):
        if self.h:
            lib().dvm_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Adjoint:
    """Adjoint phi of a State, linearised at the state's f when created: advance the state only
    after the adjoint work that needs that f is done."""

    _rank = 3

    def __init__(self, state: State, functional="drag", _handle=None):
        self.state = state
        self.functional = functional
        if _handle is not None:
            self.h = _handle
        else:
            h = C.c_void_p()
            _check(lib().dvm_adjoint_create(state.h, FUNCTIONAL[functional], C.byref(h)))
            self.h = h
        state.ctx._adopt(self)

    def set(self, phi):
        phi = _arr(phi, self.state.shape())
        _check(lib().dvm_adjoint_set(self.h, _p(phi)))

    def get(self):
        phi = np.empty(self.state.shape())
        _check(lib().dvm_adjoint_get(self.h, _p(phi)))
        return phi

    def copy_from(self, other: "Adjoint"):
        """Device-to-device warm start: phi of `other` (same shape and storage) becomes this adjoint's phi."""
        _check(lib().dvm_adjoint_copy_from(self.h, other.h))

    def iterate(self, n: int):
        r = np.empty(max(n, 1))
        _check(lib().dvm_adjoint_iterate(self.h, n, _p(r)))
        return r[:n]

    def close(self):
        if self.h:
            lib().dvm_adjoint_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------------- calls
def primal_solve(ctx: Context, mesh: Mesh, grid: VGrid, Kn, Ma, Tw=1.0, aoa=0.0, tol=1e-8, max_iter=100000,
                 storage="fp32", state: State | None = None, stall_window=0, accel=None, refine_tol=0.0,
                 refine_max=0, refine_sweeps=0, predict=0, predict_omega=0.0, predict_reuse=0, predict_precond=0):
    """Steady solve of Eq. (numerpr_gov); warm-starts from `state` if given.  accel = (m, K) turns on
    Anderson mixing of depth m every K sweeps.  predict > 0 turns on the macroscopic prediction after every
    block of sweeps (that many GMRES steps on the moment system; predict_precond = 1 preconditions them
    with a multigrid V-cycle instead of the diagonal blocks).  refine_tol > 0 (FP32
    storage) adds mixed-precision refinement to that FP64 residual after the sweeps.  Returns (state, result)."""
    flow = Flow(Kn, Ma, Tw, aoa)
    opts = SolveOpts(tol, max_iter, stall_window, *_accel(accel), refine_tol, refine_max, refine_sweeps,
                     predict_omega, predict, predict_reuse, predict_precond)
    h = C.c_void_p(state.h.value if state is not None else None)
    res = PrimalResult()
    st = lib().dvm_primal_solve(ctx.h, mesh.h, grid.h, C.byref(flow), C.byref(opts), STORAGE[storage],
                                C.byref(h), C.byref(res))
    if state is None and h.value:
        state = State(ctx, mesh, grid, Kn, Ma, Tw, aoa, storage, _handle=h)
    _check(st, ok=(DVM_OK, DVM_NOT_CONVERGED, DVM_ERR_STAGNATED))
    return state, res


def adjoint_solve(ctx: Context, state: State, functional="drag", tol=1e-8, max_iter=100000,
                  adjoint: Adjoint | None = None, stall_window=0, accel=None, predict=0, predict_omega=0.0,
                  predict_precond=0):
    """Steady solve of the discrete adjoint for `functional`; accel and predict as in primal_solve (the
    prediction by the transposed moment system)."""
    opts = SolveOpts(tol, max_iter, stall_window, *_accel(accel), 0.0, 0, 0, predict_omega, predict, 0, predict_precond)
    h = C.c_void_p(adjoint.h.value if adjoint is not None else None)
    res = AdjointResult()
    st = lib().dvm_adjoint_solve(ctx.h, state.h, FUNCTIONAL[functional], C.byref(opts), C.byref(h), C.byref(res))
    if adjoint is None and h.value:
        adjoint = Adjoint(state, functional, _handle=h)
    _check(st, ok=(DVM_OK, DVM_NOT_CONVERGED, DVM_ERR_STAGNATED))
    return adjoint, res


def sensitivity(ctx: Context, state: State, adjoint: Adjoint, dwall_dalpha, s_j=None, mode="full",
                node_grad: bool = False, noalloc: bool = False):
    """dJ/dalpha for wall-node tangents dwall_dalpha [P][ni][2] (interior nodes move by (1-s_j)).
    noalloc=True calls dvm_sensitivity_noalloc, which keeps its scratch in a static device array."""
    dwall = _arr(dwall_dalpha)
    P = dwall.shape[0]
    ni, nj = state.mesh.ni, state.mesh.nj
    if dwall.shape != (P, ni, 2):
        raise ValueError(f"dwall_dalpha must be [P, {ni}, 2]")
    sj = None if s_j is None else _arr(s_j)
    if mode == "full" and (sj is None or sj.shape != (nj + 1,)):
        raise ValueError("full mode needs s_j of length nj+1")
    g = np.zeros(max(P, 1))
    ng = None
    if node_grad:
        ng = np.zeros((ni, 2)) if mode == "paper" else np.zeros((nj + 1, ni, 2))
    fn = lib().dvm_sensitivity_noalloc if noalloc else lib().dvm_sensitivity
    _check(fn(ctx.h, state.h, adjoint.h, P, _p(dwall), _p(sj), SENS[mode], _p(g), _p(ng)))
    return (g[:P], ng) if node_grad else g[:P]


def volume_constraint(ctx: Context, mesh: Mesh, v_min: float, dwall_dalpha):
    """Q = (1/2) sum over wall elements of x . n A + V_min (n into the solid) and dQ/dalpha."""
    dwall = _arr(dwall_dalpha)
    P = dwall.shape[0]
    Q = C.c_double()
    g = np.zeros(max(P, 1))
    _check(lib().dvm_volume_constraint(ctx.h, mesh.h, float(v_min), P, _p(dwall), C.byref(Q), _p(g)))
    return Q.value, g[:P]
