"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module holds none of the DVM method's arithmetic (no moments, Maxwellians, fluxes, cell
geometry or adjoint terms).  It only places points:

* the airfoil surface: the public NACA 4-digit symmetric thickness law with the closed
  (sharp) trailing edge, as used for the initial shapes of Sec. 4.2 and Sec. 4.3;
* the Hicks-Henne bump basis that moves the surface vertically with the horizontal
  coordinate held fixed (the fixed-xi assumption of Sec. 3.3);
* a structured O-mesh: wall nodes (i periodic, counter-clockwise, upper surface first),
  far-field circle of radius 10 chords centred at mid-chord, and an algebraic radial blend
  x(i,j) = x_w(i) + s_j (x_ff(i) - x_w(i)) with geometric growth from a first spacing of
  1e-3 chord (the first-layer height of Sec. 4.2);
* velocity quadratures (uniform trapezoid or Gauss-Legendre per axis) in units of the
  free-stream sound speed a_inf = sqrt(5/3) (rho_inf = 1, R T_inf = 1, monatomic gamma = 5/3);
* the five workload recipes and a request-trace generator for the serving workload.

Everything is a pure function of its arguments and a numpy seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

A_INF = math.sqrt(5.0 / 3.0)      # free-stream sound speed for rho=1, RT=1, gamma=5/3
SEED_BASE = 20250923


# --------------------------------------------------------------------------- airfoil surface
def naca4_thickness(x: np.ndarray, t: float = 0.12) -> np.ndarray:
    """Half thickness of the symmetric NACA 4-digit section, closed trailing edge.

    Public NACA definition with the x^4 coefficient -0.1036, which closes the section at x=1.
    """
    x = np.clip(np.asarray(x, dtype=np.float64), 0.0, 1.0)
    return 5.0 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x**2
                      + 0.2843 * x**3 - 0.1036 * x**4)


def hicks_henne_basis(xi: np.ndarray, n_per_side: int, power: int = 3) -> np.ndarray:
    """Hicks-Henne bumps b_p(xi) = sin(pi xi^{m_p})^power, peaks h_p spread by a cosine law.

    Returns an array [n_per_side, len(xi)].  b_p vanishes at xi=0 and xi=1, so the leading and
    trailing edges never move.
    """
    xi = np.clip(np.asarray(xi, dtype=np.float64), 0.0, 1.0)
    p = np.arange(1, n_per_side + 1, dtype=np.float64)
    h = 0.5 * (1.0 - np.cos(np.pi * p / (n_per_side + 1)))
    m = np.log(0.5) / np.log(h)
    with np.errstate(divide="ignore", invalid="ignore"):
        b = np.sin(np.pi * xi[None, :] ** m[:, None]) ** power
    return np.where(np.isfinite(b), b, 0.0)


def wall_nodes(ni: int, alpha: np.ndarray, thickness: float = 0.12):
    """Wall nodes of the O-mesh and their derivative with respect to the bump amplitudes.

    Node m sits at theta_m = 2 pi m / ni, xi_m = (1 + cos theta_m)/2 (m=0 is the trailing edge),
    counter-clockwise with the upper surface first.  The first half of ``alpha`` thickens the
    upper surface (+b_p), the second half the lower surface (-b_p): positive amplitude thickens.

    Returns (xw [ni,2], dxw [P, ni, 2]).
    """
    alpha = np.asarray(alpha, dtype=np.float64).reshape(-1)
    P = alpha.size
    if P % 2:
        raise ValueError("the number of bump amplitudes must be even (upper/lower pairs)")
    theta = 2.0 * np.pi * np.arange(ni) / ni
    xi = 0.5 * (1.0 + np.cos(theta))
    side = np.sign(np.round(np.sin(theta), 14))            # +1 upper, -1 lower, 0 at LE/TE
    yt = naca4_thickness(xi, thickness)
    xw = np.stack([xi, side * yt], axis=1)
    dxw = np.zeros((P, ni, 2))
    if P:
        b = hicks_henne_basis(xi, P // 2)
        up = side > 0
        lo = side < 0
        for p in range(P // 2):
            dxw[p, up, 1] = b[p, up]
            dxw[P // 2 + p, lo, 1] = -b[p, lo]
        xw = xw + np.einsum("p,pmc->mc", alpha, dxw)
    return xw, dxw


def far_nodes(ni: int, radius: float = 10.0, center=(0.5, 0.0)) -> np.ndarray:
    theta = 2.0 * np.pi * np.arange(ni) / ni
    return np.stack([center[0] + radius * np.cos(theta), center[1] + radius * np.sin(theta)], 1)


def radial_blend(nj: int, first: float = 1e-3, radius: float = 10.0) -> np.ndarray:
    """s_j = (q^j - 1)/(q^nj - 1), q found by bisection so that s_1 * radius = first."""
    target = first / radius
    if nj == 1:
        return np.array([0.0, 1.0])
    lin = 1.0 / nj
    if target >= lin:                      # uniform spacing already coarse enough
        return np.linspace(0.0, 1.0, nj + 1)
    lo, hi = 1.0 + 1e-12, 10.0
    for _ in range(200):
        q = 0.5 * (lo + hi)
        s1 = (q - 1.0) / (q**nj - 1.0)
        if s1 > target:
            lo = q
        else:
            hi = q
    q = 0.5 * (lo + hi)
    j = np.arange(nj + 1, dtype=np.float64)
    s = (q**j - 1.0) / (q**nj - 1.0)
    s[0], s[-1] = 0.0, 1.0
    return s


@dataclass
class OMesh:
    ni: int
    nj: int
    nodes: np.ndarray        # [(nj+1), ni, 2]; j=0 on the wall, j=nj on the far field
    s: np.ndarray            # [nj+1] radial blend
    dwall: np.ndarray        # [P, ni, 2] d(wall nodes)/d(alpha)
    alpha: np.ndarray        # [P]

    @property
    def ncell(self) -> int:
        return self.ni * self.nj

    def dnodes(self) -> np.ndarray:
        """d(all nodes)/d(alpha) [P, nj+1, ni, 2] under the radial blend."""
        return (1.0 - self.s)[None, :, None, None] * self.dwall[:, None, :, :]


def omesh(ni: int, nj: int, alpha=None, first: float = 1e-3, radius: float = 10.0,
          thickness: float = 0.12) -> OMesh:
    alpha = np.zeros(8) if alpha is None else np.asarray(alpha, dtype=np.float64)
    xw, dxw = wall_nodes(ni, alpha, thickness)
    xf = far_nodes(ni, radius)
    s = radial_blend(nj, first, radius)
    nodes = xw[None, :, :] + s[:, None, None] * (xf - xw)[None, :, :]
    return OMesh(ni, nj, np.ascontiguousarray(nodes), s, dxw, alpha)


# --------------------------------------------------------------------------- CST parameterisation
CST_NB = 6


def cst_count(nb: int = CST_NB) -> int:
    """Design variables of the CST section: N1, N2, A_u[0..nb], A_l[0..nb], eta_T,u, eta_T,l."""
    return 2 * nb + 6


def _bernstein(xi: np.ndarray, nb: int) -> np.ndarray:
    """S_beta(xi) = C(nb, beta) xi^beta (1 - xi)^(nb - beta), [nb+1, len(xi)]."""
    return np.stack([math.comb(nb, b) * xi ** b * (1.0 - xi) ** (nb - b) for b in range(nb + 1)])


def cst_wall_nodes(ni: int, params, nb: int = CST_NB):
    """Wall nodes of the CST section (Sec. 3.3, Eq. cstsuf, cst_classfunc, cst_shapefunc) at the
    fixed abscissae of the O-mesh, xi_m = (1 + cos theta_m)/2, upper surface first, and their
    derivatives with respect to the design variables.

    eta = C(xi) S(xi) + xi eta_T with C = xi^N1 (1 - xi)^N2 and S = sum_beta A_beta S_beta(xi) on each
    surface; params = (N1, N2, A_u[0..nb], A_l[0..nb], eta_T,u, eta_T,l).  x stays fixed (only eta
    moves).  dC/dN1 = ln(xi) C and dC/dN2 = ln(1 - xi) C vanish where C does (xi = 0 or 1 with N > 0).

    Returns (xw [ni,2], dxw [2nb+6, ni, 2]).
    """
    q = np.asarray(params, dtype=np.float64).reshape(-1)
    if q.size != cst_count(nb):
        raise ValueError(f"CST with nb={nb} has {cst_count(nb)} design variables")
    N1, N2 = q[0], q[1]
    Au, Al = q[2:3 + nb], q[3 + nb:4 + 2 * nb]
    tu, tl = q[4 + 2 * nb], q[5 + 2 * nb]
    theta = 2.0 * np.pi * np.arange(ni) / ni
    xi = 0.5 * (1.0 + np.cos(theta))
    xi = np.clip(xi, 0.0, 1.0)
    side = np.sign(np.round(np.sin(theta), 14))
    up = side > 0
    lo = side < 0
    Bs = _bernstein(xi, nb)
    with np.errstate(divide="ignore", invalid="ignore"):
        C = np.where((xi > 0) & (xi < 1), xi ** N1 * (1.0 - xi) ** N2, 0.0)
        l1 = np.where(xi > 0, np.log(np.where(xi > 0, xi, 1.0)), 0.0)
        l2 = np.where(xi < 1, np.log(np.where(xi < 1, 1.0 - xi, 1.0)), 0.0)
    Su, Sl = Au @ Bs, Al @ Bs
    eta = np.zeros(ni)
    eta[up] = C[up] * Su[up] + xi[up] * tu
    eta[lo] = C[lo] * Sl[lo] + xi[lo] * tl
    P = cst_count(nb)
    d = np.zeros((P, ni))
    d[0, up] = l1[up] * C[up] * Su[up]
    d[0, lo] = l1[lo] * C[lo] * Sl[lo]
    d[1, up] = l2[up] * C[up] * Su[up]
    d[1, lo] = l2[lo] * C[lo] * Sl[lo]
    d[2:3 + nb][:, up] = C[up] * Bs[:, up]
    d[3 + nb:4 + 2 * nb][:, lo] = C[lo] * Bs[:, lo]
    d[4 + 2 * nb, up] = xi[up]
    d[5 + 2 * nb, lo] = xi[lo]
    xw = np.stack([xi, eta], 1)
    dxw = np.zeros((P, ni, 2))
    dxw[:, :, 1] = d
    return xw, dxw


def cst_fit(ni: int, target_eta: np.ndarray, nb: int = CST_NB, sharp_te: bool = True):
    """Eq. (cstini): the CST design variables whose nodes best fit the given wall ordinates (least
    squares over the nodes, xi fixed).  With N1, N2 fixed the fit is linear in A and eta_T; N1 and N2
    are then refined by Gauss-Newton on all variables.  sharp_te fixes eta_T = 0."""
    P = cst_count(nb)
    q = np.zeros(P)
    q[0], q[1] = 0.5, 1.0                          # round nose, sharp trailing edge
    free = np.ones(P, bool)
    if sharp_te:
        free[4 + 2 * nb:] = False
    for it in range(60):
        xw, dxw = cst_wall_nodes(ni, q, nb)
        r = xw[:, 1] - target_eta
        Jm = dxw[:, :, 1].T[:, free]
        if it == 0:                                   # linear stage: A only
            lin = free.copy()
            lin[:2] = False
            step = np.linalg.lstsq(dxw[:, :, 1].T[:, lin], -r, rcond=None)[0]
            q[lin] += step
            continue
        step = np.linalg.lstsq(Jm, -r, rcond=None)[0]
        q[free] += step
        q[0] = max(q[0], 0.01)
        q[1] = max(q[1], 0.01)
        if np.abs(step).max() < 1e-13:
            break
    return q


def omesh_from_wall(ni: int, nj: int, xw: np.ndarray, dxw: np.ndarray, alpha, first: float = 1e-3,
                    radius: float = 10.0) -> OMesh:
    xf = far_nodes(ni, radius)
    s = radial_blend(nj, first, radius)
    nodes = xw[None, :, :] + s[:, None, None] * (xf - xw)[None, :, :]
    return OMesh(ni, nj, np.ascontiguousarray(nodes), s, dxw, np.asarray(alpha, dtype=np.float64))


def omesh_cst(ni: int, nj: int, params, nb: int = CST_NB, first: float = 1e-3, radius: float = 10.0) -> OMesh:
    """O-mesh around the CST section of `params` (dwall = d(wall nodes)/d(params))."""
    xw, dxw = cst_wall_nodes(ni, params, nb)
    return omesh_from_wall(ni, nj, xw, dxw, params, first, radius)


def cst_naca(ni: int, nb: int = CST_NB, thickness: float = 0.12):
    """CST variables of the base section (symmetric NACA 4-digit thickness law) by Eq. (cstini)."""
    xw, _ = wall_nodes(ni, np.zeros(0), thickness)
    return cst_fit(ni, xw[:, 1], nb)


def ellipse_mesh(ni: int, nj: int, thickness: float, aoa_deg: float, first: float = 1e-3,
                 radius: float = 10.0) -> OMesh:
    """O-mesh around a thin ellipse of unit chord rotated by aoa (nose up), for the
    free-molecular check.  No shape parameters."""
    theta = 2.0 * np.pi * np.arange(ni) / ni
    x = 0.5 * np.cos(theta)
    y = 0.5 * thickness * np.sin(theta)
    a = math.radians(aoa_deg)
    xr = 0.5 + x * math.cos(a) + y * math.sin(a)
    yr = -x * math.sin(a) + y * math.cos(a)
    xw = np.stack([xr, yr], 1)
    xf = far_nodes(ni, radius)
    s = radial_blend(nj, first, radius)
    nodes = xw[None] + s[:, None, None] * (xf - xw)[None]
    return OMesh(ni, nj, np.ascontiguousarray(nodes), s, np.zeros((0, ni, 2)), np.zeros(0))


# --------------------------------------------------------------------------- velocity grids
@dataclass
class VGrid:
    vx: np.ndarray
    vy: np.ndarray
    w: np.ndarray

    @property
    def nv(self) -> int:
        return self.vx.size


def axis_rule(n: int, half_width: float, rule: str):
    if rule == "trapezoid":
        x = np.linspace(-half_width, half_width, n)
        h = x[1] - x[0]
        w = np.full(n, h)
        w[0] = w[-1] = 0.5 * h
    elif rule == "gauss":
        t, wt = np.polynomial.legendre.leggauss(n)
        x = half_width * t
        w = half_width * wt
    else:
        raise ValueError(rule)
    return x, w


def velocity_grid(n: int, range_ainf: float, rule: str = "trapezoid", ny: int | None = None) -> VGrid:
    """Tensor grid, vx fastest (k = iy*nx + ix), on [-L, L]^2 with L = range_ainf * a_inf."""
    ny = n if ny is None else ny
    L = range_ainf * A_INF
    x, wx = axis_rule(n, L, rule)
    y, wy = axis_rule(ny, L, rule)
    VX, VY = np.meshgrid(x, y, indexing="xy")
    W = np.outer(wy, wx)
    return VGrid(VX.reshape(-1).copy(), VY.reshape(-1).copy(), W.reshape(-1).copy())


def velocity_grid_explicit(vx, vy, w) -> VGrid:
    return VGrid(np.asarray(vx, np.float64).copy(), np.asarray(vy, np.float64).copy(),
                 np.asarray(w, np.float64).copy())


# --------------------------------------------------------------------------- flow + workloads
@dataclass
class Flow:
    Kn: float
    Ma: float
    Tw: float = 1.0          # wall temperature over free-stream temperature
    aoa: float = 0.0         # free-stream direction (radians)


@dataclass
class Workload:
    name: str
    mesh: OMesh
    grid: VGrid
    flow: Flow
    tol: float
    storage: str             # "fp64" | "fp32" | "bf16"
    extra: dict = field(default_factory=dict)

    @property
    def pairs(self) -> int:
        return self.mesh.ncell * self.grid.nv


def config(index: int) -> Workload:
    """The five workload recipes (index 0..4), seeded by SEED_BASE + index."""
    rng = np.random.default_rng(SEED_BASE + index)
    if index == 0:
        mesh = omesh(64, 32, np.zeros(8))
        return Workload("naca0012-omesh64x32-v16x16-Kn1-Ma0.5-fp64", mesh,
                        velocity_grid(16, 4.0, "trapezoid"), Flow(1.0, 0.5), 1e-8, "fp64")
    if index == 1:
        mesh = omesh(256, 128, rng.uniform(-0.005, 0.005, 16))
        return Workload("naca0012-16bumps-omesh256x128-gl48x48-Kn0.1-Ma0.8-fp32", mesh,
                        velocity_grid(48, 6.0, "gauss"), Flow(0.1, 0.8), 1e-6, "fp32")
    if index == 2:
        # U(-0.005, 0.005) amplitudes fold the 384-node section at its sharp trailing edge: scaled
        # by the same validity factor as the served requests
        raw = rng.uniform(-0.005, 0.005, 24)
        mesh = omesh(384, 192, raw * valid_amplitude_scale(384, raw))
        return Workload("naca0012-24bumps-omesh384x192-v64x64-Kn0.001-Ma2-fp32", mesh,
                        velocity_grid(64, 8.0, "trapezoid"), Flow(0.001, 2.0), 1e-6, "fp32")
    if index == 3:
        return Workload("served-trace-128", omesh(64, 32, np.zeros(24)),
                        velocity_grid(24, 4.0), Flow(0.1, 0.5), 1e-6, "fp32",
                        extra={"trace": request_trace(128, rng)})
    if index == 4:
        mesh = omesh(256, 128, np.zeros(24))
        return Workload("lbfgs-24bumps-omesh256x128-gl48x48", mesh,
                        velocity_grid(48, 6.0, "gauss"), Flow(0.1, 0.8), 1e-6, "bf16",
                        extra={"Kn_list": [0.01, 0.1, 1.0], "iters": 12})
    raise ValueError(index)


def range_for_mach(Ma: float) -> float:
    return 4.0 if Ma <= 0.6 else (6.0 if Ma <= 1.2 else 8.0)


def valid_amplitude_scale(ni: int, alpha: np.ndarray, keep: float = 0.5, margin: float = 0.75) -> float:
    """Largest factor <= 1 (times `margin`) by which `alpha` may be applied so that no wall node moves
    toward the chord by more than (1 - keep) of its local half-thickness.  Without such a bound,
    random bumps of 1% chord push a surface through the chord where the sharp trailing edge is
    thinner than the bump, the section self-intersects and the radial mesh lines cross."""
    alpha = np.asarray(alpha, dtype=np.float64)
    theta = 2.0 * np.pi * np.arange(ni) / ni
    xi = 0.5 * (1.0 + np.cos(theta))
    side = np.sign(np.round(np.sin(theta), 14))
    yt = naca4_thickness(xi)
    _, dxw = wall_nodes(ni, np.zeros_like(alpha))
    inward = -side * np.einsum("p,pm->m", alpha, dxw[:, :, 1])
    m = (side != 0) & (inward > 0)
    s = 1.0 if not m.any() else min(1.0, float(np.min((1.0 - keep) * yt[m] / inward[m])))
    return margin * s


def request_trace(n: int, rng: np.random.Generator, rate_hz: float = 20.0):
    """Served-solve requests: Poisson arrivals, random airfoil, Kn, Ma, mesh and velocity grid.
    Bump amplitudes are drawn U(-0.01, 0.01) and the vector is scaled by valid_amplitude_scale."""
    meshes = [(64, 32), (128, 64), (192, 96)]
    grids = [24, 32, 48]
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    out = []
    for r in range(n):
        ni, nj = meshes[rng.integers(3)]
        nv = grids[rng.integers(3)]
        Kn = 10.0 ** rng.uniform(-3.0, 1.0)
        Ma = rng.uniform(0.3, 2.0)
        raw = rng.uniform(-0.01, 0.01, 24)
        alpha = raw * valid_amplitude_scale(ni, raw)
        out.append({"t": float(t[r]), "ni": ni, "nj": nj, "nv": nv, "Kn": float(Kn),
                    "Ma": float(Ma), "alpha": alpha, "alpha_drawn": raw, "range": range_for_mach(Ma)})
    return out


def random_state(ncell: int, grid: VGrid, rng: np.random.Generator, noise: float = 0.1):
    """A positive, smooth-in-velocity field f[ncell, nv, 2] for single-iteration parity checks:
    per-cell Gaussians with random centre, width and weight times (1 + noise * U(-1,1))."""
    nv = grid.nv
    a = rng.uniform(0.5, 1.5, ncell)
    cx = rng.uniform(-0.8, 0.8, ncell)
    cy = rng.uniform(-0.8, 0.8, ncell)
    s2 = rng.uniform(0.7, 1.4, ncell)
    d = rng.uniform(0.3, 0.7, ncell)
    r2 = (grid.vx[None, :] - cx[:, None]) ** 2 + (grid.vy[None, :] - cy[:, None]) ** 2
    f1 = a[:, None] / (2 * np.pi * s2[:, None]) * np.exp(-r2 / (2 * s2[:, None]))
    f1 = f1 * (1.0 + noise * rng.uniform(-1.0, 1.0, (ncell, nv)))
    f2 = d[:, None] * f1 * (1.0 + noise * rng.uniform(-1.0, 1.0, (ncell, nv)))
    return np.ascontiguousarray(np.stack([f1, f2], axis=-1))


def random_adjoint(ncell: int, nv: int, rng: np.random.Generator):
    return np.ascontiguousarray(rng.uniform(-1.0, 1.0, (ncell, nv, 2)))
