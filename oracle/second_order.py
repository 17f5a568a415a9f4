"""TEST INFRASTRUCTURE (oracle): the second-order spatial reconstruction, in plain numpy.

The first-order residual R1 of the oracle (Eq. numerpr_gov with upwind face values) gains, on every
interior face, the linear reconstruction of the upwind cell:

    F2_e = F1_e + grad f_up . (x_e - x_up),   up = own cell if a_e = S_e . v > 0, else the neighbour,

with the unlimited Gauss gradient of Eq. (gaussgrad),

    grad f_c = (1 / V_c) sum_e fbar_e S_e,   fbar_e = (f_c + f_nb) / 2 on interior faces, and on the
    wall and far-field faces the first-order face value (own f where a_e > 0; the diffuse-wall
    Maxwellian F_rhow gbar, or the free-stream Maxwellian, where a_e <= 0).

x_c is the mean of the cell's four corners and x_e the midpoint of the face.  Boundary faces keep
their first-order values.  So R2 = R1 + dR with

    dR_c = sum_{interior e} a_e grad f_up . (x_e - x_up),

which is affine in f: the far-field values are constants, and the wall values are linear in f through
F_rhow.  Its transpose is therefore a constant matrix, assembled here column by column from dR itself
for small problems.  The point-implicit sweep keeps the first-order diagonal D:
f <- f - (R1(f) + dR) / D, with dR taken from the state at the start of each group of `period`
sweeps and frozen inside the group (defect correction: each group is a few first-order sweeps on
R1(f) = -dR).  period = 1 recomputes dR every sweep; with the unlimited reconstruction that plain
iteration can diverge in weakly collisional modes, while frozen groups of a few sweeps converge to the
same fixed point R1 + dR = 0.  The adjoint transposes R2: Ra = ((dR2/df)^T (w phi) + dJ/df) / w, with
the transposed defect frozen the same way.  The wall functional is unchanged (boundary face values
are first order).

Nothing here is shared with the CUDA path.
"""
from __future__ import annotations

import copy

import numpy as np

from . import oracle as O


class SecondOrder:
    """dR, its transpose and the second-order Jacobi sweeps of one oracle Problem."""

    def __init__(self, pr: O.Problem):
        self.pr = pr
        ni, nj, nv = pr.ni, pr.nj, pr.nv
        self.ni, self.nj, self.nv = ni, nj, nv
        V, S = pr.geometry()
        self.V, self.S = V, S                                        # [nc], [nc, 4, 2]
        X = pr.nodes                                                 # [(nj+1), ni, 2]
        ip = (np.arange(ni) + 1) % ni
        P = np.stack([X[:-1, :, :], X[1:, :, :], X[1:, ip, :], X[:-1, ip, :]], 2)  # [nj, ni, 4, 2]
        P = P.reshape(ni * nj, 4, 2)
        self.xc = P.mean(1)                                          # [nc, 2]
        self.xe = 0.5 * (P + np.roll(P, -1, axis=1))                 # face e: P_e -> P_{e+1}
        # neighbours: face 0 (i-1), 1 (j+1 or far field), 2 (i+1), 3 (j-1 or wall); -1 far, -2 wall
        c = np.arange(ni * nj)
        i, j = c % ni, c // ni
        self.nb = np.stack([j * ni + (i - 1) % ni,
                            np.where(j < nj - 1, (j + 1) * ni + i, -1),
                            j * ni + (i + 1) % ni,
                            np.where(j > 0, (j - 1) * ni + i, -2)], 1)
        vx, vy = pr.vx, pr.vy
        self._a = None
        self.f_far = pr.freestream()[0].copy()                       # [nv, 2]
        Tw = pr.Tw
        g1 = np.exp(-(vx ** 2 + vy ** 2) / (2 * Tw)) / (2 * np.pi * Tw)
        self.gbar = np.stack([g1, 0.5 * Tw * g1], 1)                 # [nv, 2], unnormalised
        self.area_wall = np.sqrt(S[:, 3, 0] ** 2 + S[:, 3, 1] ** 2)

    def face_weights(self, cells=None):
        """a_e = A_e n_e . v_k of the listed cells' faces, [n, 4, nv]."""
        c = slice(None) if cells is None else np.asarray(cells)
        S = self.S[c]
        return S[:, :, 0, None] * self.pr.vx[None, None, :] + S[:, :, 1, None] * self.pr.vy[None, None, :]

    @property
    def a(self):
        if self._a is None:
            self._a = self.face_weights()
        return self._a

    # ------------------------------------------------------------------ face values and gradients
    def _cells(self, cells):
        return np.arange(self.pr.ncell) if cells is None else np.asarray(cells)

    def _boundary_values(self, f, cells=None):
        """First-order values on the far-field (face 1) and wall (face 3) faces of the listed cells
        (all by default), [n, nv, 2] each."""
        c = self._cells(cells)
        w = self.pr.w
        fc = f[c]
        a = self.face_weights(c)
        far = np.where((a[:, 1, :] > 0)[..., None], fc, self.f_far[None])
        vn = a[:, 3, :] / self.area_wall[c, None]                      # v . n on the wall face
        D = -np.sum(np.where(vn <= 0, w[None] * vn * self.gbar[None, :, 0], 0.0), 1)
        Fw = np.sum(np.where(vn > 0, w[None] * vn * fc[:, :, 0], 0.0), 1)
        gw = (Fw / D)[:, None, None] * self.gbar[None]
        wall = np.where((a[:, 3, :] > 0)[..., None], fc, gw)
        return far, wall

    def gradients(self, f, cells=None):
        """Gauss gradient of Eq. (gaussgrad) per cell, velocity and component of the listed cells (all
        by default): [n, nv, 2 comp, 2 xy]."""
        c = self._cells(cells)
        far, wall = self._boundary_values(f, c)
        fc = f[c]
        gsum = np.zeros(fc.shape + (2,), dtype=np.result_type(fc, self.S))
        for e in range(4):
            n = self.nb[c, e]
            inside = n >= 0
            fbar = np.where(inside[:, None, None], 0.5 * (fc + f[np.where(inside, n, 0)]), 0.0)
            if e == 1:
                fbar = np.where(inside[:, None, None], fbar, far)
            if e == 3:
                fbar = np.where(inside[:, None, None], fbar, wall)
            gsum += fbar[..., None] * self.S[c, e, None, None, :]
        return gsum / self.V[c, None, None, None]

    def delta_r(self, f, cells=None):
        """dR = R2 - R1 of the listed cells (all by default), [n, nv, 2]."""
        f = np.asarray(f, dtype=np.float64)
        c = self._cells(cells)
        if cells is None:
            U = c
        else:
            nbs = self.nb[c].ravel()
            U = np.unique(np.concatenate([c, nbs[nbs >= 0]]))
        G = self.gradients(f, U)
        pos = np.full(self.pr.ncell, -1)
        pos[U] = np.arange(U.size)
        Gc = G[pos[c]]
        a_all = self.face_weights(c)
        out = np.zeros((c.size,) + f.shape[1:], dtype=np.result_type(f, self.S))
        for e in range(4):
            n = self.nb[c, e]
            inside = n >= 0
            ns = np.where(inside, n, c)
            a = a_all[:, e, :]                                        # [n, nv]
            own = np.einsum("cvkx,cx->cvk", Gc, self.xe[c, e] - self.xc[c])
            nbr = np.einsum("cvkx,cx->cvk", G[pos[ns]], self.xe[c, e] - self.xc[ns])
            corr = np.where((a > 0)[..., None], own, nbr)
            out += np.where(inside[:, None, None], a[..., None] * corr, 0.0)
        return out

    def face_values(self, f, e):
        """First- and second-order values on face e of every cell (interior faces), [nc, nv, 2] x 2."""
        G = self.gradients(f)
        n = self.nb[:, e]
        ns = np.where(n >= 0, n, 0)
        a = self.a[:, e, :]
        up_own = (a > 0)[..., None]
        F1 = np.where(up_own, f, f[ns])
        own = np.einsum("cvkx,cx->cvk", G, self.xe[:, e] - self.xc)
        nbr = np.einsum("cvkx,cx->cvk", G[ns], self.xe[:, e] - self.xc[ns])
        return F1, F1 + np.where(up_own, own, nbr)

    # ------------------------------------------------------------------ geometry and its derivative
    def geometry_of(self, nodes):
        """Face vectors A n [nc, 4, 2], volumes [nc], cell centres [nc, 2] and face midpoints [nc, 4, 2]
        of the O-mesh with the given nodes [(nj+1), ni, 2] (real or complex): face e runs from
        corner P_e to P_{e+1}, A n = (dy, -dx) along it, V by the shoelace formula."""
        ni, nj = self.ni, self.nj
        ip = (np.arange(ni) + 1) % ni
        P = np.stack([nodes[:-1, :, :], nodes[1:, :, :], nodes[1:, ip, :], nodes[:-1, ip, :]], 2).reshape(ni * nj, 4, 2)
        Q = np.roll(P, -1, axis=1)
        S = np.stack([Q[..., 1] - P[..., 1], -(Q[..., 0] - P[..., 0])], -1)
        V = 0.5 * np.sum(P[..., 0] * Q[..., 1] - Q[..., 0] * P[..., 1], axis=1)
        return S, V, P.mean(1), 0.5 * (P + Q)

    def delta_r_shape_dir(self, f, dnodes, h=1e-30):
        """Derivative of dR along a node motion dnodes [(nj+1), ni, 2] at fixed f, by a complex step
        of size h in the nodes (dR is analytic in them away from a_e = 0): [nc, nv, 2]."""
        S, V, xc, xe = self.geometry_of(self.pr.nodes + 1j * h * np.asarray(dnodes))
        c = copy.copy(self)
        c.S, c.V, c.xc, c.xe, c._a = S, V, xc, xe, None
        c.area_wall = np.sqrt(S[:, 3, 0] ** 2 + S[:, 3, 1] ** 2)
        return np.imag(c.delta_r(np.asarray(f, dtype=np.float64))) / h

    def sens_full(self, f, phi, dnodes):
        """dJ/dalpha_p of the second-order discrete problem at its steady state f and adjoint phi
        ((dR2/df)^T (w phi) = -dJ/df): dJ/dalpha = dJ/dalpha|_f + sum w phi . dR2/dalpha, the first-order
        part from the oracle's full discrete sensitivity with this phi, plus sum w phi . d(dR)/dalpha.
        dnodes: [P, (nj+1), ni, 2]."""
        g = self.pr.sens_full(f, phi, dnodes)
        w = self.pr.w[None, :, None]
        return np.array([g[p] + np.sum(w * phi * self.delta_r_shape_dir(f, dnodes[p])) for p in range(len(dnodes))])

    # ------------------------------------------------------------------ linear structure
    def matrix(self):
        """dR(f) = L f + b: L assembled column by column (small problems only), b = dR(0)."""
        n = self.pr.ncell * self.nv * 2
        b = self.delta_r(np.zeros(self.pr.fshape())).ravel()
        L = np.zeros((n, n))
        for col in range(n):
            e = np.zeros(n)
            e[col] = 1.0
            L[:, col] = self.delta_r(e.reshape(self.pr.fshape())).ravel() - b
        return L, b

    # ------------------------------------------------------------------ sweeps
    def diagonal(self, f):
        """First-order point-implicit diagonal D = V/tau + sum_e max(a_e, 0), [nc, nv]."""
        return self.pr.diagonal(f)

    def residual(self, f):
        R1, _ = self.pr.residual(f)
        return R1 + self.delta_r(f)

    def jacobi(self, f, source=None, defect=None):
        """One point-implicit sweep f - (R1(f) + dR + source) / D; dR = delta_r(f) unless a frozen
        defect is given."""
        f = np.asarray(f, dtype=np.float64)
        D = self.diagonal(f)
        R1, _ = self.pr.residual(f)
        R = R1 + (self.delta_r(f) if defect is None else defect)
        if source is not None:
            R = R + source
        return f - R / D[..., None]

    def solve(self, f0=None, source=None, tol=1e-13, max_sweeps=20000, period=20):
        """Second-order steady state by point-implicit sweeps with the defect frozen over groups of
        `period` sweeps (small problems).  Stops when a sweep moves f by less than tol max|f|."""
        f = self.pr.freestream() if f0 is None else np.array(f0, dtype=np.float64)
        for it in range(max_sweeps):
            if it % period == 0:
                dR = self.delta_r(f)
            fn = self.jacobi(f, source, dR)
            step = np.abs(fn - f).max()
            f = fn
            if step < tol * np.abs(f).max():
                return f, it + 1
        return f, max_sweeps

    def adjoint_defect(self, phi, L):
        """Transposed defect (dR/df)^T (w phi) / w, [nc, nv, 2]."""
        w = self.pr.w[None, :, None]
        return (L.T @ (w * phi).ravel()).reshape(phi.shape) / w

    def adjoint_defect_cells(self, phi, cells):
        """(dR/df)^T (w phi) / w at the listed cells, each at least three rows from the wall (large
        problems).  There dR does not reach the wall value, so it is diagonal in velocity and
        component, and one probe per component gives a whole column block: with h the unit state on
        component kappa of cell m, E_{m,k,kappa} = sum_c phi_{c,k,kappa} (dR(h) - dR(0))_{c,k,kappa}
        over the cells c whose dR sees f_m (m, its neighbours and theirs)."""
        cells = np.asarray(cells)
        ni = self.ni
        if np.any(cells // ni < 3):
            raise ValueError("adjoint_defect_cells: cells must be three or more rows from the wall")
        h = np.zeros(self.pr.fshape())
        out = np.zeros((cells.size, self.nv, 2))
        for i, m in enumerate(cells):
            ring = {int(m)}
            for _ in range(2):
                ring |= {int(n) for r in ring for n in self.nb[r] if n >= 0}
            R = np.array(sorted(ring))
            b = self.delta_r(h, R)
            for kap in range(2):
                h[m, :, kap] = 1.0
                col = self.delta_r(h, R) - b
                h[m, :, kap] = 0.0
                out[i, :, kap] = np.sum(phi[R, :, kap] * col[:, :, kap], axis=0)
        return out

    def adjoint_solve(self, f, tol=1e-13, max_sweeps=20000, period=20):
        L, _ = self.matrix()
        phi = np.zeros(self.pr.fshape())
        for it in range(max_sweeps):
            if it % period == 0:
                E = self.adjoint_defect(phi, L)
            pn = self.adjoint_jacobi(f, phi, defect=E)
            step = np.abs(pn - phi).max()
            phi = pn
            if step < tol * max(np.abs(phi).max(), 1e-300):
                return phi, it + 1
        return phi, max_sweeps

    def adjoint_jacobi(self, f, phi, L=None, defect=None):
        """One point-implicit sweep of the second-order adjoint: phi - Ra / D with
        Ra = (dR1/df)^T (w phi) / w + dJ/df / w + E, E = (dR/df)^T (w phi) / w from L (matrix(), passed
        to avoid rebuilding it) unless a frozen defect E is given."""
        f = np.asarray(f, dtype=np.float64)
        w = self.pr.w[None, :, None]
        if defect is None:
            if L is None:
                L, _ = self.matrix()
            defect = self.adjoint_defect(phi, L)
        Ra = (self.pr.apply_RT(f, (w * phi)) + self.pr.functional_grad(f)) / w + defect
        D = self.diagonal(f)
        return phi - Ra / D[..., None]
