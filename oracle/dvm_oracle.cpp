/*
 * FP64 CPU oracle for the steady discrete-velocity (DVM) BGK problem on a body-fitted O-mesh,
 * its exact discrete adjoint and the boundary sensitivities of Yuan & Wu, "Adjoint shape
 * optimization from the continuum to free-molecular gas flows" (arXiv 2501.00923).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * load this library.  It shares no code, header or table with the CUDA library; both are fed by
 * the seeded input generators only.  Plain loops, FP64 throughout, no blocking or fusion.
 *
 * Units and readings (stated once, used everywhere):
 *   rho_inf = 1, R T_inf = 1, chord = l_ref = 1; the reduced 2D model of a monatomic gas
 *   (energy rho E = rho|u|^2/2 + 3/2 rho R T, Eq. (macint_reduce) with the moment tensor Psi).
 *   tau = mu/p with mu ~ sqrt(T) (Sec. 2.1)  =>  tau = tau_inf / (rho sqrt(T)),
 *   tau_inf from the Knudsen definition Eq. (kndefine): tau_inf = (5/16) Kn sqrt(2 pi).
 *   Free stream: rho=1, T=1, u = Ma sqrt(5/3) (cos aoa, sin aoa).
 *   Interface values: first-order upwind (the paper's DUGKS interface of Sec. 3.1 is not
 *   given in the paper; first order keeps the discrete problem exactly differentiable).
 *
 * Mesh: cell c = j*ni + i, corners P0=X(j,i), P1=X(j+1,i), P2=X(j+1,i+1), P3=X(j,i+1) (i
 * periodic).  Face e runs P_e -> P_{e+1}; its vector S_e = A_e n_e = (dy, -dx) points out of the
 * cell.  Face 0 borders (i-1,j), face 1 (i,j+1) or the far field, face 2 (i+1,j), face 3 (i,j-1)
 * or the wall.  On the wall face, n points into the solid as in Sec. 3.2.
 *
 * Unknowns f[c][k][2] = (f1, f2) (Eq. f_reduce); weights w_k are the velocity quadrature.
 * Discrete primal residual, Eq. (numerpr_gov), first-order upwind:
 *   R_{c,k} = sum_e a_{e,k} F_{e,k} + (V_c/tau_c) (f_{c,k} - g_{c,k}),  a_{e,k} = S_e . v_k
 *   F_{e,k} = f_{c,k} if a > 0, else the upwind value: the neighbour cell, the far-field
 *   Maxwellian (Eq. bc_drlt / drlt_maxwell) or the wall Maxwellian g_w = F_rhow gbar_w
 *   (Eq. formula_bgk_fdw0, formula_bgk_fdw and the discrete form above Eq. barg).
 * Functional, Eq. (formula_opt) discretised as Eq. (numer_J):
 *   J = sum_l sum_k w_k m_k (v_k . S_l) f1_{l,k},  m_k = d . v_k + h |v_k|^2 / 2: the moment m_J of
 *   Eq. (formula_opt); d = force direction with h = 0 (drag: d = e1), or d = 0, h = 1 for the heat
 * Discrete adjoint in the paper's sign (Lagrangian L = J + sum w phi . R, Eq. lagrangian):
 *   (dR/df)^T (w phi) = -(dJ/df)^T,   dJ/dalpha = dJ/dalpha|_f + sum w phi . dR/dalpha|_f.
 */
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double kPi = 3.14159265358979323846;
enum { WALL = -1, FAR = -2 };

/* ---------------------------------------------------------------- forward-mode dual numbers */
struct Dual {
    double v, d;
    Dual() : v(0.0), d(0.0) {}
    Dual(double a) : v(a), d(0.0) {}
    Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, a.d * e); }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, 0.5 * a.d / s); }
inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }
using std::exp;
using std::sqrt;

/* ---------------------------------------------------------------- problem description */
struct Prob {
    int ni, nj, nv;
    const double* nodes;  /* [(nj+1)][ni][2] */
    const double* vx;
    const double* vy;
    const double* w;
    double Kn, Ma, Tw, aoa;
    double dir[3];        /* m_J(v) = dir[0] vx + dir[1] vy + dir[2] |v|^2/2 */
    int conservative;     /* 1: the cell Maxwellian matches the cell's discrete moments exactly */
};

inline double moment_J(const double* dir, double vx, double vy) {
    return dir[0] * vx + dir[1] * vy + dir[2] * 0.5 * (vx * vx + vy * vy);
}

struct Consts {
    double tau_inf, u1, u2, Tw;
    std::vector<double> fd1, fd2; /* far-field Maxwellian g_M(1, u_inf, 1) at each v_k */
    std::vector<double> gw1;      /* unnormalised wall Maxwellian g_M1(1, 0, T_w) at each v_k */
};

/* reduced Maxwellian, Eq. (maxwell_reduce) */
template <class S>
void maxwellian(S rho, S u1, S u2, S T, double vx, double vy, S& g1, S& g2) {
    S c2 = (vx - u1) * (vx - u1) + (vy - u2) * (vy - u2);
    g1 = rho / (2.0 * kPi * T) * exp(-c2 / (2.0 * T));
    g2 = 0.5 * T * g1;
}

Consts make_consts(const Prob& p) {
    Consts K;
    K.tau_inf = 5.0 / 16.0 * p.Kn * std::sqrt(2.0 * kPi); /* Eq. (kndefine) with RT=1, l_ref=1 */
    double ainf = std::sqrt(5.0 / 3.0);
    K.u1 = p.Ma * ainf * std::cos(p.aoa);
    K.u2 = p.Ma * ainf * std::sin(p.aoa);
    K.Tw = p.Tw;
    K.fd1.resize(p.nv); K.fd2.resize(p.nv); K.gw1.resize(p.nv);
    for (int k = 0; k < p.nv; ++k) {
        double g1, g2;
        maxwellian<double>(1.0, K.u1, K.u2, 1.0, p.vx[k], p.vy[k], g1, g2);
        K.fd1[k] = g1; K.fd2[k] = g2;
        maxwellian<double>(1.0, 0.0, 0.0, p.Tw, p.vx[k], p.vy[k], g1, g2);
        K.gw1[k] = g1;
    }
    return K;
}

/* ---------------------------------------------------------------- geometry */
template <class S>
struct Geo {
    int ni, nj;
    std::vector<S> V;        /* [ncell] */
    std::vector<S> Sx, Sy;   /* [ncell*4] outward face vectors A n */
};

template <class S>
void build_geo(int ni, int nj, const S* X, Geo<S>& g) {
    g.ni = ni; g.nj = nj;
    int nc = ni * nj;
    g.V.assign(nc, S(0.0));
    g.Sx.assign(nc * 4, S(0.0));
    g.Sy.assign(nc * 4, S(0.0));
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            int ip = (i + 1) % ni, c = j * ni + i;
            const S* P[4] = {X + 2 * (j * ni + i), X + 2 * ((j + 1) * ni + i),
                             X + 2 * ((j + 1) * ni + ip), X + 2 * (j * ni + ip)};
            S area(0.0);
            for (int e = 0; e < 4; ++e) {
                const S* A = P[e];
                const S* B = P[(e + 1) % 4];
                area += 0.5 * (A[0] * B[1] - B[0] * A[1]);   /* shoelace */
                g.Sx[4 * c + e] = B[1] - A[1];
                g.Sy[4 * c + e] = -(B[0] - A[0]);
            }
            g.V[c] = area;
        }
}

int neighbour(int ni, int nj, int c, int e) {
    int i = c % ni, j = c / ni;
    switch (e) {
        case 0: return j * ni + (i - 1 + ni) % ni;
        case 1: return j + 1 < nj ? (j + 1) * ni + i : FAR;
        case 2: return j * ni + (i + 1) % ni;
        default: return j > 0 ? (j - 1) * ni + i : WALL;
    }
}

/* ---------------------------------------------------------------- cell-level kinetics */
/* W = sum_k w_k Psi_k . f_k, Eq. (macint_reduce) */
template <class S>
void cell_moments(const Prob& p, const S* fc, S W[4]) {
    for (int m = 0; m < 4; ++m) W[m] = S(0.0);
    for (int k = 0; k < p.nv; ++k) {
        double vx = p.vx[k], vy = p.vy[k], w = p.w[k];
        S f1 = fc[2 * k], f2 = fc[2 * k + 1];
        W[0] += w * f1;
        W[1] += w * vx * f1;
        W[2] += w * vy * f1;
        W[3] += w * (0.5 * (vx * vx + vy * vy) * f1 + f2);
    }
}

/* (rho, u, T) from W with E = |u|^2/2 + 3/2 T (gamma = 5/3) */
template <class S>
void primitives(const S W[4], S& rho, S& u1, S& u2, S& T) {
    rho = W[0];
    u1 = W[1] / rho;
    u2 = W[2] / rho;
    T = (2.0 / 3.0) * (W[3] / rho - 0.5 * (u1 * u1 + u2 * u2));
}

/* Solve the 4x4 system A x = b in place (Gaussian elimination, pivots chosen on the values). */
template <class S>
void solve4(S A[4][4], S b[4], S x[4]) {
    int piv[4] = {0, 1, 2, 3};
    for (int col = 0; col < 4; ++col) {
        int best = col;
        for (int r = col + 1; r < 4; ++r)
            if (std::fabs(val(A[piv[r]][col])) > std::fabs(val(A[piv[best]][col]))) best = r;
        std::swap(piv[col], piv[best]);
        for (int r = col + 1; r < 4; ++r) {
            S m = A[piv[r]][col] / A[piv[col]][col];
            for (int c2 = col; c2 < 4; ++c2) A[piv[r]][c2] -= m * A[piv[col]][c2];
            b[piv[r]] -= m * b[piv[col]];
        }
    }
    for (int col = 3; col >= 0; --col) {
        S acc = b[piv[col]];
        for (int c2 = col + 1; c2 < 4; ++c2) acc -= A[piv[col]][c2] * x[c2];
        x[col] = acc / A[piv[col]][col];
    }
}

/* Parameters (rho, u1, u2, T) of the cell Maxwellian g in the collision term.  Plain: the
 * primitives of W.  Conservative: the parameters whose discrete Maxwellian has exactly the cell's
 * discrete moments, sum_k w_k Psi_k g_k = W (Psi = 1, vx, vy and |v|^2/2 on g1 plus 1 on g2), by
 * Newton's method from the primitives.  With dual numbers the converged iteration carries the
 * implicit derivative (dM/dp)^{-1} dW, so the transposed operator and the sensitivities follow. */
template <class S>
void maxwell_params(const Prob& p, const S W[4], S& rho, S& u1, S& u2, S& T) {
    primitives(W, rho, u1, u2, T);
    if (!p.conservative) return;
    int extra = -1;
    for (int it = 0; it < 60; ++it) {
        S M[4] = {S(0.0), S(0.0), S(0.0), S(0.0)};
        S J[4][4];
        for (int m = 0; m < 4; ++m)
            for (int q = 0; q < 4; ++q) J[m][q] = S(0.0);
        for (int k = 0; k < p.nv; ++k) {
            double vx = p.vx[k], vy = p.vy[k], w = p.w[k], h = 0.5 * (vx * vx + vy * vy);
            S g1, g2;
            maxwellian(rho, u1, u2, T, vx, vy, g1, g2);
            S cx = vx - u1, cy = vy - u2;
            S c2 = cx * cx + cy * cy;
            S d1[4] = {g1 / rho, g1 * cx / T, g1 * cy / T, g1 * (c2 / (2.0 * T * T) - 1.0 / T)};
            const double psi[3] = {1.0, vx, vy};
            for (int m = 0; m < 3; ++m) {
                M[m] += w * psi[m] * g1;
                for (int q = 0; q < 4; ++q) J[m][q] += w * psi[m] * d1[q];
            }
            M[3] += w * (h * g1 + g2);
            for (int q = 0; q < 4; ++q) {
                S d2 = 0.5 * T * d1[q];                       /* g2 = T g1 / 2 */
                if (q == 3) d2 += 0.5 * g1;
                J[3][q] += w * (h * d1[q] + d2);
            }
        }
        S r[4] = {M[0] - W[0], M[1] - W[1], M[2] - W[2], M[3] - W[3]};
        S x[4];
        solve4(J, r, x);
        rho -= x[0]; u1 -= x[1]; u2 -= x[2]; T -= x[3];
        double step = std::fabs(val(x[0])) / std::fabs(val(rho)) + std::fabs(val(x[3])) / std::fabs(val(T)) +
                      std::fabs(val(x[1])) + std::fabs(val(x[2]));
        if (extra < 0 && step < 1e-14) extra = 2;    /* values converged: two more steps for the duals */
        if (extra >= 0 && extra-- == 0) break;
    }
}

template <class S>
S relax_time(double tau_inf, S rho, S T) { return tau_inf / (rho * sqrt(T)); }

/* Wall face of cell c (j = 0, face 3): unit normal into the solid, area, the discrete incoming
 * mass flux F_rhow = sum_{a>0} w (v.n) f1 and the normaliser D = -sum_{a<=0} w (v.n) g_M1(1,0,T_w)
 * of gbar_w, Eq. (barg). */
template <class S>
struct WallFace { S A, nx, ny, Fw, D; };

template <class S>
WallFace<S> wall_face(const Prob& p, const Consts& K, const Geo<S>& g, const S* fc, int c) {
    WallFace<S> wf;
    S sx = g.Sx[4 * c + 3], sy = g.Sy[4 * c + 3];
    wf.A = sqrt(sx * sx + sy * sy);
    wf.nx = sx / wf.A;
    wf.ny = sy / wf.A;
    wf.Fw = S(0.0);
    wf.D = S(0.0);
    for (int k = 0; k < p.nv; ++k) {
        S vn = p.vx[k] * wf.nx + p.vy[k] * wf.ny;
        if (val(vn) > 0.0) wf.Fw += p.w[k] * vn * fc[2 * k];
        else wf.D -= p.w[k] * vn * K.gw1[k];
    }
    return wf;
}

/* ---------------------------------------------------------------- residual, Eq. (numerpr_gov) */
template <class S>
void residual_cell(const Prob& p, const Consts& K, const Geo<S>& g, const S* f, int c, S* Rc) {
    const int nv = p.nv;
    const S* fc = f + (size_t)c * nv * 2;
    S W[4], rho, u1, u2, T, gr, gu1, gu2, gT;
    cell_moments(p, fc, W);
    primitives(W, rho, u1, u2, T);
    maxwell_params(p, W, gr, gu1, gu2, gT);
    S Vt = g.V[c] / relax_time(K.tau_inf, rho, T);
    bool wall = (c / p.ni) == 0;
    WallFace<S> wf;
    if (wall) wf = wall_face(p, K, g, fc, c);
    for (int k = 0; k < nv; ++k) {
        double vx = p.vx[k], vy = p.vy[k];
        S g1, g2;
        maxwellian(gr, gu1, gu2, gT, vx, vy, g1, g2);
        S R1 = Vt * (fc[2 * k] - g1);
        S R2 = Vt * (fc[2 * k + 1] - g2);
        for (int e = 0; e < 4; ++e) {
            S a = g.Sx[4 * c + e] * vx + g.Sy[4 * c + e] * vy;
            S F1, F2;
            if (val(a) > 0.0) {
                F1 = fc[2 * k]; F2 = fc[2 * k + 1];
            } else {
                int nb = neighbour(p.ni, p.nj, c, e);
                if (nb >= 0) {
                    F1 = f[((size_t)nb * nv + k) * 2]; F2 = f[((size_t)nb * nv + k) * 2 + 1];
                } else if (nb == FAR) {
                    F1 = S(K.fd1[k]); F2 = S(K.fd2[k]);
                } else {
                    S gb1 = K.gw1[k] / wf.D;       /* gbar_w, Eq. (barg) */
                    F1 = wf.Fw * gb1;
                    F2 = wf.Fw * (0.5 * K.Tw) * gb1;
                }
            }
            R1 += a * F1;
            R2 += a * F2;
        }
        Rc[2 * k] = R1;
        Rc[2 * k + 1] = R2;
    }
}

template <class S>
void residual_all(const Prob& p, const Consts& K, const Geo<S>& g, const S* f, S* R) {
    int nc = p.ni * p.nj;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nc; ++c) residual_cell(p, K, g, f, c, R + (size_t)c * p.nv * 2);
}

/* D_{c,k} = V_c/tau_c + sum_{e: a>0} a_{e,k}: the diagonal of the point-implicit update */
void diagonal_all(const Prob& p, const Consts& K, const Geo<double>& g, const double* f, double* Dg) {
    int nc = p.ni * p.nj, nv = p.nv;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nc; ++c) {
        double W[4], rho, u1, u2, T;
        cell_moments(p, f + (size_t)c * nv * 2, W);
        primitives(W, rho, u1, u2, T);
        double Vt = g.V[c] / relax_time(K.tau_inf, rho, T);
        for (int k = 0; k < nv; ++k) {
            double d = Vt;
            for (int e = 0; e < 4; ++e) {
                double a = g.Sx[4 * c + e] * p.vx[k] + g.Sy[4 * c + e] * p.vy[k];
                if (a > 0.0) d += a;
            }
            Dg[(size_t)c * nv + k] = d;
        }
    }
}

/* w-weighted norm of R/V: sqrt(sum_{c,k,comp} w_k (R/V_c)^2) */
double residual_norm(const Prob& p, const Geo<double>& g, const double* R) {
    int nc = p.ni * p.nj, nv = p.nv;
    double s = 0.0;
    for (int c = 0; c < nc; ++c) {
        double iv = 1.0 / g.V[c];
        for (int k = 0; k < nv; ++k) {
            double r1 = R[((size_t)c * nv + k) * 2] * iv, r2 = R[((size_t)c * nv + k) * 2 + 1] * iv;
            s += p.w[k] * (r1 * r1 + r2 * r2);
        }
    }
    return std::sqrt(s);
}

/* ---------------------------------------------------------------- functional, Eq. (numer_J) */
template <class S>
S functional(const Prob& p, const Consts& K, const Geo<S>& g, const S* f) {
    S J(0.0);
    int nv = p.nv;
    for (int i = 0; i < p.ni; ++i) {
        int c = i; /* j = 0 */
        const S* fc = f + (size_t)c * nv * 2;
        WallFace<S> wf = wall_face(p, K, g, fc, c);
        S sx = g.Sx[4 * c + 3], sy = g.Sy[4 * c + 3];
        for (int k = 0; k < nv; ++k) {
            double vx = p.vx[k], vy = p.vy[k];
            double m = moment_J(p.dir, vx, vy);
            S a = sx * vx + sy * vy;
            S f1l = val(a) > 0.0 ? fc[2 * k] : wf.Fw * (K.gw1[k] / wf.D);
            J += p.w[k] * m * a * f1l;
        }
    }
    return J;
}

/* dJ/df, written out from the definition above: for wall cells and a_k > 0,
 * dJ/df1_k = w_k [ m_k a_k + (v_k.n) M ],  M = sum_{a<=0} w m a gbar1  (the reflected part
 * of J depends on f only through F_rhow). */
void functional_grad(const Prob& p, const Consts& K, const Geo<double>& g, const double* f, double* dJ) {
    int nv = p.nv;
    std::memset(dJ, 0, sizeof(double) * (size_t)p.ni * p.nj * nv * 2);
    for (int i = 0; i < p.ni; ++i) {
        int c = i;
        const double* fc = f + (size_t)c * nv * 2;
        WallFace<double> wf = wall_face(p, K, g, fc, c);
        double sx = g.Sx[4 * c + 3], sy = g.Sy[4 * c + 3];
        double M = 0.0;
        for (int k = 0; k < nv; ++k) {
            double a = sx * p.vx[k] + sy * p.vy[k];
            if (!(a > 0.0)) M += p.w[k] * moment_J(p.dir, p.vx[k], p.vy[k]) * a * K.gw1[k] / wf.D;
        }
        for (int k = 0; k < nv; ++k) {
            double a = sx * p.vx[k] + sy * p.vy[k];
            if (a > 0.0) {
                double m = moment_J(p.dir, p.vx[k], p.vy[k]);
                double vn = p.vx[k] * wf.nx + p.vy[k] * wf.ny;
                dJ[((size_t)c * nv + k) * 2] = p.w[k] * (m * a + vn * M);
            }
        }
    }
}

void collision_partials(const Prob& p, const Consts& K, const Geo<double>& g, const double* f,
                        std::vector<double>& dC);

/* ---------------------------------------------------------------- explicit transpose (dR/df)^T lam
 * Scatter form: every term of R_{c,k,comp} sends lam_{c,k,comp} times its partial derivative to
 * the unknown it depends on.  The collision partials d/dW of (V/tau(W))(f - g(W)) come from dual
 * numbers in each W component (collision_partials), then are chained through dW/df = w_k Psi_k. */
void apply_RT(const Prob& p, const Consts& K, const Geo<double>& g, const double* f,
              const double* dC, const double* lam, double* out) {
    const int nv = p.nv, nc = p.ni * p.nj;
    std::memset(out, 0, sizeof(double) * (size_t)nc * nv * 2);
    for (int c = 0; c < nc; ++c) {
        const double* fc = f + (size_t)c * nv * 2;
        const double* lc = lam + (size_t)c * nv * 2;
        double* oc = out + (size_t)c * nv * 2;
        /* transport terms */
        bool wall = (c / p.ni) == 0;
        WallFace<double> wf;
        if (wall) wf = wall_face(p, K, g, fc, c);
        double Lam = 0.0;
        for (int e = 0; e < 4; ++e) {
            int nb = neighbour(p.ni, p.nj, c, e);
            for (int k = 0; k < nv; ++k) {
                double a = g.Sx[4 * c + e] * p.vx[k] + g.Sy[4 * c + e] * p.vy[k];
                for (int q = 0; q < 2; ++q) {
                    double l = lc[2 * k + q];
                    if (a > 0.0) oc[2 * k + q] += a * l;
                    else if (nb >= 0) out[((size_t)nb * nv + k) * 2 + q] += a * l;
                    else if (nb == WALL) {
                        double gb = K.gw1[k] / wf.D * (q == 0 ? 1.0 : 0.5 * K.Tw);
                        Lam += a * l * gb;     /* d(F_rhow gbar)/d f1_{k'} = gbar w_k' (v_k'.n) */
                    }
                }
            }
        }
        if (wall)
            for (int k = 0; k < nv; ++k) {
                double vn = p.vx[k] * wf.nx + p.vy[k] * wf.ny;
                if (vn > 0.0) oc[2 * k] += Lam * p.w[k] * vn;
            }
        /* collision terms (V/tau)(f - g) */
        double W[4], rho, u1, u2, T;
        cell_moments(p, fc, W);
        primitives(W, rho, u1, u2, T);
        double Vt = g.V[c] / relax_time(K.tau_inf, rho, T);
        for (int k = 0; k < nv; ++k) {
            oc[2 * k] += Vt * lc[2 * k];
            oc[2 * k + 1] += Vt * lc[2 * k + 1];
        }
        double s[4];
        for (int m = 0; m < 4; ++m) {
            const double* dc = dC + (((size_t)c * 4 + m) * nv) * 2;
            double acc = 0.0;
            for (int k = 0; k < nv; ++k) acc += lc[2 * k] * dc[2 * k] + lc[2 * k + 1] * dc[2 * k + 1];
            s[m] = acc;
        }
        for (int k = 0; k < nv; ++k) {
            double vx = p.vx[k], vy = p.vy[k], w = p.w[k];
            oc[2 * k] += w * (s[0] + s[1] * vx + s[2] * vy + s[3] * 0.5 * (vx * vx + vy * vy));
            oc[2 * k + 1] += w * s[3];
        }
    }
}

/* ---------------------------------------------------------------- primal solver (own iteration)
 * Nonlinear Gauss-Seidel, in place, alternating the four sweep directions of the O-mesh.  Each
 * cell update is the point-implicit solve of its own rows with the current neighbour values and
 * the cell's current moments. */
void gs_update_cell(const Prob& p, const Consts& K, const Geo<double>& g, const double* f, int c, double* dst) {
    const int nv = p.nv;
    const double* fc = f + (size_t)c * nv * 2;
    double W[4], rho, u1, u2, T, gr, gu1, gu2, gT;
    cell_moments(p, fc, W);
    primitives(W, rho, u1, u2, T);
    maxwell_params(p, W, gr, gu1, gu2, gT);
    double Vt = g.V[c] / relax_time(K.tau_inf, rho, T);
    bool wall = (c / p.ni) == 0;
    WallFace<double> wf;
    if (wall) wf = wall_face(p, K, g, fc, c);
    std::vector<double> nf(2 * nv);
    for (int k = 0; k < nv; ++k) {
        double vx = p.vx[k], vy = p.vy[k], g1, g2;
        maxwellian<double>(gr, gu1, gu2, gT, vx, vy, g1, g2);
        double d = Vt, r1 = Vt * g1, r2 = Vt * g2;
        for (int e = 0; e < 4; ++e) {
            double a = g.Sx[4 * c + e] * vx + g.Sy[4 * c + e] * vy;
            if (a > 0.0) { d += a; continue; }
            int nb = neighbour(p.ni, p.nj, c, e);
            double F1, F2;
            if (nb >= 0) { F1 = f[((size_t)nb * nv + k) * 2]; F2 = f[((size_t)nb * nv + k) * 2 + 1]; }
            else if (nb == FAR) { F1 = K.fd1[k]; F2 = K.fd2[k]; }
            else { double gb = K.gw1[k] / wf.D; F1 = wf.Fw * gb; F2 = wf.Fw * 0.5 * K.Tw * gb; }
            r1 -= a * F1;
            r2 -= a * F2;
        }
        nf[2 * k] = r1 / d;
        nf[2 * k + 1] = r2 / d;
    }
    std::memcpy(dst, nf.data(), sizeof(double) * 2 * nv);
}

void gs_sweep(const Prob& p, const Consts& K, const Geo<double>& g, double* f, int dir) {
    int ni = p.ni, nj = p.nj;
    bool jup = (dir & 1) == 0, iup = (dir & 2) == 0;
    for (int jj = 0; jj < nj; ++jj) {
        int j = jup ? jj : nj - 1 - jj;
        for (int ii = 0; ii < ni; ++ii) {
            int i = iup ? ii : ni - 1 - ii;
            gs_update_cell(p, K, g, f, j * ni + i, f + (size_t)(j * ni + i) * p.nv * 2);
        }
    }
}

/* ---------------------------------------------------------------- adjoint solver (own iteration)
 * Gauss-Seidel on the transposed rows, written in gather form for cell c (all k, comp):
 *   D phi = -dJ/(w) + sum_{e:a>0, interior} a phi_nb - q . Psi - [wall, a_wall>0, comp 1] (v.n) Lam
 * with q_m = sum lam d[(V/tau)(f-g)]/dW_m (from duals) and Lam = sum_{a_wall<=0} w a phi.gbar.
 * Convergence is measured with the scatter-form apply_RT above, not with this update. */
/* d[(V/tau)(f - g(W))]_{k,comp} / dW_m for every cell, from dual numbers in each W component:
 * dC[((c*4 + m)*nv + k)*2 + comp].  f is fixed during an adjoint solve, so this is built once. */
void collision_partials_cell(const Prob& p, const Consts& K, const Geo<double>& g, const double* f, int c,
                             double* dCc /* [4][nv][2] */) {
    const int nv = p.nv;
    const double* fc = f + (size_t)c * nv * 2;
    double W[4];
    cell_moments(p, fc, W);
    for (int m = 0; m < 4; ++m) {
        Dual Wd[4];
        for (int n = 0; n < 4; ++n) Wd[n] = Dual(W[n], n == m ? 1.0 : 0.0);
        Dual rd, ud1, ud2, Td, gr, gu1, gu2, gT;
        primitives(Wd, rd, ud1, ud2, Td);
        maxwell_params(p, Wd, gr, gu1, gu2, gT);
        Dual Vtd = Dual(g.V[c]) / relax_time(K.tau_inf, rd, Td);
        double* out = dCc + (size_t)m * nv * 2;
        for (int k = 0; k < nv; ++k) {
            Dual g1, g2;
            maxwellian(gr, gu1, gu2, gT, p.vx[k], p.vy[k], g1, g2);
            out[2 * k] = (Vtd * (Dual(fc[2 * k]) - g1)).d;
            out[2 * k + 1] = (Vtd * (Dual(fc[2 * k + 1]) - g2)).d;
        }
    }
}

void collision_partials(const Prob& p, const Consts& K, const Geo<double>& g, const double* f,
                        std::vector<double>& dC) {
    const int nv = p.nv, nc = p.ni * p.nj;
    dC.assign((size_t)nc * 4 * nv * 2, 0.0);
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nc; ++c) collision_partials_cell(p, K, g, f, c, &dC[(size_t)c * 4 * nv * 2]);
}

void adjoint_gs_update_cell(const Prob& p, const Consts& K, const Geo<double>& g, const double* f,
                            const double* jsrc, const double* dCc, const double* phi, int c, double* dst) {
    const int nv = p.nv;
    const double* fc = f + (size_t)c * nv * 2;
    const double* pc = phi + (size_t)c * nv * 2;
    double W[4], rho, u1, u2, T;
    cell_moments(p, fc, W);
    primitives(W, rho, u1, u2, T);
    double Vt = g.V[c] / relax_time(K.tau_inf, rho, T);
    double q[4];
    for (int m = 0; m < 4; ++m) {
        const double* dc = dCc + (size_t)m * nv * 2;
        double acc = 0.0;
        for (int k = 0; k < nv; ++k) acc += p.w[k] * (pc[2 * k] * dc[2 * k] + pc[2 * k + 1] * dc[2 * k + 1]);
        q[m] = acc;
    }
    bool wall = (c / p.ni) == 0;
    WallFace<double> wf;
    double Lam = 0.0;
    if (wall) {
        wf = wall_face(p, K, g, fc, c);
        for (int k = 0; k < nv; ++k) {
            double a = g.Sx[4 * c + 3] * p.vx[k] + g.Sy[4 * c + 3] * p.vy[k];
            if (!(a > 0.0)) {
                double gb1 = K.gw1[k] / wf.D, gb2 = 0.5 * K.Tw * gb1;
                Lam += p.w[k] * a * (pc[2 * k] * gb1 + pc[2 * k + 1] * gb2);
            }
        }
    }
    std::vector<double> np(2 * nv);
    for (int k = 0; k < nv; ++k) {
        double vx = p.vx[k], vy = p.vy[k];
        double d = Vt;
        double r1 = -jsrc[((size_t)c * nv + k) * 2] / p.w[k];
        double r2 = -jsrc[((size_t)c * nv + k) * 2 + 1] / p.w[k];
        for (int e = 0; e < 4; ++e) {
            double a = g.Sx[4 * c + e] * vx + g.Sy[4 * c + e] * vy;
            if (!(a > 0.0)) continue;
            d += a;
            int nb = neighbour(p.ni, p.nj, c, e);
            if (nb >= 0) {
                r1 += a * phi[((size_t)nb * nv + k) * 2];
                r2 += a * phi[((size_t)nb * nv + k) * 2 + 1];
            }
        }
        r1 -= q[0] + q[1] * vx + q[2] * vy + q[3] * 0.5 * (vx * vx + vy * vy);
        r2 -= q[3];
        if (wall) {
            double vn = vx * wf.nx + vy * wf.ny;
            if (vn > 0.0) r1 -= vn * Lam;
        }
        np[2 * k] = r1 / d;
        np[2 * k + 1] = r2 / d;
    }
    std::memcpy(dst, np.data(), sizeof(double) * 2 * nv);
}

/* adjoint residual in phi units: Ra = ((dR/df)^T (w phi) + dJ/df) / w */
void adjoint_residual(const Prob& p, const Consts& K, const Geo<double>& g, const double* f,
                      const double* dC, const double* jsrc, const double* phi, double* Ra) {
    size_t n = (size_t)p.ni * p.nj * p.nv;
    std::vector<double> lam(2 * n);
    for (size_t ck = 0; ck < n; ++ck) {
        double w = p.w[ck % p.nv];
        lam[2 * ck] = w * phi[2 * ck];
        lam[2 * ck + 1] = w * phi[2 * ck + 1];
    }
    apply_RT(p, K, g, f, dC, lam.data(), Ra);
    for (size_t ck = 0; ck < n; ++ck) {
        double w = p.w[ck % p.nv];
        Ra[2 * ck] = (Ra[2 * ck] + jsrc[2 * ck]) / w;
        Ra[2 * ck + 1] = (Ra[2 * ck + 1] + jsrc[2 * ck + 1]) / w;
    }
}

std::vector<double> to_vec(const double* a, size_t n) { return std::vector<double>(a, a + n); }

Geo<double> geo_of(const Prob& p) {
    Geo<double> g;
    build_geo<double>(p.ni, p.nj, p.nodes, g);
    return g;
}

} /* namespace */

/* =============================================================================== C entry points */
extern "C" {

typedef struct {
    int ni, nj, nv;
    const double* nodes;
    const double* vx;
    const double* vy;
    const double* w;
    double Kn, Ma, Tw, aoa;
    double dir[3];
    int conservative;
} orc_problem;

static Prob to_prob(const orc_problem* q) {
    Prob p;
    p.ni = q->ni; p.nj = q->nj; p.nv = q->nv; p.nodes = q->nodes;
    p.vx = q->vx; p.vy = q->vy; p.w = q->w;
    p.Kn = q->Kn; p.Ma = q->Ma; p.Tw = q->Tw; p.aoa = q->aoa;
    p.dir[0] = q->dir[0]; p.dir[1] = q->dir[1]; p.dir[2] = q->dir[2];
    p.conservative = q->conservative;
    return p;
}

int orc_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* cell volumes [ncell] and outward face vectors [ncell][4][2] */
int orc_geometry(const orc_problem* q, double* V, double* S) {
    Prob p = to_prob(q);
    Geo<double> g = geo_of(p);
    int nc = p.ni * p.nj;
    for (int c = 0; c < nc; ++c) {
        V[c] = g.V[c];
        for (int e = 0; e < 4; ++e) { S[8 * c + 2 * e] = g.Sx[4 * c + e]; S[8 * c + 2 * e + 1] = g.Sy[4 * c + e]; }
    }
    return 0;
}

/* free-stream initial state f = g_M(1, u_inf, 1) in every cell */
int orc_freestream(const orc_problem* q, double* f) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    size_t nc = (size_t)p.ni * p.nj;
    for (size_t c = 0; c < nc; ++c)
        for (int k = 0; k < p.nv; ++k) { f[(c * p.nv + k) * 2] = K.fd1[k]; f[(c * p.nv + k) * 2 + 1] = K.fd2[k]; }
    return 0;
}

/* per-cell moments W [ncell][4] */
int orc_moments(const orc_problem* q, const double* f, double* W) {
    Prob p = to_prob(q);
    int nc = p.ni * p.nj;
    for (int c = 0; c < nc; ++c) cell_moments(p, f + (size_t)c * p.nv * 2, W + 4 * c);
    return 0;
}

/* collision term per cell g(W(f)) - f, for the conservation check */
int orc_collision(const orc_problem* q, const double* f, double* Q) {
    Prob p = to_prob(q);
    int nc = p.ni * p.nj;
    for (int c = 0; c < nc; ++c) {
        const double* fc = f + (size_t)c * p.nv * 2;
        double W[4], rho, u1, u2, T;
        cell_moments(p, fc, W);
        maxwell_params(p, W, rho, u1, u2, T);
        for (int k = 0; k < p.nv; ++k) {
            double g1, g2;
            maxwellian<double>(rho, u1, u2, T, p.vx[k], p.vy[k], g1, g2);
            Q[((size_t)c * p.nv + k) * 2] = g1 - fc[2 * k];
            Q[((size_t)c * p.nv + k) * 2 + 1] = g2 - fc[2 * k + 1];
        }
    }
    return 0;
}

int orc_residual(const orc_problem* q, const double* f, double* R, double* norm) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> g = geo_of(p);
    residual_all(p, K, g, f, R);
    if (norm) *norm = residual_norm(p, g, R);
    return 0;
}

/* residual and its directional derivative along df (dual numbers in f) */
int orc_residual_dir(const orc_problem* q, const double* f, const double* df, double* R, double* dR) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> gd = geo_of(p);
    Geo<Dual> g;
    g.ni = gd.ni; g.nj = gd.nj;
    for (double v : gd.V) g.V.push_back(Dual(v));
    for (double v : gd.Sx) g.Sx.push_back(Dual(v));
    for (double v : gd.Sy) g.Sy.push_back(Dual(v));
    size_t n = (size_t)p.ni * p.nj * p.nv * 2;
    std::vector<Dual> fd(n), Rd(n);
    for (size_t i = 0; i < n; ++i) fd[i] = Dual(f[i], df[i]);
    residual_all(p, K, g, fd.data(), Rd.data());
    for (size_t i = 0; i < n; ++i) { R[i] = Rd[i].v; dR[i] = Rd[i].d; }
    return 0;
}

/* functional J and its directional derivative along df */
int orc_functional_dir(const orc_problem* q, const double* f, const double* df, double* J, double* dJ) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> gd = geo_of(p);
    Geo<Dual> g;
    g.ni = gd.ni; g.nj = gd.nj;
    for (double v : gd.V) g.V.push_back(Dual(v));
    for (double v : gd.Sx) g.Sx.push_back(Dual(v));
    for (double v : gd.Sy) g.Sy.push_back(Dual(v));
    size_t n = (size_t)p.ni * p.nj * p.nv * 2;
    std::vector<Dual> fd(n);
    for (size_t i = 0; i < n; ++i) fd[i] = Dual(f[i], df ? df[i] : 0.0);
    Dual Jd = functional(p, K, g, fd.data());
    *J = Jd.v;
    if (dJ) *dJ = Jd.d;
    return 0;
}

double orc_functional(const orc_problem* q, const double* f) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> g = geo_of(p);
    return functional(p, K, g, f);
}

int orc_functional_grad(const orc_problem* q, const double* f, double* dJ) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> g = geo_of(p);
    functional_grad(p, K, g, f, dJ);
    return 0;
}

int orc_apply_RT(const orc_problem* q, const double* f, const double* lam, double* out) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> g = geo_of(p);
    std::vector<double> dC;
    collision_partials(p, K, g, f, dC);
    apply_RT(p, K, g, f, dC.data(), lam, out);
    return 0;
}

/* the point-implicit diagonal D = V/tau + sum_e max(a_e, 0) at the state f, [ncell][nv] */
int orc_diagonal(const orc_problem* q, const double* f, double* D) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> g = geo_of(p);
    diagonal_all(p, K, g, f, D);
    return 0;
}

/* point-implicit (Jacobi) update of every cell: f_new = f - R(f)/D.  Returns the residual norm of
 * the input state in *norm. */
int orc_jacobi(const orc_problem* q, const double* f, double* fnew, double* norm) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> g = geo_of(p);
    size_t n = (size_t)p.ni * p.nj * p.nv;
    std::vector<double> R(2 * n), Dg(n);
    residual_all(p, K, g, f, R.data());
    diagonal_all(p, K, g, f, Dg.data());
    for (size_t ck = 0; ck < n; ++ck) {
        fnew[2 * ck] = f[2 * ck] - R[2 * ck] / Dg[ck];
        fnew[2 * ck + 1] = f[2 * ck + 1] - R[2 * ck + 1] / Dg[ck];
    }
    if (norm) *norm = residual_norm(p, g, R.data());
    return 0;
}

/* point-implicit (Jacobi) update of the adjoint: phi_new = phi - Ra/D with the scatter-form
 * adjoint residual Ra.  *norm = w-weighted norm of Ra/V of the input. */
int orc_adjoint_jacobi(const orc_problem* q, const double* f, const double* phi, double* phinew, double* norm) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> g = geo_of(p);
    size_t n = (size_t)p.ni * p.nj * p.nv;
    std::vector<double> js(2 * n), Ra(2 * n), Dg(n), dC;
    functional_grad(p, K, g, f, js.data());
    collision_partials(p, K, g, f, dC);
    adjoint_residual(p, K, g, f, dC.data(), js.data(), phi, Ra.data());
    diagonal_all(p, K, g, f, Dg.data());
    for (size_t ck = 0; ck < n; ++ck) {
        phinew[2 * ck] = phi[2 * ck] - Ra[2 * ck] / Dg[ck];
        phinew[2 * ck + 1] = phi[2 * ck + 1] - Ra[2 * ck + 1] / Dg[ck];
    }
    if (norm) *norm = residual_norm(p, g, Ra.data());
    return 0;
}

/* Point-implicit (Jacobi) update of selected cells only, out[n][nv][2]: the cell update of the
 * Gauss-Seidel solver applied to the unmodified state (so it equals one Jacobi sweep there). */
int orc_jacobi_cells(const orc_problem* q, const double* f, int n, const int* cells, double* out) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> g = geo_of(p);
#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < n; ++s) gs_update_cell(p, K, g, f, cells[s], out + (size_t)s * p.nv * 2);
    return 0;
}

/* Adjoint point-implicit update of selected cells (gather form, see adjoint_gs_update_cell). */
int orc_adjoint_jacobi_cells(const orc_problem* q, const double* f, const double* phi, int n, const int* cells,
                             double* out) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> g = geo_of(p);
    std::vector<double> js((size_t)p.ni * p.nj * p.nv * 2);
    functional_grad(p, K, g, f, js.data());
#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < n; ++s) {
        std::vector<double> dCc((size_t)4 * p.nv * 2);
        collision_partials_cell(p, K, g, f, cells[s], dCc.data());
        adjoint_gs_update_cell(p, K, g, f, js.data(), dCc.data(), phi, cells[s], out + (size_t)s * p.nv * 2);
    }
    return 0;
}

/* Solve R(f) = 0 in place by Gauss-Seidel sweeps until |R|/r0 <= tol, r0 = |R(free stream)|.
 * Returns 0 when converged, 4 otherwise. */
int orc_primal_solve(const orc_problem* q, double* f, double tol, int max_sweeps, double* rel, int* sweeps) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> g = geo_of(p);
    size_t n = (size_t)p.ni * p.nj * p.nv * 2;
    std::vector<double> R(n), fs(n);
    orc_freestream(q, fs.data());
    residual_all(p, K, g, fs.data(), R.data());
    double r0 = residual_norm(p, g, R.data());
    double r = 0.0;
    int s = 0;
    for (; s <= max_sweeps; ++s) {
        if (s % 4 == 0 || s == max_sweeps) {
            residual_all(p, K, g, f, R.data());
            r = residual_norm(p, g, R.data()) / r0;
            if (r <= tol || !std::isfinite(r) || s == max_sweeps) break;
        }
        gs_sweep(p, K, g, f, s % 4);
    }
    *rel = r;
    *sweeps = s;
    return (r <= tol) ? 0 : 4;
}

/* Solve the discrete adjoint (dR/df)^T (w phi) = -dJ/df in place; |Ra|/|Ra(phi=0)| <= tol. */
int orc_adjoint_solve(const orc_problem* q, const double* f, double* phi, double tol, int max_sweeps,
                      double* rel, int* sweeps) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> g = geo_of(p);
    size_t n = (size_t)p.ni * p.nj * p.nv * 2;
    std::vector<double> js(n), Ra(n), zero(n, 0.0), dC;
    functional_grad(p, K, g, f, js.data());
    collision_partials(p, K, g, f, dC);
    adjoint_residual(p, K, g, f, dC.data(), js.data(), zero.data(), Ra.data());
    double r0 = residual_norm(p, g, Ra.data());
    double r = 0.0;
    int s = 0;
    for (; s <= max_sweeps; ++s) {
        if (s % 4 == 0 || s == max_sweeps) {
            adjoint_residual(p, K, g, f, dC.data(), js.data(), phi, Ra.data());
            r = residual_norm(p, g, Ra.data()) / r0;
            if (r <= tol || !std::isfinite(r) || s == max_sweeps) break;
        }
        int ni = p.ni, nj = p.nj;
        bool jup = (s & 1) == 0, iup = (s & 2) == 0;
        for (int jj = 0; jj < nj; ++jj) {
            int j = jup ? jj : nj - 1 - jj;
            for (int ii = 0; ii < ni; ++ii) {
                int i = iup ? ii : ni - 1 - ii;
                int c = j * ni + i;
                adjoint_gs_update_cell(p, K, g, f, js.data(), dC.data() + (size_t)c * 4 * p.nv * 2, phi, c,
                                       phi + (size_t)c * p.nv * 2);
            }
        }
    }
    *rel = r;
    *sweeps = s;
    return (r <= tol) ? 0 : 4;
}

/* Full-discrete sensitivity: dJ/dalpha_p = dJ/dalpha_p|_f + sum_{c,k,comp} w phi dR/dalpha_p|_f,
 * with dR/dalpha and dJ/dalpha from dual numbers carried through the geometry along the node
 * tangent dnodes[p] = d(all nodes)/d(alpha_p), [P][(nj+1)][ni][2]. */
int orc_sens_full(const orc_problem* q, const double* f, const double* phi, int P,
                  const double* dnodes, double* grad) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    size_t nn = (size_t)(p.nj + 1) * p.ni * 2;
    size_t n = (size_t)p.ni * p.nj * p.nv * 2;
    std::vector<Dual> fd(n), Rd(n), Xd(nn);
    for (size_t i = 0; i < n; ++i) fd[i] = Dual(f[i]);
    for (int ip = 0; ip < P; ++ip) {
        for (size_t i = 0; i < nn; ++i) Xd[i] = Dual(p.nodes[i], dnodes[ip * nn + i]);
        Geo<Dual> g;
        build_geo<Dual>(p.ni, p.nj, Xd.data(), g);
        residual_all(p, K, g, fd.data(), Rd.data());
        Dual J = functional(p, K, g, fd.data());
        double s = J.d;
        for (size_t ck = 0; ck < n / 2; ++ck) {
            double w = p.w[ck % p.nv];
            s += w * (phi[2 * ck] * Rd[2 * ck].d + phi[2 * ck + 1] * Rd[2 * ck + 1].d);
        }
        grad[ip] = s;
    }
    return 0;
}

/* Eq. (sens_nod) for one node x_a of a 2-node surface element with other node x_b and unit
 * normal n: dA/dx_a [2], dn/dx_a [2][2] (row = component of n, column = component of x_a). */
int orc_sens_nod(const double* xa, const double* xb, const double* n, double* dA, double* dn) {
    double ex = xa[0] - xb[0], ey = xa[1] - xb[1];
    double A = std::sqrt(ex * ex + ey * ey);
    dA[0] = ex / A;
    dA[1] = ey / A;
    double cross = ex * n[1] - ey * n[0];
    double sg = cross > 0.0 ? 1.0 : (cross < 0.0 ? -1.0 : 0.0);
    dn[0] = sg / A * (-n[0] * n[1]);
    dn[1] = sg / A * (-n[1] * n[1]);
    dn[2] = sg / A * (n[0] * n[0]);
    dn[3] = sg / A * (n[0] * n[1]);
    return 0;
}

/* The paper's boundary sensitivity (Sec. 3.2).  For each wall element l (cell c = l, face 3):
 *   f_{l,k}   = f_c on Xi+ (a > 0), g_w = F_rhow gbar_w on Xi-            (face values)
 *   grad f_{l,k} = (1/V_c) sum_e F_{e,k} S_e                               Eq. (gaussgrad)
 *   phi_w,l,k = (-(v.n)(phi1 + m), -(v.n) phi2) on Xi-                     Eq. (formula_adjointbgk)
 *   dL/dA  = sum_k w m (v.n) f1                                            Eq. (sens_J_itf), dB/dA = 0
 *   dL/dx  = sum_k w m (v.n) A grad f1
 *          + sum_{Xi-} w [ A phi_w . grad f - A (phi_w . gbar) sum_{Xi+} w' (v'.n) grad f1' ]  Eq. (sens_B_itf)
 *   dL/dn  = sum_k w m v A f1 - sum_{Xi-} w A (phi_w . gbar) sum_k' w' v' f1'  Eq. (sens_B_itf)
 *            (the factor A_l in the second term follows from B_{w,l,k} ~ A_l, Eq. numer_B)
 * then Eq. (sens_nod) to the two nodes of each element and the chain rule with dwall[P][ni][2].
 * elem[ni][5] receives (dL/dA, dL/dx1, dL/dx2, dL/dn1, dL/dn2); node_grad[ni][2] dL/dx_m. */
int orc_sens_paper(const orc_problem* q, const double* f, const double* phi, int P, const double* dwall,
                   double* grad, double* node_grad, double* elem) {
    Prob p = to_prob(q);
    Consts K = make_consts(p);
    Geo<double> g = geo_of(p);
    const int nv = p.nv, ni = p.ni;
    std::vector<double> ng(2 * ni, 0.0);
    std::vector<double> F1(4 * nv), F2(4 * nv), gx1(nv), gy1(nv), gx2(nv), gy2(nv);
    for (int l = 0; l < ni; ++l) {
        int c = l;
        const double* fc = f + (size_t)c * nv * 2;
        const double* pc = phi + (size_t)c * nv * 2;
        WallFace<double> wf = wall_face(p, K, g, fc, c);
        double A = wf.A, nx = wf.nx, ny = wf.ny;
        /* interface values of all four faces, as in the residual */
        for (int e = 0; e < 4; ++e) {
            int nb = neighbour(p.ni, p.nj, c, e);
            for (int k = 0; k < nv; ++k) {
                double a = g.Sx[4 * c + e] * p.vx[k] + g.Sy[4 * c + e] * p.vy[k];
                double v1, v2;
                if (a > 0.0) { v1 = fc[2 * k]; v2 = fc[2 * k + 1]; }
                else if (nb >= 0) { v1 = f[((size_t)nb * nv + k) * 2]; v2 = f[((size_t)nb * nv + k) * 2 + 1]; }
                else if (nb == FAR) { v1 = K.fd1[k]; v2 = K.fd2[k]; }
                else { double gb = K.gw1[k] / wf.D; v1 = wf.Fw * gb; v2 = wf.Fw * 0.5 * K.Tw * gb; }
                F1[e * nv + k] = v1;
                F2[e * nv + k] = v2;
            }
        }
        for (int k = 0; k < nv; ++k) {
            double sx1 = 0, sy1 = 0, sx2 = 0, sy2 = 0;
            for (int e = 0; e < 4; ++e) {
                sx1 += F1[e * nv + k] * g.Sx[4 * c + e];
                sy1 += F1[e * nv + k] * g.Sy[4 * c + e];
                sx2 += F2[e * nv + k] * g.Sx[4 * c + e];
                sy2 += F2[e * nv + k] * g.Sy[4 * c + e];
            }
            gx1[k] = sx1 / g.V[c]; gy1[k] = sy1 / g.V[c];
            gx2[k] = sx2 / g.V[c]; gy2[k] = sy2 / g.V[c];
        }
        /* wall-face values f_{l,k} are the face-3 interface values */
        const double* fl1 = &F1[3 * nv];
        /* sums over the Xi+ / all velocities used by the B_w derivatives */
        double Gp_x = 0, Gp_y = 0;   /* sum_{Xi+} w (v.n) grad f1 */
        double Vf_x = 0, Vf_y = 0;   /* sum_k w v f1_l */
        for (int k = 0; k < nv; ++k) {
            double vn = p.vx[k] * nx + p.vy[k] * ny;
            if (vn > 0.0) { Gp_x += p.w[k] * vn * gx1[k]; Gp_y += p.w[k] * vn * gy1[k]; }
            Vf_x += p.w[k] * p.vx[k] * fl1[k];
            Vf_y += p.w[k] * p.vy[k] * fl1[k];
        }
        double dA = 0, dxx = 0, dxy = 0, dnx = 0, dny = 0;
        for (int k = 0; k < nv; ++k) {
            double vx = p.vx[k], vy = p.vy[k], w = p.w[k];
            double m = moment_J(p.dir, vx, vy);
            double vn = vx * nx + vy * ny;
            /* J part, Eq. (sens_J_itf) */
            dA += w * m * vn * fl1[k];
            dxx += w * m * vn * A * gx1[k];
            dxy += w * m * vn * A * gy1[k];
            dnx += w * m * vx * A * fl1[k];
            dny += w * m * vy * A * fl1[k];
            if (!(vn > 0.0)) {
                /* B_w part on Xi-, Eq. (sens_B_itf) */
                double pw1 = -vn * (pc[2 * k] + m), pw2 = -vn * pc[2 * k + 1];
                double gb1 = K.gw1[k] / wf.D, gb2 = 0.5 * K.Tw * gb1;
                double pg = pw1 * gb1 + pw2 * gb2;
                dxx += w * (A * (pw1 * gx1[k] + pw2 * gx2[k]) - A * pg * Gp_x);
                dxy += w * (A * (pw1 * gy1[k] + pw2 * gy2[k]) - A * pg * Gp_y);
                dnx -= w * A * pg * Vf_x;
                dny -= w * A * pg * Vf_y;
            }
        }
        if (elem) {
            elem[5 * l + 0] = dA; elem[5 * l + 1] = dxx; elem[5 * l + 2] = dxy;
            elem[5 * l + 3] = dnx; elem[5 * l + 4] = dny;
        }
        /* element -> its two wall nodes, Eq. (sens_nod): nodes (0,l) and (0,l+1) */
        int na[2] = {l, (l + 1) % ni};
        for (int s = 0; s < 2; ++s) {
            const double* xa = p.nodes + 2 * na[s];
            const double* xb = p.nodes + 2 * na[1 - s];
            double n2[2] = {nx, ny}, dAx[2], dnx2[4];
            orc_sens_nod(xa, xb, n2, dAx, dnx2);
            ng[2 * na[s]] += dA * dAx[0] + 0.5 * dxx + dnx * dnx2[0] + dny * dnx2[2];
            ng[2 * na[s] + 1] += dA * dAx[1] + 0.5 * dxy + dnx * dnx2[1] + dny * dnx2[3];
        }
    }
    if (node_grad) std::memcpy(node_grad, ng.data(), sizeof(double) * 2 * ni);
    for (int ip = 0; ip < P; ++ip) {
        double s = 0.0;
        for (int m = 0; m < 2 * ni; ++m) s += ng[m] * dwall[(size_t)ip * 2 * ni + m];
        grad[ip] = s;
    }
    return 0;
}

/* Volume constraint of Eq. (formula_opt): Q = (1/D) sum_l x_l . n_l A_l + V_min (D = 2, n_l into the
 * solid, x_l the element midpoint; exact for straight elements), and its node sensitivity
 * Eq. (sens_con_nod): dQ/dx_m = sum over the elements z containing node m of (1/D) A_z n_z.
 * dQ[ni][2] receives dQ/dx of the wall nodes; dQda[P] the contraction with dwall[P][ni][2]. */
double orc_volume_constraint(const orc_problem* q, double vmin, int P, const double* dwall, double* dQ, double* dQda) {
    Prob p = to_prob(q);
    Geo<double> g = geo_of(p);
    const int ni = p.ni;
    double Q = vmin;
    std::vector<double> node(2 * ni, 0.0);
    for (int l = 0; l < ni; ++l) {
        const double* xa = p.nodes + 2 * l;
        const double* xb = p.nodes + 2 * ((l + 1) % ni);
        const double xm = 0.5 * (xa[0] + xb[0]), ym = 0.5 * (xa[1] + xb[1]);
        const double Sx = g.Sx[4 * l + 3], Sy = g.Sy[4 * l + 3];   /* A_l n_l, into the solid */
        Q += 0.5 * (xm * Sx + ym * Sy);
        for (int m : {l, (l + 1) % ni}) {
            node[2 * m] += 0.5 * Sx;
            node[2 * m + 1] += 0.5 * Sy;
        }
    }
    if (dQ) std::memcpy(dQ, node.data(), sizeof(double) * 2 * ni);
    if (dQda)
        for (int ip = 0; ip < P; ++ip) {
            double s2 = 0.0;
            for (int m = 0; m < 2 * ni; ++m) s2 += node[m] * dwall[(size_t)ip * 2 * ni + m];
            dQda[ip] = s2;
        }
    return Q;
}

/* Wall functional of one face for given wall-cell values (used by the free-molecular check):
 * J_l = sum_k w m a f1_l with f1_l = f1 on a > 0 and F_rhow gbar1 otherwise. */
double orc_wall_face_functional(const double* S, int nv, const double* vx, const double* vy,
                                const double* w, const double* f1, double Tw, const double* dir) {
    double A = std::sqrt(S[0] * S[0] + S[1] * S[1]), nx = S[0] / A, ny = S[1] / A;
    double Fw = 0.0, D = 0.0;
    for (int k = 0; k < nv; ++k) {
        double vn = vx[k] * nx + vy[k] * ny, g1, g2;
        maxwellian<double>(1.0, 0.0, 0.0, Tw, vx[k], vy[k], g1, g2);
        if (vn > 0.0) Fw += w[k] * vn * f1[k];
        else D -= w[k] * vn * g1;
    }
    double J = 0.0;
    for (int k = 0; k < nv; ++k) {
        double a = S[0] * vx[k] + S[1] * vy[k], g1, g2;
        maxwellian<double>(1.0, 0.0, 0.0, Tw, vx[k], vy[k], g1, g2);
        double m = moment_J(dir, vx[k], vy[k]);
        J += w[k] * m * a * (a > 0.0 ? f1[k] : Fw * g1 / D);
    }
    return J;
}

} /* extern "C" */
