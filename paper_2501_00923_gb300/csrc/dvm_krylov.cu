// GMRES on the moment system of the macroscopic prediction: A x = b for the primal sweeps and the
// refinement's correction sweeps, A^T x = b for the adjoint sweeps.  A has a 4x4 block per cell and
// one per face neighbour: the diagonal block D_c (the cell's outflow blocks summed, plus the wall's
// re-emission) and the coupling -OUT[nb][e'] of the neighbour's outflow through the shared face
// (see k_coarse_assemble).  Block-Jacobi alone diverges on large subsonic meshes (its iteration is
// non-normal and not contractive there), so the blocks serve as the right preconditioner of one GMRES
// cycle of m Arnoldi steps (classical Gram-Schmidt, applied twice), which minimises the residual over
// the Krylov space and cannot amplify it.
//
// Every scalar of the solve stays in device memory: no host synchronisation inside it, and a fixed
// sequence of launches.  Dot products are summed in a fixed order (a fixed grid of blocks, then one
// block over their partial sums), so the solve is bitwise reproducible.
#include "dvm_internal.h"

namespace dvm {
namespace {

constexpr int kKT = 256;      // threads per block
constexpr int kKB = 256;      // blocks of the dot-product kernel (= kKT: one reduction pass sums them)

__device__ __forceinline__ double kr_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a block of kKT threads in a fixed order; the result is valid in thread 0.
__device__ __forceinline__ double kr_block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = kr_warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = threadIdx.x < kKT / 32 ? sh[threadIdx.x] : 0.0;
    if (wid == 0) v = kr_warp_sum(v);
    __syncthreads();
    return v;
}

__device__ __forceinline__ double dot4(double4 a, double4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }

// z = M^{-1} v for one cell: M = D (primal) or D^T (adjoint); dinv holds D^{-1} row-major.
__device__ __forceinline__ void kr_precond(const double* __restrict__ d, double4 v, bool tr, double z[4]) {
    const double vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
        z[i] = tr ? d[i] * vv[0] + d[4 + i] * vv[1] + d[8 + i] * vv[2] + d[12 + i] * vv[3]
                  : d[4 * i] * vv[0] + d[4 * i + 1] * vv[1] + d[4 * i + 2] * vv[2] + d[4 * i + 3] * vv[3];
}

// w = A M^{-1} v = v - sum_e C_e z_nb(e), z = M^{-1} v (the diagonal block cancels its preconditioner).
// Primal: C_e = OUT[nb][e^2] (faces 0/2 and 1/3 of neighbouring cells are the same face); adjoint:
// C_e = OUT[c][e]^T.
__global__ void __launch_bounds__(kKT) k_kr_matvec(int ncell, const int4* __restrict__ nb, const double* __restrict__ out,
                                                   const double* __restrict__ dinv, const double4* __restrict__ v,
                                                   double4* __restrict__ w, int tr) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double4 vc = v[c];
    double r[4] = {vc.x, vc.y, vc.z, vc.w};
    const int4 n4 = nb[c];
    const int nbs[4] = {n4.x, n4.y, n4.z, n4.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int n = nbs[e];
        if (n < 0) continue;
        double z[4];
        kr_precond(dinv + (size_t)n * 16, v[n], tr != 0, z);
        if (tr) {
            const double* o = out + ((size_t)c * 4 + e) * 16;
#pragma unroll
            for (int i = 0; i < 4; ++i) r[i] -= o[i] * z[0] + o[4 + i] * z[1] + o[8 + i] * z[2] + o[12 + i] * z[3];
        } else {
            const double* o = out + ((size_t)n * 4 + (e ^ 2)) * 16;
#pragma unroll
            for (int i = 0; i < 4; ++i) r[i] -= o[4 * i] * z[0] + o[4 * i + 1] * z[1] + o[4 * i + 2] * z[2] + o[4 * i + 3] * z[3];
        }
    }
    w[c] = make_double4(r[0], r[1], r[2], r[3]);
}

// part[i][block] = partial sums of <V_i, w> for i < nvec (V_i = V + i ncell), over a fixed grid.
__global__ void __launch_bounds__(kKT) k_kr_dots(int ncell, int nvec, const double4* __restrict__ V,
                                                 const double4* __restrict__ w, double* __restrict__ part) {
    __shared__ double sh[kKT / 32];
    for (int i = 0; i < nvec; ++i) {
        const double4* vi = V + (size_t)i * ncell;
        double s = 0.0;
        for (int c = blockIdx.x * kKT + threadIdx.x; c < ncell; c += kKB * kKT) s += dot4(vi[c], w[c]);
        s = kr_block_sum(s, sh);
        if (threadIdx.x == 0) part[(size_t)i * kKB + blockIdx.x] = s;
    }
}

// out[i] = sum of part[i][:] (fixed order); col[i] = out[i] (add = 0) or col[i] += out[i] (add = 1).
__global__ void __launch_bounds__(kKT) k_kr_reduce(int nvec, const double* __restrict__ part, double* __restrict__ out,
                                                   double* __restrict__ col, int add) {
    __shared__ double sh[kKT / 32];
    for (int i = 0; i < nvec; ++i) {
        const double s = kr_block_sum(part[(size_t)i * kKB + threadIdx.x], sh);
        if (threadIdx.x == 0) {
            out[i] = s;
            if (col) col[i] = add ? col[i] + s : s;
        }
    }
}

// w -= sum_{i < nvec} h[i] V_i.
__global__ void __launch_bounds__(kKT) k_kr_orth(int ncell, int nvec, const double4* __restrict__ V,
                                                 const double* __restrict__ h, double4* __restrict__ w) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    double4 a = w[c];
    for (int i = 0; i < nvec; ++i) {
        const double hi = h[i];
        const double4 b = V[(size_t)i * ncell + c];
        a.x -= hi * b.x; a.y -= hi * b.y; a.z -= hi * b.z; a.w -= hi * b.w;
    }
    w[c] = a;
}

// vnext = w / |w| with |w|^2 in nrm2[0]; *hsub = |w| (the subdiagonal of the Hessenberg matrix, or the
// initial residual norm).  A zero or non-finite norm leaves vnext = 0 (the Krylov space is exhausted).
__global__ void __launch_bounds__(kKT) k_kr_normalize(int ncell, const double* __restrict__ nrm2,
                                                      const double4* __restrict__ w, double4* __restrict__ vnext,
                                                      double* __restrict__ hsub) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const double n = sqrt(nrm2[0]);
    const bool ok = n > 0.0 && isfinite(n);
    if (c == 0) *hsub = ok ? n : 0.0;
    if (c >= ncell) return;
    const double inv = ok ? 1.0 / n : 0.0;
    const double4 a = w[c];
    vnext[c] = make_double4(a.x * inv, a.y * inv, a.z * inv, a.w * inv);
}

__global__ void k_kr_neg(int ncell, const double4* __restrict__ b, double4* __restrict__ w) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double4 a = b[c];
    w[c] = make_double4(-a.x, -a.y, -a.z, -a.w);
}

// min |beta e1 - H y| by Givens rotations (one thread; m <= kMaxKrylov).  H is stored by columns,
// column j at H + j (m + 1), rows 0..j+1; it is overwritten with R.  A pivot below 1e-13 of the largest
// ends the basis there (the remaining y are 0).
__global__ void k_kr_lsq(int m, double* __restrict__ H, const double* __restrict__ beta, double* __restrict__ y) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double g[kMaxKrylov + 1], cs[kMaxKrylov], sn[kMaxKrylov];
    g[0] = *beta;
    for (int i = 1; i <= m; ++i) g[i] = 0.0;
    double rmax = 0.0;
    int mm = m;
    for (int j = 0; j < m; ++j) {
        double* h = H + (size_t)j * (m + 1);
        for (int i = 0; i < j; ++i) {
            const double a = h[i], b = h[i + 1];
            h[i] = cs[i] * a + sn[i] * b;
            h[i + 1] = -sn[i] * a + cs[i] * b;
        }
        const double a = h[j], b = h[j + 1], r = hypot(a, b);
        cs[j] = r > 0.0 ? a / r : 1.0;
        sn[j] = r > 0.0 ? b / r : 0.0;
        h[j] = r;
        h[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        rmax = fmax(rmax, r);
        if (!(r > 1e-13 * rmax) || !isfinite(r)) { mm = j; break; }
    }
    for (int j = 0; j < m; ++j) y[j] = 0.0;
    for (int j = mm - 1; j >= 0; --j) {
        double s = g[j];
        for (int k = j + 1; k < mm; ++k) s -= H[(size_t)k * (m + 1) + j] * y[k];
        y[j] = s / H[(size_t)j * (m + 1) + j];
    }
}

// x = M^{-1} sum_j y_j V_j.
__global__ void __launch_bounds__(kKT) k_kr_combine(int ncell, int m, const double4* __restrict__ V,
                                                    const double* __restrict__ y, const double* __restrict__ dinv,
                                                    int tr, double4* __restrict__ x) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    double4 u = make_double4(0.0, 0.0, 0.0, 0.0);
    for (int j = 0; j < m; ++j) {
        const double yj = y[j];
        const double4 b = V[(size_t)j * ncell + c];
        u.x += yj * b.x; u.y += yj * b.y; u.z += yj * b.z; u.w += yj * b.w;
    }
    double z[4];
    kr_precond(dinv + (size_t)c * 16, u, tr != 0, z);
    x[c] = make_double4(z[0], z[1], z[2], z[3]);
}

// ---------------------------------------------------------------------------------- multigrid
// Neighbour of cell c = j ni + i across face e (0: i-1, 1: j+1, 2: i+1, 3: j-1; periodic in i, -1 at
// the far field and the wall), the convention of the O-mesh's neighbour table.
__device__ __forceinline__ int mg_nb(int c, int e, int ni, int nj) {
    const int i = c % ni, j = c / ni;
    if (e == 0) return j * ni + (i + ni - 1) % ni;
    if (e == 2) return j * ni + (i + 1) % ni;
    if (e == 1) return j + 1 < nj ? c + ni : -1;
    return j > 0 ? c - ni : -1;
}

// 4x4 inverse by Gauss-Jordan with partial pivoting (row-major); false (and zeros) when singular.
__device__ bool inv4(const double* a, double* out) {
    double m[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) { m[i][j] = a[4 * i + j]; m[i][4 + j] = i == j ? 1.0 : 0.0; }
    double amax = 0.0;
    for (int i = 0; i < 16; ++i) amax = fmax(amax, fabs(a[i]));
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r) if (fabs(m[r][col]) > fabs(m[piv][col])) piv = r;
        if (!(fabs(m[piv][col]) > 1e-14 * amax)) {
            for (int i = 0; i < 16; ++i) out[i] = 0.0;
            return false;
        }
        if (piv != col)
            for (int k = 0; k < 8; ++k) { const double t = m[col][k]; m[col][k] = m[piv][k]; m[piv][k] = t; }
        const double ip = 1.0 / m[col][col];
        for (int k = 0; k < 8; ++k) m[col][k] *= ip;
        for (int r = 0; r < 4; ++r) {
            if (r == col) continue;
            const double f = m[r][col];
            for (int k = 0; k < 8; ++k) m[r][k] -= f * m[col][k];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) out[4 * i + j] = m[i][4 + j];
    return true;
}

// y = B v (tr: B^T v) for a row-major 4x4 block.
__device__ __forceinline__ void mv4(const double* B, const double v[4], bool tr, double y[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
        y[i] = tr ? B[i] * v[0] + B[4 + i] * v[1] + B[8 + i] * v[2] + B[12 + i] * v[3]
                  : B[4 * i] * v[0] + B[4 * i + 1] * v[1] + B[4 * i + 2] * v[2] + B[4 * i + 3] * v[3];
}

__device__ __forceinline__ void ld4(const double4* p, int c, double v[4]) {
    const double4 a = p[c];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

// (A x)_c at one level: D x_c + sum_e C[c][e] x_nb (tr: D^T x_c + sum_e C[nb][e ^ 2]^T x_nb).
__device__ __forceinline__ void mg_ax(int c, int ni, int nj, const double* __restrict__ D, const double* __restrict__ C,
                                     const double4* __restrict__ x, bool tr, double y[4]) {
    double v[4], t[4];
    ld4(x, c, v);
    mv4(D + (size_t)c * 16, v, tr, y);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int n = mg_nb(c, e, ni, nj);
        if (n < 0) continue;
        ld4(x, n, v);
        mv4(tr ? C + ((size_t)n * 4 + (e ^ 2)) * 16 : C + ((size_t)c * 4 + e) * 16, v, tr, t);
        y[0] += t[0]; y[1] += t[1]; y[2] += t[2]; y[3] += t[3];
    }
}

// The fine level from the assembled blocks: D = (D^{-1})^{-1}, C[c][e] = -OUT[nb][e ^ 2].
__global__ void __launch_bounds__(kKT) k_mg_fine(int nc, int ni, int nj, const double* __restrict__ out,
                                                 const double* __restrict__ dinv, double* __restrict__ D,
                                                 double* __restrict__ Dinv, double* __restrict__ C) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double a[16], b[16];
    for (int k = 0; k < 16; ++k) a[k] = dinv[(size_t)c * 16 + k];
    inv4(a, b);
    for (int k = 0; k < 16; ++k) { D[(size_t)c * 16 + k] = b[k]; Dinv[(size_t)c * 16 + k] = a[k]; }
    for (int e = 0; e < 4; ++e) {
        const int n = mg_nb(c, e, ni, nj);
        double* o = C + ((size_t)c * 4 + e) * 16;
        const double* src = n >= 0 ? out + ((size_t)n * 4 + (e ^ 2)) * 16 : nullptr;
        for (int k = 0; k < 16; ++k) o[k] = src ? -src[k] : 0.0;
    }
}

// Galerkin coarse level (P piecewise constant over 2x2 children, R = P^T): D sums the children's
// diagonal blocks and their couplings to each other, C[e] the children's couplings across face e.
__global__ void __launch_bounds__(kKT) k_mg_coarsen(int ncC, int niC, int niF, const double* __restrict__ DF,
                                                    const double* __restrict__ CF, double* __restrict__ DC,
                                                    double* __restrict__ CC) {
    const int C_ = blockIdx.x * blockDim.x + threadIdx.x;
    if (C_ >= ncC) return;
    const int I = C_ % niC, J = C_ / niC;
    double d[16], cc[4][16];
    for (int k = 0; k < 16; ++k) { d[k] = 0.0; cc[0][k] = cc[1][k] = cc[2][k] = cc[3][k] = 0.0; }
    for (int cj = 0; cj < 2; ++cj)
        for (int ci = 0; ci < 2; ++ci) {
            const int f = (2 * J + cj) * niF + 2 * I + ci;
            for (int k = 0; k < 16; ++k) d[k] += DF[(size_t)f * 16 + k];
            for (int e = 0; e < 4; ++e) {
                const bool internal = (e == 0 && ci == 1) || (e == 2 && ci == 0) || (e == 1 && cj == 0) || (e == 3 && cj == 1);
                const double* src = CF + ((size_t)f * 4 + e) * 16;
                double* dst = internal ? d : cc[e];
                for (int k = 0; k < 16; ++k) dst[k] += src[k];
            }
        }
    for (int k = 0; k < 16; ++k) DC[(size_t)C_ * 16 + k] = d[k];
    for (int e = 0; e < 4; ++e)
        for (int k = 0; k < 16; ++k) CC[((size_t)C_ * 4 + e) * 16 + k] = cc[e][k];
}

__global__ void __launch_bounds__(kKT) k_mg_invert(int nc, const double* __restrict__ D, double* __restrict__ Dinv) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double a[16], b[16];
    for (int k = 0; k < 16; ++k) a[k] = D[(size_t)c * 16 + k];
    inv4(a, b);
    for (int k = 0; k < 16; ++k) Dinv[(size_t)c * 16 + k] = b[k];
}

// Damped block-Jacobi smoothing: xn = xo + w D^{-1} (b - A xo) (xo = nullptr: from zero).
__global__ void __launch_bounds__(kKT) k_mg_smooth(int nc, int ni, int nj, const double* __restrict__ D,
                                                   const double* __restrict__ Dinv, const double* __restrict__ C,
                                                   const double4* __restrict__ xo, const double4* __restrict__ b,
                                                   double4* __restrict__ xn, double w, int tr) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double r[4], ax[4] = {0.0, 0.0, 0.0, 0.0}, y[4];
    ld4(b, c, r);
    if (xo) mg_ax(c, ni, nj, D, C, xo, tr != 0, ax);
    for (int k = 0; k < 4; ++k) r[k] -= ax[k];
    mv4(Dinv + (size_t)c * 16, r, tr != 0, y);
    double x0[4] = {0.0, 0.0, 0.0, 0.0};
    if (xo) ld4(xo, c, x0);
    xn[c] = make_double4(x0[0] + w * y[0], x0[1] + w * y[1], x0[2] + w * y[2], x0[3] + w * y[3]);
}

// r = b - A x.
__global__ void __launch_bounds__(kKT) k_mg_residual(int nc, int ni, int nj, const double* __restrict__ D,
                                                     const double* __restrict__ C, const double4* __restrict__ x,
                                                     const double4* __restrict__ b, double4* __restrict__ r, int tr) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double ax[4], bb[4];
    mg_ax(c, ni, nj, D, C, x, tr != 0, ax);
    ld4(b, c, bb);
    r[c] = make_double4(bb[0] - ax[0], bb[1] - ax[1], bb[2] - ax[2], bb[3] - ax[3]);
}

// w = A x at one level.
__global__ void __launch_bounds__(kKT) k_mg_apply(int nc, int ni, int nj, const double* __restrict__ D,
                                                  const double* __restrict__ C, const double4* __restrict__ x,
                                                  double4* __restrict__ w, int tr) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double ax[4];
    mg_ax(c, ni, nj, D, C, x, tr != 0, ax);
    w[c] = make_double4(ax[0], ax[1], ax[2], ax[3]);
}

// bC = R rF (the sum over the 2x2 children).
__global__ void __launch_bounds__(kKT) k_mg_restrict(int ncC, int niC, int niF, const double4* __restrict__ rF,
                                                     double4* __restrict__ bC) {
    const int C_ = blockIdx.x * blockDim.x + threadIdx.x;
    if (C_ >= ncC) return;
    const int I = C_ % niC, J = C_ / niC;
    double4 s = make_double4(0.0, 0.0, 0.0, 0.0);
    for (int cj = 0; cj < 2; ++cj)
        for (int ci = 0; ci < 2; ++ci) {
            const double4 a = rF[(size_t)(2 * J + cj) * niF + 2 * I + ci];
            s.x += a.x; s.y += a.y; s.z += a.z; s.w += a.w;
        }
    bC[C_] = s;
}

// xF += P xC.
__global__ void __launch_bounds__(kKT) k_mg_prolong(int ncF, int niF, int niC, const double4* __restrict__ xC,
                                                    double4* __restrict__ xF) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= ncF) return;
    const int i = f % niF, j = f / niF;
    const double4 a = xC[(size_t)(j / 2) * niC + i / 2];
    double4 x = xF[f];
    x.x += a.x; x.y += a.y; x.z += a.z; x.w += a.w;
    xF[f] = x;
}

// u = sum_j y_j V_j.
__global__ void __launch_bounds__(kKT) k_kr_lincomb(int ncell, int m, const double4* __restrict__ V,
                                                    const double* __restrict__ y, double4* __restrict__ u) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    double4 a = make_double4(0.0, 0.0, 0.0, 0.0);
    for (int j = 0; j < m; ++j) {
        const double yj = y[j];
        const double4 b = V[(size_t)j * ncell + c];
        a.x += yj * b.x; a.y += yj * b.y; a.z += yj * b.z; a.w += yj * b.w;
    }
    u[c] = a;
}

__global__ void k_copy4(int n, const double4* __restrict__ a, double4* __restrict__ b) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) b[c] = a[c];
}

constexpr double kMGSmooth = 0.7;       // damping of the block-Jacobi smoother
constexpr int kMGCoarsest = 30;         // smoothing sweeps on the coarsest level (even)

inline int kr_cdiv(int a, int b) { return (a + b - 1) / b; }

}  // namespace

size_t krylov_part_count(int m) { return (size_t)(m + 1) * kKB; }

int mg_plan(int ni, int nj, int* nis, int* njs) {
    int n = 0;
    nis[n] = ni; njs[n] = nj; ++n;
    while (n < kMaxMGLevels && ni % 2 == 0 && nj % 2 == 0 && ni / 2 >= 3 && ni * nj > 64) {
        ni /= 2; nj /= 2;
        nis[n] = ni; njs[n] = nj; ++n;
    }
    return n;
}

cudaError_t launch_mg_setup(const DevMesh& msh, const double* out, const double* dinv, const MGWork& mg, cudaStream_t s) {
    if (mg.nlev < 1) return cudaErrorInvalidValue;
    const MGLevel& f = mg.lev[0];
    k_mg_fine<<<kr_cdiv(f.nc, kKT), kKT, 0, s>>>(f.nc, f.ni, f.nj, out, dinv, f.D, f.Dinv, f.C);
    for (int l = 1; l < mg.nlev; ++l) {
        const MGLevel& F = mg.lev[l - 1];
        const MGLevel& Cl = mg.lev[l];
        k_mg_coarsen<<<kr_cdiv(Cl.nc, kKT), kKT, 0, s>>>(Cl.nc, Cl.ni, F.ni, F.D, F.C, Cl.D, Cl.C);
        k_mg_invert<<<kr_cdiv(Cl.nc, kKT), kKT, 0, s>>>(Cl.nc, Cl.D, Cl.Dinv);
    }
    return cudaGetLastError();
}

// One V(1,1) cycle from zero at level l for the right-hand side b; returns the buffer holding the result.
static double4* mg_vcycle(const MGWork& mg, int l, const double4* b, int tr, cudaStream_t s) {
    const MGLevel& L = mg.lev[l];
    const int gb = kr_cdiv(L.nc, kKT);
    if (l == mg.nlev - 1) {                     // coarsest: smoothing sweeps, ping-pong x <-> r
        k_mg_smooth<<<gb, kKT, 0, s>>>(L.nc, L.ni, L.nj, L.D, L.Dinv, L.C, nullptr, b, L.x, kMGSmooth, tr);
        double4 *src = L.x, *dst = L.r;
        for (int k = 1; k < kMGCoarsest; ++k) {
            k_mg_smooth<<<gb, kKT, 0, s>>>(L.nc, L.ni, L.nj, L.D, L.Dinv, L.C, src, b, dst, kMGSmooth, tr);
            double4* t = src; src = dst; dst = t;
        }
        return src;
    }
    const MGLevel& Cl = mg.lev[l + 1];
    k_mg_smooth<<<gb, kKT, 0, s>>>(L.nc, L.ni, L.nj, L.D, L.Dinv, L.C, nullptr, b, L.x, kMGSmooth, tr);
    k_mg_residual<<<gb, kKT, 0, s>>>(L.nc, L.ni, L.nj, L.D, L.C, L.x, b, L.r, tr);
    k_mg_restrict<<<kr_cdiv(Cl.nc, kKT), kKT, 0, s>>>(Cl.nc, Cl.ni, L.ni, L.r, Cl.b);
    const double4* xc = mg_vcycle(mg, l + 1, Cl.b, tr, s);
    k_mg_prolong<<<gb, kKT, 0, s>>>(L.nc, L.ni, Cl.ni, xc, L.x);
    k_mg_smooth<<<gb, kKT, 0, s>>>(L.nc, L.ni, L.nj, L.D, L.Dinv, L.C, L.x, b, L.r, kMGSmooth, tr);
    return L.r;
}

void krylov_release_graphs(KrylovWork& K) {
    for (int t = 0; t < 2; ++t) {
        if (K.graph[t]) cudaGraphExecDestroy(K.graph[t]);
        K.graph[t] = nullptr;
        K.key_m[t] = 0;
    }
}

static cudaError_t enqueue_gmres(const DevMesh& msh, const double* out, const double* dinv, const double4* rhs_neg,
                                 bool transpose, int m, const KrylovWork& K, double4* x, cudaStream_t s,
                                 const MGWork* mg) {
    const int nc = msh.ncell, gb = kr_cdiv(nc, kKT), tr = transpose ? 1 : 0;
    double* nrm2 = K.scal;             // scratch: |w|^2
    double* beta = K.scal + 1;         // |b|
    double* hh = K.scal + 2;           // scratch: one Gram-Schmidt pass's coefficients (m + 1)
    // r0 = b (x0 = 0), V_0 = b / |b|
    k_kr_neg<<<gb, kKT, 0, s>>>(nc, rhs_neg, K.w);
    k_kr_dots<<<kKB, kKT, 0, s>>>(nc, 1, K.w, K.w, K.part);
    k_kr_reduce<<<1, kKT, 0, s>>>(1, K.part, nrm2, nullptr, 0);
    k_kr_normalize<<<gb, kKT, 0, s>>>(nc, nrm2, K.w, K.V, beta);
    for (int j = 0; j < m; ++j) {
        double* col = K.H + (size_t)j * (m + 1);
        if (mg) {                       // w = A M^{-1} V_j, M^{-1} one V-cycle
            const double4* z = mg_vcycle(*mg, 0, K.V + (size_t)j * nc, tr, s);
            const MGLevel& L = mg->lev[0];
            k_mg_apply<<<gb, kKT, 0, s>>>(nc, L.ni, L.nj, L.D, L.C, z, K.w, tr);
        } else {
            k_kr_matvec<<<gb, kKT, 0, s>>>(nc, msh.nb, out, dinv, K.V + (size_t)j * nc, K.w, tr);
        }
        for (int pass = 0; pass < 2; ++pass) {
            k_kr_dots<<<kKB, kKT, 0, s>>>(nc, j + 1, K.V, K.w, K.part);
            k_kr_reduce<<<1, kKT, 0, s>>>(j + 1, K.part, hh, col, pass);
            k_kr_orth<<<gb, kKT, 0, s>>>(nc, j + 1, K.V, hh, K.w);
        }
        k_kr_dots<<<kKB, kKT, 0, s>>>(nc, 1, K.w, K.w, K.part);
        k_kr_reduce<<<1, kKT, 0, s>>>(1, K.part, nrm2, nullptr, 0);
        k_kr_normalize<<<gb, kKT, 0, s>>>(nc, nrm2, K.w, K.V + (size_t)(j + 1) * nc, col + j + 1);
    }
    k_kr_lsq<<<1, 32, 0, s>>>(m, K.H, beta, K.y);
    if (mg) {                           // x = M^{-1} sum_j y_j V_j
        k_kr_lincomb<<<gb, kKT, 0, s>>>(nc, m, K.V, K.y, K.w);
        const double4* z = mg_vcycle(*mg, 0, K.w, tr, s);
        k_copy4<<<gb, kKT, 0, s>>>(nc, z, x);
    } else {
        k_kr_combine<<<gb, kKT, 0, s>>>(nc, m, K.V, K.y, dinv, tr, x);
    }
    return cudaGetLastError();
}

cudaError_t launch_coarse_gmres(const DevMesh& msh, const double* out, const double* dinv, const double4* rhs_neg,
                                bool transpose, int m, KrylovWork& K, double4* x, bool use_graph, cudaStream_t s,
                                const MGWork* mg) {
    if (m < 1 || m > kMaxKrylov || !K.V || !K.w || !K.part || !K.H || !K.scal || !K.y) return cudaErrorInvalidValue;
    if (mg && (mg->nlev < 1 || mg->lev[0].nc != msh.ncell)) return cudaErrorInvalidValue;
    if (!use_graph || s == nullptr) return enqueue_gmres(msh, out, dinv, rhs_neg, transpose, m, K, x, s, mg);
    const int t = transpose ? 1 : 0;
    const void* key[5] = {out, dinv, rhs_neg, x, mg};
    bool hit = K.graph[t] && K.key_m[t] == m;
    for (int i = 0; i < 5 && hit; ++i) hit = K.key[t][i] == key[i];
    if (!hit) {
        if (K.graph[t]) {                 // a replay of the old graph may still be in flight
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
            cudaGraphExecDestroy(K.graph[t]);
        }
        K.graph[t] = nullptr;
        K.key_m[t] = 0;
        cudaGraph_t g;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const cudaError_t ce = enqueue_gmres(msh, out, dinv, rhs_neg, transpose, m, K, x, s, mg);
        e = cudaStreamEndCapture(s, &g);
        if (ce != cudaSuccess) { if (e == cudaSuccess) cudaGraphDestroy(g); return ce; }
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(&K.graph[t], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { K.graph[t] = nullptr; return e; }
        for (int i = 0; i < 5; ++i) K.key[t][i] = key[i];
        K.key_m[t] = m;
    }
    return cudaGraphLaunch(K.graph[t], s);
}

int krylov_launches(int m) { return 6 + 10 * m; }

}  // namespace dvm
