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

inline int kr_cdiv(int a, int b) { return (a + b - 1) / b; }

}  // namespace

size_t krylov_part_count(int m) { return (size_t)(m + 1) * kKB; }

void krylov_release_graphs(KrylovWork& K) {
    for (int t = 0; t < 2; ++t) {
        if (K.graph[t]) cudaGraphExecDestroy(K.graph[t]);
        K.graph[t] = nullptr;
        K.key_m[t] = 0;
    }
}

static cudaError_t enqueue_gmres(const DevMesh& msh, const double* out, const double* dinv, const double4* rhs_neg,
                                 bool transpose, int m, const KrylovWork& K, double4* x, cudaStream_t s) {
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
        k_kr_matvec<<<gb, kKT, 0, s>>>(nc, msh.nb, out, dinv, K.V + (size_t)j * nc, K.w, tr);
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
    k_kr_combine<<<gb, kKT, 0, s>>>(nc, m, K.V, K.y, dinv, tr, x);
    return cudaGetLastError();
}

cudaError_t launch_coarse_gmres(const DevMesh& msh, const double* out, const double* dinv, const double4* rhs_neg,
                                bool transpose, int m, KrylovWork& K, double4* x, bool use_graph, cudaStream_t s) {
    if (m < 1 || m > kMaxKrylov || !K.V || !K.w || !K.part || !K.H || !K.scal || !K.y) return cudaErrorInvalidValue;
    if (!use_graph || s == nullptr) return enqueue_gmres(msh, out, dinv, rhs_neg, transpose, m, K, x, s);
    const int t = transpose ? 1 : 0;
    const void* key[4] = {out, dinv, rhs_neg, x};
    bool hit = K.graph[t] && K.key_m[t] == m;
    for (int i = 0; i < 4 && hit; ++i) hit = K.key[t][i] == key[i];
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
        const cudaError_t ce = enqueue_gmres(msh, out, dinv, rhs_neg, transpose, m, K, x, s);
        e = cudaStreamEndCapture(s, &g);
        if (ce != cudaSuccess) { if (e == cudaSuccess) cudaGraphDestroy(g); return ce; }
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(&K.graph[t], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { K.graph[t] = nullptr; return e; }
        for (int i = 0; i < 4; ++i) K.key[t][i] = key[i];
        K.key_m[t] = m;
    }
    return cudaGraphLaunch(K.graph[t], s);
}

int krylov_launches(int m) { return 6 + 10 * m; }

}  // namespace dvm
