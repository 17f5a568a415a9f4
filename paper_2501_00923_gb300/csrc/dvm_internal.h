// Internal declarations of the DVM CUDA library: device-side data of meshes, velocity grids,
// states and adjoints, and the kernel launchers.  Not part of the C ABI (see include/dvm.h).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstddef>
#include <cstdint>
#include <type_traits>

namespace dvm {

constexpr int kWall = -1;            // neighbour code of a wall face
constexpr int kFar = -2;             // neighbour code of a far-field face
constexpr int kWarpsPerBlock = 8;    // one warp per cell, 8 cells per 256-thread block
constexpr int kPad = 4;              // velocity count padded to a multiple of this

// Geometry of an O-mesh on the device.  Face e of cell c: 0 -> (i-1,j), 1 -> (i,j+1) or far field,
// 2 -> (i+1,j), 3 -> (i,j-1) or wall.  S = A n points out of the cell (into the solid on the wall).
struct DevMesh {
    int ni = 0, nj = 0, ncell = 0;
    int4* nb = nullptr;         // [ncell]  (face0, face1, face2, face3) neighbour or kWall/kFar
    double2* Sd = nullptr;      // [ncell*4]
    double* Vd = nullptr;       // [ncell]
    float2* Sf = nullptr;       // [ncell*4]
    float* Vf = nullptr;        // [ncell]
    double2* nodes = nullptr;   // [(nj+1)*ni]
};

// Velocity list padded with zero-weight, zero-velocity entries: (vx, vy, w, |v|^2/2).
struct DevGrid {
    int nv = 0, nvp = 0;
    double4* vd = nullptr;      // [nvp]
    float4* vf = nullptr;       // [nvp]
    float4* vpa = nullptr;      // per velocity pair p (padded to a multiple of 128 pairs): (vx, vx', vy, vy')
    float4* vpb = nullptr;      // (w, w', h, h'), h = |v|^2/2
};

// The moment of the functional, Eq. (formula_opt): m_J(v) = dx vx + dy vy + h |v|^2 / 2 (a force along
// (dx, dy) with h = 0; the heat with dx = dy = 0, h = 1).
struct MomentJ {
    double dx = 1.0, dy = 0.0, h = 0.0;
};

// Per-flow tables for one state.
struct DevFlow {
    double tau_inf = 0, u1 = 0, u2 = 0, Tw = 1, Ma = 0, aoa = 0;
    double2* fdd = nullptr;     // [nvp] far-field Maxwellian (g1, g2)
    float2* fdf = nullptr;
    double* gwd = nullptr;      // [nvp] wall Maxwellian g_M1(1, 0, Tw), unnormalised
    float* gwf = nullptr;
    double* wallD = nullptr;    // [ni] normaliser D_l = -sum_{a<=0} w (v.n) g_M1
    double* wallM = nullptr;    // [ni] M_l = sum_{a<=0} w m a g_M1 / D_l for the drag direction
};

// Tiled-TMA descriptors of one distribution buffer viewed as [nj][ni][16-byte chunks]: boxes of
// 32 chunks x 1 cell x 10 rows (a column with its halo rows) and x 8 rows (a side column).
struct TmaMaps {
    alignas(64) CUtensorMap col;
    alignas(64) CUtensorMap side;
};
cudaError_t make_tmamaps(void* base, int ni, int nj, int nq, TmaMaps* out);

// Arguments of the primal sweep.  TS = storage type, TC = compute type.
template <class TS, class TC>
struct PrimalArgs {
    int ncell, nq;                          // nq = nvp / KV  (16-byte chunks per cell)
    int ni, nj;
    const int4* nb;
    const typename std::conditional<sizeof(TC) == 8, double2, float2>::type* S;
    const TC* V;
    const typename std::conditional<sizeof(TC) == 8, double4, float4>::type* vt;
    const float4* vpa;                      // paired velocity table (FP32 arithmetic): (vx, vy) pairs
    const float4* vpb;                      // (w, h) pairs
    const typename std::conditional<sizeof(TC) == 8, double2, float2>::type* fd;
    const TC* gw;
    const double* wallD;
    double inv_tau_inf;
    TC halfTw, dirx, diry;
    const TS* f_old;
    TS* f_new;
    const double4* prim_old;
    double4* prim_new;
    const double4* maxw_old;                // parameters of the cell Maxwellian: prim_old, or the fit
    const double* Fw_old;
    double* Fw_new;
    double* Jpart;
    double* respart;
    int* err;                               // set when a staged copy never completed
    const TS* defect;                       // second order: dR(f_old), subtracted before the division by D
    // Refinement (linearised sweep of a correction e, FP32 storage): f_old/f_new hold e; prim_old is
    // the linearisation point; lin_src the increment s of one FP64 sweep; lin_f the FP32 state at the
    // linearisation point; dW_old/dW_new the moment sums of e (the sweep writes them instead of prim_new).
    const TS* lin_src;
    const TS* lin_f;
    const double4* dW_old;
    double4* dW_new;
    // Velocity-space shard (the state holds a slice of the velocity grid): the sweep writes the raw
    // velocity sums of its slice here instead of finishing the moments (layout: see shard_count()).
    double* part;
    // Macroscopic prediction: the residual sweep (kRes) also writes the moments sum_k w Psi_k R_k of its
    // input's residual per cell, or nothing when null.
    double4* rW;
};

// Partial sums of one velocity shard, doubles: [4 ncell] moment sums (sum w f1, w f1 vx, w f1 vy,
// w (f1 |v|^2/2 + f2)); [ncell] residual sum w (R/V)^2; [ni] wall density F_rhow; [ni] outflow drag;
// [ni] wall normaliser D_l; [ni] M_l D_l.  Adding the shards' buffers gives those of the whole grid.
inline size_t shard_count(int ncell, int ni) { return 5 * (size_t)ncell + 4 * (size_t)ni; }

// Second-order reconstruction (Eq. gaussgrad): the gradient (or, for the adjoint, the transposed
// reconstruction weights mu) and the defect live in buffers of the state's storage and layout.
template <class TS, class TC>
struct SOArgs {
    int ncell, nq, ni;
    const int4* nb;
    const typename std::conditional<sizeof(TC) == 8, double2, float2>::type* S;
    const TC* V;
    const typename std::conditional<sizeof(TC) == 8, double4, float4>::type* vt;
    const typename std::conditional<sizeof(TC) == 8, double2, float2>::type* fd;
    const TC* gw;
    const double* wallD;
    TC halfTw;
    const double2* nodes;                   // [(nj+1)][ni]
    const TS* in;                           // f (primal) or phi (adjoint)
    const double* Fw;                       // wall density of f (primal)
    TS* gx;                                 // d/dx (primal gradient) or the x part of mu (adjoint)
    TS* gy;
    TS* out;                                // dR (primal) or (dR/df)^T (w phi) / w (adjoint)
};

// Per-cell constants of the adjoint linearisation (see k_adjoint_cellconst).
template <class TC>
struct alignas(sizeof(TC) * 4) AdjCell {
    TC n0, inv2T, halfT, Vt, u1, u2, ir, iT, iT2h, c0, c3, j30, j31, j32, j33, irg;
};

template <class TS, class TC>
struct AdjointArgs {
    int ncell, nq;
    int ni, nj;
    const int4* nb;
    const typename std::conditional<sizeof(TC) == 8, double2, float2>::type* S;
    const TC* V;
    const typename std::conditional<sizeof(TC) == 8, double4, float4>::type* vt;
    const float4* vpa;                      // paired velocity table (FP32 arithmetic): (vx, vy) pairs
    const float4* vpb;                      // (w, h) pairs
    const TC* gw;
    const double* wallD;
    const double* wallM;                    // for the functional's direction
    double inv_tau_inf;
    TC halfTw, dirx, diry, heat;             // m_J = dirx vx + diry vy + heat |v|^2/2
    const TS* f;                            // primal state (fixed)
    const AdjCell<TC>* cell;                // constants of the linearisation at that state
    const TS* phi_old;
    TS* phi_new;
    const double4* Z_old;                   // collision coupling (W space) of the previous sweep
    double4* Z_new;
    const double* Lam_old;                  // wall coupling of the previous sweep
    double* Lam_new;
    double* respart;
    int* err;
    const TS* defect;                       // second order: (dR/df)^T (w phi_old) / w, subtracted likewise
    const double* Kinv;                     // conservative Maxwellian: dp/dW per cell ([16]), else null
};

// Descriptors of the batched sweeps: the arguments and tensor maps of one request for both
// parities (slot 0 reads the buffer that is current when the tick starts).  64-byte aligned (the
// tensor maps are read from global memory by the tiled-TMA unit).
template <class TS>
struct alignas(64) PrimalBatchDesc {
    TmaMaps maps[2];
    PrimalArgs<TS, typename std::conditional<sizeof(TS) == 8, double, float>::type> args[2];
};
template <class TS>
struct alignas(64) AdjointBatchDesc {
    TmaMaps phi_maps[2];
    TmaMaps f_maps;
    AdjointArgs<TS, typename std::conditional<sizeof(TS) == 8, double, float>::type> args[2];
};
// Residual/drag reduction of one request (see k_finalize).
struct FinalizeDesc {
    const double* respart;
    int ncell, ni;
    const double* Jpart;
    const double* Fw;
    const double* M;
};

// ---------------------------------------------------------------------------------- launchers
// All launchers enqueue on `s` and return cudaGetLastError().
cudaError_t launch_flow_tables(const DevGrid& g, DevFlow& fl, cudaStream_t s);
// raw = true: wallM receives M_l D_l (the unnormalised sum, which adds across velocity shards).
cudaError_t launch_wall_setup(const DevMesh& m, const DevGrid& g, const DevFlow& fl, MomentJ mj,
                              double* wallD, double* wallM, cudaStream_t s, bool raw = false);
cudaError_t launch_fill_freestream(int storage, void* f, int ncell, const DevGrid& g, const DevFlow& fl,
                                   cudaStream_t s);
cudaError_t launch_moments(int storage, const void* f, const DevMesh& m, const DevGrid& g, double4* prim,
                           double* Fw, cudaStream_t s);
// Velocity shards: the raw moment sums and wall density of f into a shard buffer (residual and drag
// entries zeroed); and the combination of the shards' summed buffer into primitives, wall density,
// residual and drag partials and the wall constants of the whole grid.
cudaError_t launch_shard_moments(int storage, const void* f, const DevMesh& m, const DevGrid& g, double* part,
                                 cudaStream_t s);
cudaError_t launch_shard_combine(const DevMesh& m, const double* total, double4* prim, double* Fw, double* respart,
                                 double* Jpart, double* wallD, double* wallM, cudaStream_t s);
// res = false: skip the residual (only the sweeps whose residual is read need it).  maps: of f_old.
cudaError_t launch_primal_sweep(int storage, const void* args, const TmaMaps& maps, bool res, cudaStream_t s);
// Residual sweep that also writes the residual's moments per cell to args.rW (macroscopic prediction).
cudaError_t launch_primal_sweep_rm(int storage, const void* args, const TmaMaps& maps, cudaStream_t s);
// Sweep of a velocity shard (args.part set): raw velocity sums of the slice into args.part.
cudaError_t launch_primal_shard_sweep(int storage, const void* args, const TmaMaps& maps, bool res, cudaStream_t s);
// Linearised correction sweep of the refinement (FP32 storage only; args: PrimalArgs<float, float> with the
// lin_* fields set, maps: of the correction e_old).
cudaError_t launch_primal_lin_sweep(const void* args, const TmaMaps& maps, bool res, bool rm, cudaStream_t s);
// Refinement elementwise steps over FP32 states of ncell x nvp velocities: f64 <- fbar + delta (FP64 storage
// layout); s <- f64_new - f64_old (FP32 layout); delta += e, then fbar <- fl(fbar + delta) and delta keeps the
// exact remainder (two-sum).
cudaError_t launch_refine_compose(const float* fbar, const float* delta, double* f64, int ncell, int nvp,
                                  cudaStream_t s);
cudaError_t launch_refine_diff(const double* f64_new, const double* f64_old, float* src, int ncell, int nvp,
                               cudaStream_t s);
cudaError_t launch_refine_update(float* fbar, float* delta, const float* e, size_t n, cudaStream_t s);
// update = false: no phi update, only the couplings (Z, Lambda) of phi_old into the *_new slots.
// phi_maps: of phi_old; f_maps: of the primal f.
cudaError_t launch_adjoint_sweep(int storage, const void* args, const TmaMaps& phi_maps, const TmaMaps& f_maps,
                                 bool update, bool res, cudaStream_t s);
// Batched sweeps over work items (request, i, j0); descs is PrimalBatchDesc<TS>[] / AdjointBatchDesc<TS>[].
// n_items blocks are launched (the table's capacity); *count (device memory) of them are in use.
cudaError_t launch_primal_sweep_batch(int storage, const void* descs, const int4* items, int n_items, const int* count,
                                      int parity, bool res, cudaStream_t s);
cudaError_t launch_adjoint_sweep_batch(int storage, const void* descs, const int4* items, int n_items, const int* count,
                                       int parity, bool res, cudaStream_t s);
cudaError_t launch_finalize_batch(const FinalizeDesc* fd, int n, const int* count, double* out, cudaStream_t s);
// maxw: parameters of the cell Maxwellian (prim itself, or the conservative fit)
cudaError_t launch_adjoint_cellconst(int storage, const double4* prim, const double4* maxw, const DevMesh& m,
                                     double inv_tau_inf, void* out, cudaStream_t s);
// A wait that nothing completes, bounded like the sweeps' waits: sets *err after the wait limit.
cudaError_t launch_wait_probe(int* err, cudaStream_t s);
// Moment-space mixing: W = (rho, rho u, rho E) per cell from the primitives, and f += g(W) - g(prim).
cudaError_t launch_prim_to_W(int ncell, const double4* prim, double* W, cudaStream_t s);
cudaError_t launch_moment_shift(int storage, void* f, const DevMesh& m, const DevGrid& g, const double4* prim,
                                const double* W, cudaStream_t s);
// Macroscopic prediction (see k_coarse_assemble): the moment-system blocks out [ncell][4 faces][4x4] and
// the inverses of the diagonal blocks dinv [ncell][4x4] at the primitives prim; one block-Jacobi
// iteration x_n = D^{-1}(-rW + sum OUT x_o) (first: from x = 0); the target moments W(prim) + s omega dW
// with s <= 1 keeping each cell's density and temperature within a relative change cap.
cudaError_t launch_coarse_assemble(int storage, const DevMesh& m, const DevGrid& g, const DevFlow& fl,
                                   const double4* prim, double* out, double* dinv, cudaStream_t s);
// GMRES on the moment system (dvm_krylov.cu): x = A^{-1} (-rhs_neg), or A^{-T} with transpose, from one
// cycle of m <= kMaxKrylov Arnoldi steps right-preconditioned by the diagonal blocks.  Device scalars only;
// with use_graph (a created stream) the launch sequence is captured once and replayed.
constexpr int kMaxKrylov = 64;
struct KrylovWork {
    double4* V = nullptr;       // [(m + 1) ncell] the Arnoldi basis
    double4* w = nullptr;       // [ncell]
    double* part = nullptr;     // [krylov_part_count(m)] partial dot products
    double* H = nullptr;        // [m (m + 1)] Hessenberg columns
    double* scal = nullptr;     // [m + 3]
    double* y = nullptr;        // [m]
    // The launch sequence of a solve depends only on pointers and sizes, so it is captured once per
    // (primal/adjoint) as a CUDA graph and replayed; key = the operands it was captured with.
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    const void* key[2][5] = {{nullptr, nullptr, nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr, nullptr, nullptr}};
    int key_m[2] = {0, 0};
};
void krylov_release_graphs(KrylovWork& K);
// Multigrid preconditioner of the moment system (dvm_krylov.cu): levels of the structured O-mesh
// coarsened 2x2 while both counts are even (Galerkin operators with piecewise-constant transfer),
// per level the 4x4 blocks of the 5-point stencil: D (diagonal), C[e] (the block that multiplies the
// neighbour across face e), D^{-1}, and three vectors.
constexpr int kMaxMGLevels = 12;
struct MGLevel {
    int ni = 0, nj = 0, nc = 0;
    double* D = nullptr;        // [16 nc]
    double* Dinv = nullptr;     // [16 nc]
    double* C = nullptr;        // [64 nc]
    double4* x = nullptr;       // [nc]
    double4* b = nullptr;
    double4* r = nullptr;
};
struct MGWork {
    int nlev = 0;
    MGLevel lev[kMaxMGLevels];
};
// The level sizes for a fine ni x nj mesh (ni, nj of every level), returns the level count.
int mg_plan(int ni, int nj, int* nis, int* njs);
// Builds every level from the assembled outflow blocks and inverse diagonal blocks of the fine mesh.
cudaError_t launch_mg_setup(const DevMesh& msh, const double* out, const double* dinv, const MGWork& mg, cudaStream_t s);
size_t krylov_part_count(int m);
int krylov_launches(int m);
cudaError_t launch_coarse_gmres(const DevMesh& msh, const double* out, const double* dinv, const double4* rhs_neg,
                                bool transpose, int m, KrylovWork& K, double4* x, bool use_graph, cudaStream_t s,
                                const MGWork* mg = nullptr);
cudaError_t launch_coarse_target(int ncell, const double4* prim, const double4* dW, double omega, double cap,
                                 double* W, cudaStream_t s);
// Residual moments of a block from its last sweep's input and output (the served batch's prediction).
cudaError_t launch_primal_restrict(int storage, const DevMesh& m, const DevGrid& g, const double4* prim_old,
                                   double inv_tau_inf, const void* f_old, const void* f_new, double4* rW,
                                   cudaStream_t s);
// Prediction of the adjoint sweeps (FP64/FP32 storage): restriction of the last sweep's residual
// D (phi_old - phi_new) with (dg/dW)^T, the update phi += omega Psi . x.
cudaError_t launch_adjoint_restrict(int storage, const DevMesh& m, const DevGrid& g, const double4* prim,
                                    double inv_tau_inf, const void* phi_o, const void* phi_n, double4* rA,
                                    cudaStream_t s);
cudaError_t launch_adjoint_shift(int storage, const DevMesh& m, const DevGrid& g, const double4* x, double omega,
                                 void* phi, cudaStream_t s);
// Prediction of a linear correction e (FP32): e += (dg/dW) s omega x (s <= 1 keeps the density and
// temperature parts within cap of the state's), then its moment sums dW and wall flux dF.
cudaError_t launch_coarse_lin_shift(const DevMesh& m, const DevGrid& g, const double4* prim, const double4* x,
                                    double omega, double cap, float* e, double4* dW, double* dF, cudaStream_t s);
// Conservative discrete Maxwellian of every cell from its primitive variables (see k_maxwell_fit).
cudaError_t launch_maxwell_fit(int storage, const DevMesh& m, const DevGrid& g, const double4* prim, double4* fit,
                               bool warm, int iters, double* Kinv, cudaStream_t s);
// out[0] = sum respart; out[1] = sum_l Jpart_l + Fw_l M_l (Fw/M may be null -> only sum Jpart)
cudaError_t launch_finalize(const double* respart, int ncell, const double* Jpart, const double* Fw,
                            const double* M, int ni, double* out, cudaStream_t s);
cudaError_t launch_functional(int storage, const void* f, const DevMesh& m, const DevGrid& g,
                              const DevFlow& fl, const double* Fw, MomentJ mj,
                              double* face_out, double* out, cudaStream_t s);
// direction 0: device storage [ncell][nvp] -> double [ncell][nv]; 1: double [ncell][nv] -> storage [ncell][nvp]
cudaError_t launch_convert(int storage, int direction, const void* src, void* dst, int ncell, int nv,
                           int nvp, cudaStream_t s);
// sensitivities
cudaError_t launch_sens_paper(int storage, const DevMesh& m, const DevGrid& g, const DevFlow& fl,
                              const void* f, const void* phi, const double* Fw, MomentJ mj,
                              double* elem, double* node_grad, cudaStream_t s);
cudaError_t launch_sens_full(int storage, const DevMesh& m, const DevGrid& g, const DevFlow& fl,
                             const void* f, const void* phi, const double4* prim, const double4* maxw, const double* Fw,
                             MomentJ mj, double2* GN, double2* GE, double2* GW,
                             double* vol, double2* node_grad, cudaStream_t s);
cudaError_t launch_contract(const double2* node_grad, int nrows, int ni, const double* s_j,
                            const double* dwall, int P, double* grad, cudaStream_t s);

// Anderson mixing of the sweeps (flat storage vectors of n elements; history in FP32, FP64 for FP64
// storage): load X <- F; collect r = G - X, the differences (ring slot `slot`) and the 2m dots into
// out (device, [2m]); mix F, X <- G - dG gamma (neg set on a negative value when `positive`);
// restore F, X <- G.
int aa_max_depth();
int aa_blocks();
cudaError_t launch_aa_load(int storage, size_t n, const void* F, void* X, cudaStream_t s);
cudaError_t launch_aa_collect(int storage, size_t n, const void* G, void* X, void* Rp, void* Gp, void* dR, void* dG,
                              int m, int cnt, int slot, int first, double* part, double* out, cudaStream_t s);
cudaError_t launch_aa_mix(int storage, size_t n, void* F, void* X, const void* Gp, const void* dG, int cnt,
                          const double* gamma, int positive, int* neg, cudaStream_t s);
cudaError_t launch_aa_restore(int storage, size_t n, void* F, void* X, const void* Gp, cudaStream_t s);

// Second order: adjoint = false -> gradient of args.in, then dR into args.out; adjoint = true -> mu of
// args.in (phi), then the transposed defect into args.out.  args is SOArgs<TS, TC>.
cudaError_t launch_second_order(int storage, const void* args, bool adjoint, cudaStream_t s);
// Full discrete sensitivity of a second-order state: adds d(sum w phi . dR)/dx to node_grad
// [(nj+1)][ni] (args: SOArgs with in = f, Fw of f; corner: [ncell][4] scratch).
cudaError_t launch_so_sens(int storage, const void* args, const void* phi, double2* corner, int ni, int nj,
                           double2* node_grad, cudaStream_t s);

// out[0] = Q, out[1 + p] = dQ/dalpha_p
cudaError_t launch_volume(const DevMesh& m, double vmin, const double* dwall, int P, double* out, cudaStream_t s);

size_t storage_bytes(int storage);   // bytes of one (f1,f2) pair

}  // namespace dvm
