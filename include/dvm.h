/*
 * dvm.h -- C ABI of the GB300 (sm_103a) library for the steady discrete-velocity (DVM) BGK
 * solve on a body-fitted O-mesh with diffuse walls, its discrete adjoint and the boundary
 * sensitivities of Yuan & Wu, "Adjoint shape optimization from the continuum to free-molecular
 * gas flows" (arXiv 2501.00923).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units: rho_inf = 1, R T_inf = 1, chord = 1, monatomic gas (gamma = 5/3); velocities in units of
 *   sqrt(R T_inf); free-stream speed Ma * sqrt(5/3).  tau = tau_inf / (rho sqrt(T)) (hard-sphere
 *   mu ~ sqrt(T), tau = mu/p, Sec. 2.1) with tau_inf = (5/16) Kn sqrt(2 pi) (Eq. kndefine).
 * Mesh: structured O-mesh, ni cells around (periodic), nj cells from the wall (j = 0) to the far
 *   field (j = nj - 1).  Nodes are passed as double [(nj+1)][ni][2], j = 0 on the wall,
 *   counter-clockwise around the body.  Cell c = j*ni + i.
 * Velocities: any list (v_k, w_k), k < nv (uniform, Gauss-Legendre or unstructured, Sec. 4.3).
 * Distribution layout (host side, every get/set call): double [ncell][nv][2] = (f1, f2) of
 *   Eq. (f_reduce), velocity fastest.  The device keeps the same order in the storage precision
 *   chosen at state creation (FP64, FP32 or BF16), the velocity count padded to a multiple of 4 with
 *   zero-weight velocities.
 * Ownership: host arrays are caller-owned and only read (or written, for outputs) during the call.
 *   Every handle is library-owned and released by its *_destroy.  Device memory comes from one
 *   stream-ordered pool per device (cudaMallocFromPoolAsync on the context's stream; freed blocks are
 *   kept by the pool and reused, so a state created after another is destroyed does not call
 *   cudaMalloc); dvm_context_destroy trims the pool.  The context's stream orders all work.
 * Errors: every call returns a dvm_status; DVM_OK = 0.  No C++ exception crosses the ABI.  After
 *   DVM_ERR_CUDA the context should be destroyed.  dvm_last_error() gives a message for the
 *   calling thread.  Calls are thread-compatible per context (one thread at a time per context).
 */
#ifndef DVM_H
#define DVM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DVM_OK = 0,
    DVM_ERR_INVALID_ARG = 1,
    DVM_ERR_OOM = 2,
    DVM_ERR_ADMISSION = 3,   /* request does not fit the context's HBM budget */
    DVM_NOT_CONVERGED = 4,   /* max_iter reached; the result still holds the last residual */
    DVM_ERR_NONFINITE = 5,   /* a residual or a moment became NaN/Inf */
    DVM_ERR_CUDA = 6,
    DVM_ERR_TIMEOUT = 7,
    DVM_ERR_STAGNATED = 8    /* residual stopped decreasing (FP32/BF16 floor) before tol */
} dvm_status;

typedef enum { DVM_STORE_FP64 = 0, DVM_STORE_FP32 = 1, DVM_STORE_BF16 = 2 } dvm_storage;
/* cell Maxwellian of the collision term (dvm_state_set_maxwellian) */
typedef enum { DVM_MAXWELL_PLAIN = 0, DVM_MAXWELL_CONSERVATIVE = 1 } dvm_maxwellian;

/* Objective of Eq. (formula_opt): J = sum_wall sum_k w m_k (v_k . n A) f1.
 * DVM_DRAG: m_k = v_k . d, d = free-stream direction (m_J = v1 at zero incidence, Sec. 2.4);
 * DVM_LIFT: d = free-stream direction rotated by +90 degrees;
 * DVM_HEAT: m_k = |v_k|^2 / 2, the heat carried by f1 into the wall (Sec. 2.4). */
typedef enum { DVM_DRAG = 0, DVM_LIFT = 1, DVM_HEAT = 2 } dvm_functional;

/* DVM_SENS_PAPER: the boundary sensitivity of Sec. 3.2 (Eq. sens_J_itf, sens_B_itf, gaussgrad,
 *   sens_nod), wall nodes only, as the paper computes it.
 * DVM_SENS_FULL: the exact derivative of the discrete J, including the interior mesh motion
 *   x(i,j) = x_w(i) + s_j (x_ff(i) - x_w(i)) (the terms the paper drops below Eq. sens_shape). */
typedef enum { DVM_SENS_PAPER = 0, DVM_SENS_FULL = 1 } dvm_sens_mode;

typedef struct dvm_context dvm_context;
typedef struct dvm_mesh dvm_mesh;
typedef struct dvm_vgrid dvm_vgrid;
typedef struct dvm_state dvm_state;
typedef struct dvm_adjoint dvm_adjoint;

enum { DVM_OPT_NO_GRAPHS = 1 };   /* launch every sweep directly (no CUDA-graph capture) */

typedef struct {
    int graph_iters;        /* sweeps captured per CUDA-graph launch (even, >= 2); 0 -> 20 */
    size_t hbm_budget;      /* bytes the context may hold for states (admission); 0 -> no limit */
    void* stream;           /* cudaStream_t to run on (e.g. torch's); NULL -> the library's own */
    int flags;              /* DVM_OPT_* */
} dvm_options;

typedef struct {
    double Kn;              /* Knudsen number with the chord and the free stream, Eq. (kndefine) */
    double Ma;              /* free-stream Mach number */
    double Tw;              /* wall temperature / free-stream temperature (u_w = 0), Eq. (formula_bgk_fdw0) */
    double aoa;             /* free-stream direction, radians */
} dvm_flow;

typedef struct {
    double tol;             /* stop when |R|/r0 <= tol; |R| = sqrt(sum_{c,k,comp} w_k (R/V_c)^2) */
    int max_iter;           /* cap on point-implicit sweeps */
    int stall_window;       /* stop with DVM_ERR_STAGNATED after this many sweeps without a 2% drop; 0 = off */
    int accel_depth;        /* 0 = plain sweeps.  m in [1, 8]: Anderson mixing of depth m applied to the map of
                               accel_period sweeps (x -> G(x); next x = G - dG gamma, gamma = argmin |r - dR gamma|
                               over the last m differences of r = G(x) - x and of G).  It accelerates the
                               iteration only: the discrete solution is the same.  The history holds 2m + 3
                               vectors of the state's size (FP32; FP64 for FP64 storage), kept with the state or
                               adjoint.  A primal mix that makes any value of f negative is undone and the history
                               restarts; so does a block residual above twice the best since the history
                               started.  On the second such restart, or when the stall window runs out
                               while mixing, the solve finishes with plain sweeps (with a stall window of
                               their own), so FP32/BF16 solves end on the plain sweeps' rounding floor */
    int accel_period;       /* sweeps between mixings (>= 1; with accel_depth > 0) */
    int accel_space;        /* what is mixed: 0 = the whole state (f, or phi for the adjoint); 1 = the cell moments
                               W = (rho, rho u, rho E) of the primal, one FP64 vector of 4 values per cell, the
                               mixed moments imposed on f by f += g(W_mixed) - g(W) (the non-equilibrium part of
                               f is kept; cells whose mixed moments lose positive density or temperature are left
                               unshifted).  The shift vanishes at a fixed point, so the solution is unchanged.
                               Adjoint solves ignore 1 and mix phi */
    double refine_tol;      /* primal solves of FP32 states (order 1, plain Maxwellian) only; 0 = off.  > 0: after the
                               sweeps stop (tolerance, stall window or cap), mixed-precision refinement of the same
                               discrete problem until the FP64 residual |R(f)|/r0 <= refine_tol.  f is carried as
                               fbar + delta, two FP32 arrays (fbar the state, delta the exact remainder of each
                               update).  A correction step takes R(fbar + delta) exactly from one FP64 sweep of
                               the composed state (its increment s = -R/D), then solves J e = -R for the correction
                               e by linearised FP32 point-implicit sweeps at fbar + delta (J the Jacobian of R:
                               upwind transport, the linearised Maxwellian and relaxation rate with lagged moment
                               couplings, the wall density), until the linear residual falls below a tenth of |R|
                               or after refine_sweeps (the residual of these sweeps can stay near |R| for hundreds
                               of sweeps at small Kn before it decays, so there is no stall exit); with
                               predict_iters > 0 every block of these sweeps is followed by the macroscopic
                               prediction of e (the same moment system at fbar + delta, linear: e += (dg/dW) dW).
                               Then delta += e and (fbar, delta) is renormalised by a two-sum.  Rounding in the
                               FP32 sweeps is relative to e, not to f, so the solution
                               reaches the FP64 one; the state ends at fl(fbar + delta) and J, Cd and residual of
                               the result are those of fbar + delta in FP64.  Temporary device memory: an FP64
                               state and four FP32 arrays of the state's size, freed at the end.  Errors:
                               DVM_ERR_INVALID_ARG for another storage, order or Maxwellian */
    int refine_max;         /* correction steps at most (0 -> 20); the refinement also stops (DVM_ERR_STAGNATED)
                               when two steps in a row leave the FP64 residual above 0.7 of the best so far (one
                               such step is allowed: far from the solution a step can raise |R| while it cuts the
                               error, by the quadratic term of R in e) */
    int refine_sweeps;      /* linearised FP32 sweeps per correction step at most (0 -> 4000) */
    double predict_omega;   /* damping of the macroscopic prediction's correction (0 -> 0.8), its initial and
                               largest value: it halves after a block whose residual grew by more than 1.5x and
                               after five predicted blocks in a row without a new best residual, and recovers by
                               1.25x after a block that set a new best */
    int predict_iters;      /* primal solves, FP64 or FP32 storage, order 1, plain Maxwellian; 0 = off; at most 64.
                               > 0: after every block of graph_iters sweeps a macroscopic prediction (the
                               prediction acceleration of Sec. 3.1 by equations for the moments): the moments of
                               the steady residual of Eq. (numerpr_gov) per cell (from the block's last sweep) are
                               cancelled by a moment correction dW solved from the discrete transport of the
                               Maxwellian derivative in moment form (4 x 4 blocks per cell and face: upwind
                               outflow at the cell's moments, inflow from the neighbour, re-emission on the wall)
                               by one GMRES cycle of this many Arnoldi steps, right-preconditioned by the diagonal
                               blocks, on the device (no host synchronisation, fixed-order sums; workspace
                               (steps + 2) x 4 doubles per cell); f is then shifted by g(W + s omega dW) - g(W), s <= 1 keeping each
                               cell's density and temperature within 30% and positive.  At small Kn the slow
                               modes of the sweeps are these moments, so this removes most of their sweeps; the
                               steady solution is unchanged (the shift vanishes at it).  FP32 storage: near
                               the rounding floor the residual moments are dominated by the rounding of the
                               relaxation term, which the moment solve amplifies into smooth errors; once two
                               blocks in a row end with a residual above twice the best so far the prediction
                               is switched off and the solve goes on with plain sweeps (with a new stall window).  With refinement, stop the FP32 sweeps
                               early (tol ~1e-5) and let the predicted refinement finish.  Memory: 88 doubles per
                               cell plus the GMRES workspace, kept with the state */
    int predict_reuse;      /* predictions between reassemblies of the moment system (0 -> 4) */
    int predict_precond;    /* preconditioner of the prediction's GMRES: 0 = the diagonal blocks (default);
                               1 = one multigrid V(1,1) cycle per step: the O-mesh coarsened 2x2 while both
                               counts are even (Galerkin levels, piecewise-constant transfer), damped
                               block-Jacobi smoothing (0.7), 30 smoothing sweeps on the coarsest level.  Its
                               steps are nearly mesh-independent, so 2-5 steps do what 40 diagonal ones do not;
                               an accurate solve of the moment system overcorrects as the cell Knudsen number
                               grows (damp it, or keep the steps few).  Memory: ~4/3 x 108 doubles per cell */
    /* Adjoint solves take predict_iters and predict_omega too: the transposed coarse problem.  The
       prolongation of the moment prediction, dW -> (dg/dW) dW, and its restriction, r -> sum_k w Psi_k r_k,
       swap roles in the w-weighted product of the adjoint sweep: lambda -> Psi . lambda and
       r_a -> sum_k w (dg_k/dW)^T r_a,k, with the transposed system A^T (assembled once at the primal
       state; its GMRES products use each cell's own outflow blocks).  phi += omega Psi . lambda,
       after which the collision and wall couplings of phi are recomputed.  The same FP32 noise rule. */
} dvm_solve_opts;

typedef struct {
    double J;               /* drag functional of Eq. (numer_J) at the final state */
    double Cd;              /* J / (rho_inf |u_inf|^2 / 2 * chord) */
    double residual;        /* |R| / r0 of the last sweep's input state */
    double r0;              /* |R| of the free-stream state */
    int iters;              /* sweeps done by this call (before any refinement) */
    int status;             /* dvm_status of the solve (of the refinement when it ran) */
    int refine_steps;       /* refinement correction steps (FP64 residual evaluations - 1) */
    int refine_sweeps;      /* linearised FP32 sweeps of the refinement */
    double residual_fp32;   /* |R|/r0 of the FP32 sweeps when they stopped (= residual without refinement) */
    double residual_fp64;   /* refinement: the FP64 residual |R|/r0 of the state the FP32 sweeps left */
    int predictions;        /* macroscopic predictions applied (one per block of sweeps) */
} dvm_primal_result;

typedef struct {
    double residual;        /* adjoint |R_a| / |R_a(phi = 0)| */
    double r0;
    int iters;
    int status;
    int predictions;        /* macroscopic predictions applied (one per block of sweeps) */
} dvm_adjoint_result;

/* ------------------------------------------------------------------------ context, B1 */
/* Create a context on CUDA device `cuda_device`.  opt may be NULL (defaults).
 * Errors: DVM_ERR_INVALID_ARG (bad device/options), DVM_ERR_CUDA. */
int dvm_context_create(dvm_context** out, int cuda_device, const dvm_options* opt);
void dvm_context_destroy(dvm_context* ctx);
/* bytes currently held by states/adjoints of this context (admission accounting) */
size_t dvm_context_bytes(const dvm_context* ctx);
const char* dvm_status_string(int status);
const char* dvm_last_error(void);
/* number of kernel launches issued by this context since creation (graph launches count each
 * captured kernel) */
uint64_t dvm_context_launches(const dvm_context* ctx);
/* number of device allocations made for this context since creation (blocks taken from the
 * library's stream-ordered pool, transient ones included) */
uint64_t dvm_context_allocations(const dvm_context* ctx);
/* Self-test of the failure path of the bounded device waits.  One kernel waits on an mbarrier that
 * nothing completes, with the same bound as the sweeps' pipeline waits (2 s of the device's global
 * timer); the wait gives up, the kernel sets the context's device flag and returns.  Returns
 * DVM_ERR_TIMEOUT (the flag is cleared) after about 2 s; the context stays usable.  No fault and no
 * hang is involved.  Errors: DVM_ERR_INVALID_ARG (NULL), DVM_ERR_CUDA. */
int dvm_selftest_wait_timeout(dvm_context* ctx);

/* ------------------------------------------------------------------------ mesh, B2 */
/* Copy the O-mesh nodes (double [(nj+1)][ni][2]) and build on the host the cell volumes, the
 * outward face vectors A n of Eq. (numerpr_gov) and the neighbour table.  Fails with
 * DVM_ERR_INVALID_ARG if ni < 3, nj < 1, or a cell has non-positive area (tangled mesh). */
int dvm_mesh_create(dvm_context* ctx, int ni, int nj, const double* nodes_xy, dvm_mesh** out);
void dvm_mesh_destroy(dvm_mesh* mesh);

/* ------------------------------------------------------------------------ velocity grid, B3 */
/* Copy an arbitrary velocity list with quadrature weights (w_k > 0).  nv >= 1. */
int dvm_vgrid_create(dvm_context* ctx, int nv, const double* vx, const double* vy, const double* w,
                     dvm_vgrid** out);
void dvm_vgrid_destroy(dvm_vgrid* grid);

/* ------------------------------------------------------------------------ primal state, B4 */
/* Allocate a primal state (two f buffers, per-cell moments, wall density) in the given storage
 * precision and set it to the free-stream Maxwellian (Eq. drlt_maxwell).  Counts against the
 * context's HBM budget (DVM_ERR_ADMISSION).  mesh and grid must outlive the state. */
int dvm_state_create(dvm_context* ctx, const dvm_mesh* mesh, const dvm_vgrid* grid,
                     const dvm_flow* flow, int storage, dvm_state** out);
void dvm_state_destroy(dvm_state* st);
/* Upload f (host double [ncell][nv][2]) and recompute the moments W (Eq. macint_reduce) and the
 * wall density F_rhow (Eq. formula_bgk_fdw) from it. */
int dvm_state_set(dvm_state* st, const double* f_host);
/* Download f (converted to double). */
int dvm_state_get(const dvm_state* st, double* f_host);
/* Device-to-device warm start: copy the current f of src into dst (no host round trip) and recompute
 * dst's moments W and wall density F_rhow (Eq. macint_reduce, formula_bgk_fdw) on dst's own mesh, as
 * dvm_state_set does after an upload.  The two states need the same context, the same mesh shape
 * (ni, nj), the same velocity count and the same storage; their meshes and flows may differ (a new
 * design of the same shape, Sec. 3.4, Steps 2-3), and the velocity lists should be the same.
 * Enqueued on the context's stream; src is only read.  Errors: DVM_ERR_INVALID_ARG (NULL or a
 * layout mismatch), DVM_ERR_CUDA. */
int dvm_state_copy_from(dvm_state* dst, const dvm_state* src);
/* Download per-cell primitive variables (rho, u1, u2, T) [ncell][4] of the current f. */
int dvm_state_moments(const dvm_state* st, double* prim_host);
/* Spatial order of the face values used by every later sweep of this state and of its adjoints.
 * order 1 (the default): first-order upwind values, Eq. (numerpr_gov).  order 2: on interior faces the
 * upwind cell's linear reconstruction F_e = f_up + grad f_up . (x_e - x_up), with the unlimited Gauss
 * gradient of Eq. (gaussgrad) (face averages inside, the first-order value on wall and far-field faces;
 * x_c the mean of the cell's corners, x_e the face midpoint).  Sweeps of order 2 are defect correction:
 * the added flux dR is taken from the sweep's input at the first sweep of every group of
 * defect_period sweeps (0 -> 20) and frozen for the rest of the group, while each sweep keeps the
 * first-order point-implicit form,
 *   f_new = [ V g/tau + sum_{a<=0} (-a) F_up - dR ] / [ V/tau + sum_{a>0} a ],
 * so a converged solve satisfies R1(f) + dR(f) = 0 whatever the period.  (A period of 1 can diverge:
 * with the unlimited reconstruction the point-implicit map is unstable in weakly collisional modes,
 * and on fine meshes the group must be long enough for its first-order sweeps to contract: 4 diverges
 * and 8 stalls on a 256x128 mesh at Kn 0.1, 16 and more converge.  Start second-order solves from a
 * converged first-order state: from the free stream the unlimited reconstruction can drive f
 * negative on coarse meshes.)
 * Adjoint sweeps take the exact transpose of dR, (dR/df)^T (w phi) / w, frozen the same way.  Boundary
 * faces, the drag and the wall density stay first order.  The first call with order 2 allocates three
 * buffers of the size of f for the state and one for each adjoint swept later (counted against the HBM
 * budget: DVM_ERR_ADMISSION).  dvm_state_set and an adjoint upload retake the defect at the next sweep;
 * the residual normaliser r0 keeps its value from state creation.
 * With order 2, DVM_SENS_FULL adds the derivative of the reconstruction's added flux with respect to
 * the nodes (face vectors, volumes, cell centres and face midpoints in the Gauss gradient and the
 * offsets, and the wall inflow values); its first call on an adjoint allocates a per-cell corner
 * buffer (4 ncell double2, counted against the HBM budget).  dvm_sensitivity_noalloc accepts only
 * DVM_SENS_PAPER for order-2 states.  dvm_batch requests stay first order.
 * Errors: DVM_ERR_INVALID_ARG (NULL, order not 1 or 2, defect_period < 0), DVM_ERR_ADMISSION,
 * DVM_ERR_OOM. */
int dvm_state_set_order(dvm_state* st, int order, int defect_period);
int dvm_state_get_order(const dvm_state* st, int* order);
/* Cell Maxwellian of the collision term for every later sweep of this state and its adjoints.
 * DVM_MAXWELL_PLAIN (the default): g of Eq. (maxwell_reduce) at the cell's primitive variables, whose
 * discrete moments on a truncated velocity grid differ slightly from the cell's.
 * DVM_MAXWELL_CONSERVATIVE: g at the parameters p = (rho, u, T) whose discrete moments equal the
 * cell's exactly, sum_k w_k Psi_k g_k(p) = W (Newton's method per cell: from the primitive variables on
 * this call and after dvm_state_set, one warm step after every sweep), so the collision term conserves
 * mass, momentum and energy on the grid itself.  The relaxation time stays that of the primitive
 * variables.  The adjoint takes the fit's implicit derivative dp/dW = (dM/dp)^{-1}, and both
 * sensitivity modes use the fitted g.  Allocates a small per-cell buffer for the state and one for
 * each adjoint (16 doubles per cell; DVM_ERR_ADMISSION); dvm_batch requests use the plain Maxwellian.
 * Errors: DVM_ERR_INVALID_ARG (NULL, unknown kind), DVM_ERR_ADMISSION, DVM_ERR_OOM, DVM_ERR_CUDA. */
int dvm_state_set_maxwellian(dvm_state* st, int kind);
int dvm_state_get_maxwellian(const dvm_state* st, int* kind);
/* Run exactly n point-implicit sweeps (Eq. numerpr_gov solved for f_{c,k} with the neighbours,
 * moments and wall density of the previous sweep):
 *   f_new = [ V g/tau + sum_{a<=0} (-a) F_up ] / [ V/tau + sum_{a>0} a ],  a = A n . v_k.
 * residual_out (optional, host double[n]) receives |R|/r0 of each sweep's input state. */
int dvm_primal_iterate(dvm_state* st, int n, double* residual_out);
/* Drag J (Eq. numer_J) of the state's current f, and the y-force for the same state. */
int dvm_state_functional(dvm_state* st, int functional, double* J);
/* Whole steady solve, B4.  *inout == NULL: create a state (storage from ctx-default FP32 unless
 * flow-specific storage was chosen with dvm_state_create) and solve from the free stream;
 * otherwise warm start from the given state (its mesh/grid/flow must match the arguments).
 * Returns the solve status (DVM_OK, DVM_NOT_CONVERGED, DVM_ERR_STAGNATED, DVM_ERR_NONFINITE). */
int dvm_primal_solve(dvm_context* ctx, const dvm_mesh* mesh, const dvm_vgrid* grid,
                     const dvm_flow* flow, const dvm_solve_opts* opts, int storage,
                     dvm_state** inout, dvm_primal_result* out);

/* ------------------------------------------------------------------------ velocity shards */
/* One steady primal solve split over velocity space (each GPU holds every cell for a slice of the
 * velocity grid).  The point-implicit sweep of Eq. (numerpr_gov) couples velocities only through
 * velocity sums: the cell moments W of Eq. (macint_reduce) that give g and tau, the wall density
 * F_rhow of Eq. (formula_bgk_fdw), the normaliser D_l of Eq. (barg), the drag of Eq. (numer_J) and
 * the residual norm.  A shard is a state created on its slice (a dvm_vgrid of those velocities) with
 * the common mesh and flow; its sweeps write the slice's partial sums instead of finishing them, the
 * caller adds the shards' buffers (an all-reduce across GPUs, or a sum on one device), and each shard
 * installs the total before its next sweep.  The totals equal those of the whole grid up to the order
 * of the additions, so the shards together follow the unsplit sweeps.
 * Buffer layout (doubles, dvm_state_shard_count of them): [4 ncell] the sums (w f1, w f1 vx, w f1 vy,
 * w (f1 |v|^2/2 + f2)) per cell; [ncell] the residual sums w (R/V)^2; [ni] F_rhow; [ni] the outflow
 * part of the drag; [ni] D_l; [ni] M_l D_l of the drag direction.  Per sweep that is
 * 8 (5 ncell + 4 ni) bytes to all-reduce.
 * dvm_state_set_shard(st, 1): first-order states with the plain Maxwellian only; fills the buffer
 *   from the current f (moments, F_rhow and the slice's D_l, M_l D_l; residual and drag entries 0).
 *   Allocates two buffers of the count (HBM budget).  (st, 0) returns the state to a grid of its own.
 * dvm_state_shard_partials: copy the buffer to `out` (host or device memory, count doubles).
 * dvm_state_shard_combine: install the summed buffer `total` (host or device memory): the primitive
 *   variables and F_rhow of the whole grid for the next sweep, and D_l, M_l of the whole grid; returns
 *   the residual sum sum w (R/V)^2 of the last sweep's input (0 after dvm_state_set_shard) and the drag
 *   of the current f (its outflow part as summed; meaningful after a sweep).
 * dvm_primal_iterate on a shard takes n = 1 (residual_out receives NaN).  dvm_primal_solve, adjoints,
 * order 2 and the conservative Maxwellian are refused on shards (DVM_ERR_INVALID_ARG).
 * Errors: DVM_ERR_INVALID_ARG (NULL, not a shard, wrong count), DVM_ERR_OOM, DVM_ERR_ADMISSION,
 * DVM_ERR_CUDA. */
int dvm_state_set_shard(dvm_state* st, int on);
size_t dvm_state_shard_count(const dvm_state* st);
int dvm_state_shard_partials(const dvm_state* st, double* out, size_t count);
int dvm_state_shard_combine(dvm_state* st, const double* total, size_t count, double* residual_sq, double* J);

/* ------------------------------------------------------------------------ adjoint, B5 */
/* Allocate the adjoint phi of `st` (same storage), zero it, linearised at the state's current f.
 * The state must not change while the adjoint is used. */
int dvm_adjoint_create(dvm_state* st, int functional, dvm_adjoint** out);
void dvm_adjoint_destroy(dvm_adjoint* adj);
int dvm_adjoint_set(dvm_adjoint* adj, const double* phi_host);
/* Device-to-device warm start of the adjoint: copy the current phi of src into dst and rebuild dst's
 * collision and wall couplings from it, as dvm_adjoint_set does after an upload.  Same layout rules as
 * dvm_state_copy_from (for the adjoints' states).  Errors: DVM_ERR_INVALID_ARG, DVM_ERR_CUDA. */
int dvm_adjoint_copy_from(dvm_adjoint* dst, const dvm_adjoint* src);
int dvm_adjoint_get(const dvm_adjoint* adj, double* phi_host);
/* Exactly n sweeps of the transposed (downwind) point-implicit update of Eq. (numerad_gov) in
 * discrete form, (dR/df)^T (w phi) = -(dJ/df)^T:
 *   D phi = -dJ/df/w + sum_{a>0, interior} a phi_nb + (V/tau) What.Psi
 *           - (V/tau^2) rhohat (dtau/dW).Psi - [wall, a>0] (v.n) Lambda
 * with What, rhohat of Eq. (adjoint_macdefines) and the wall coupling of Eq. (formula_adjointbgk)
 * taken from the previous sweep.  residual_out as for the primal. */
int dvm_adjoint_iterate(dvm_adjoint* adj, int n, double* residual_out);
int dvm_adjoint_solve(dvm_context* ctx, dvm_state* st, int functional, const dvm_solve_opts* opts,
                      dvm_adjoint** inout, dvm_adjoint_result* out);

/* ------------------------------------------------------------------------ sensitivity, B6 */
/* dJ/dalpha_p for n_params shape parameters that move the wall nodes by dwall_dalpha
 * (double [n_params][ni][2], caller-owned) and the interior nodes by (1 - s_j) times that
 * (s_j: double [nj+1], s_0 = 0, s_nj = 1; used by DVM_SENS_FULL only).  grad_out: double[n_params].
 * node_grad_out (optional): DVM_SENS_PAPER -> dJ/dx of the wall nodes, double [ni][2];
 * DVM_SENS_FULL -> dJ/dx of every node, double [(nj+1)][ni][2].
 * The first call on an adjoint allocates its scratch (per-cell face sums, node gradient, tangents;
 * counted against the HBM budget) and later calls reuse it. */
int dvm_sensitivity(dvm_context* ctx, const dvm_state* st, const dvm_adjoint* adj, int n_params,
                    const double* dwall_dalpha, const double* s_j, int mode, double* grad_out,
                    double* node_grad_out);

/* Volume constraint of Eq. (formula_opt), Q = (1/D) int_wall x . n dGamma + V_min with n into the
 * solid and D = 2 (Q <= 0 keeps the section area >= V_min), evaluated exactly on the straight wall
 * elements, and dQ/dalpha_p from the node sensitivity of Eq. (sens_con_nod) contracted with
 * dwall_dalpha [n_params][ni][2].  dQ_dalpha: double[n_params], caller-owned. */
int dvm_volume_constraint(dvm_context* ctx, const dvm_mesh* mesh, double v_min, int n_params,
                          const double* dwall_dalpha, double* Q, double* dQ_dalpha);

/* ------------------------------------------------------------------------ served batch, B7 */
/* Continuous batching of whole solve requests (primal solve, adjoint solve, sensitivity) on one
 * context.  Requests are admitted in arrival order while their device footprint fits the batch's
 * HBM budget; every tick advances each admitted request by `sweeps_per_tick` point-implicit
 * sweeps of its current phase in one batched launch per sweep (all requests of the tick share the
 * launch; the launches read their work lists and counts from device tables of fixed capacity, so the
 * tick's sweeps, reductions and read-back are one captured CUDA graph, re-captured only when a table
 * outgrows its capacity, and the tables are re-uploaded only when the admitted set changes), then
 * checks convergence; a converged primal moves to its adjoint, a converged adjoint to
 * its sensitivity, and the request retires, freeing its memory.  Requests that arrive while others
 * run are admitted at the next tick.  A request's result does not depend on what else is in the
 * batch (same kernels, same per-request arithmetic, fixed reduction order).
 * Warm start: a request with warm_key != 0 starts its f and phi from those of the last retired
 * request with the same key and the same mesh/grid/storage, when that is still cached. */
typedef struct dvm_batch dvm_batch;

typedef struct {
    size_t hbm_budget;          /* bytes for admitted requests and the warm cache; 0 -> no limit */
    int sweeps_per_tick;        /* even, >= 2 */
    int max_active;             /* cap on admitted requests; 0 -> no cap */
} dvm_batch_options;

typedef struct {
    int ni, nj;
    const double* nodes_xy;     /* [(nj+1)][ni][2], copied at submit */
    int nv;
    const double* vx;           /* [nv], copied */
    const double* vy;
    const double* w;
    dvm_flow flow;
    int storage;                /* dvm_storage */
    double tol;                 /* primal and adjoint relative residual targets */
    double adjoint_tol;
    int max_iter;               /* per phase; a phase that reaches it moves on (status NOT_CONVERGED) */
    int functional;             /* dvm_functional */
    int n_params;               /* sensitivity parameters; 0 -> no adjoint/sensitivity */
    const double* dwall_dalpha; /* [n_params][ni][2], copied */
    const double* s_j;          /* [nj+1], copied (DVM_SENS_FULL) */
    int sens_mode;              /* dvm_sens_mode */
    uint64_t warm_key;          /* 0 -> no warm start */
    int stall_window;           /* > 0: a phase ends with DVM_ERR_STAGNATED once its residual has not
                                   fallen below 0.98 x its best for this many sweeps (as dvm_solve_opts) */
    int predict_iters;          /* > 0 (FP64/FP32 storage): the macroscopic prediction of dvm_solve_opts after
                                   every tick that leaves the phase running, primal and (transposed) adjoint,
                                   with this many GMRES steps (<= 64); its residual moments come from the
                                   tick's last sweep (input and output), its damping and FP32 noise rule are
                                   the request's own.  The request's result then still does not depend on
                                   the rest of the batch.  Device memory: counted in the admission footprint */
    double predict_omega;       /* initial damping of the prediction (0 -> 0.8) */
} dvm_request;

typedef struct {
    int done;                   /* 1 when retired */
    int status;                 /* DVM_OK, DVM_NOT_CONVERGED (a phase hit max_iter), or an error */
    int phase;                  /* 0 queued, 1 primal, 2 adjoint, 3 retired */
    int primal_iters, adjoint_iters;
    double J, Cd, residual, adjoint_residual;
    int warm_started;
    int predictions;            /* macroscopic predictions applied (primal + adjoint) */
} dvm_request_result;

/* Counters of a batch since creation: */
typedef struct {
    uint64_t ticks;             /* ticks that ran sweeps */
    uint64_t graph_launches;    /* ticks whose sweeps, reductions and read-back ran as one CUDA-graph launch */
    uint64_t graph_builds;      /* captures of that graph: the first tick, and a table outgrowing its capacity */
    uint64_t table_uploads;     /* ticks that rebuilt and uploaded the descriptor tables (the admitted set or a
                                   request's phase changed); other ticks reuse the tables on the device */
    int peak_active;            /* most requests admitted at once */
    size_t peak_bytes;          /* most device memory held by admitted requests and the warm cache (footprints) */
} dvm_batch_stats;

int dvm_batch_create(dvm_context* ctx, const dvm_batch_options* opt, dvm_batch** out);
/* Frees every request and the cache.  Destroy a batch before its context. */
void dvm_batch_destroy(dvm_batch* b);
/* Queue a request (host arrays copied).  Fails with DVM_ERR_ADMISSION if it can never fit the budget. */
int dvm_batch_submit(dvm_batch* b, const dvm_request* req, uint64_t* ticket);
/* Admit what fits, run one tick, retire what converged.  n_active/n_queued (optional) report the
 * state after the tick. */
int dvm_batch_tick(dvm_batch* b, int* n_active, int* n_queued);
/* Result of a request; grad_out (optional, [n_params]) receives dJ/dalpha once retired.  A retired
 * request is forgotten after it has been polled with forget = 1. */
int dvm_batch_poll(dvm_batch* b, uint64_t ticket, dvm_request_result* out, double* grad_out, int forget);
/* Copy the batch's counters.  Errors: DVM_ERR_INVALID_ARG (NULL). */
int dvm_batch_get_stats(const dvm_batch* b, dvm_batch_stats* out);

/* Same result as dvm_sensitivity, for callers that must not allocate device memory during the
 * call (e.g. a serving loop whose device memory is reserved once, up front, by another allocator,
 * or a host thread that must not stall on cudaMalloc's implicit synchronisation).  The paper has no
 * counterpart: this is a property of the library, not of the method.
 * Scratch: a static 8 MiB device array, present on every GPU that loads the library until the
 * process exits.  A request whose intermediates exceed it (about 150 000 cells in the full mode)
 * fails with DVM_ERR_INVALID_ARG and a message giving the size needed.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.
 * All calls share the array and its contents persist between calls; each call writes every entry it
 * reads, so nothing is cleared.  Calls whose GPU work overlaps (other contexts or threads on the same
 * device) race on the array: serialise them.  Host arrays are as for dvm_sensitivity. */
int dvm_sensitivity_noalloc(dvm_context* ctx, const dvm_state* st, const dvm_adjoint* adj, int n_params,
                            const double* dwall_dalpha, const double* s_j, int mode, double* grad_out,
                            double* node_grad_out);

#ifdef __cplusplus
}
#endif
#endif /* DVM_H */
