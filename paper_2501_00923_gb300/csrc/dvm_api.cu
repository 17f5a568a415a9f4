// Host side of the C ABI declared in include/dvm.h: handles, geometry preprocessing, the sweep
// loops (captured as CUDA graphs), convergence control and the sensitivity driver.  Every step of
// the DVM path runs in the kernels of dvm_kernels.cu; this file only prepares arguments,
// allocates device memory and moves small results.
#include "dvm.h"
#include "dvm_internal.h"

#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

using namespace dvm;

struct dvm_context {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int graph_iters = 20;
    size_t budget = 0;
    size_t bytes = 0;
    uint64_t launches = 0;
    uint64_t allocs = 0;        // device allocations made for this context (pool blocks)
    double* pinned = nullptr;   // 64 doubles for small device->host results
    int* derr = nullptr;        // device flag: a kernel's bounded wait ran out
    int flags = 0;
};

struct dvm_mesh {
    dvm_context* ctx = nullptr;
    DevMesh d;
    std::vector<double> nodes;
};

struct dvm_vgrid {
    dvm_context* ctx = nullptr;
    DevGrid d;
};

// Anderson-mixing history of one solve (allocated on the first accelerated solve of a state or
// adjoint): the iterate X at the start of the current block of sweeps, the previous residual and
// image, the rings of their differences, and the Gram matrix of the residual differences.
struct AAState {
    int m = 0, storage = 0;
    size_t n = 0, bytes = 0;
    void *X = nullptr, *Rp = nullptr, *Gp = nullptr, *dR = nullptr, *dG = nullptr;
    double *part = nullptr, *out = nullptr, *gamma = nullptr;
    int* neg = nullptr;
    int cnt = 0, slot = 0, steps = 0;       // columns in use, next ring slot, blocks since (re)start
    int mixes = 0, rejects = 0, restarts = 0;
    double best = INFINITY;                 // lowest block residual since the history started
    std::vector<double> H;                  // m x m: dR_i . dR_j
};

struct dvm_state {
    dvm_context* ctx = nullptr;
    const dvm_mesh* mesh = nullptr;
    const dvm_vgrid* grid = nullptr;
    dvm_flow flow{};
    int storage = 1;
    DevFlow fl;
    void* f[2] = {nullptr, nullptr};
    double4* prim[2] = {nullptr, nullptr};
    double* Fw[2] = {nullptr, nullptr};
    double* Jpart = nullptr;
    double* respart = nullptr;
    double* out = nullptr;      // [2]: sum respart, J
    double* scratch = nullptr;  // [ni + 2] functional scratch
    int cur = 0;
    double r0 = 0.0;
    size_t bytes = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_n = 0;
    int graph_cur = -1;
    uint64_t version = 0;       // bumped whenever f changes (sweeps, uploads)
    TmaMaps maps[2];            // tiled-TMA descriptors of f[0], f[1]
    AAState* aa = nullptr;
    int order = 1;              // spatial order of the face values (2: linear reconstruction)
    int graph_order = 1;        // order the captured graph was built for
    void* so[3] = {nullptr, nullptr, nullptr};   // second order: gradient x, y and the frozen defect
    int so_period = 20;         // sweeps per defect (defect correction groups)
    int so_phase = 0;           // sweeps since the defect was taken (0: take it at the next sweep)
    int graph_phase = 0;        // so_phase at the start of the captured graph
    int graph_so = 0;           // reconstruction launches inside the captured graph
    bool capturing = false;
    int maxwell = 0;            // 1: conservative discrete Maxwellian (fitted to the cell's discrete moments)
    double4* fit = nullptr;     // its parameters for the current f
    AAState* aaW = nullptr;     // moment-space mixing: history over the cell moments
    double* Wbuf = nullptr;     // [ncell][4] FP64 moments
    // macroscopic prediction (dvm_solve_opts.predict_iters > 0; see k_coarse_assemble)
    bool predict = false;       // the residual sweep of each block also writes the residual's moments
    double* co_out = nullptr;   // [ncell][4][16] outflow blocks of the moment system
    double* co_dinv = nullptr;  // [ncell][16] inverses of its diagonal blocks
    double4* co_rW = nullptr;   // [ncell] moments of the residual
    double4* co_x = nullptr;    // [ncell] the moment correction
    KrylovWork co_kr;           // GMRES workspace for up to co_m Arnoldi steps
    int co_m = 0;
    MGWork co_mg;               // multigrid levels of the moment system (dvm_solve_opts.predict_precond = 1)
    int shard = 0;              // 1: a velocity shard (sweeps write partial sums; see dvm_state_set_shard)
    double* part = nullptr;     // [shard_count] this shard's partial sums
    double* part_total = nullptr;   // [shard_count] the summed buffer of all shards
};

struct dvm_adjoint {
    dvm_state* st = nullptr;
    int functional = DVM_DRAG;
    MomentJ mj;                 // m_J of the functional
    double* wallM = nullptr;
    void* cell = nullptr;       // AdjCell<TC>[ncell]: linearisation constants
    uint64_t st_version = ~0ull; // state version the constants and couplings belong to
    void* phi[2] = {nullptr, nullptr};
    double4* Z[2] = {nullptr, nullptr};
    double* Lam[2] = {nullptr, nullptr};
    double* respart = nullptr;
    double* out = nullptr;
    int cur = 0;
    double r0 = 0.0;
    size_t bytes = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_n = 0;
    int graph_cur = -1;
    int graph_st_cur = -1;
    int graph_order = 1;
    int graph_phase = 0;
    int graph_so = 0;
    bool capturing = false;
    void* so_def = nullptr;     // second order: frozen transposed defect (dR/df)^T (w phi) / w
    int so_phase = 0;
    double* Kinv = nullptr;     // conservative Maxwellian: dp/dW per cell, [ncell][4][4]
    TmaMaps maps[2];            // tiled-TMA descriptors of phi[0], phi[1]
    // sensitivity scratch, allocated on first use
    double2 *GN = nullptr, *GE = nullptr, *GW = nullptr, *node_grad = nullptr, *so_corner = nullptr;
    double *vol = nullptr, *elem = nullptr, *dwall = nullptr, *sj = nullptr, *grad = nullptr;
    int sens_P = 0;
    AAState* aa = nullptr;
};

namespace {

thread_local std::string g_err;

// Live-handle registry: every handle is registered at creation and removed by its destroy call, so a
// destroy of an unknown (already released) handle is a no-op, and a context's destroy can release
// whatever its caller left behind, in dependency order.
enum HandleKind { kCtx = 1, kMesh, kGrid, kState, kAdjoint, kBatch };
struct LiveEntry { int kind; const dvm_context* ctx; const void* parent; };
std::mutex g_live_mu;
std::unordered_map<const void*, LiveEntry> g_live;

void live_add(const void* h, int kind, const dvm_context* ctx, const void* parent = nullptr) {
    std::lock_guard<std::mutex> lk(g_live_mu);
    g_live[h] = LiveEntry{kind, ctx, parent};
}
bool live_take(const void* h, int kind) {
    std::lock_guard<std::mutex> lk(g_live_mu);
    auto it = g_live.find(h);
    if (it == g_live.end() || it->second.kind != kind) return false;
    g_live.erase(it);
    return true;
}
std::vector<const void*> live_children(int kind, const dvm_context* ctx, const void* parent = nullptr) {
    std::lock_guard<std::mutex> lk(g_live_mu);
    std::vector<const void*> out;
    for (auto& kv : g_live)
        if (kv.second.kind == kind && (ctx == nullptr || kv.second.ctx == ctx) &&
            (parent == nullptr || kv.second.parent == parent))
            out.push_back(kv.first);
    return out;
}

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int fail_cuda(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return DVM_ERR_CUDA;
}

#define CK(x)                                          \
    do {                                               \
        cudaError_t e_ = (x);                          \
        if (e_ != cudaSuccess) return fail_cuda(e_, #x); \
    } while (0)

// Device memory of states, adjoints, meshes and grids: stream-ordered allocations on the context's
// stream from one pool per device that keeps freed blocks (release threshold at its maximum), so a
// state created after another is destroyed reuses its memory without cudaMalloc or cudaFree, and a
// free never waits for the device.  Every block is freed on the stream it was allocated on, after
// the work queued there that uses it.  dvm_context_destroy trims the pool.
std::mutex g_pool_mu;
std::unordered_map<int, cudaMemPool_t> g_pools;
std::unordered_map<void*, cudaStream_t> g_block_stream;

cudaError_t device_pool(int device, cudaMemPool_t* out) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(device);
    if (it != g_pools.end()) { *out = it->second; return cudaSuccess; }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = ~0ull;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) { cudaMemPoolDestroy(pool); return e; }
    g_pools[device] = pool;
    *out = pool;
    return cudaSuccess;
}

template <class T>
int dalloc(dvm_context* ctx, T** p, size_t count, size_t* acc = nullptr) {
    size_t b = count * sizeof(T);
    if (b == 0) b = sizeof(T);
    cudaMemPool_t pool;
    cudaError_t e = device_pool(ctx->device, &pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)p, b, pool, ctx->stream);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(DVM_ERR_OOM, "device allocation failed: out of device memory");
    }
    if (e != cudaSuccess) return fail_cuda(e, "device allocation");
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        g_block_stream[(void*)*p] = ctx->stream;
    }
    ctx->allocs += 1;
    if (acc) *acc += b;
    return DVM_OK;
}

void dfree(void* p) {
    if (!p) return;
    cudaStream_t s = nullptr;
    bool pooled = false;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        auto it = g_block_stream.find(p);
        if (it != g_block_stream.end()) { s = it->second; pooled = true; g_block_stream.erase(it); }
    }
    if (pooled) cudaFreeAsync(p, s);
    else cudaFree(p);
}

// Return the pool's unused blocks to the device (after the context's work has finished).
void trim_pool(int device) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(device);
    if (it != g_pools.end()) cudaMemPoolTrimTo(it->second, 0);
}

// NVTX range over one library call (solve phases, sensitivity, batch tick) for timeline tools;
// header-only, inert unless a profiler is attached.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

double dir_angle(const dvm_flow& fl, int functional) {
    return fl.aoa + (functional == DVM_LIFT ? 0.5 * M_PI : 0.0);
}

// m_J of a functional (Eq. formula_opt): a force along the free stream (drag) or normal to it
// (lift), or the heat (m_J = |v|^2/2).
MomentJ moment_of(const dvm_flow& fl, int functional) {
    MomentJ mj;
    if (functional == DVM_HEAT) {
        mj.dx = mj.dy = 0.0;
        mj.h = 1.0;
    } else {
        const double ang = dir_angle(fl, functional);
        mj.dx = cos(ang);
        mj.dy = sin(ang);
    }
    return mj;
}

// ------------------------------------------------------------------ argument builders
template <class TS, class TC>
PrimalArgs<TS, TC> primal_args(const dvm_state* st, int src) {
    PrimalArgs<TS, TC> a{};
    const DevMesh& m = st->mesh->d;
    const DevGrid& g = st->grid->d;
    constexpr int KV = 16 / (2 * (int)sizeof(TS));
    a.ncell = m.ncell;
    a.ni = m.ni;
    a.nj = m.nj;
    a.nq = g.nvp / KV;
    a.nb = m.nb;
    if constexpr (sizeof(TC) == 8) {
        a.S = m.Sd; a.V = m.Vd; a.vt = g.vd; a.fd = st->fl.fdd; a.gw = st->fl.gwd;
    } else {
        a.S = m.Sf; a.V = m.Vf; a.vt = g.vf; a.vpa = g.vpa; a.vpb = g.vpb; a.fd = st->fl.fdf; a.gw = st->fl.gwf;
    }
    a.wallD = st->fl.wallD;
    a.inv_tau_inf = 1.0 / st->fl.tau_inf;
    a.halfTw = (TC)(0.5 * st->fl.Tw);
    const double ang = dir_angle(st->flow, DVM_DRAG);
    a.dirx = (TC)cos(ang);
    a.diry = (TC)sin(ang);
    a.f_old = (const TS*)st->f[src];
    a.f_new = (TS*)st->f[1 - src];
    a.prim_old = st->prim[src];
    a.prim_new = st->prim[1 - src];
    a.maxw_old = st->maxwell ? st->fit : st->prim[src];
    a.Fw_old = st->Fw[src];
    a.Fw_new = st->Fw[1 - src];
    a.Jpart = st->Jpart;
    a.respart = st->respart;
    a.err = st->ctx->derr;
    a.defect = st->order == 2 ? (const TS*)st->so[2] : nullptr;
    a.part = st->shard ? st->part : nullptr;
    a.rW = st->predict ? st->co_rW : nullptr;
    return a;
}

template <class TS, class TC>
AdjointArgs<TS, TC> adjoint_args(const dvm_adjoint* ad, int src) {
    AdjointArgs<TS, TC> a{};
    const dvm_state* st = ad->st;
    const DevMesh& m = st->mesh->d;
    const DevGrid& g = st->grid->d;
    constexpr int KV = 16 / (2 * (int)sizeof(TS));
    a.ncell = m.ncell;
    a.ni = m.ni;
    a.nj = m.nj;
    a.nq = g.nvp / KV;
    a.nb = m.nb;
    if constexpr (sizeof(TC) == 8) {
        a.S = m.Sd; a.V = m.Vd; a.vt = g.vd; a.gw = st->fl.gwd;
    } else {
        a.S = m.Sf; a.V = m.Vf; a.vt = g.vf; a.vpa = g.vpa; a.vpb = g.vpb; a.gw = st->fl.gwf;
    }
    a.wallD = st->fl.wallD;
    a.wallM = ad->wallM;
    a.inv_tau_inf = 1.0 / st->fl.tau_inf;
    a.halfTw = (TC)(0.5 * st->fl.Tw);
    a.dirx = (TC)ad->mj.dx;
    a.diry = (TC)ad->mj.dy;
    a.heat = (TC)ad->mj.h;
    a.f = (const TS*)st->f[st->cur];
    a.cell = (const AdjCell<TC>*)ad->cell;
    a.phi_old = (const TS*)ad->phi[src];
    a.phi_new = (TS*)ad->phi[1 - src];
    a.Z_old = ad->Z[src];
    a.Z_new = ad->Z[1 - src];
    a.Lam_old = ad->Lam[src];
    a.Lam_new = ad->Lam[1 - src];
    a.respart = ad->respart;
    a.err = st->ctx->derr;
    a.defect = st->order == 2 ? (const TS*)ad->so_def : nullptr;
    a.Kinv = st->maxwell ? ad->Kinv : nullptr;
    return a;
}

// Second-order reconstruction of `in` (f of the state, or an adjoint phi) into the state's scratch.
template <class TS, class TC>
SOArgs<TS, TC> so_args(const dvm_state* st, const void* in, const double* Fw, void* out) {
    SOArgs<TS, TC> a{};
    const DevMesh& m = st->mesh->d;
    const DevGrid& g = st->grid->d;
    constexpr int KV = 16 / (2 * (int)sizeof(TS));
    a.ncell = m.ncell;
    a.nq = g.nvp / KV;
    a.ni = m.ni;
    a.nb = m.nb;
    if constexpr (sizeof(TC) == 8) {
        a.S = m.Sd; a.V = m.Vd; a.vt = g.vd; a.fd = st->fl.fdd; a.gw = st->fl.gwd;
    } else {
        a.S = m.Sf; a.V = m.Vf; a.vt = g.vf; a.fd = st->fl.fdf; a.gw = st->fl.gwf;
    }
    a.wallD = st->fl.wallD;
    a.halfTw = (TC)(0.5 * st->fl.Tw);
    a.nodes = m.nodes;
    a.in = (const TS*)in;
    a.Fw = Fw;
    a.gx = (TS*)st->so[0];
    a.gy = (TS*)st->so[1];
    a.out = (TS*)out;
    return a;
}

cudaError_t enqueue_second_order(const dvm_state* st, const void* in, const double* Fw, void* out, bool adjoint) {
    cudaStream_t s = st->ctx->stream;
    switch (st->storage) {
        case DVM_STORE_FP64: { auto a = so_args<double, double>(st, in, Fw, out); return launch_second_order(0, &a, adjoint, s); }
        case DVM_STORE_FP32: { auto a = so_args<float, float>(st, in, Fw, out); return launch_second_order(1, &a, adjoint, s); }
        default: { auto a = so_args<__nv_bfloat16, float>(st, in, Fw, out); return launch_second_order(2, &a, adjoint, s); }
    }
}

// Identity of the discretisation a captured graph was built for (spatial order, Maxwellian).
int scheme_of(const dvm_state* st) { return 2 * st->order + st->maxwell + 8 * (st->predict ? 1 : 0); }

// Defect correction: the defect is taken from the sweep's input at the first sweep of each group of
// so_period sweeps and frozen for the rest of the group.  Counts its launches (into the graph's count
// while a graph is being captured).
cudaError_t enqueue_defect_if_due(dvm_state* st, int& phase, bool& capturing, int& graph_so, const void* in,
                                  const double* Fw, void* out, bool adjoint) {
    cudaError_t e = cudaSuccess;
    if (!out || !st->so[0] || !st->so[1]) return cudaErrorInvalidValue;   // buffers of order 2 missing
    if (phase == 0) {
        e = enqueue_second_order(st, in, Fw, out, adjoint);
        if (capturing) graph_so += 2;
        else st->ctx->launches += 2;
    }
    phase = (phase + 1) % st->so_period;
    return e;
}

cudaError_t enqueue_primal(dvm_state* st, int src, bool res = true) {
    if (st->order == 2) {
        cudaError_t e = enqueue_defect_if_due(st, st->so_phase, st->capturing, st->graph_so, st->f[src], st->Fw[src],
                                              st->so[2], false);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e;
    auto launch = st->shard ? launch_primal_shard_sweep : launch_primal_sweep;
    const bool rm = st->predict && res && st->order == 1 && !st->shard;   // residual moments for the prediction
    switch (st->storage) {
        case DVM_STORE_FP64: { auto a = primal_args<double, double>(st, src);
                               e = rm ? launch_primal_sweep_rm(0, &a, st->maps[src], st->ctx->stream)
                                      : launch(0, &a, st->maps[src], res, st->ctx->stream); break; }
        case DVM_STORE_FP32: { auto a = primal_args<float, float>(st, src);
                               e = rm ? launch_primal_sweep_rm(1, &a, st->maps[src], st->ctx->stream)
                                      : launch(1, &a, st->maps[src], res, st->ctx->stream); break; }
        default: { auto a = primal_args<__nv_bfloat16, float>(st, src);
                   e = rm ? launch_primal_sweep_rm(2, &a, st->maps[src], st->ctx->stream)
                          : launch(2, &a, st->maps[src], res, st->ctx->stream); break; }
    }
    if (e == cudaSuccess && st->maxwell) {
        // the next sweep's Maxwellian: one Newton step from the previous fit
        e = launch_maxwell_fit(st->storage, st->mesh->d, st->grid->d, st->prim[1 - src], st->fit, true, 1, nullptr,
                               st->ctx->stream);
        if (st->capturing) st->graph_so += 1;
        else st->ctx->launches += 1;
    }
    return e;
}

cudaError_t enqueue_adjoint(dvm_adjoint* ad, int src, bool update = true, bool res = true) {
    cudaStream_t s = ad->st->ctx->stream;
    if (update && ad->st->order == 2) {
        cudaError_t e = enqueue_defect_if_due(ad->st, ad->so_phase, ad->capturing, ad->graph_so, ad->phi[src], nullptr,
                                              ad->so_def, true);
        if (e != cudaSuccess) return e;
    }
    const TmaMaps& pm = ad->maps[src];
    const TmaMaps& fm = ad->st->maps[ad->st->cur];
    switch (ad->st->storage) {
        case DVM_STORE_FP64: { auto a = adjoint_args<double, double>(ad, src); return launch_adjoint_sweep(0, &a, pm, fm, update, res, s); }
        case DVM_STORE_FP32: { auto a = adjoint_args<float, float>(ad, src); return launch_adjoint_sweep(1, &a, pm, fm, update, res, s); }
        default: { auto a = adjoint_args<__nv_bfloat16, float>(ad, src); return launch_adjoint_sweep(2, &a, pm, fm, update, res, s); }
    }
}

// Recompute the linearisation constants from the state's current moments.
cudaError_t adjoint_relinearise(dvm_adjoint* ad) {
    const dvm_state* st = ad->st;
    cudaError_t e = cudaSuccess;
    if (st->maxwell && ad->Kinv) {
        e = launch_maxwell_fit(st->storage, st->mesh->d, st->grid->d, st->prim[st->cur], st->fit, true, 0, ad->Kinv,
                               st->ctx->stream);
        st->ctx->launches += 1;
    }
    if (e == cudaSuccess)
        e = launch_adjoint_cellconst(st->storage, st->prim[st->cur], st->maxwell ? st->fit : st->prim[st->cur],
                                     st->mesh->d, 1.0 / st->fl.tau_inf,
                                             ad->cell, st->ctx->stream);
    st->ctx->launches += 1;
    ad->st_version = st->version;
    return e;
}

// Rebuild the couplings (Z, Lambda) of phi[cur] in place: a non-updating pass whose outputs land in
// the slot the next sweep reads.
cudaError_t refresh_adjoint_couplings(dvm_adjoint* ad) {
    ad->so_phase = 0;           // phi changed outside the sweeps: retake the second-order defect
    // the non-updating pass reads phi[cur] and writes Z/Lam of slot 1-cur; copy them to slot cur
    cudaError_t e = enqueue_adjoint(ad, ad->cur, false);
    const DevMesh& m = ad->st->mesh->d;
    cudaStream_t s = ad->st->ctx->stream;
    if (e == cudaSuccess) e = cudaMemcpyAsync(ad->Z[ad->cur], ad->Z[1 - ad->cur], m.ncell * sizeof(double4), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ad->Lam[ad->cur], ad->Lam[1 - ad->cur], m.ni * sizeof(double), cudaMemcpyDeviceToDevice, s);
    ad->st->ctx->launches += 1;
    return e;
}

cudaError_t enqueue_primal_finalize(dvm_state* st, int dst_state, double* out) {
    const DevMesh& m = st->mesh->d;
    return launch_finalize(st->respart, m.ncell, st->Jpart, st->Fw[dst_state], st->fl.wallM, m.ni, out,
                           st->ctx->stream);
}

cudaError_t enqueue_adjoint_finalize(dvm_adjoint* ad, double* out) {
    const DevMesh& m = ad->st->mesh->d;
    return launch_finalize(ad->respart, m.ncell, nullptr, nullptr, nullptr, m.ni, out, ad->st->ctx->stream);
}

int check_finite(double v, const char* what) {
    if (!std::isfinite(v)) return fail(DVM_ERR_NONFINITE, std::string(what) + " is not finite");
    return DVM_OK;
}

// Run n primal sweeps without a graph; hist (device, [2n]) receives (sum respart, J) per sweep.
int run_primal_plain(dvm_state* st, int n, double* hist) {
    st->version += (uint64_t)n;
    for (int i = 0; i < n; ++i) {
        CK(enqueue_primal(st, st->cur));
        CK(enqueue_primal_finalize(st, 1 - st->cur, hist ? hist + 2 * i : st->out));
        st->cur = 1 - st->cur;
        st->ctx->launches += 2;
    }
    return DVM_OK;
}

int run_adjoint_plain(dvm_adjoint* ad, int n, double* hist) {
    for (int i = 0; i < n; ++i) {
        CK(enqueue_adjoint(ad, ad->cur));
        CK(enqueue_adjoint_finalize(ad, hist ? hist + 2 * i : ad->out));
        ad->cur = 1 - ad->cur;
        ad->st->ctx->launches += 2;
    }
    return DVM_OK;
}

// ---------------------------------------------------------------- Anderson mixing (host side)
void aa_free(dvm_context* ctx, AAState*& A) {
    if (!A) return;
    dfree(A->X); dfree(A->Rp); dfree(A->Gp); dfree(A->dR); dfree(A->dG);
    dfree(A->part); dfree(A->out); dfree(A->gamma); dfree(A->neg);
    ctx->bytes -= A->bytes;
    delete A;
    A = nullptr;
}

// History for n-element vectors of the given storage and depth m (reused when they match).
int aa_ensure(dvm_context* ctx, AAState*& A, int storage, size_t n, int m) {
    if (A && A->m == m && A->n == n && A->storage == storage) return DVM_OK;
    aa_free(ctx, A);
    A = new (std::nothrow) AAState();
    if (!A) return fail(DVM_ERR_OOM, "host allocation");
    A->m = m; A->n = n; A->storage = storage;
    const size_t eb = storage == DVM_STORE_FP64 ? 8 : 4;
    void** vec[5] = {&A->X, &A->Rp, &A->Gp, &A->dR, &A->dG};
    const size_t len[5] = {n, n, n, (size_t)m * n, (size_t)m * n};
    int rc = DVM_OK;
    for (int i = 0; i < 5 && !rc; ++i) {
        unsigned char* p = nullptr;
        rc = dalloc(ctx, &p, len[i] * eb, &A->bytes);
        *vec[i] = p;
    }
    if (!rc) rc = dalloc(ctx, &A->part, (size_t)aa_blocks() * 2 * m, &A->bytes);
    if (!rc) rc = dalloc(ctx, &A->out, 2 * (size_t)m, &A->bytes);
    if (!rc) rc = dalloc(ctx, &A->gamma, (size_t)m, &A->bytes);
    if (!rc) rc = dalloc(ctx, &A->neg, 1, &A->bytes);
    ctx->bytes += A->bytes;
    if (rc) {
        aa_free(ctx, A);
        return rc;
    }
    A->H.assign((size_t)m * m, 0.0);
    return DVM_OK;
}

// Start a solve (or restart the history): X <- F, empty history.
int aa_begin(dvm_context* ctx, AAState* A, const void* F) {
    A->cnt = A->slot = A->steps = 0;
    A->best = INFINITY;
    CK(launch_aa_load(A->storage, A->n, F, A->X, ctx->stream));
    ctx->launches += 1;
    return DVM_OK;
}

// Safeguard: a block residual above twice the best since the history started means the mixing is
// steering the iteration off (near the rounding floor of FP32 storage, for instance).
bool aa_restart_if_growing(AAState* A, double r) {
    if (A->steps > 1 && r > 2.0 * A->best) {
        A->restarts += 1;
        return true;
    }
    A->best = std::min(A->best, r);
    return false;
}

// Solve (H + eps I) gamma = b for the cnt columns in use (Cholesky, eps = 1e-10 of the mean diagonal).
bool aa_solve(const std::vector<double>& Hm, int m, int cnt, const double* b, double* gamma) {
    std::vector<double> A((size_t)cnt * cnt), L((size_t)cnt * cnt, 0.0);
    double tr = 0.0;
    for (int i = 0; i < cnt; ++i) tr += Hm[(size_t)i * m + i];
    if (!(tr > 0.0) || !std::isfinite(tr)) return false;
    const double eps = 1e-10 * tr / cnt;
    for (int i = 0; i < cnt; ++i)
        for (int j = 0; j < cnt; ++j) A[(size_t)i * cnt + j] = Hm[(size_t)i * m + j] + (i == j ? eps : 0.0);
    for (int j = 0; j < cnt; ++j) {
        double d = A[(size_t)j * cnt + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * cnt + k] * L[(size_t)j * cnt + k];
        if (!(d > 0.0)) return false;
        L[(size_t)j * cnt + j] = sqrt(d);
        for (int i = j + 1; i < cnt; ++i) {
            double v = A[(size_t)i * cnt + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * cnt + k] * L[(size_t)j * cnt + k];
            L[(size_t)i * cnt + j] = v / L[(size_t)j * cnt + j];
        }
    }
    std::vector<double> y(cnt);
    for (int i = 0; i < cnt; ++i) {
        double v = b[i];
        for (int k = 0; k < i; ++k) v -= L[(size_t)i * cnt + k] * y[k];
        y[i] = v / L[(size_t)i * cnt + i];
    }
    for (int i = cnt - 1; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < cnt; ++k) v -= L[(size_t)k * cnt + i] * gamma[k];
        gamma[i] = v / L[(size_t)i * cnt + i];
    }
    for (int i = 0; i < cnt; ++i)
        if (!std::isfinite(gamma[i])) return false;
    return true;
}

// One mixing step after a block of sweeps left G in F.  *mixed = true when F now holds the mixed
// iterate (then the caller refreshes what depends on F).  positive: F is a distribution, and a mix
// that makes a value negative is undone (the adjoint has no sign).
int aa_step(dvm_context* ctx, AAState* A, void* F, bool positive, bool* mixed) {
    *mixed = false;
    cudaStream_t s = ctx->stream;
    const int m = A->m;
    const bool first = A->steps == 0;
    const int slot = A->slot, cnt = first ? 0 : std::min(A->cnt + 1, m);
    CK(launch_aa_collect(A->storage, A->n, F, A->X, A->Rp, A->Gp, A->dR, A->dG, m, cnt, slot, first ? 1 : 0,
                         A->part, A->out, s));
    ctx->launches += first ? 1 : 2;
    A->steps += 1;
    if (first) return DVM_OK;
    std::vector<double> o(2 * (size_t)m);
    CK(cudaMemcpyAsync(o.data(), A->out, o.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < cnt; ++i) {
        A->H[(size_t)slot * m + i] = o[i];
        A->H[(size_t)i * m + slot] = o[i];
    }
    A->cnt = cnt;
    A->slot = (slot + 1) % m;
    std::vector<double> gam(m, 0.0);
    if (!aa_solve(A->H, m, cnt, o.data() + m, gam.data())) return DVM_OK;   // keep G, history goes on
    int zero = 0, neg = 0;
    CK(cudaMemcpyAsync(A->gamma, gam.data(), m * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(A->neg, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    CK(launch_aa_mix(A->storage, A->n, F, A->X, A->Gp, A->dG, cnt, A->gamma, positive ? 1 : 0, A->neg, s));
    CK(cudaMemcpyAsync(&neg, A->neg, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->launches += 1;
    if (neg) {                         // a negative distribution value: undo, restart the history
        CK(launch_aa_restore(A->storage, A->n, F, A->X, A->Gp, s));
        ctx->launches += 1;
        A->cnt = A->slot = A->steps = 0;
        A->rejects += 1;
        return DVM_OK;
    }
    A->mixes += 1;
    *mixed = true;
    return DVM_OK;
}

int check_solve_opts(const dvm_solve_opts* o) {
    if (o->max_iter < 0 || !(o->tol >= 0.0)) return fail(DVM_ERR_INVALID_ARG, "bad solve options");
    if (o->accel_depth < 0 || o->accel_depth > aa_max_depth() || (o->accel_depth > 0 && o->accel_period < 1))
        return fail(DVM_ERR_INVALID_ARG, "accel_depth must be in [0, 8] and accel_period >= 1");
    if (o->accel_space != 0 && o->accel_space != 1) return fail(DVM_ERR_INVALID_ARG, "accel_space must be 0 or 1");
    if (!(o->refine_tol >= 0.0) || o->refine_max < 0 || o->refine_sweeps < 0)
        return fail(DVM_ERR_INVALID_ARG, "refine_tol, refine_max and refine_sweeps must be >= 0");
    if (o->predict_iters < 0 || o->predict_iters > kMaxKrylov || o->predict_reuse < 0 ||
        !(o->predict_omega >= 0.0 && o->predict_omega <= 1.0))
        return fail(DVM_ERR_INVALID_ARG, "predict_iters must be in [0, 64], predict_reuse >= 0, predict_omega in [0, 1]");
    if (o->predict_iters > 0 && o->accel_depth > 0)
        return fail(DVM_ERR_INVALID_ARG, "the macroscopic prediction and Anderson mixing exclude each other");
    if (o->predict_precond != 0 && o->predict_precond != 1)
        return fail(DVM_ERR_INVALID_ARG, "predict_precond must be 0 (block-Jacobi) or 1 (multigrid)");
    return DVM_OK;
}

bool graphs_ok(const dvm_context* ctx) { return ctx->stream != nullptr && !(ctx->flags & DVM_OPT_NO_GRAPHS); }

// Capture K (even) sweeps + one finalize.  Buffers return to the same parity after K sweeps.
int build_primal_graph(dvm_state* st, int K) {
    if (st->graph && st->graph_n == K && st->graph_cur == st->cur && st->graph_order == scheme_of(st) &&
        st->graph_phase == st->so_phase)
        return DVM_OK;
    if (st->graph) { cudaGraphExecDestroy(st->graph); st->graph = nullptr; }
    cudaStream_t s = st->ctx->stream;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int cur = st->cur;
    const int phase0 = st->so_phase;
    st->capturing = true;
    st->graph_so = 0;
    for (int i = 0; i < K; ++i) {
        enqueue_primal(st, cur, i == K - 1);
        if (i == K - 1) enqueue_primal_finalize(st, 1 - cur, st->out);
        cur = 1 - cur;
    }
    st->capturing = false;
    st->so_phase = phase0;      // the sweeps run when the graph is launched
    st->graph_phase = phase0;
    CK(cudaStreamEndCapture(s, &g));
    cudaError_t e = cudaGraphInstantiate(&st->graph, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    st->graph_n = K;
    st->graph_cur = st->cur;
    st->graph_order = scheme_of(st);
    return DVM_OK;
}

int build_adjoint_graph(dvm_adjoint* ad, int K) {
    if (ad->graph && ad->graph_n == K && ad->graph_cur == ad->cur && ad->graph_st_cur == ad->st->cur &&
        ad->graph_order == scheme_of(ad->st) && ad->graph_phase == ad->so_phase)
        return DVM_OK;
    if (ad->graph) { cudaGraphExecDestroy(ad->graph); ad->graph = nullptr; }
    cudaStream_t s = ad->st->ctx->stream;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int cur = ad->cur;
    const int phase0 = ad->so_phase;
    ad->capturing = true;
    ad->graph_so = 0;
    for (int i = 0; i < K; ++i) {
        enqueue_adjoint(ad, cur, true, i == K - 1);
        if (i == K - 1) enqueue_adjoint_finalize(ad, ad->out);
        cur = 1 - cur;
    }
    ad->capturing = false;
    ad->so_phase = phase0;
    ad->graph_phase = phase0;
    CK(cudaStreamEndCapture(s, &g));
    cudaError_t e = cudaGraphInstantiate(&ad->graph, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    ad->graph_n = K;
    ad->graph_cur = ad->cur;
    ad->graph_st_cur = ad->st->cur;
    ad->graph_order = scheme_of(ad->st);
    return DVM_OK;
}

// Read and clear the device error flag (after the stream has been synchronised).
int check_device_flag(dvm_context* ctx) {
    int e = 0;
    CK(cudaMemcpy(&e, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        CK(cudaMemset(ctx->derr, 0, sizeof(int)));
        return fail(DVM_ERR_TIMEOUT, "a staged copy of a sweep did not complete within the wait limit");
    }
    return DVM_OK;
}

// read out[0..1] of the device into the pinned buffer and wait
int fetch2(dvm_context* ctx, const double* dout, double* r) {
    CK(cudaMemcpyAsync(ctx->pinned, dout, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->pinned + 2, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    r[0] = ctx->pinned[0];
    r[1] = ctx->pinned[1];
    int e = 0;
    memcpy(&e, ctx->pinned + 2, sizeof(int));
    if (e) {
        CK(cudaMemset(ctx->derr, 0, sizeof(int)));
        return fail(DVM_ERR_TIMEOUT, "a staged copy of a sweep did not complete within the wait limit");
    }
    return DVM_OK;
}

}  // namespace

// ======================================================================================== C ABI
extern "C" {

const char* dvm_status_string(int s) {
    switch (s) {
        case DVM_OK: return "DVM_OK";
        case DVM_ERR_INVALID_ARG: return "DVM_ERR_INVALID_ARG";
        case DVM_ERR_OOM: return "DVM_ERR_OOM";
        case DVM_ERR_ADMISSION: return "DVM_ERR_ADMISSION";
        case DVM_NOT_CONVERGED: return "DVM_NOT_CONVERGED";
        case DVM_ERR_NONFINITE: return "DVM_ERR_NONFINITE";
        case DVM_ERR_CUDA: return "DVM_ERR_CUDA";
        case DVM_ERR_TIMEOUT: return "DVM_ERR_TIMEOUT";
        case DVM_ERR_STAGNATED: return "DVM_ERR_STAGNATED";
        default: return "DVM_UNKNOWN_STATUS";
    }
}

const char* dvm_last_error(void) { return g_err.c_str(); }

int dvm_context_create(dvm_context** out, int cuda_device, const dvm_options* opt) {
    if (!out) return fail(DVM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDeviceCount");
    if (cuda_device < 0 || cuda_device >= ndev) return fail(DVM_ERR_INVALID_ARG, "no such CUDA device");
    if (opt && opt->graph_iters != 0 && (opt->graph_iters < 2 || opt->graph_iters % 2))
        return fail(DVM_ERR_INVALID_ARG, "graph_iters must be even and >= 2");
    DeviceGuard dg(cuda_device);
    dvm_context* c = new (std::nothrow) dvm_context();
    if (!c) return fail(DVM_ERR_OOM, "host allocation");
    c->device = cuda_device;
    if (opt) {
        if (opt->graph_iters) c->graph_iters = opt->graph_iters;
        c->budget = opt->hbm_budget;
        c->stream = (cudaStream_t)opt->stream;
        c->flags = opt->flags;
    }
    if (!opt || !opt->stream) {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; return fail_cuda(e, "cudaStreamCreate"); }
        c->own_stream = true;
    }
    e = cudaMallocHost((void**)&c->pinned, 64 * sizeof(double));
    if (e != cudaSuccess) { if (c->own_stream) cudaStreamDestroy(c->stream); delete c; return fail_cuda(e, "cudaMallocHost"); }
    e = cudaMalloc((void**)&c->derr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->derr, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFreeHost(c->pinned);
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return fail_cuda(e, "error flag");
    }
    live_add(c, kCtx, c);
    *out = c;
    return DVM_OK;
}

void dvm_context_destroy(dvm_context* c) {
    if (!c) return;
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        auto it = g_live.find(c);
        if (it == g_live.end() || it->second.kind != kCtx) return;
    }
    for (const void* h : live_children(kBatch, c)) dvm_batch_destroy((dvm_batch*)h);
    for (const void* h : live_children(kAdjoint, c)) dvm_adjoint_destroy((dvm_adjoint*)h);
    for (const void* h : live_children(kState, c)) dvm_state_destroy((dvm_state*)h);
    for (const void* h : live_children(kGrid, c)) dvm_vgrid_destroy((dvm_vgrid*)h);
    for (const void* h : live_children(kMesh, c)) dvm_mesh_destroy((dvm_mesh*)h);
    if (!live_take(c, kCtx)) return;
    DeviceGuard dg(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->derr) cudaFree(c->derr);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    trim_pool(c->device);
    delete c;
}

int dvm_selftest_wait_timeout(dvm_context* ctx) {
    if (!ctx) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(ctx->device);
    CK(launch_wait_probe(ctx->derr, ctx->stream));
    ctx->launches += 1;
    CK(cudaStreamSynchronize(ctx->stream));
    return check_device_flag(ctx);
}

size_t dvm_context_bytes(const dvm_context* c) { return c ? c->bytes : 0; }
uint64_t dvm_context_launches(const dvm_context* c) { return c ? c->launches : 0; }
uint64_t dvm_context_allocations(const dvm_context* c) { return c ? c->allocs : 0; }

// ------------------------------------------------------------------------------------- mesh
int dvm_mesh_create(dvm_context* ctx, int ni, int nj, const double* X, dvm_mesh** out) {
    if (!ctx || !X || !out) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (ni < 3 || nj < 1) return fail(DVM_ERR_INVALID_ARG, "mesh needs ni >= 3 and nj >= 1");
    DeviceGuard dg(ctx->device);
    const int nc = ni * nj;
    std::vector<int4> nb(nc);
    std::vector<double2> S(4 * (size_t)nc);
    std::vector<double> V(nc);
    std::vector<float2> Sf(4 * (size_t)nc);
    std::vector<float> Vf(nc);
    auto node = [&](int j, int i) { return double2{X[2 * ((size_t)j * ni + i)], X[2 * ((size_t)j * ni + i) + 1]}; };
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            const int c = j * ni + i, ir = (i + 1) % ni, il = (i + ni - 1) % ni;
            // corners counter-clockwise: (j,i), (j+1,i), (j+1,i+1), (j,i+1)
            const double2 q[4] = {node(j, i), node(j + 1, i), node(j + 1, ir), node(j, ir)};
            double area2 = 0.0;
            for (int e = 0; e < 4; ++e) {
                const double2 a = q[e], b = q[(e + 1) & 3];
                area2 += a.x * b.y - b.x * a.y;
                S[4 * (size_t)c + e] = double2{b.y - a.y, a.x - b.x};
                Sf[4 * (size_t)c + e] = float2{(float)(b.y - a.y), (float)(a.x - b.x)};
            }
            V[c] = 0.5 * area2;
            Vf[c] = (float)V[c];
            if (!(V[c] > 0.0)) {
                char msg[128];
                snprintf(msg, sizeof msg, "cell (i=%d, j=%d) has non-positive area %g", i, j, V[c]);
                return fail(DVM_ERR_INVALID_ARG, msg);
            }
            nb[c] = int4{j * ni + il, j + 1 < nj ? (j + 1) * ni + i : kFar, j * ni + ir, j > 0 ? (j - 1) * ni + i : kWall};
        }
    dvm_mesh* m = new (std::nothrow) dvm_mesh();
    if (!m) return fail(DVM_ERR_OOM, "host allocation");
    m->ctx = ctx;
    m->d.ni = ni; m->d.nj = nj; m->d.ncell = nc;
    m->nodes.assign(X, X + 2 * (size_t)(nj + 1) * ni);
    int rc = DVM_OK;
    if ((rc = dalloc(ctx, &m->d.nb, nc)) || (rc = dalloc(ctx, &m->d.Sd, 4 * (size_t)nc)) ||
        (rc = dalloc(ctx, &m->d.Vd, nc)) || (rc = dalloc(ctx, &m->d.Sf, 4 * (size_t)nc)) ||
        (rc = dalloc(ctx, &m->d.Vf, nc)) || (rc = dalloc(ctx, &m->d.nodes, (size_t)(nj + 1) * ni))) {
        live_add(m, kMesh, ctx);
        dvm_mesh_destroy(m);
        return rc;
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d.nb, nb.data(), nc * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d.Sd, S.data(), S.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d.Vd, V.data(), nc * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d.Sf, Sf.data(), Sf.size() * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d.Vf, Vf.data(), nc * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d.nodes, X, (size_t)(nj + 1) * ni * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);     // the host arrays are local
    if (e != cudaSuccess) { live_add(m, kMesh, ctx); dvm_mesh_destroy(m); return fail_cuda(e, "mesh upload"); }
    live_add(m, kMesh, ctx);
    *out = m;
    return DVM_OK;
}

void dvm_mesh_destroy(dvm_mesh* m) {
    if (!m || !live_take(m, kMesh)) return;
    DeviceGuard dg(m->ctx->device);
    dfree(m->d.nb); dfree(m->d.Sd); dfree(m->d.Vd); dfree(m->d.Sf); dfree(m->d.Vf); dfree(m->d.nodes);
    delete m;
}

// ------------------------------------------------------------------------------------- velocity grid
int dvm_vgrid_create(dvm_context* ctx, int nv, const double* vx, const double* vy, const double* w, dvm_vgrid** out) {
    if (!ctx || !vx || !vy || !w || !out) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (nv < 1) return fail(DVM_ERR_INVALID_ARG, "nv must be >= 1");
    for (int k = 0; k < nv; ++k)
        if (!(w[k] > 0.0) || !std::isfinite(vx[k]) || !std::isfinite(vy[k]))
            return fail(DVM_ERR_INVALID_ARG, "weights must be positive and velocities finite");
    DeviceGuard dg(ctx->device);
    const int nvp = (nv + kPad - 1) / kPad * kPad;
    std::vector<double4> vd(nvp, double4{0, 0, 0, 0});
    const int npair = (nvp / 2 + 127) / 128 * 128;            // whole stage rows of pairs
    std::vector<float4> vf(nvp, float4{0, 0, 0, 0}), vpa(npair, float4{0, 0, 0, 0}), vpb(npair, float4{0, 0, 0, 0});
    for (int k = 0; k < nv; ++k) {
        vd[k] = double4{vx[k], vy[k], w[k], 0.5 * (vx[k] * vx[k] + vy[k] * vy[k])};
        vf[k] = float4{(float)vx[k], (float)vy[k], (float)w[k], (float)vd[k].w};
    }
    for (int p = 0; p < nvp / 2; ++p) {
        const float4 a = vf[2 * p], b = vf[2 * p + 1];
        vpa[p] = float4{a.x, b.x, a.y, b.y};
        vpb[p] = float4{a.z, b.z, a.w, b.w};
    }
    dvm_vgrid* g = new (std::nothrow) dvm_vgrid();
    if (!g) return fail(DVM_ERR_OOM, "host allocation");
    g->ctx = ctx;
    g->d.nv = nv;
    g->d.nvp = nvp;
    int rc;
    live_add(g, kGrid, ctx);
    if ((rc = dalloc(ctx, &g->d.vd, nvp)) || (rc = dalloc(ctx, &g->d.vf, nvp)) || (rc = dalloc(ctx, &g->d.vpa, npair)) ||
        (rc = dalloc(ctx, &g->d.vpb, npair))) {
        dvm_vgrid_destroy(g);
        return rc;
    }
    cudaError_t e = cudaMemcpyAsync(g->d.vd, vd.data(), nvp * sizeof(double4), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->d.vf, vf.data(), nvp * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->d.vpa, vpa.data(), npair * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->d.vpb, vpb.data(), npair * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);     // the host arrays are local
    if (e != cudaSuccess) { dvm_vgrid_destroy(g); return fail_cuda(e, "grid upload"); }
    *out = g;
    return DVM_OK;
}

void dvm_vgrid_destroy(dvm_vgrid* g) {
    if (!g || !live_take(g, kGrid)) return;
    DeviceGuard dg(g->ctx->device);
    dfree(g->d.vd); dfree(g->d.vf); dfree(g->d.vpa); dfree(g->d.vpb);
    delete g;
}

// ------------------------------------------------------------------------------------- state
void dvm_state_destroy(dvm_state* st) {
    if (!st) return;
    for (const void* h : live_children(kAdjoint, nullptr, st)) dvm_adjoint_destroy((dvm_adjoint*)h);
    if (!live_take(st, kState)) return;
    DeviceGuard dg(st->ctx->device);
    cudaStreamSynchronize(st->ctx->stream);
    if (st->graph) cudaGraphExecDestroy(st->graph);
    for (int b = 0; b < 2; ++b) { dfree(st->f[b]); dfree(st->prim[b]); dfree(st->Fw[b]); }
    dfree(st->Jpart); dfree(st->respart); dfree(st->out); dfree(st->scratch);
    for (void* p : st->so) dfree(p);
    dfree(st->fit);
    dfree(st->fl.fdd); dfree(st->fl.fdf); dfree(st->fl.gwd); dfree(st->fl.gwf); dfree(st->fl.wallD); dfree(st->fl.wallM);
    aa_free(st->ctx, st->aa);
    aa_free(st->ctx, st->aaW);
    dfree(st->Wbuf);
    dfree(st->part);
    dfree(st->part_total);
    dfree(st->co_out); dfree(st->co_dinv); dfree(st->co_rW); dfree(st->co_x);
    krylov_release_graphs(st->co_kr);
    for (int l = 0; l < st->co_mg.nlev; ++l) {
        MGLevel& L = st->co_mg.lev[l];
        dfree(L.D); dfree(L.Dinv); dfree(L.C); dfree(L.x); dfree(L.b); dfree(L.r);
    }
    dfree(st->co_kr.V); dfree(st->co_kr.w); dfree(st->co_kr.part); dfree(st->co_kr.H); dfree(st->co_kr.scal);
    dfree(st->co_kr.y);
    st->ctx->bytes -= st->bytes;
    delete st;
}

static size_t state_bytes(const dvm_mesh* m, const dvm_vgrid* g, int storage) {
    return 2 * (size_t)m->d.ncell * g->d.nvp * storage_bytes(storage) + (size_t)m->d.ncell * (2 * 32 + 8) +
           (size_t)m->d.ni * 48 + (size_t)g->d.nvp * 48;
}

int dvm_state_create(dvm_context* ctx, const dvm_mesh* mesh, const dvm_vgrid* grid, const dvm_flow* flow,
                     int storage, dvm_state** out) {
    if (!ctx || !mesh || !grid || !flow || !out) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (storage < 0 || storage > 2) return fail(DVM_ERR_INVALID_ARG, "unknown storage");
    if (!(flow->Kn > 0.0) || !(flow->Ma >= 0.0) || !(flow->Tw > 0.0) || !std::isfinite(flow->aoa))
        return fail(DVM_ERR_INVALID_ARG, "flow needs Kn > 0, Ma >= 0, Tw > 0");
    if (mesh->ctx != ctx || grid->ctx != ctx) return fail(DVM_ERR_INVALID_ARG, "mesh/grid from another context");
    const size_t need = state_bytes(mesh, grid, storage);
    if (ctx->budget && ctx->bytes + need > ctx->budget)
        return fail(DVM_ERR_ADMISSION, "state does not fit the context's HBM budget");
    DeviceGuard dg(ctx->device);
    dvm_state* st = new (std::nothrow) dvm_state();
    if (!st) return fail(DVM_ERR_OOM, "host allocation");
    st->ctx = ctx; st->mesh = mesh; st->grid = grid; st->flow = *flow; st->storage = storage;
    live_add(st, kState, ctx);
    const DevMesh& m = mesh->d;
    const DevGrid& g = grid->d;
    st->fl.tau_inf = 5.0 / 16.0 * flow->Kn * sqrt(2.0 * M_PI);
    const double U = flow->Ma * sqrt(5.0 / 3.0);
    st->fl.u1 = U * cos(flow->aoa);
    st->fl.u2 = U * sin(flow->aoa);
    st->fl.Tw = flow->Tw;
    st->fl.Ma = flow->Ma;
    st->fl.aoa = flow->aoa;
    size_t acc = 0;
    const size_t pair = storage_bytes(storage), nfp = (size_t)m.ncell * g.nvp;
    int rc = DVM_OK;
    auto bail = [&](int r) { st->bytes = 0; dvm_state_destroy(st); return r; };
    for (int b = 0; b < 2 && !rc; ++b) {
        rc = dalloc(ctx, (unsigned char**)&st->f[b], nfp * pair, &acc);
        if (!rc) rc = dalloc(ctx, &st->prim[b], m.ncell, &acc);
        if (!rc) rc = dalloc(ctx, &st->Fw[b], m.ni, &acc);
    }
    if (!rc) rc = dalloc(ctx, &st->Jpart, m.ni, &acc);
    if (!rc) rc = dalloc(ctx, &st->respart, m.ncell, &acc);
    if (!rc) rc = dalloc(ctx, &st->out, 2, &acc);
    if (!rc) rc = dalloc(ctx, &st->scratch, (size_t)m.ni + 2, &acc);
    if (!rc) rc = dalloc(ctx, &st->fl.fdd, g.nvp, &acc);
    if (!rc) rc = dalloc(ctx, &st->fl.fdf, g.nvp, &acc);
    if (!rc) rc = dalloc(ctx, &st->fl.gwd, g.nvp, &acc);
    if (!rc) rc = dalloc(ctx, &st->fl.gwf, g.nvp, &acc);
    if (!rc) rc = dalloc(ctx, &st->fl.wallD, m.ni, &acc);
    if (!rc) rc = dalloc(ctx, &st->fl.wallM, m.ni, &acc);
    if (rc) return bail(rc);
    st->bytes = acc;
    ctx->bytes += acc;
    {
        const int nq = g.nvp * (int)pair / 16;
        for (int b = 0; b < 2; ++b) {
            cudaError_t me = make_tmamaps(st->f[b], m.ni, m.nj, nq, &st->maps[b]);
            if (me != cudaSuccess) return bail(fail_cuda(me, "tensor map of f"));
        }
    }
    cudaStream_t s = ctx->stream;
    cudaError_t e = launch_flow_tables(g, st->fl, s);
    if (e == cudaSuccess) e = launch_wall_setup(m, g, st->fl, moment_of(*flow, DVM_DRAG), st->fl.wallD, st->fl.wallM, s);
    if (e == cudaSuccess) e = launch_fill_freestream(storage, st->f[0], m.ncell, g, st->fl, s);
    if (e == cudaSuccess) e = launch_moments(storage, st->f[0], m, g, st->prim[0], st->Fw[0], s);
    ctx->launches += 5;
    if (e != cudaSuccess) return bail(fail_cuda(e, "state setup"));
    // r0: residual of the free-stream state, from one sweep whose output is discarded
    e = enqueue_primal(st, 0);
    if (e == cudaSuccess) e = enqueue_primal_finalize(st, 1, st->out);
    ctx->launches += 2;
    if (e != cudaSuccess) return bail(fail_cuda(e, "r0 sweep"));
    double r[2];
    if ((rc = fetch2(ctx, st->out, r))) return bail(rc);
    st->r0 = sqrt(r[0]);
    if (!std::isfinite(st->r0) || st->r0 <= 0.0) return bail(fail(DVM_ERR_NONFINITE, "free-stream residual not finite"));
    *out = st;
    return DVM_OK;
}

int dvm_state_set(dvm_state* st, const double* f_host) {
    if (!st || !f_host) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(st->ctx->device);
    const DevMesh& m = st->mesh->d;
    const DevGrid& g = st->grid->d;
    double* tmp = nullptr;
    const size_t n = (size_t)m.ncell * g.nv * 2;
    int rc = dalloc(st->ctx, &tmp, n);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(tmp, f_host, n * sizeof(double), cudaMemcpyHostToDevice, st->ctx->stream);
    if (e == cudaSuccess) e = launch_convert(st->storage, 1, tmp, st->f[st->cur], m.ncell, g.nv, g.nvp, st->ctx->stream);
    if (e == cudaSuccess) e = launch_moments(st->storage, st->f[st->cur], m, g, st->prim[st->cur], st->Fw[st->cur], st->ctx->stream);
    if (e == cudaSuccess && st->maxwell) {
        e = launch_maxwell_fit(st->storage, m, g, st->prim[st->cur], st->fit, false, 8, nullptr, st->ctx->stream);
        st->ctx->launches += 1;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st->ctx->stream);
    st->ctx->launches += 2;
    st->version += 1;
    st->so_phase = 0;
    dfree(tmp);
    if (e != cudaSuccess) return fail_cuda(e, "state upload");
    return DVM_OK;
}

int dvm_state_get(const dvm_state* st, double* f_host) {
    if (!st || !f_host) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(st->ctx->device);
    const DevMesh& m = st->mesh->d;
    const DevGrid& g = st->grid->d;
    double* tmp = nullptr;
    const size_t n = (size_t)m.ncell * g.nv * 2;
    int rc = dalloc(st->ctx, &tmp, n);
    if (rc) return rc;
    cudaError_t e = launch_convert(st->storage, 0, st->f[st->cur], tmp, m.ncell, g.nv, g.nvp, st->ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f_host, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, st->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st->ctx->stream);
    st->ctx->launches += 1;
    dfree(tmp);
    if (e != cudaSuccess) return fail_cuda(e, "state download");
    return DVM_OK;
}

// Shape check shared by the device-to-device copies: same context, cell layout, velocity count and
// storage.
static int same_layout(const dvm_state* a, const dvm_state* b) {
    if (a->ctx != b->ctx) return fail(DVM_ERR_INVALID_ARG, "states of different contexts");
    if (a->mesh->d.ni != b->mesh->d.ni || a->mesh->d.nj != b->mesh->d.nj)
        return fail(DVM_ERR_INVALID_ARG, "meshes of different shapes");
    if (a->grid->d.nv != b->grid->d.nv) return fail(DVM_ERR_INVALID_ARG, "velocity grids of different sizes");
    if (a->storage != b->storage) return fail(DVM_ERR_INVALID_ARG, "different storage precisions");
    return DVM_OK;
}

int dvm_state_copy_from(dvm_state* dst, const dvm_state* src) {
    if (!dst || !src) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    if (dst == src) return DVM_OK;
    int rc = same_layout(dst, src);
    if (rc) return rc;
    DeviceGuard dg(dst->ctx->device);
    const DevMesh& m = dst->mesh->d;
    const DevGrid& g = dst->grid->d;
    cudaStream_t s = dst->ctx->stream;
    const size_t bytes = (size_t)m.ncell * g.nvp * storage_bytes(dst->storage);
    cudaError_t e = cudaMemcpyAsync(dst->f[dst->cur], src->f[src->cur], bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = launch_moments(dst->storage, dst->f[dst->cur], m, g, dst->prim[dst->cur], dst->Fw[dst->cur], s);
    dst->ctx->launches += 1;
    if (e == cudaSuccess && dst->maxwell) {
        e = launch_maxwell_fit(dst->storage, m, g, dst->prim[dst->cur], dst->fit, false, 8, nullptr, s);
        dst->ctx->launches += 1;
    }
    dst->version += 1;
    dst->so_phase = 0;
    if (e != cudaSuccess) return fail_cuda(e, "state copy");
    return DVM_OK;
}

int dvm_state_moments(const dvm_state* st, double* prim_host) {
    if (!st || !prim_host) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(st->ctx->device);
    CK(cudaMemcpyAsync(prim_host, st->prim[st->cur], st->mesh->d.ncell * sizeof(double4), cudaMemcpyDeviceToHost,
                       st->ctx->stream));
    CK(cudaStreamSynchronize(st->ctx->stream));
    return DVM_OK;
}

int dvm_state_set_order(dvm_state* st, int order, int defect_period) {
    if (!st) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    if (st->shard && order != 1) return fail(DVM_ERR_INVALID_ARG, "velocity shards are first order");
    if (order != 1 && order != 2) return fail(DVM_ERR_INVALID_ARG, "order must be 1 or 2");
    if (defect_period < 0) return fail(DVM_ERR_INVALID_ARG, "defect_period must be >= 0");
    if (order == 2 && !st->so[0]) {
        dvm_context* ctx = st->ctx;
        const size_t nb = (size_t)st->mesh->d.ncell * st->grid->d.nvp * storage_bytes(st->storage);
        if (ctx->budget && ctx->bytes + 3 * nb > ctx->budget)
            return fail(DVM_ERR_ADMISSION, "second-order buffers do not fit the context's HBM budget");
        DeviceGuard dg(ctx->device);
        size_t acc = 0;
        int rc = DVM_OK;
        for (int b = 0; b < 3 && !rc; ++b) rc = dalloc(ctx, (unsigned char**)&st->so[b], nb, &acc);
        if (rc) {
            for (void*& p : st->so) { dfree(p); p = nullptr; }
            return rc;
        }
        st->bytes += acc;
        ctx->bytes += acc;
    }
    st->order = order;
    st->so_period = defect_period > 0 ? defect_period : 20;
    st->so_phase = 0;
    return DVM_OK;
}

// The adjoint's frozen defect buffer, allocated when a sweep of a second-order state first needs it.
static int adjoint_so_ensure(dvm_adjoint* ad) {
    dvm_context* ctx = ad->st->ctx;
    if (ad->st->maxwell && !ad->Kinv) {
        const size_t nb = (size_t)ad->st->mesh->d.ncell * 16 * sizeof(double);
        if (ctx->budget && ctx->bytes + nb > ctx->budget)
            return fail(DVM_ERR_ADMISSION, "the adjoint's Maxwellian Jacobians do not fit the context's HBM budget");
        size_t acc = 0;
        int rc = dalloc(ctx, &ad->Kinv, (size_t)ad->st->mesh->d.ncell * 16, &acc);
        if (rc) return rc;
        ad->bytes += acc;
        ctx->bytes += acc;
        ad->st_version = ~0ull;   // relinearise with the Jacobians
    }
    if (ad->st->order != 2 || ad->so_def) return DVM_OK;
    const size_t nb = (size_t)ad->st->mesh->d.ncell * ad->st->grid->d.nvp * storage_bytes(ad->st->storage);
    if (ctx->budget && ctx->bytes + nb > ctx->budget)
        return fail(DVM_ERR_ADMISSION, "second-order adjoint buffer does not fit the context's HBM budget");
    size_t acc = 0;
    int rc = dalloc(ctx, (unsigned char**)&ad->so_def, nb, &acc);
    if (rc) return rc;
    ad->bytes += acc;
    ctx->bytes += acc;
    ad->so_phase = 0;
    return DVM_OK;
}

int dvm_state_get_order(const dvm_state* st, int* order) {
    if (!st || !order) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    *order = st->order;
    return DVM_OK;
}

int dvm_state_set_maxwellian(dvm_state* st, int kind) {
    if (!st) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    if (st->shard && kind != DVM_MAXWELL_PLAIN) return fail(DVM_ERR_INVALID_ARG, "velocity shards use the plain Maxwellian");
    if (kind != DVM_MAXWELL_PLAIN && kind != DVM_MAXWELL_CONSERVATIVE) return fail(DVM_ERR_INVALID_ARG, "unknown Maxwellian");
    dvm_context* ctx = st->ctx;
    DeviceGuard dg(ctx->device);
    if (kind == DVM_MAXWELL_CONSERVATIVE && !st->fit) {
        const size_t nb = (size_t)st->mesh->d.ncell * sizeof(double4);
        if (ctx->budget && ctx->bytes + nb > ctx->budget)
            return fail(DVM_ERR_ADMISSION, "the fitted Maxwellian does not fit the context's HBM budget");
        size_t acc = 0;
        int rc = dalloc(ctx, &st->fit, st->mesh->d.ncell, &acc);
        if (rc) return rc;
        st->bytes += acc;
        ctx->bytes += acc;
    }
    st->maxwell = kind;
    st->version += 1;           // adjoints relinearise
    if (kind == DVM_MAXWELL_CONSERVATIVE) {
        CK(launch_maxwell_fit(st->storage, st->mesh->d, st->grid->d, st->prim[st->cur], st->fit, false, 8, nullptr,
                              ctx->stream));
        ctx->launches += 1;
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return DVM_OK;
}

int dvm_state_get_maxwellian(const dvm_state* st, int* kind) {
    if (!st || !kind) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    *kind = st->maxwell;
    return DVM_OK;
}

int dvm_primal_iterate(dvm_state* st, int n, double* residual_out) {
    if (!st || n < 0) return fail(DVM_ERR_INVALID_ARG, "bad argument");
    if (n == 0) return DVM_OK;
    DeviceGuard dg(st->ctx->device);
    if (st->shard) {              // one sweep into the partial sums; the caller combines the shards
        if (n != 1) return fail(DVM_ERR_INVALID_ARG, "a velocity shard sweeps once between combinations");
        CK(enqueue_primal(st, st->cur, true));
        st->cur = 1 - st->cur;
        st->version += 1;
        st->ctx->launches += 1;
        CK(cudaStreamSynchronize(st->ctx->stream));
        if (residual_out) residual_out[0] = NAN;
        return check_device_flag(st->ctx);
    }
    double* hist = nullptr;
    int rc = dalloc(st->ctx, &hist, 2 * (size_t)n);
    if (rc) return rc;
    rc = run_primal_plain(st, n, hist);
    if (!rc) {
        std::vector<double> h(2 * (size_t)n);
        cudaError_t e = cudaMemcpyAsync(h.data(), hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st->ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st->ctx->stream);
        if (e != cudaSuccess) rc = fail_cuda(e, "residual history");
        if (!rc) rc = check_device_flag(st->ctx);
        for (int i = 0; i < n && !rc; ++i) {
            const double r = sqrt(h[2 * i]) / st->r0;
            if (residual_out) residual_out[i] = r;
            if (!std::isfinite(r)) rc = fail(DVM_ERR_NONFINITE, "residual is not finite");
        }
    }
    dfree(hist);
    return rc;
}

int dvm_state_functional(dvm_state* st, int functional, double* J) {
    if (!st || !J) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(st->ctx->device);
    if (functional < DVM_DRAG || functional > DVM_HEAT) return fail(DVM_ERR_INVALID_ARG, "unknown functional");
    CK(launch_functional(st->storage, st->f[st->cur], st->mesh->d, st->grid->d, st->fl, st->Fw[st->cur],
                         moment_of(st->flow, functional), st->scratch, st->scratch + st->mesh->d.ni,
                         st->ctx->stream));
    st->ctx->launches += 2;
    double r[2];
    int rc = fetch2(st->ctx, st->scratch + st->mesh->d.ni, r);
    if (rc) return rc;
    *J = r[1];
    return DVM_OK;
}

// ---------------------------------------------------------------- mixed-precision refinement
// f = fbar + delta (fbar: the FP32 state, delta: an FP32 remainder).  Each correction step takes the
// exact residual R(fbar + delta) from one FP64 sweep of the composed state (increment s = -R/D), solves
// J e = -R by linearised FP32 sweeps (k_primal_lin_sweep) and adds e to delta, renormalised into fbar.
namespace {

// Damping of the prediction, adapted from block to block: a correction the moment model misjudges
// (a mode it takes as nearly free while the kinetic sweeps damp it) raises the next block's residual,
// at once or slowly.  The damping halves after a block that grew the residual by more than 1.5x, and
// after five predicted blocks in a row without a new best residual (a slow growth); after a block that
// set a new best it recovers by 1.25x up to its initial value.  As it goes to 0 the sweeps are plain.
struct PredictDamping {
    double w0, w;
    double r_prev = INFINITY, best = INFINITY;
    int since_best = 0;
    bool after_prediction = false;
    explicit PredictDamping(double omega) : w0(omega), w(omega) {}
    void block(double r) {
        if (after_prediction) {
            if (r > 1.5 * r_prev) w *= 0.5;
            if (r < 0.98 * best) {
                w = std::min(w0, 1.25 * w);
                since_best = 0;
            } else if (++since_best >= 5) {
                w *= 0.5;
                since_best = 0;
            }
        }
        best = std::min(best, r);
        r_prev = r;
        after_prediction = false;
    }
};

// Buffers of the macroscopic prediction, allocated on the first predicted solve and kept with the state
// (the GMRES workspace grows with the Arnoldi steps asked for).
static int predict_ensure(dvm_state* st, int m) {
    dvm_context* ctx = st->ctx;
    const size_t nc = (size_t)st->mesh->d.ncell;
    size_t acc = 0;
    int rc;
    if (!st->co_out) {                    // all or nothing: co_out marks the set as present
        double *out = nullptr, *dinv = nullptr, *W = st->Wbuf;
        double4 *rW = nullptr, *x = nullptr;
        size_t a0 = 0;
        if ((rc = dalloc(ctx, &out, 64 * nc, &a0)) || (rc = dalloc(ctx, &dinv, 16 * nc, &a0)) ||
            (rc = dalloc(ctx, &rW, nc, &a0)) || (rc = dalloc(ctx, &x, nc, &a0)) ||
            (!W && (rc = dalloc(ctx, &W, 4 * nc, &a0)))) {
            dfree(out); dfree(dinv); dfree(rW); dfree(x);
            if (W != st->Wbuf) dfree(W);
            return rc;
        }
        st->co_out = out; st->co_dinv = dinv; st->co_rW = rW; st->co_x = x; st->Wbuf = W;
        acc += a0;
    }
    if (m > st->co_m) {
        KrylovWork& K = st->co_kr;
        const size_t old = st->co_m > 0 ? (size_t)(st->co_m + 1) * nc * sizeof(double4) + nc * sizeof(double4) +
                                              (krylov_part_count(st->co_m) + (size_t)st->co_m * (st->co_m + 1) +
                                               (size_t)(st->co_m + 3) + (size_t)st->co_m) * sizeof(double)
                                        : 0;
        if (K.graph[0] || K.graph[1]) {   // a replay may still be in flight
            CK(cudaStreamSynchronize(ctx->stream));
            krylov_release_graphs(K);
        }
        dfree(K.V); dfree(K.w); dfree(K.part); dfree(K.H); dfree(K.scal); dfree(K.y);
        K = KrylovWork();
        st->co_m = 0;
        st->bytes -= old;
        ctx->bytes -= old;
        if ((rc = dalloc(ctx, &K.V, (size_t)(m + 1) * nc, &acc)) || (rc = dalloc(ctx, &K.w, nc, &acc)) ||
            (rc = dalloc(ctx, &K.part, krylov_part_count(m), &acc)) ||
            (rc = dalloc(ctx, &K.H, (size_t)m * (m + 1), &acc)) || (rc = dalloc(ctx, &K.scal, (size_t)m + 3, &acc)) ||
            (rc = dalloc(ctx, &K.y, (size_t)m, &acc))) {
            st->bytes += acc;
            ctx->bytes += acc;
            return rc;
        }
        st->co_m = m;
    }
    st->bytes += acc;
    ctx->bytes += acc;
    return DVM_OK;
}

// Multigrid levels of the moment system, allocated on first use and kept with the state.
static int mg_ensure(dvm_state* st) {
    if (st->co_mg.nlev > 0) return DVM_OK;
    dvm_context* ctx = st->ctx;
    int nis[kMaxMGLevels], njs[kMaxMGLevels];
    const int n = mg_plan(st->mesh->d.ni, st->mesh->d.nj, nis, njs);
    MGWork W;
    size_t acc = 0;
    int rc = DVM_OK;
    for (int l = 0; l < n && !rc; ++l) {
        MGLevel& L = W.lev[l];
        L.ni = nis[l]; L.nj = njs[l]; L.nc = nis[l] * njs[l];
        const size_t nc = (size_t)L.nc;
        if ((rc = dalloc(ctx, &L.D, 16 * nc, &acc)) || (rc = dalloc(ctx, &L.Dinv, 16 * nc, &acc)) ||
            (rc = dalloc(ctx, &L.C, 64 * nc, &acc)) || (rc = dalloc(ctx, &L.x, nc, &acc)) ||
            (rc = dalloc(ctx, &L.b, nc, &acc)) || (rc = dalloc(ctx, &L.r, nc, &acc)))
            break;
    }
    if (rc) {
        for (int l = 0; l < n; ++l) {
            MGLevel& L = W.lev[l];
            dfree(L.D); dfree(L.Dinv); dfree(L.C); dfree(L.x); dfree(L.b); dfree(L.r);
        }
        return rc;
    }
    W.nlev = n;
    st->co_mg = W;
    st->bytes += acc;
    ctx->bytes += acc;
    return DVM_OK;
}

// The moment system at the moments prim, and its multigrid levels when the solve uses them.
static cudaError_t assemble_coarse(dvm_state* st, const double4* prim, bool mg) {
    cudaStream_t s = st->ctx->stream;
    cudaError_t e = launch_coarse_assemble(st->storage, st->mesh->d, st->grid->d, st->fl, prim, st->co_out,
                                           st->co_dinv, s);
    st->ctx->launches += 1;
    if (e == cudaSuccess && mg) {
        e = launch_mg_setup(st->mesh->d, st->co_out, st->co_dinv, st->co_mg, s);
        st->ctx->launches += 2 * st->co_mg.nlev - 1;
    }
    return e;
}

// One macroscopic prediction after a block whose last sweep wrote the moments of its residual to co_rW:
// (re)assemble the moment system at the current moments if asked, solve it for dW by GMRES (m steps),
// the limited target moments, the Maxwellian shift of f to them, and the moments of the shifted f.
static int predict_step(dvm_state* st, int m, double omega, bool assemble, bool mg = false) {
    const DevMesh& msh = st->mesh->d;
    const DevGrid& g = st->grid->d;
    cudaStream_t s = st->ctx->stream;
    const int c = st->cur;
    if (assemble) CK(assemble_coarse(st, st->prim[c], mg));
    CK(launch_coarse_gmres(msh, st->co_out, st->co_dinv, st->co_rW, false, m, st->co_kr, st->co_x, graphs_ok(st->ctx), s,
                           mg ? &st->co_mg : nullptr));
    CK(launch_coarse_target(msh.ncell, st->prim[c], st->co_x, omega, 0.3, st->Wbuf, s));
    CK(launch_moment_shift(st->storage, st->f[c], msh, g, st->prim[c], st->Wbuf, s));
    CK(launch_moments(st->storage, st->f[c], msh, g, st->prim[c], st->Fw[c], s));
    st->ctx->launches += krylov_launches(m) + 3;
    st->version += 1;
    return DVM_OK;
}

struct RefineWork {
    dvm_context* ctx = nullptr;
    dvm_state* s64 = nullptr;
    float* delta = nullptr;
    float* e[2] = {nullptr, nullptr};
    float* src = nullptr;
    double4* dW[2] = {nullptr, nullptr};
    double* dF[2] = {nullptr, nullptr};
    double* Jp = nullptr;
    double* rp = nullptr;
    double* out = nullptr;
    TmaMaps maps[2];
    ~RefineWork() {
        if (ctx) cudaStreamSynchronize(ctx->stream);
        for (int b = 0; b < 2; ++b) { dfree(e[b]); dfree(dW[b]); dfree(dF[b]); }
        dfree(delta); dfree(src); dfree(Jp); dfree(rp); dfree(out);
        if (s64) dvm_state_destroy(s64);
    }
};

int refine_primal(dvm_state* st, const dvm_solve_opts* o, dvm_primal_result* res) {
    if (st->storage != DVM_STORE_FP32 || st->order != 1 || st->maxwell)
        return fail(DVM_ERR_INVALID_ARG, "refinement needs an FP32 state of order 1 with the plain Maxwellian");
    Range nvtx("dvm_primal_refine");
    dvm_context* ctx = st->ctx;
    cudaStream_t s = ctx->stream;
    const DevMesh& m = st->mesh->d;
    const DevGrid& g = st->grid->d;
    const size_t nf = (size_t)m.ncell * g.nvp * 2;       // floats of one FP32 state buffer
    RefineWork W;
    W.ctx = ctx;
    int rc = dvm_state_create(ctx, st->mesh, st->grid, &st->flow, DVM_STORE_FP64, &W.s64);
    if (rc) return rc;
    dvm_state* s64 = W.s64;
    if ((rc = dalloc(ctx, &W.delta, nf)) || (rc = dalloc(ctx, &W.src, nf)) || (rc = dalloc(ctx, &W.Jp, m.ni)) ||
        (rc = dalloc(ctx, &W.rp, m.ncell)) || (rc = dalloc(ctx, &W.out, 2)))
        return rc;
    for (int b = 0; b < 2; ++b) {
        if ((rc = dalloc(ctx, &W.e[b], nf)) || (rc = dalloc(ctx, &W.dW[b], m.ncell)) || (rc = dalloc(ctx, &W.dF[b], m.ni)))
            return rc;
        CK(make_tmamaps(W.e[b], m.ni, m.nj, g.nvp / 2, &W.maps[b]));
    }
    CK(cudaMemsetAsync(W.delta, 0, nf * sizeof(float), s));
    const bool pred = o->predict_iters > 0;     // the macroscopic prediction of the correction sweeps
    if (pred && (rc = predict_ensure(st, o->predict_iters))) return rc;
    const bool mg = pred && o->predict_precond == 1;
    if (mg && (rc = mg_ensure(st))) return rc;
    const double omega = o->predict_omega > 0.0 ? o->predict_omega : 0.8;
    int predictions = 0;
    PredictDamping damp(omega);
    const int max_steps = o->refine_max > 0 ? o->refine_max : 20;
    const int max_sweeps = o->refine_sweeps > 0 ? o->refine_sweeps : 4000;
    constexpr int kBlock = 20;             // linearised sweeps between residual checks
    double r64 = INFINITY, best = INFINITY, J64 = 0.0;
    int steps = 0, sweeps = 0, misses = 0, status = DVM_NOT_CONVERGED;
    float* fbar = static_cast<float*>(st->f[st->cur]);
    for (;;) {
        // exact residual of fbar + delta: compose it in the FP64 state and sweep that once
        const int c64 = s64->cur;
        CK(launch_refine_compose(fbar, W.delta, static_cast<double*>(s64->f[c64]), m.ncell, g.nvp, s));
        CK(launch_moments(DVM_STORE_FP64, s64->f[c64], m, g, s64->prim[c64], s64->Fw[c64], s));
        ctx->launches += 2;
        s64->version += 1;
        if ((rc = dvm_state_functional(s64, DVM_DRAG, &J64))) return rc;
        CK(enqueue_primal(s64, c64, true));
        CK(enqueue_primal_finalize(s64, 1 - c64, s64->out));
        ctx->launches += 2;
        double ro[2];
        if ((rc = fetch2(ctx, s64->out, ro))) return rc;
        r64 = sqrt(ro[0]) / st->r0;
        if (steps == 0) res->residual_fp64 = r64;
        if (!std::isfinite(r64) || !std::isfinite(J64)) { status = fail(DVM_ERR_NONFINITE, "refinement residual is not finite"); break; }
        if (r64 <= o->refine_tol) { status = DVM_OK; break; }
        if (steps >= max_steps) { status = DVM_NOT_CONVERGED; break; }
        // a step far from the solution can raise the residual while it cuts the error (the quadratic
        // term of the residual in the correction): stagnation is two steps in a row without a cut to 0.7
        if (r64 > 0.7 * best) {
            if (++misses >= 2) { status = DVM_ERR_STAGNATED; break; }
        } else {
            misses = 0;
        }
        best = std::min(best, r64);
        // s = -R/D from that sweep; e solves J e = -R by linearised sweeps from e = 0
        CK(launch_refine_diff(static_cast<const double*>(s64->f[1 - c64]), static_cast<const double*>(s64->f[c64]),
                              W.src, m.ncell, g.nvp, s));
        CK(cudaMemsetAsync(W.e[0], 0, nf * sizeof(float), s));
        CK(cudaMemsetAsync(W.dW[0], 0, m.ncell * sizeof(double4), s));
        CK(cudaMemsetAsync(W.dF[0], 0, m.ni * sizeof(double), s));
        ctx->launches += 1;
        // no stall exit: upwind transport makes these sweeps strongly non-normal at small Kn, and the
        // linear residual can stay near (or above) |R| for hundreds of sweeps before it decays
        int ec = 0, n = 0;
        const double target = 0.1 * r64 * st->r0;
        if (pred) {         // the moment system of the correction, linearised at fbar + delta
            CK(assemble_coarse(st, s64->prim[c64], mg));
        }
        while (n < max_sweeps) {
            const int k = std::min(kBlock, max_sweeps - n);
            for (int i = 0; i < k; ++i) {
                const bool rm = pred && i == k - 1;
                PrimalArgs<float, float> a = primal_args<float, float>(st, st->cur);
                a.f_old = W.e[ec]; a.f_new = W.e[1 - ec];
                a.prim_old = a.maxw_old = s64->prim[c64];
                a.prim_new = nullptr;
                a.Fw_old = W.dF[ec]; a.Fw_new = W.dF[1 - ec];
                a.Jpart = W.Jp; a.respart = W.rp;
                a.defect = nullptr;
                a.lin_src = W.src; a.lin_f = fbar;
                a.dW_old = W.dW[ec]; a.dW_new = W.dW[1 - ec];
                a.rW = rm ? st->co_rW : nullptr;
                CK(launch_primal_lin_sweep(&a, W.maps[ec], i == k - 1, rm, s));
                ec = 1 - ec;
            }
            CK(launch_finalize(W.rp, m.ncell, nullptr, nullptr, nullptr, m.ni, W.out, s));
            ctx->launches += k + 1;
            n += k;
            double lo[2];
            if ((rc = fetch2(ctx, W.out, lo))) return rc;
            const double rin = sqrt(lo[0]);
            if (!std::isfinite(rin)) return fail(DVM_ERR_NONFINITE, "refinement correction is not finite");
            if (rin <= target) break;
            if (pred) damp.block(rin);
            if (pred && n < max_sweeps) {
                CK(launch_coarse_gmres(m, st->co_out, st->co_dinv, st->co_rW, false, o->predict_iters, st->co_kr,
                                       st->co_x, graphs_ok(ctx), s, mg ? &st->co_mg : nullptr));
                CK(launch_coarse_lin_shift(m, g, s64->prim[c64], st->co_x, damp.w, 0.3, W.e[ec], W.dW[ec], W.dF[ec], s));
                ctx->launches += krylov_launches(o->predict_iters) + 1;
                damp.after_prediction = true;
                predictions += 1;
            }
        }
        CK(launch_refine_update(fbar, W.delta, W.e[ec], nf, s));
        ctx->launches += 1;
        steps += 1;
        sweeps += n;
    }
    // the state holds fl(fbar + delta): its moments and wall density follow it
    CK(launch_moments(st->storage, st->f[st->cur], m, g, st->prim[st->cur], st->Fw[st->cur], s));
    ctx->launches += 1;
    st->version += 1;
    res->J = J64;
    const double U = st->flow.Ma * sqrt(5.0 / 3.0);
    res->Cd = U > 0.0 ? J64 / (0.5 * U * U) : J64;
    res->residual = r64;
    res->refine_steps = steps;
    res->refine_sweeps = sweeps;
    res->predictions += predictions;
    res->status = status;
    return status;
}

}  // namespace

// ------------------------------------------------------------------ velocity shards
int dvm_state_set_shard(dvm_state* st, int on) {
    if (!st || (on != 0 && on != 1)) return fail(DVM_ERR_INVALID_ARG, "bad argument");
    DeviceGuard dg(st->ctx->device);
    dvm_context* ctx = st->ctx;
    const DevMesh& m = st->mesh->d;
    const DevGrid& g = st->grid->d;
    cudaStream_t s = ctx->stream;
    if (on) {
        if (st->order != 1 || st->maxwell)
            return fail(DVM_ERR_INVALID_ARG, "velocity shards take first-order states with the plain Maxwellian");
        const size_t n = shard_count(m.ncell, m.ni);
        if (!st->part) {
            size_t acc = 0;
            int rc;
            if ((rc = dalloc(ctx, &st->part, n, &acc)) || (rc = dalloc(ctx, &st->part_total, n, &acc))) return rc;
            st->bytes += acc;
            ctx->bytes += acc;
        }
        CK(launch_shard_moments(st->storage, st->f[st->cur], m, g, st->part, s));
        CK(launch_wall_setup(m, g, st->fl, moment_of(st->flow, DVM_DRAG), st->part + 5 * (size_t)m.ncell + 2 * m.ni,
                             st->part + 5 * (size_t)m.ncell + 3 * m.ni, s, true));
        ctx->launches += 2;
    } else if (st->shard) {        // back to a whole grid of its own: its own wall constants and moments
        CK(launch_wall_setup(m, g, st->fl, moment_of(st->flow, DVM_DRAG), st->fl.wallD, st->fl.wallM, s));
        CK(launch_moments(st->storage, st->f[st->cur], m, g, st->prim[st->cur], st->Fw[st->cur], s));
        ctx->launches += 2;
        st->version += 1;
    }
    st->shard = on;
    CK(cudaStreamSynchronize(s));
    return DVM_OK;
}

size_t dvm_state_shard_count(const dvm_state* st) {
    return st ? shard_count(st->mesh->d.ncell, st->mesh->d.ni) : 0;
}

int dvm_state_shard_partials(const dvm_state* st, double* out, size_t count) {
    if (!st || !out) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    if (!st->shard) return fail(DVM_ERR_INVALID_ARG, "not a velocity shard");
    if (count != shard_count(st->mesh->d.ncell, st->mesh->d.ni)) return fail(DVM_ERR_INVALID_ARG, "wrong count");
    DeviceGuard dg(st->ctx->device);
    CK(cudaMemcpyAsync(out, st->part, count * sizeof(double), cudaMemcpyDefault, st->ctx->stream));
    CK(cudaStreamSynchronize(st->ctx->stream));
    return DVM_OK;
}

int dvm_state_shard_combine(dvm_state* st, const double* total, size_t count, double* residual_sq, double* J) {
    if (!st || !total) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    if (!st->shard) return fail(DVM_ERR_INVALID_ARG, "not a velocity shard");
    const DevMesh& m = st->mesh->d;
    if (count != shard_count(m.ncell, m.ni)) return fail(DVM_ERR_INVALID_ARG, "wrong count");
    DeviceGuard dg(st->ctx->device);
    cudaStream_t s = st->ctx->stream;
    CK(cudaMemcpyAsync(st->part_total, total, count * sizeof(double), cudaMemcpyDefault, s));
    CK(launch_shard_combine(m, st->part_total, st->prim[st->cur], st->Fw[st->cur], st->respart, st->Jpart,
                            st->fl.wallD, st->fl.wallM, s));
    CK(enqueue_primal_finalize(st, st->cur, st->out));
    st->ctx->launches += 2;
    st->version += 1;
    double r[2];
    int rc = fetch2(st->ctx, st->out, r);
    if (rc) return rc;
    if (residual_sq) *residual_sq = r[0];
    if (J) *J = r[1];
    return DVM_OK;
}

int dvm_primal_solve(dvm_context* ctx, const dvm_mesh* mesh, const dvm_vgrid* grid, const dvm_flow* flow,
                     const dvm_solve_opts* opts, int storage, dvm_state** inout, dvm_primal_result* res) {
    if (!ctx || !mesh || !grid || !flow || !opts || !inout || !res) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    Range nvtx("dvm_primal_solve");
    int rc0;
    if ((rc0 = check_solve_opts(opts))) return rc0;
    DeviceGuard dg(ctx->device);
    std::memset(res, 0, sizeof(*res));
    int rc;
    if (!*inout) {
        if ((rc = dvm_state_create(ctx, mesh, grid, flow, storage, inout))) return rc;
    } else {
        const dvm_state* s = *inout;
        if (s->mesh != mesh || s->grid != grid || s->ctx != ctx)
            return fail(DVM_ERR_INVALID_ARG, "warm-start state belongs to another mesh/grid/context");
        if (s->flow.Kn != flow->Kn || s->flow.Ma != flow->Ma || s->flow.Tw != flow->Tw || s->flow.aoa != flow->aoa)
            return fail(DVM_ERR_INVALID_ARG, "warm-start state has another flow; create a new state");
    }
    dvm_state* st = *inout;
    if (st->shard) return fail(DVM_ERR_INVALID_ARG, "a velocity shard is swept with dvm_primal_iterate and combined");
    if (opts->refine_tol > 0.0 && (st->storage != DVM_STORE_FP32 || st->order != 1 || st->maxwell))
        return fail(DVM_ERR_INVALID_ARG, "refinement needs an FP32 state of order 1 with the plain Maxwellian");
    const bool accel = opts->accel_depth > 0;
    const int K = accel ? opts->accel_period : ctx->graph_iters;
    const bool use_graph = graphs_ok(ctx) && K % 2 == 0;
    const bool wspace = accel && opts->accel_space == 1;
    const int nc = st->mesh->d.ncell;
    const bool predict = opts->predict_iters > 0;
    if (predict && (st->order != 1 || st->maxwell || st->storage == DVM_STORE_BF16))
        return fail(DVM_ERR_INVALID_ARG,
                    "the macroscopic prediction needs an FP64 or FP32 state of order 1 with the plain Maxwellian");
    if (predict && (rc = predict_ensure(st, opts->predict_iters))) return rc;
    const bool use_mg = predict && opts->predict_precond == 1;
    if (use_mg && (rc = mg_ensure(st))) return rc;
    st->predict = predict;
    const int reuse = opts->predict_reuse > 0 ? opts->predict_reuse : 4;
    const double omega = opts->predict_omega > 0.0 ? opts->predict_omega : 0.8;
    int predictions = 0;
    bool predicting = predict;
    double pred_best = INFINITY;
    int pred_high = 0;
    PredictDamping damp(omega);
    if (accel && !wspace) {
        const size_t n = (size_t)nc * st->grid->d.nvp * 2;
        if ((rc = aa_ensure(ctx, st->aa, st->storage, n, opts->accel_depth))) return rc;
        if ((rc = aa_begin(ctx, st->aa, st->f[st->cur]))) return rc;
    }
    if (wspace) {               // the cell moments as one FP64 vector
        if ((rc = aa_ensure(ctx, st->aaW, DVM_STORE_FP64, 4 * (size_t)nc, opts->accel_depth))) return rc;
        if (!st->Wbuf) {
            size_t acc = 0;
            if ((rc = dalloc(ctx, &st->Wbuf, 4 * (size_t)nc, &acc))) return rc;
            st->bytes += acc;
            ctx->bytes += acc;
        }
        CK(launch_prim_to_W(nc, st->prim[st->cur], st->Wbuf, ctx->stream));
        ctx->launches += 1;
        if ((rc = aa_begin(ctx, st->aaW, st->Wbuf))) return rc;
    }
    bool mixing = accel;
    int restarts = 0;
    int it = 0;
    double r = INFINITY, best = INFINITY, J = 0.0;
    int best_it = 0;
    int status = DVM_NOT_CONVERGED;
    while (it < opts->max_iter) {
        const int k = std::min(K, opts->max_iter - it);
        if (use_graph && k == K) {
            if ((rc = build_primal_graph(st, K))) return rc;
            CK(cudaGraphLaunch(st->graph, ctx->stream));
            ctx->launches += K + 1 + st->graph_so;
            if (st->order == 2) st->so_phase = (st->so_phase + K) % st->so_period;
            st->version += (uint64_t)K;
        } else if ((rc = run_primal_plain(st, k, nullptr))) {
            return rc;
        }
        it += k;
        double o[2];
        if ((rc = fetch2(ctx, st->out, o))) return rc;
        r = sqrt(o[0]) / st->r0;
        J = o[1];
        if (!std::isfinite(r) || !std::isfinite(J)) { status = DVM_ERR_NONFINITE; fail(status, "residual is not finite"); break; }
        if (r <= opts->tol) { status = DVM_OK; break; }
        if (r < 0.98 * best) { best = r; best_it = it; }
        if (opts->stall_window > 0 && it - best_it >= opts->stall_window) {
            if (!mixing) { status = DVM_ERR_STAGNATED; break; }
            mixing = false;                 // a stall while mixing: finish with plain sweeps, new window
            best = r;
            best_it = it;
        }
        if (predicting && st->storage != DVM_STORE_FP64) {
            // FP32 storage: near the rounding floor the residual moments are dominated by the rounding
            // of the relaxation term (V/tau times a storage ulp of f, large against transport at small Kn),
            // which the moment solve amplifies; residuals well above the best seen, two blocks in a row,
            // show it, and the solve finishes with plain sweeps under a stall window of their own
            pred_high = r > 2.0 * pred_best ? pred_high + 1 : 0;
            if (pred_high >= 2) {
                predicting = false;
                st->predict = false;
                best = r;
                best_it = it;
            }
            pred_best = std::min(pred_best, r);
        }
        if (predicting) damp.block(r);
        if (predicting && k == K && it < opts->max_iter) {
            if ((rc = predict_step(st, opts->predict_iters, damp.w, predictions % reuse == 0, use_mg))) return rc;
            damp.after_prediction = true;
            predictions += 1;
        }
        if (mixing && k == K && it < opts->max_iter && wspace) {
            // moments after the block are G(x); mix them, impose the mixed moments on f by a
            // Maxwellian shift, and restart the next block from the moments f then has
            bool mixed = false;
            CK(launch_prim_to_W(nc, st->prim[st->cur], st->Wbuf, ctx->stream));
            ctx->launches += 1;
            if (aa_restart_if_growing(st->aaW, r)) {
                if (++restarts >= 2) mixing = false;
                else if ((rc = aa_begin(ctx, st->aaW, st->Wbuf))) return rc;
            } else if ((rc = aa_step(ctx, st->aaW, st->Wbuf, false, &mixed))) {
                return rc;
            }
            if (mixed) {
                CK(launch_moment_shift(st->storage, st->f[st->cur], st->mesh->d, st->grid->d, st->prim[st->cur],
                                       st->Wbuf, ctx->stream));
                CK(launch_moments(st->storage, st->f[st->cur], st->mesh->d, st->grid->d, st->prim[st->cur],
                                  st->Fw[st->cur], ctx->stream));
                CK(launch_prim_to_W(nc, st->prim[st->cur], st->Wbuf, ctx->stream));
                CK(launch_aa_load(DVM_STORE_FP64, 4 * (size_t)nc, st->Wbuf, st->aaW->X, ctx->stream));
                ctx->launches += 4;
                if (st->maxwell) {
                    CK(launch_maxwell_fit(st->storage, st->mesh->d, st->grid->d, st->prim[st->cur], st->fit, true, 3,
                                          nullptr, ctx->stream));
                    ctx->launches += 1;
                }
                st->so_phase = 0;
                st->version += 1;
            }
        } else if (mixing && k == K && it < opts->max_iter) {
            bool mixed = false;
            if (aa_restart_if_growing(st->aa, r)) {   // the history misleads: start it again here,
                if (++restarts >= 2) mixing = false;    // and on the second time finish with plain sweeps
                else if ((rc = aa_begin(ctx, st->aa, st->f[st->cur]))) return rc;
            } else if ((rc = aa_step(ctx, st->aa, st->f[st->cur], true, &mixed))) {
                return rc;
            }
            if (mixed) {
                st->so_phase = 0;
                CK(launch_moments(st->storage, st->f[st->cur], st->mesh->d, st->grid->d, st->prim[st->cur],
                                  st->Fw[st->cur], ctx->stream));
                if (st->maxwell) {
                    CK(launch_maxwell_fit(st->storage, st->mesh->d, st->grid->d, st->prim[st->cur], st->fit, true, 3,
                                          nullptr, ctx->stream));
                    ctx->launches += 1;
                }
                ctx->launches += 1;
                st->version += 1;
            }
        }
    }
    if (opts->max_iter == 0) {
        if ((rc = dvm_state_functional(st, DVM_DRAG, &J))) return rc;
        r = NAN;
    }
    res->J = J;
    const double U = flow->Ma * sqrt(5.0 / 3.0);
    res->Cd = U > 0.0 ? J / (0.5 * U * U) : J;
    res->residual = r;
    res->residual_fp32 = r;
    res->r0 = st->r0;
    res->iters = it;
    res->status = status;
    res->predictions = predictions;
    st->predict = false;
    if (opts->refine_tol > 0.0 && status != DVM_ERR_NONFINITE) return refine_primal(st, opts, res);
    return status;
}

// ------------------------------------------------------------------------------------- adjoint
void dvm_adjoint_destroy(dvm_adjoint* ad) {
    if (!ad || !live_take(ad, kAdjoint)) return;
    DeviceGuard dg(ad->st->ctx->device);
    cudaStreamSynchronize(ad->st->ctx->stream);
    if (ad->graph) cudaGraphExecDestroy(ad->graph);
    for (int b = 0; b < 2; ++b) { dfree(ad->phi[b]); dfree(ad->Z[b]); dfree(ad->Lam[b]); }
    dfree(ad->respart); dfree(ad->out); dfree(ad->wallM); dfree(ad->cell);
    dfree(ad->GN); dfree(ad->GE); dfree(ad->GW); dfree(ad->node_grad); dfree(ad->vol); dfree(ad->elem);
    dfree(ad->dwall); dfree(ad->sj); dfree(ad->grad); dfree(ad->so_def); dfree(ad->Kinv); dfree(ad->so_corner);
    aa_free(ad->st->ctx, ad->aa);
    ad->st->ctx->bytes -= ad->bytes;
    delete ad;
}

static int adjoint_reset(dvm_adjoint* ad) {
    const DevMesh& m = ad->st->mesh->d;
    const DevGrid& g = ad->st->grid->d;
    cudaStream_t s = ad->st->ctx->stream;
    ad->cur = 0;
    ad->so_phase = 0;
    CK(cudaMemsetAsync(ad->phi[0], 0, (size_t)m.ncell * g.nvp * storage_bytes(ad->st->storage), s));
    CK(cudaMemsetAsync(ad->Z[0], 0, m.ncell * sizeof(double4), s));
    CK(cudaMemsetAsync(ad->Lam[0], 0, m.ni * sizeof(double), s));
    return DVM_OK;
}

int dvm_adjoint_create(dvm_state* st, int functional, dvm_adjoint** out) {
    if (!st || !out) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    if (st->shard) return fail(DVM_ERR_INVALID_ARG, "adjoints of velocity shards are not provided");
    if (functional < DVM_DRAG || functional > DVM_HEAT) return fail(DVM_ERR_INVALID_ARG, "unknown functional");
    *out = nullptr;
    dvm_context* ctx = st->ctx;
    DeviceGuard dg(ctx->device);
    const DevMesh& m = st->mesh->d;
    const DevGrid& g = st->grid->d;
    const size_t need = (size_t)m.ncell * g.nvp * storage_bytes(st->storage) * 2 + (size_t)m.ncell * 72;
    if (ctx->budget && ctx->bytes + need > ctx->budget)
        return fail(DVM_ERR_ADMISSION, "adjoint does not fit the context's HBM budget");
    dvm_adjoint* ad = new (std::nothrow) dvm_adjoint();
    if (!ad) return fail(DVM_ERR_OOM, "host allocation");
    ad->st = st;
    ad->functional = functional;
    live_add(ad, kAdjoint, st->ctx, st);
    ad->mj = moment_of(st->flow, functional);
    size_t acc = 0;
    int rc = DVM_OK;
    for (int b = 0; b < 2 && !rc; ++b) {
        rc = dalloc(ctx, (unsigned char**)&ad->phi[b], (size_t)m.ncell * g.nvp * storage_bytes(st->storage), &acc);
        if (!rc) rc = dalloc(ctx, &ad->Z[b], m.ncell, &acc);
        if (!rc) rc = dalloc(ctx, &ad->Lam[b], m.ni, &acc);
    }
    if (!rc) rc = dalloc(ctx, &ad->respart, m.ncell, &acc);
    if (!rc) rc = dalloc(ctx, &ad->out, 2, &acc);
    if (!rc) rc = dalloc(ctx, &ad->wallM, m.ni, &acc);
    if (!rc) rc = dalloc(ctx, (unsigned char**)&ad->cell,
                         (size_t)m.ncell * 16 * (st->storage == DVM_STORE_FP64 ? sizeof(double) : sizeof(float)), &acc);
    if (rc) { dvm_adjoint_destroy(ad); return rc; }
    ad->bytes = acc;
    ctx->bytes += acc;
    {
        const int nq = g.nvp * (int)storage_bytes(st->storage) / 16;
        for (int b = 0; b < 2; ++b) {
            cudaError_t me = make_tmamaps(ad->phi[b], m.ni, m.nj, nq, &ad->maps[b]);
            if (me != cudaSuccess) { dvm_adjoint_destroy(ad); return fail_cuda(me, "tensor map of phi"); }
        }
    }
    // M_l of this functional's direction (the normaliser D_l is the state's; recomputed into scratch)
    double* dtmp = nullptr;
    if ((rc = dalloc(ctx, &dtmp, m.ni))) { dvm_adjoint_destroy(ad); return rc; }
    cudaError_t e = launch_wall_setup(m, g, st->fl, ad->mj, dtmp, ad->wallM, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx->launches += 1;
    dfree(dtmp);
    if (e != cudaSuccess) { dvm_adjoint_destroy(ad); return fail_cuda(e, "adjoint setup"); }
    if ((rc = adjoint_reset(ad))) { dvm_adjoint_destroy(ad); return rc; }
    if ((rc = adjoint_so_ensure(ad))) { dvm_adjoint_destroy(ad); return rc; }
    if ((e = adjoint_relinearise(ad)) != cudaSuccess) { dvm_adjoint_destroy(ad); return fail_cuda(e, "adjoint constants"); }
    // r0: adjoint residual at phi = 0 from one discarded sweep
    e = enqueue_adjoint(ad, 0);
    if (e == cudaSuccess) e = enqueue_adjoint_finalize(ad, ad->out);
    ctx->launches += 2;
    if (e != cudaSuccess) { dvm_adjoint_destroy(ad); return fail_cuda(e, "adjoint r0"); }
    double r[2];
    if ((rc = fetch2(ctx, ad->out, r))) { dvm_adjoint_destroy(ad); return rc; }
    ad->so_phase = 0;          // the r0 sweep is discarded
    ad->r0 = sqrt(r[0]);
    if (!std::isfinite(ad->r0)) { dvm_adjoint_destroy(ad); return fail(DVM_ERR_NONFINITE, "adjoint source not finite"); }
    if (ad->r0 == 0.0) ad->r0 = 1.0;
    *out = ad;
    return DVM_OK;
}

int dvm_adjoint_set(dvm_adjoint* ad, const double* phi_host) {
    if (!ad || !phi_host) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(ad->st->ctx->device);
    const DevMesh& m = ad->st->mesh->d;
    const DevGrid& g = ad->st->grid->d;
    cudaStream_t s = ad->st->ctx->stream;
    double* tmp = nullptr;
    const size_t n = (size_t)m.ncell * g.nv * 2;
    int rc = dalloc(ad->st->ctx, &tmp, n);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(tmp, phi_host, n * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_convert(ad->st->storage, 1, tmp, ad->phi[ad->cur], m.ncell, g.nv, g.nvp, s);
    if (e == cudaSuccess) e = refresh_adjoint_couplings(ad);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(tmp);
    if (e != cudaSuccess) return fail_cuda(e, "adjoint upload");
    return DVM_OK;
}

int dvm_adjoint_get(const dvm_adjoint* ad, double* phi_host) {
    if (!ad || !phi_host) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(ad->st->ctx->device);
    const DevMesh& m = ad->st->mesh->d;
    const DevGrid& g = ad->st->grid->d;
    cudaStream_t s = ad->st->ctx->stream;
    double* tmp = nullptr;
    const size_t n = (size_t)m.ncell * g.nv * 2;
    int rc = dalloc(ad->st->ctx, &tmp, n);
    if (rc) return rc;
    cudaError_t e = launch_convert(ad->st->storage, 0, ad->phi[ad->cur], tmp, m.ncell, g.nv, g.nvp, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(phi_host, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(tmp);
    if (e != cudaSuccess) return fail_cuda(e, "adjoint download");
    return DVM_OK;
}

int dvm_adjoint_copy_from(dvm_adjoint* dst, const dvm_adjoint* src) {
    if (!dst || !src) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    if (dst == src) return DVM_OK;
    int rc = same_layout(dst->st, src->st);
    if (rc) return rc;
    DeviceGuard dg(dst->st->ctx->device);
    const DevMesh& m = dst->st->mesh->d;
    const DevGrid& g = dst->st->grid->d;
    cudaStream_t s = dst->st->ctx->stream;
    const size_t bytes = (size_t)m.ncell * g.nvp * storage_bytes(dst->st->storage);
    cudaError_t e = cudaMemcpyAsync(dst->phi[dst->cur], src->phi[src->cur], bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = refresh_adjoint_couplings(dst);
    if (e != cudaSuccess) return fail_cuda(e, "adjoint copy");
    return DVM_OK;
}

static int adjoint_follow_state(dvm_adjoint* ad) {
    if (ad->st_version == ad->st->version) return DVM_OK;
    CK(adjoint_relinearise(ad));
    CK(refresh_adjoint_couplings(ad));
    return DVM_OK;
}

int dvm_adjoint_iterate(dvm_adjoint* ad, int n, double* residual_out) {
    if (!ad || n < 0) return fail(DVM_ERR_INVALID_ARG, "bad argument");
    if (n == 0) return DVM_OK;
    DeviceGuard dg(ad->st->ctx->device);
    int rc0 = adjoint_so_ensure(ad);            // buffers first: a new Jacobian buffer forces relinearisation
    if (!rc0) rc0 = adjoint_follow_state(ad);
    if (rc0) return rc0;
    double* hist = nullptr;
    int rc = dalloc(ad->st->ctx, &hist, 2 * (size_t)n);
    if (rc) return rc;
    rc = run_adjoint_plain(ad, n, hist);
    if (!rc) {
        std::vector<double> h(2 * (size_t)n);
        cudaError_t e = cudaMemcpyAsync(h.data(), hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ad->st->ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ad->st->ctx->stream);
        if (e != cudaSuccess) rc = fail_cuda(e, "residual history");
        if (!rc) rc = check_device_flag(ad->st->ctx);
        for (int i = 0; i < n && !rc; ++i) {
            const double r = sqrt(h[2 * i]) / ad->r0;
            if (residual_out) residual_out[i] = r;
            if (!std::isfinite(r)) rc = fail(DVM_ERR_NONFINITE, "adjoint residual is not finite");
        }
    }
    dfree(hist);
    return rc;
}

int dvm_adjoint_solve(dvm_context* ctx, dvm_state* st, int functional, const dvm_solve_opts* opts,
                      dvm_adjoint** inout, dvm_adjoint_result* res) {
    if (!ctx || !st || !opts || !inout || !res) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    if (st->ctx != ctx) return fail(DVM_ERR_INVALID_ARG, "state from another context");
    if (int rc0 = check_solve_opts(opts)) return rc0;
    Range nvtx("dvm_adjoint_solve");
    DeviceGuard dg(ctx->device);
    std::memset(res, 0, sizeof(*res));
    int rc;
    if (!*inout) {
        if ((rc = dvm_adjoint_create(st, functional, inout))) return rc;
    } else if ((*inout)->st != st || (*inout)->functional != functional) {
        return fail(DVM_ERR_INVALID_ARG, "warm-start adjoint belongs to another state/functional");
    }
    dvm_adjoint* ad = *inout;
    const bool predict = opts->predict_iters > 0;
    if (predict && (st->order != 1 || st->maxwell || st->storage == DVM_STORE_BF16))
        return fail(DVM_ERR_INVALID_ARG,
                    "the macroscopic prediction needs an FP64 or FP32 state of order 1 with the plain Maxwellian");
    if ((rc = adjoint_so_ensure(ad))) return rc;
    if ((rc = adjoint_follow_state(ad))) return rc;
    const bool accel = opts->accel_depth > 0;
    const int K = accel ? opts->accel_period : ctx->graph_iters;
    const bool use_graph = graphs_ok(ctx) && K % 2 == 0;
    const double omega = opts->predict_omega > 0.0 ? opts->predict_omega : 0.8;
    if (predict) {              // the moment system at the (fixed) primal state
        if ((rc = predict_ensure(st, opts->predict_iters))) return rc;
        if (opts->predict_precond == 1 && (rc = mg_ensure(st))) return rc;
        CK(assemble_coarse(st, st->prim[st->cur], opts->predict_precond == 1));
    }
    bool predicting = predict;
    double pred_best = INFINITY;
    int pred_high = 0;
    int predictions = 0;
    PredictDamping damp(omega);
    if (accel) {
        const size_t n = (size_t)st->mesh->d.ncell * st->grid->d.nvp * 2;
        if ((rc = aa_ensure(ctx, ad->aa, st->storage, n, opts->accel_depth))) return rc;
        if ((rc = aa_begin(ctx, ad->aa, ad->phi[ad->cur]))) return rc;
    }
    bool mixing = accel;
    int restarts = 0;
    int it = 0, best_it = 0;
    double r = INFINITY, best = INFINITY;
    int status = DVM_NOT_CONVERGED;
    while (it < opts->max_iter) {
        const int k = std::min(K, opts->max_iter - it);
        if (use_graph && k == K) {
            if ((rc = build_adjoint_graph(ad, K))) return rc;
            CK(cudaGraphLaunch(ad->graph, ctx->stream));
            ctx->launches += K + 1 + ad->graph_so;
            if (st->order == 2) ad->so_phase = (ad->so_phase + K) % st->so_period;
        } else if ((rc = run_adjoint_plain(ad, k, nullptr))) {
            return rc;
        }
        it += k;
        double o[2];
        if ((rc = fetch2(ctx, ad->out, o))) return rc;
        r = sqrt(o[0]) / ad->r0;
        if (!std::isfinite(r)) { status = DVM_ERR_NONFINITE; fail(status, "adjoint residual is not finite"); break; }
        if (r <= opts->tol) { status = DVM_OK; break; }
        if (r < 0.98 * best) { best = r; best_it = it; }
        if (opts->stall_window > 0 && it - best_it >= opts->stall_window) {
            if (!mixing) { status = DVM_ERR_STAGNATED; break; }
            mixing = false;                 // a stall while mixing: finish with plain sweeps, new window
            best = r;
            best_it = it;
        }
        if (mixing && k == K && it < opts->max_iter) {
            bool mixed = false;
            if (aa_restart_if_growing(ad->aa, r)) {
                if (++restarts >= 2) mixing = false;
                else if ((rc = aa_begin(ctx, ad->aa, ad->phi[ad->cur]))) return rc;
            } else if ((rc = aa_step(ctx, ad->aa, ad->phi[ad->cur], false, &mixed))) {
                return rc;
            }
            if (mixed) CK(refresh_adjoint_couplings(ad));
        }
        if (predicting && st->storage != DVM_STORE_FP64) {     // FP32 noise floor: as in the primal solve
            pred_high = r > 2.0 * pred_best ? pred_high + 1 : 0;
            if (pred_high >= 2) {
                predicting = false;
                best = r;
                best_it = it;
            }
            pred_best = std::min(pred_best, r);
        }
        if (predicting) damp.block(r);
        if (predicting && k == K && it < opts->max_iter) {
            // after a block the last sweep read phi[1 - cur] and wrote phi[cur]
            const DevMesh& m = st->mesh->d;
            cudaStream_t s = ctx->stream;
            const int n = opts->predict_iters;
            CK(launch_adjoint_restrict(st->storage, m, st->grid->d, st->prim[st->cur], 1.0 / st->fl.tau_inf,
                                       ad->phi[1 - ad->cur], ad->phi[ad->cur], st->co_rW, s));
            CK(launch_coarse_gmres(m, st->co_out, st->co_dinv, st->co_rW, true, n, st->co_kr, st->co_x, graphs_ok(ctx), s,
                                   opts->predict_precond == 1 ? &st->co_mg : nullptr));
            CK(launch_adjoint_shift(st->storage, m, st->grid->d, st->co_x, damp.w, ad->phi[ad->cur], s));
            CK(refresh_adjoint_couplings(ad));
            ctx->launches += krylov_launches(n) + 2;
            damp.after_prediction = true;
            predictions += 1;
        }
    }
    res->residual = r;
    res->r0 = ad->r0;
    res->iters = it;
    res->status = status;
    res->predictions = predictions;
    return status;
}

// ------------------------------------------------------------------------------------- sensitivity
int dvm_sensitivity(dvm_context* ctx, const dvm_state* st, const dvm_adjoint* cad, int P, const double* dwall,
                    const double* s_j, int mode, double* grad_out, double* node_grad_out) {
    if (!ctx || !st || !cad || (P > 0 && (!dwall || !grad_out))) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    if (mode != DVM_SENS_PAPER && mode != DVM_SENS_FULL) return fail(DVM_ERR_INVALID_ARG, "unknown mode");
    if (mode == DVM_SENS_FULL && !s_j) return fail(DVM_ERR_INVALID_ARG, "full mode needs s_j");
    if (cad->st != st || st->ctx != ctx) return fail(DVM_ERR_INVALID_ARG, "adjoint/state/context mismatch");
    if (P < 0) return fail(DVM_ERR_INVALID_ARG, "n_params < 0");
    DeviceGuard dg(ctx->device);
    Range nvtx("dvm_sensitivity");
    dvm_adjoint* ad = const_cast<dvm_adjoint*>(cad);
    const DevMesh& m = st->mesh->d;
    const DevGrid& g = st->grid->d;
    cudaStream_t s = ctx->stream;
    int rc = DVM_OK;
    const int nnodes = (m.nj + 1) * m.ni;
    if (!ad->GN) {
        size_t acc = 0;
        if ((rc = dalloc(ctx, &ad->GN, m.ncell, &acc)) || (rc = dalloc(ctx, &ad->GE, m.ncell, &acc)) ||
            (rc = dalloc(ctx, &ad->GW, m.ni, &acc)) || (rc = dalloc(ctx, &ad->node_grad, nnodes, &acc)) ||
            (rc = dalloc(ctx, &ad->vol, m.ncell, &acc)) || (rc = dalloc(ctx, &ad->elem, 5 * (size_t)m.ni, &acc)) ||
            (rc = dalloc(ctx, &ad->sj, m.nj + 1, &acc)))
            return rc;
        ad->bytes += acc;
        ctx->bytes += acc;
    }
    if (P > ad->sens_P) {
        dfree(ad->dwall); dfree(ad->grad);
        ad->dwall = nullptr; ad->grad = nullptr;
        if ((rc = dalloc(ctx, &ad->dwall, (size_t)P * m.ni * 2)) || (rc = dalloc(ctx, &ad->grad, P))) return rc;
        ad->sens_P = P;
    }
    if (P > 0) CK(cudaMemcpyAsync(ad->dwall, dwall, (size_t)P * m.ni * 2 * sizeof(double), cudaMemcpyHostToDevice, s));
    const void* f = st->f[st->cur];
    const void* phi = ad->phi[ad->cur];
    if (mode == DVM_SENS_PAPER) {
        CK(launch_sens_paper(st->storage, m, g, st->fl, f, phi, st->Fw[st->cur], ad->mj, ad->elem,
                             (double*)ad->node_grad, s));
        CK(launch_contract(ad->node_grad, 1, m.ni, nullptr, ad->dwall, P, ad->grad, s));
        ctx->launches += 2 + (P > 0);
        if (node_grad_out)
            CK(cudaMemcpyAsync(node_grad_out, ad->node_grad, (size_t)m.ni * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    } else {
        CK(cudaMemcpyAsync(ad->sj, s_j, (m.nj + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(launch_sens_full(st->storage, m, g, st->fl, f, phi, st->prim[st->cur],
                            st->maxwell ? st->fit : st->prim[st->cur], st->Fw[st->cur], ad->mj,
                            ad->GN, ad->GE, ad->GW, ad->vol, ad->node_grad, s));
        if (st->order == 2) {          // + d(sum w phi . dR)/dx of the reconstruction
            if (!ad->so_corner) {
                size_t acc = 0;
                if ((rc = dalloc(ctx, &ad->so_corner, 4 * (size_t)m.ncell, &acc))) return rc;
                ad->bytes += acc;
                ctx->bytes += acc;
            }
            switch (st->storage) {
                case DVM_STORE_FP64: { auto a = so_args<double, double>(st, f, st->Fw[st->cur], nullptr);
                                       CK(launch_so_sens(0, &a, phi, ad->so_corner, m.ni, m.nj, ad->node_grad, s)); break; }
                case DVM_STORE_FP32: { auto a = so_args<float, float>(st, f, st->Fw[st->cur], nullptr);
                                       CK(launch_so_sens(1, &a, phi, ad->so_corner, m.ni, m.nj, ad->node_grad, s)); break; }
                default: { auto a = so_args<__nv_bfloat16, float>(st, f, st->Fw[st->cur], nullptr);
                           CK(launch_so_sens(2, &a, phi, ad->so_corner, m.ni, m.nj, ad->node_grad, s)); break; }
            }
            ctx->launches += 2;
        }
        CK(launch_contract(ad->node_grad, m.nj + 1, m.ni, ad->sj, ad->dwall, P, ad->grad, s));
        ctx->launches += 2 + (P > 0);
        if (node_grad_out)
            CK(cudaMemcpyAsync(node_grad_out, ad->node_grad, (size_t)nnodes * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    if (P > 0) CK(cudaMemcpyAsync(grad_out, ad->grad, P * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return DVM_OK;
}

}  // extern "C"

extern "C" int dvm_volume_constraint(dvm_context* ctx, const dvm_mesh* mesh, double v_min, int P,
                                     const double* dwall, double* Q, double* dQ_dalpha) {
    if (!ctx || !mesh || !Q || (P > 0 && (!dwall || !dQ_dalpha)) || P < 0) return fail(DVM_ERR_INVALID_ARG, "bad argument");
    DeviceGuard dg(ctx->device);
    double* d = nullptr;
    const size_t nw = (size_t)P * mesh->d.ni * 2;
    int rc = dalloc(ctx, &d, nw + 1 + P);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (P > 0) e = cudaMemcpyAsync(d, dwall, nw * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = launch_volume(mesh->d, v_min, d, P, d + nw, ctx->stream);
    std::vector<double> h(1 + P);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d + nw, (1 + P) * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx->launches += 1;
    dfree(d);
    if (e != cudaSuccess) return fail_cuda(e, "volume constraint");
    *Q = h[0];
    for (int p = 0; p < P; ++p) dQ_dalpha[p] = h[1 + p];
    return DVM_OK;
}

// ======================================================================= no-allocation variant
// dvm_sensitivity_noalloc keeps every intermediate of the sensitivity reduction in the static
// device array below instead of device memory from cudaMalloc.  It exists for callers that must not
// allocate device memory during the call (for example a serving loop whose device memory is carved
// out once, up front, by another allocator, or a host thread that must not stall on cudaMalloc's
// implicit device synchronisation).  The array costs kNoAllocScratchBytes on every GPU that loads
// this library, for the life of the process.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on `device`, looked up once per device with that device
// current (the host-side symbol is only a stand-in and must never be handed to a kernel).
int noalloc_scratch(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return fail(DVM_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[device]) {
        DeviceGuard dg(device);
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return fail_cuda(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
        g_noalloc_addr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_addr[device]);
    return DVM_OK;
}

struct ScratchCarver {
    unsigned char* base;
    size_t used = 0;
    template <class T>
    T* take(size_t count) {
        used = (used + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base ? base + used : nullptr);
        used += count * sizeof(T);
        return p;
    }
};

}  // namespace

extern "C" int dvm_sensitivity_noalloc(dvm_context* ctx, const dvm_state* st, const dvm_adjoint* ad, int P,
                                       const double* dwall, const double* s_j, int mode, double* grad_out,
                                       double* node_grad_out) {
    if (!ctx || !st || !ad || (P > 0 && (!dwall || !grad_out))) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    if (mode != DVM_SENS_PAPER && mode != DVM_SENS_FULL) return fail(DVM_ERR_INVALID_ARG, "unknown mode");
    if (mode == DVM_SENS_FULL && !s_j) return fail(DVM_ERR_INVALID_ARG, "full mode needs s_j");
    if (ad->st != st || st->ctx != ctx) return fail(DVM_ERR_INVALID_ARG, "adjoint/state/context mismatch");
    if (P < 0) return fail(DVM_ERR_INVALID_ARG, "n_params < 0");
    if (mode == DVM_SENS_FULL && st->order != 1)
        return fail(DVM_ERR_INVALID_ARG, "the scratch-free full gradient is first-order only; use dvm_sensitivity");
    const DevMesh& m = st->mesh->d;
    const DevGrid& g = st->grid->d;
    const int nnodes = (m.nj + 1) * m.ni;
    // layout first (base = nullptr), so an oversized request is rejected before any device work
    ScratchCarver probe{nullptr};
    probe.take<double2>(m.ncell); probe.take<double2>(m.ncell); probe.take<double2>(m.ni);
    probe.take<double2>(nnodes); probe.take<double>(m.ncell); probe.take<double>(5 * (size_t)m.ni);
    probe.take<double>((size_t)P * m.ni * 2); probe.take<double>(m.nj + 1); probe.take<double>(P > 0 ? P : 1);
    if (probe.used > kNoAllocScratchBytes) {
        char msg[160];
        snprintf(msg, sizeof msg, "dvm_sensitivity_noalloc needs %zu bytes of scratch; the static limit is %zu",
                 probe.used, kNoAllocScratchBytes);
        return fail(DVM_ERR_INVALID_ARG, msg);
    }
    DeviceGuard dg(ctx->device);
    unsigned char* base = nullptr;
    int rc = noalloc_scratch(ctx->device, &base);
    if (rc) return rc;
    ScratchCarver sc{base};
    double2* GN = sc.take<double2>(m.ncell);
    double2* GE = sc.take<double2>(m.ncell);
    double2* GW = sc.take<double2>(m.ni);
    double2* node_grad = sc.take<double2>(nnodes);
    double* vol = sc.take<double>(m.ncell);
    double* elem = sc.take<double>(5 * (size_t)m.ni);
    double* dw = sc.take<double>((size_t)P * m.ni * 2);
    double* sj = sc.take<double>(m.nj + 1);
    double* grad = sc.take<double>(P > 0 ? P : 1);
    // every scratch entry read below is written earlier in the same call: nothing needs clearing
    cudaStream_t s = ctx->stream;
    if (P > 0) CK(cudaMemcpyAsync(dw, dwall, (size_t)P * m.ni * 2 * sizeof(double), cudaMemcpyHostToDevice, s));
    const void* f = st->f[st->cur];
    const void* phi = ad->phi[ad->cur];
    if (mode == DVM_SENS_PAPER) {
        CK(launch_sens_paper(st->storage, m, g, st->fl, f, phi, st->Fw[st->cur], ad->mj, elem,
                             (double*)node_grad, s));
        CK(launch_contract(node_grad, 1, m.ni, nullptr, dw, P, grad, s));
        if (node_grad_out)
            CK(cudaMemcpyAsync(node_grad_out, node_grad, (size_t)m.ni * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    } else {
        CK(cudaMemcpyAsync(sj, s_j, (m.nj + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(launch_sens_full(st->storage, m, g, st->fl, f, phi, st->prim[st->cur],
                            st->maxwell ? st->fit : st->prim[st->cur], st->Fw[st->cur], ad->mj,
                            GN, GE, GW, vol, node_grad, s));
        CK(launch_contract(node_grad, m.nj + 1, m.ni, sj, dw, P, grad, s));
        if (node_grad_out)
            CK(cudaMemcpyAsync(node_grad_out, node_grad, (size_t)nnodes * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    ctx->launches += 2 + (P > 0);
    if (P > 0) CK(cudaMemcpyAsync(grad_out, grad, P * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return DVM_OK;
}

// ======================================================================= served batch (continuous batching)
namespace {

struct BatchReq {
    uint64_t ticket = 0;
    dvm_request r{};
    std::vector<double> nodes, vx, vy, w, dwall, sj;
    int phase = 0;              // 0 queued, 1 primal, 2 adjoint, 3 retired
    int status = DVM_OK;
    int pstatus = DVM_OK, astatus = DVM_OK;
    dvm_mesh* mesh = nullptr;
    dvm_vgrid* grid = nullptr;
    dvm_state* st = nullptr;
    dvm_adjoint* ad = nullptr;
    int pit = 0, ait = 0;
    double res = NAN, ares = NAN, J = 0.0;
    double best = INFINITY;     // best residual of the current phase, and the sweep it was reached at
    int best_it = 0;
    int warm = 0;
    std::vector<double> grad;
    size_t footprint = 0;
    // macroscopic prediction of the current phase (dvm_request.predict_iters)
    bool predicting = false;
    int predictions = 0, phase_predictions = 0, pred_high = 0;
    double pred_best = INFINITY;
    PredictDamping damp{0.8};
};

struct WarmEntry {
    uint64_t key = 0, stamp = 0;
    int ni = 0, nj = 0, nv = 0, storage = 0;
    dvm_mesh* mesh = nullptr;
    dvm_vgrid* grid = nullptr;
    dvm_state* st = nullptr;
    dvm_adjoint* ad = nullptr;
    size_t footprint = 0;
};

size_t request_footprint(const dvm_request& r) {
    const size_t nc = (size_t)r.ni * r.nj, nvp = (size_t)(r.nv + kPad - 1) / kPad * kPad;
    const size_t pair = storage_bytes(r.storage), tc = r.storage == DVM_STORE_FP64 ? 8 : 4;
    size_t b = 2 * nc * nvp * pair + nc * 72 + (size_t)r.ni * 48 + nvp * 48;          // state
    b += nc * (4 * 16 + 4 * 8 + 16 + 8 + 4) + (size_t)(r.nj + 1) * r.ni * 16 + nvp * 48;  // mesh + grid
    if (r.n_params > 0)
        b += 2 * nc * nvp * pair + nc * (72 + 16 * tc) + nc * 40 + (size_t)(r.nj + 1) * r.ni * 16 +
             (size_t)r.n_params * r.ni * 16;                                              // adjoint + sensitivity
    if (r.predict_iters > 0)                                                              // the prediction's buffers
        b += nc * 8 * (64 + 16 + 4 + 4 + 4) + nc * 32 * (size_t)(r.predict_iters + 2) +
             8 * ((size_t)(r.predict_iters + 1) * 256 + (size_t)r.predict_iters * (r.predict_iters + 2) + 8);
    return b;
}

}  // namespace

struct dvm_batch {
    dvm_context* ctx = nullptr;
    dvm_batch_options opt{};
    uint64_t next = 1, stamp = 0;
    size_t used = 0;
    std::deque<BatchReq*> queue;
    std::vector<BatchReq*> active;
    std::unordered_map<uint64_t, BatchReq*> all;
    std::vector<WarmEntry> cache;
    // Device tables of the admitted set, in six segments k = 2 storage + (0 primal, 1 adjoint): work
    // items and descriptors per segment, a finalize descriptor and two results per request, and the
    // counts in use.  Capacities only grow, so the launches of a tick (grids of the capacities, counts
    // read from the device) keep their shape, and one captured graph serves every tick until a table
    // outgrows its capacity.
    int cap_items[6] = {0, 0, 0, 0, 0, 0};
    int cap_desc[6] = {0, 0, 0, 0, 0, 0};
    int cap_act = 0;
    size_t item_off[6] = {0, 0, 0, 0, 0, 0};
    int4* items = nullptr;
    void* desc[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    FinalizeDesc* fdesc = nullptr;
    double* dout = nullptr;
    int* counts = nullptr;           // [8]: items in use per segment, then the requests in use
    double* hout = nullptr;          // pinned [2 cap_act]: the results the tick reads back
    unsigned char* host = nullptr;   // pinned staging of the tables
    size_t host_cap = 0;
    std::vector<uint64_t> sig;       // (ticket, phase) of the admitted set whose tables are on the device
    cudaGraphExec_t graph = nullptr;
    int graph_M = 0;
    bool graph_stale = true;
    dvm_batch_stats stats{};
};

namespace {

// Replace a device table by one of `bytes` (its contents are rewritten before the next use).
template <class T>
int realloc_device(T** p, size_t bytes) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(bytes, 64));
    if (e != cudaSuccess) return fail_cuda(e, "batch table");
    return DVM_OK;
}

int grow_host(dvm_batch* b, size_t bytes) {
    if (bytes <= b->host_cap) return DVM_OK;
    if (b->host) cudaFreeHost(b->host);
    b->host = nullptr;
    size_t nb = std::max(bytes, b->host_cap * 2);
    CK(cudaMallocHost((void**)&b->host, nb));
    b->host_cap = nb;
    return DVM_OK;
}

void destroy_objects(dvm_adjoint*& ad, dvm_state*& st, dvm_vgrid*& g, dvm_mesh*& m) {
    dvm_adjoint_destroy(ad); ad = nullptr;
    dvm_state_destroy(st); st = nullptr;
    dvm_vgrid_destroy(g); g = nullptr;
    dvm_mesh_destroy(m); m = nullptr;
}

bool evict_one(dvm_batch* b) {
    if (b->cache.empty()) return false;
    size_t lru = 0;
    for (size_t i = 1; i < b->cache.size(); ++i)
        if (b->cache[i].stamp < b->cache[lru].stamp) lru = i;
    WarmEntry& e = b->cache[lru];
    destroy_objects(e.ad, e.st, e.grid, e.mesh);
    b->used -= e.footprint;
    b->cache.erase(b->cache.begin() + lru);
    return true;
}

WarmEntry* find_warm(dvm_batch* b, const dvm_request& r) {
    if (!r.warm_key) return nullptr;
    for (auto& e : b->cache)
        if (e.key == r.warm_key && e.ni == r.ni && e.nj == r.nj && e.nv == r.nv && e.storage == r.storage) return &e;
    return nullptr;
}

int admit(dvm_batch* b, BatchReq* q) {
    dvm_context* ctx = b->ctx;
    const dvm_request& r = q->r;
    int rc;
    if ((rc = dvm_mesh_create(ctx, r.ni, r.nj, q->nodes.data(), &q->mesh))) return rc;
    if ((rc = dvm_vgrid_create(ctx, r.nv, q->vx.data(), q->vy.data(), q->w.data(), &q->grid))) return rc;
    if ((rc = dvm_state_create(ctx, q->mesh, q->grid, &r.flow, r.storage, &q->st))) return rc;
    if (WarmEntry* e = find_warm(b, r)) {
        dvm_state* st = q->st;
        const size_t bytes = (size_t)st->mesh->d.ncell * st->grid->d.nvp * storage_bytes(st->storage);
        CK(cudaMemcpyAsync(st->f[st->cur], e->st->f[e->st->cur], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(launch_moments(st->storage, st->f[st->cur], st->mesh->d, st->grid->d, st->prim[st->cur], st->Fw[st->cur],
                          ctx->stream));
        ctx->launches += 1;
        st->version += 1;
        q->warm = 1;
        e->stamp = ++b->stamp;
    }
    if (r.predict_iters > 0) {
        if ((rc = predict_ensure(q->st, r.predict_iters))) return rc;
        q->predicting = true;
        q->damp = PredictDamping(r.predict_omega > 0.0 ? r.predict_omega : 0.8);
    }
    q->phase = 1;
    return DVM_OK;
}

void retire(dvm_batch* b, BatchReq* q) {
    q->status = q->pstatus != DVM_OK ? q->pstatus : q->astatus;
    q->phase = 3;
    if (q->r.warm_key && q->status != DVM_ERR_NONFINITE) {
        if (WarmEntry* e = find_warm(b, q->r)) {
            destroy_objects(e->ad, e->st, e->grid, e->mesh);
            b->used -= e->footprint;
            b->cache.erase(b->cache.begin() + (e - b->cache.data()));
        }
        WarmEntry e;
        e.key = q->r.warm_key; e.stamp = ++b->stamp;
        e.ni = q->r.ni; e.nj = q->r.nj; e.nv = q->r.nv; e.storage = q->r.storage;
        e.mesh = q->mesh; e.grid = q->grid; e.st = q->st; e.ad = q->ad;
        e.footprint = q->footprint;
        b->cache.push_back(e);
        q->mesh = nullptr; q->grid = nullptr; q->st = nullptr; q->ad = nullptr;
    } else {
        destroy_objects(q->ad, q->st, q->grid, q->mesh);
        b->used -= q->footprint;
    }
}

int start_adjoint(dvm_batch* b, BatchReq* q) {
    int rc;
    if ((rc = dvm_adjoint_create(q->st, q->r.functional, &q->ad))) return rc;
    if (WarmEntry* e = find_warm(b, q->r)) {
        if (e->ad) {
            dvm_adjoint* ad = q->ad;
            const size_t bytes = (size_t)q->st->mesh->d.ncell * q->st->grid->d.nvp * storage_bytes(q->st->storage);
            CK(cudaMemcpyAsync(ad->phi[ad->cur], e->ad->phi[e->ad->cur], bytes, cudaMemcpyDeviceToDevice,
                               b->ctx->stream));
            CK(refresh_adjoint_couplings(ad));
        }
    }
    if (q->r.predict_iters > 0) {         // the transposed moment system at the converged primal state
        dvm_state* st = q->st;
        CK(launch_coarse_assemble(st->storage, st->mesh->d, st->grid->d, st->fl, st->prim[st->cur], st->co_out,
                                  st->co_dinv, b->ctx->stream));
        b->ctx->launches += 1;
        q->predicting = true;
        q->phase_predictions = 0;
        q->pred_high = 0;
        q->pred_best = INFINITY;
        q->damp = PredictDamping(q->r.predict_omega > 0.0 ? q->r.predict_omega : 0.8);
    }
    q->phase = 2;
    return DVM_OK;
}

// The macroscopic prediction of a served request after a tick that leaves its phase running: the same
// steps as a predicted dvm_primal_solve / dvm_adjoint_solve block, with the residual moments taken from
// the tick's last sweep (input f[1 - cur], output f[cur]; phi likewise).
int batch_predict(dvm_batch* b, BatchReq* q) {
    dvm_context* ctx = b->ctx;
    cudaStream_t s = ctx->stream;
    dvm_state* st = q->st;
    const double r = q->phase == 1 ? q->res : q->ares;
    if (st->storage != DVM_STORE_FP64) {            // FP32 noise rule of the solves
        q->pred_high = r > 2.0 * q->pred_best ? q->pred_high + 1 : 0;
        if (q->pred_high >= 2) {
            q->predicting = false;
            q->best = r;
            q->best_it = q->phase == 1 ? q->pit : q->ait;
            return DVM_OK;
        }
        q->pred_best = std::min(q->pred_best, r);
    }
    q->damp.block(r);
    const int m = q->r.predict_iters;
    const DevMesh& msh = st->mesh->d;
    if (q->phase == 1) {
        const int c = st->cur;
        CK(launch_primal_restrict(st->storage, msh, st->grid->d, st->prim[1 - c], 1.0 / st->fl.tau_inf, st->f[1 - c],
                                  st->f[c], st->co_rW, s));
        ctx->launches += 1;
        int rc = predict_step(st, m, q->damp.w, q->phase_predictions % 4 == 0);
        if (rc) return rc;
    } else {
        dvm_adjoint* ad = q->ad;
        CK(launch_adjoint_restrict(st->storage, msh, st->grid->d, st->prim[st->cur], 1.0 / st->fl.tau_inf,
                                   ad->phi[1 - ad->cur], ad->phi[ad->cur], st->co_rW, s));
        CK(launch_coarse_gmres(msh, st->co_out, st->co_dinv, st->co_rW, true, m, st->co_kr, st->co_x, graphs_ok(ctx), s));
        CK(launch_adjoint_shift(st->storage, msh, st->grid->d, st->co_x, q->damp.w, ad->phi[ad->cur], s));
        CK(refresh_adjoint_couplings(ad));
        ctx->launches += krylov_launches(m) + 3;
    }
    q->damp.after_prediction = true;
    q->phase_predictions += 1;
    q->predictions += 1;
    return DVM_OK;
}

template <class TS>
void fill_primal_desc(PrimalBatchDesc<TS>* d, dvm_state* st) {
    using TC = typename std::conditional<sizeof(TS) == 8, double, float>::type;
    d->maps[0] = st->maps[st->cur];
    d->maps[1] = st->maps[1 - st->cur];
    d->args[0] = primal_args<TS, TC>(st, st->cur);
    d->args[1] = primal_args<TS, TC>(st, 1 - st->cur);
}

template <class TS>
void fill_adjoint_desc(AdjointBatchDesc<TS>* d, dvm_adjoint* ad) {
    using TC = typename std::conditional<sizeof(TS) == 8, double, float>::type;
    d->phi_maps[0] = ad->maps[ad->cur];
    d->phi_maps[1] = ad->maps[1 - ad->cur];
    d->f_maps = ad->st->maps[ad->st->cur];
    d->args[0] = adjoint_args<TS, TC>(ad, ad->cur);
    d->args[1] = adjoint_args<TS, TC>(ad, 1 - ad->cur);
}

size_t pdesc_size(int storage) {
    return storage == 0 ? sizeof(PrimalBatchDesc<double>)
                        : (storage == 1 ? sizeof(PrimalBatchDesc<float>) : sizeof(PrimalBatchDesc<__nv_bfloat16>));
}
size_t adesc_size(int storage) {
    return storage == 0 ? sizeof(AdjointBatchDesc<double>)
                        : (storage == 1 ? sizeof(AdjointBatchDesc<float>) : sizeof(AdjointBatchDesc<__nv_bfloat16>));
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" {

int dvm_batch_create(dvm_context* ctx, const dvm_batch_options* opt, dvm_batch** out) {
    if (!ctx || !opt || !out) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    if (opt->sweeps_per_tick < 2 || opt->sweeps_per_tick % 2) return fail(DVM_ERR_INVALID_ARG, "sweeps_per_tick must be even and >= 2");
    if (!ctx->stream) return fail(DVM_ERR_INVALID_ARG, "the batch needs a context with a stream");
    dvm_batch* b = new (std::nothrow) dvm_batch();
    if (!b) return fail(DVM_ERR_OOM, "host allocation");
    b->ctx = ctx;
    b->opt = *opt;
    live_add(b, kBatch, ctx);
    *out = b;
    return DVM_OK;
}

void dvm_batch_destroy(dvm_batch* b) {
    if (!b || !live_take(b, kBatch)) return;
    DeviceGuard dg(b->ctx->device);
    cudaStreamSynchronize(b->ctx->stream);
    for (auto& kv : b->all) {
        BatchReq* q = kv.second;
        destroy_objects(q->ad, q->st, q->grid, q->mesh);
        delete q;
    }
    for (auto& e : b->cache) destroy_objects(e.ad, e.st, e.grid, e.mesh);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (int k = 0; k < 6; ++k) if (b->desc[k]) cudaFree(b->desc[k]);
    if (b->items) cudaFree(b->items);
    if (b->fdesc) cudaFree(b->fdesc);
    if (b->dout) cudaFree(b->dout);
    if (b->counts) cudaFree(b->counts);
    if (b->hout) cudaFreeHost(b->hout);
    if (b->host) cudaFreeHost(b->host);
    delete b;
}

int dvm_batch_submit(dvm_batch* b, const dvm_request* r, uint64_t* ticket) {
    if (!b || !r || !ticket) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    if (r->ni < 3 || r->nj < 1 || r->nv < 1 || !r->nodes_xy || !r->vx || !r->vy || !r->w)
        return fail(DVM_ERR_INVALID_ARG, "request needs a mesh and a velocity grid");
    if (r->storage < 0 || r->storage > 2 || r->max_iter < 0) return fail(DVM_ERR_INVALID_ARG, "bad request options");
    if (r->predict_iters < 0 || r->predict_iters > kMaxKrylov || !(r->predict_omega >= 0.0 && r->predict_omega <= 1.0) ||
        (r->predict_iters > 0 && r->storage == DVM_STORE_BF16))
        return fail(DVM_ERR_INVALID_ARG, "predict_iters must be in [0, 64] (FP64/FP32 storage), predict_omega in [0, 1]");
    if (r->n_params > 0 && (!r->dwall_dalpha || (r->sens_mode == DVM_SENS_FULL && !r->s_j)))
        return fail(DVM_ERR_INVALID_ARG, "sensitivity needs dwall_dalpha (and s_j in full mode)");
    BatchReq* q = new (std::nothrow) BatchReq();
    if (!q) return fail(DVM_ERR_OOM, "host allocation");
    q->r = *r;
    q->nodes.assign(r->nodes_xy, r->nodes_xy + 2 * (size_t)(r->nj + 1) * r->ni);
    q->vx.assign(r->vx, r->vx + r->nv);
    q->vy.assign(r->vy, r->vy + r->nv);
    q->w.assign(r->w, r->w + r->nv);
    if (r->n_params > 0) {
        q->dwall.assign(r->dwall_dalpha, r->dwall_dalpha + 2 * (size_t)r->n_params * r->ni);
        if (r->s_j) q->sj.assign(r->s_j, r->s_j + r->nj + 1);
    }
    q->r.nodes_xy = q->nodes.data(); q->r.vx = q->vx.data(); q->r.vy = q->vy.data(); q->r.w = q->w.data();
    q->r.dwall_dalpha = q->dwall.empty() ? nullptr : q->dwall.data();
    q->r.s_j = q->sj.empty() ? nullptr : q->sj.data();
    q->footprint = request_footprint(q->r);
    if (b->opt.hbm_budget && q->footprint > b->opt.hbm_budget) {
        delete q;
        return fail(DVM_ERR_ADMISSION, "request larger than the batch's HBM budget");
    }
    q->ticket = b->next++;
    b->all[q->ticket] = q;
    b->queue.push_back(q);
    *ticket = q->ticket;
    return DVM_OK;
}

int dvm_batch_tick(dvm_batch* b, int* n_active, int* n_queued) {
    if (!b) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    dvm_context* ctx = b->ctx;
    DeviceGuard dg(ctx->device);
    Range nvtx("dvm_batch_tick");
    const int M = b->opt.sweeps_per_tick;
    int rc;
    // 1. admission, arrival order
    while (!b->queue.empty()) {
        BatchReq* q = b->queue.front();
        if (b->opt.max_active && (int)b->active.size() >= b->opt.max_active) break;
        if (b->opt.hbm_budget && b->used + q->footprint > b->opt.hbm_budget) {
            if (evict_one(b)) continue;
            break;
        }
        b->queue.pop_front();
        b->used += q->footprint;
        rc = admit(b, q);
        if (rc) {                                    // this request fails, the batch goes on
            q->pstatus = rc;
            destroy_objects(q->ad, q->st, q->grid, q->mesh);
            b->used -= q->footprint;
            q->status = rc;
            q->phase = 3;
            continue;
        }
        b->active.push_back(q);
    }
    // 2. the admitted set in six segments (storage, phase); tables grow to fit it
    std::vector<BatchReq*> seg[6];
    for (BatchReq* q : b->active) seg[2 * q->r.storage + (q->phase == 1 ? 0 : 1)].push_back(q);
    const size_t nact = b->active.size();
    b->stats.peak_active = std::max(b->stats.peak_active, (int)nact);
    b->stats.peak_bytes = std::max(b->stats.peak_bytes, b->used);
    if (nact > 0) {
        cudaStream_t s = ctx->stream;
        size_t need[6];
        bool grown_items = false;
        for (int k = 0; k < 6; ++k) {
            need[k] = 0;
            for (BatchReq* q : seg[k]) need[k] += (size_t)q->r.ni * ((q->r.nj + kWarpsPerBlock - 1) / kWarpsPerBlock);
            if ((int)need[k] > b->cap_items[k]) {
                b->cap_items[k] = (int)std::max<size_t>(need[k], std::max(2 * (size_t)b->cap_items[k], (size_t)256));
                grown_items = true;
            }
            if ((int)seg[k].size() > b->cap_desc[k]) {
                b->cap_desc[k] = std::max((int)seg[k].size(), std::max(2 * b->cap_desc[k], 4));
                const size_t dsz = (k & 1) ? adesc_size(k / 2) : pdesc_size(k / 2);
                if ((rc = realloc_device((unsigned char**)&b->desc[k], b->cap_desc[k] * dsz))) return rc;
                b->graph_stale = true;
            }
        }
        if (grown_items) {
            size_t tot = 0;
            for (int k = 0; k < 6; ++k) { b->item_off[k] = tot; tot += (size_t)b->cap_items[k]; }
            if ((rc = realloc_device(&b->items, tot * sizeof(int4)))) return rc;
            b->graph_stale = true;
        }
        if ((int)nact > b->cap_act) {
            b->cap_act = std::max((int)nact, std::max(2 * b->cap_act, 16));
            if ((rc = realloc_device(&b->fdesc, b->cap_act * sizeof(FinalizeDesc))) ||
                (rc = realloc_device(&b->dout, 2 * (size_t)b->cap_act * sizeof(double))))
                return rc;
            if (b->hout) cudaFreeHost(b->hout);
            b->hout = nullptr;
            CK(cudaMallocHost((void**)&b->hout, 2 * (size_t)b->cap_act * sizeof(double)));
            b->graph_stale = true;
        }
        if (!b->counts && (rc = realloc_device(&b->counts, 8 * sizeof(int)))) return rc;
        if (b->graph_stale) b->sig.clear();
        // 3. tables: rebuilt and uploaded only when the admitted set or a phase changed
        std::vector<uint64_t> sig;
        sig.reserve(nact);
        for (BatchReq* q : b->active) sig.push_back(4 * q->ticket + (uint64_t)q->phase);
        if (sig != b->sig) {
            size_t off_d[6], hb = 0;
            for (int k = 0; k < 6; ++k) {
                off_d[k] = hb;
                hb = align_up(hb + seg[k].size() * ((k & 1) ? adesc_size(k / 2) : pdesc_size(k / 2)), 128);
            }
            const size_t off_items = hb;
            size_t n_items = 0;
            for (int k = 0; k < 6; ++k) n_items += need[k];
            hb = align_up(hb + n_items * sizeof(int4), 128);
            const size_t off_fd = hb;
            hb = align_up(hb + nact * sizeof(FinalizeDesc), 128);
            const size_t off_cnt = hb;
            hb += 8 * sizeof(int);
            if ((rc = grow_host(b, hb))) return rc;
            int4* hitems = reinterpret_cast<int4*>(b->host + off_items);
            int* hcnt = reinterpret_cast<int*>(b->host + off_cnt);
            size_t it = 0;
            for (int k = 0; k < 6; ++k) {
                const int t = k / 2;
                const size_t it0 = it;
                for (size_t r = 0; r < seg[k].size(); ++r) {
                    BatchReq* q = seg[k][r];
                    if (k & 1) {
                        unsigned char* d = b->host + off_d[k] + r * adesc_size(t);
                        if (t == 0) fill_adjoint_desc(reinterpret_cast<AdjointBatchDesc<double>*>(d), q->ad);
                        else if (t == 1) fill_adjoint_desc(reinterpret_cast<AdjointBatchDesc<float>*>(d), q->ad);
                        else fill_adjoint_desc(reinterpret_cast<AdjointBatchDesc<__nv_bfloat16>*>(d), q->ad);
                    } else {
                        unsigned char* d = b->host + off_d[k] + r * pdesc_size(t);
                        if (t == 0) fill_primal_desc(reinterpret_cast<PrimalBatchDesc<double>*>(d), q->st);
                        else if (t == 1) fill_primal_desc(reinterpret_cast<PrimalBatchDesc<float>*>(d), q->st);
                        else fill_primal_desc(reinterpret_cast<PrimalBatchDesc<__nv_bfloat16>*>(d), q->st);
                    }
                    const DevMesh& m = q->st->mesh->d;
                    for (int i = 0; i < m.ni; ++i)
                        for (int j0 = 0; j0 < m.nj; j0 += kWarpsPerBlock) hitems[it++] = int4{(int)r, i, j0, 0};
                }
                hcnt[k] = (int)(it - it0);
                if (!seg[k].empty()) {
                    const size_t dsz = (k & 1) ? adesc_size(t) : pdesc_size(t);
                    CK(cudaMemcpyAsync(b->desc[k], b->host + off_d[k], seg[k].size() * dsz, cudaMemcpyHostToDevice, s));
                    CK(cudaMemcpyAsync(b->items + b->item_off[k], hitems + it0, (it - it0) * sizeof(int4),
                                       cudaMemcpyHostToDevice, s));
                }
            }
            hcnt[6] = (int)nact;
            hcnt[7] = 0;
            FinalizeDesc* hfd = reinterpret_cast<FinalizeDesc*>(b->host + off_fd);
            for (size_t k = 0; k < nact; ++k) {
                BatchReq* q = b->active[k];
                const DevMesh& m = q->st->mesh->d;
                if (q->phase == 1) hfd[k] = FinalizeDesc{q->st->respart, m.ncell, m.ni, q->st->Jpart, q->st->Fw[q->st->cur], q->st->fl.wallM};
                else hfd[k] = FinalizeDesc{q->ad->respart, m.ncell, m.ni, nullptr, nullptr, nullptr};
            }
            CK(cudaMemcpyAsync(b->fdesc, hfd, nact * sizeof(FinalizeDesc), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(b->counts, hcnt, 8 * sizeof(int), cudaMemcpyHostToDevice, s));
            b->sig.swap(sig);
            b->stats.table_uploads += 1;
        }
        // M sweeps of every admitted request (one batched launch per segment and sweep), the residual
        // and drag reduction, and the read-back: one graph launch, or the same launches directly
        int kernels = 1;
        for (int k = 0; k < 6; ++k) kernels += b->cap_items[k] > 0 ? M : 0;
        auto enqueue = [&]() -> cudaError_t {
            cudaError_t e = cudaSuccess;
            for (int sw = 0; sw < M && e == cudaSuccess; ++sw) {
                const bool res = sw == M - 1;
                for (int t = 0; t < 3 && e == cudaSuccess; ++t) {
                    e = launch_primal_sweep_batch(t, b->desc[2 * t], b->items + b->item_off[2 * t], b->cap_items[2 * t],
                                                  b->counts + 2 * t, sw & 1, res, s);
                    if (e == cudaSuccess)
                        e = launch_adjoint_sweep_batch(t, b->desc[2 * t + 1], b->items + b->item_off[2 * t + 1],
                                                       b->cap_items[2 * t + 1], b->counts + 2 * t + 1, sw & 1, res, s);
                }
            }
            if (e == cudaSuccess) e = launch_finalize_batch(b->fdesc, b->cap_act, b->counts + 6, b->dout, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(b->hout, b->dout, 2 * (size_t)b->cap_act * sizeof(double), cudaMemcpyDeviceToHost, s);
            return e;
        };
        if (graphs_ok(ctx)) {
            if (!b->graph || b->graph_stale || b->graph_M != M) {
                if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
                cudaGraph_t gr;
                CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                cudaError_t ce = enqueue();
                cudaError_t ee = cudaStreamEndCapture(s, &gr);
                CK(ce);
                CK(ee);
                cudaError_t ie = cudaGraphInstantiate(&b->graph, gr, 0);
                cudaGraphDestroy(gr);
                CK(ie);
                b->graph_M = M;
                b->graph_stale = false;
                b->stats.graph_builds += 1;
            }
            CK(cudaGraphLaunch(b->graph, s));
            b->stats.graph_launches += 1;
        } else {
            CK(enqueue());
        }
        ctx->launches += kernels;
        b->stats.ticks += 1;
        CK(cudaStreamSynchronize(s));
        if ((rc = check_device_flag(ctx))) return rc;
        const double* hout = b->hout;
        // 4. convergence and phase changes
        std::vector<BatchReq*> keep;
        for (size_t k = 0; k < nact; ++k) {
            BatchReq* q = b->active[k];
            const double r2 = hout[2 * k], J = hout[2 * k + 1];
            bool leave = false;
            if (q->phase == 1) {
                q->pit += M;
                q->st->version += (uint64_t)M;
                q->res = sqrt(r2) / q->st->r0;
                q->J = J;
                if (q->res < 0.98 * q->best) { q->best = q->res; q->best_it = q->pit; }
                const bool stalled = q->r.stall_window > 0 && q->pit - q->best_it >= q->r.stall_window;
                if (!std::isfinite(q->res) || !std::isfinite(J)) { q->pstatus = DVM_ERR_NONFINITE; leave = true; }
                else if (q->res <= q->r.tol || q->pit >= q->r.max_iter || stalled) {
                    q->pstatus = q->res <= q->r.tol ? DVM_OK : stalled ? DVM_ERR_STAGNATED : DVM_NOT_CONVERGED;
                    q->best = INFINITY;
                    q->best_it = 0;
                    // the fused partials carry the drag; another functional is evaluated on the final state
                    if (q->r.functional != DVM_DRAG && (rc = dvm_state_functional(q->st, q->r.functional, &q->J)))
                        q->pstatus = rc;
                    if (q->r.n_params > 0) {
                        if ((rc = start_adjoint(b, q))) { q->astatus = rc; leave = true; }
                    } else {
                        leave = true;
                    }
                }
            } else {
                q->ait += M;
                q->ares = sqrt(r2) / q->ad->r0;
                if (q->ares < 0.98 * q->best) { q->best = q->ares; q->best_it = q->ait; }
                const bool stalled = q->r.stall_window > 0 && q->ait - q->best_it >= q->r.stall_window;
                if (!std::isfinite(q->ares)) { q->astatus = DVM_ERR_NONFINITE; leave = true; }
                else if (q->ares <= q->r.adjoint_tol || q->ait >= q->r.max_iter || stalled) {
                    q->astatus = q->ares <= q->r.adjoint_tol ? DVM_OK : stalled ? DVM_ERR_STAGNATED : DVM_NOT_CONVERGED;
                    q->grad.assign(q->r.n_params, 0.0);
                    rc = dvm_sensitivity(ctx, q->st, q->ad, q->r.n_params, q->r.dwall_dalpha, q->r.s_j, q->r.sens_mode,
                                         q->grad.data(), nullptr);
                    if (rc) q->astatus = rc;
                    leave = true;
                }
            }
            // a primal that just moved to its adjoint starts predicting after the adjoint's first tick
            const bool moved = q->phase == 2 && q->ait == 0;
            if (!leave && q->predicting && !moved && (rc = batch_predict(b, q))) {
                if (q->phase == 1) q->pstatus = rc;
                else q->astatus = rc;
                leave = true;
            }
            if (leave) retire(b, q);
            else keep.push_back(q);
        }
        b->active.swap(keep);
    }
    if (n_active) *n_active = (int)b->active.size();
    if (n_queued) *n_queued = (int)b->queue.size();
    return DVM_OK;
}

int dvm_batch_get_stats(const dvm_batch* b, dvm_batch_stats* out) {
    if (!b || !out) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    *out = b->stats;
    return DVM_OK;
}

int dvm_batch_poll(dvm_batch* b, uint64_t ticket, dvm_request_result* out, double* grad_out, int forget) {
    if (!b || !out) return fail(DVM_ERR_INVALID_ARG, "NULL argument");
    auto itq = b->all.find(ticket);
    if (itq == b->all.end()) return fail(DVM_ERR_INVALID_ARG, "unknown ticket");
    BatchReq* q = itq->second;
    std::memset(out, 0, sizeof(*out));
    out->done = q->phase == 3;
    out->phase = q->phase;
    out->status = q->phase == 3 ? q->status : DVM_OK;
    out->primal_iters = q->pit;
    out->adjoint_iters = q->ait;
    out->J = q->J;
    const double U = q->r.flow.Ma * sqrt(5.0 / 3.0);
    out->Cd = U > 0.0 ? q->J / (0.5 * U * U) : q->J;
    out->residual = q->res;
    out->adjoint_residual = q->ares;
    out->warm_started = q->warm;
    out->predictions = q->predictions;
    if (out->done && grad_out && !q->grad.empty()) std::memcpy(grad_out, q->grad.data(), q->grad.size() * sizeof(double));
    if (out->done && forget) {
        b->all.erase(itq);
        delete q;
    }
    return DVM_OK;
}

}  // extern "C"
