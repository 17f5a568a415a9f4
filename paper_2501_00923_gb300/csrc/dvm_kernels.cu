// CUDA kernels (sm_103a) of the DVM-BGK primal sweep, the transposed adjoint sweep, the wall
// reductions and the boundary sensitivities (Yuan & Wu, arXiv 2501.00923, Sec. 2-3).
//
// Layout: f[cell][k] = (f1, f2) pairs in the storage type, velocity fastest, nv padded to a
// multiple of 4.  One warp owns one cell and walks its velocities in 16-byte chunks (1 pair in
// FP64, 2 in FP32, 4 in BF16), so every load and store of a warp is 512 contiguous bytes.  Because
// a warp holds all velocities of its cell, the velocity-space reductions (moments W, the wall
// density F_rhow, the adjoint What / rhohat / Lambda, the residual) finish inside the warp with
// no cross-block step: per-lane FP32 Kahan sums (FP64 sums for FP64 storage) combined in FP64 by a
// fixed butterfly, so results are deterministic.
#include "dvm_internal.h"

#include <algorithm>
#include <cstring>
#include <type_traits>

// Tile parameters of the sweeps (see the pipeline section): chunks per lane per stage and stages.
// 2 chunks per lane, 2 stages and 3 resident blocks per SM were the fastest of (1,4,3), (1,4,4),
// (2,3,2), (2,2,3) and (2,4,2) on the 256x128-cell, 48x48-velocity workload.
#ifndef DVM_CPL
#define DVM_CPL 2
#endif
#ifndef DVM_STAGES
#define DVM_STAGES 2
#endif
// Resident 256-thread blocks per SM asked of the second-order reconstruction kernels.
#ifndef DVM_SO_BLOCKS
#define DVM_SO_BLOCKS 1
#endif

namespace dvm {
namespace {

constexpr double kPi = 3.14159265358979323846;

template <class T> struct Vec;
template <> struct Vec<float> { using v2 = float2; using v4 = float4; };
template <> struct Vec<double> { using v2 = double2; using v4 = double4; };

// ------------------------------------------------------------------ 16-byte chunks of (f1,f2)
template <class TS> struct Pack;
template <> struct Pack<double> {
    using TC = double;
    static constexpr int KV = 1;
    __device__ static void unpack(const uint4& r, double (&a)[1], double (&b)[1]) {
        a[0] = __hiloint2double((int)r.y, (int)r.x);
        b[0] = __hiloint2double((int)r.w, (int)r.z);
    }
    __device__ static uint4 pack(const double (&a)[1], const double (&b)[1]) {
        uint4 r;
        r.x = (unsigned)__double2loint(a[0]); r.y = (unsigned)__double2hiint(a[0]);
        r.z = (unsigned)__double2loint(b[0]); r.w = (unsigned)__double2hiint(b[0]);
        return r;
    }
};
// FP32 chunks hold (f1_k, f1_k+1, f2_k, f2_k+1): the two velocities of one component sit in one
// register pair, the operand of the paired FP32 instructions (FFMA2 and friends).
template <> struct Pack<float> {
    using TC = float;
    static constexpr int KV = 2;
    __device__ static void unpack(const uint4& r, float (&a)[2], float (&b)[2]) {
        a[0] = __uint_as_float(r.x); a[1] = __uint_as_float(r.y);
        b[0] = __uint_as_float(r.z); b[1] = __uint_as_float(r.w);
    }
    __device__ static uint4 pack(const float (&a)[2], const float (&b)[2]) {
        return make_uint4(__float_as_uint(a[0]), __float_as_uint(a[1]), __float_as_uint(b[0]),
                          __float_as_uint(b[1]));
    }
};
template <> struct Pack<__nv_bfloat16> {
    using TC = float;
    static constexpr int KV = 4;
    __device__ static void unpack(const uint4& r, float (&a)[4], float (&b)[4]) {
        const unsigned wd[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            a[i] = __uint_as_float(wd[i] << 16);
            b[i] = __uint_as_float(wd[i] & 0xffff0000u);
        }
    }
    __device__ static uint4 pack(const float (&a)[4], const float (&b)[4]) {
        unsigned wd[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 h = __floats2bfloat162_rn(a[i], b[i]);
            unsigned u;
            memcpy(&u, &h, 4);
            wd[i] = u;
        }
        return make_uint4(wd[0], wd[1], wd[2], wd[3]);
    }
};

// Element index of f1 of velocity k of cell c; f2 follows at + kComp<TS>.
template <class TS> constexpr int kComp = std::is_same<TS, float>::value ? 2 : 1;
template <class TS> __device__ __forceinline__ size_t fpos(size_t c, int nvp, int k) {
    if (std::is_same<TS, float>::value) return (c * nvp + (k & ~1)) * 2 + (k & 1);
    return (c * nvp + k) * 2;
}

// ------------------------------------------------------------------ accumulators
template <class T> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ void add(double x) { s += x; }
    __device__ double get() const { return s; }
};
// Kahan-compensated FP32 sum: error independent of the number of terms.
template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ double get() const { return (double)s - (double)c; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint4 ldg16(const uint4* p) { return __ldg(p); }
__device__ __forceinline__ void stg16(uint4* p, const uint4& v) { __stcs(p, v); }

template <class TC> __device__ __forceinline__ TC dexp(TC x);
template <> __device__ __forceinline__ float dexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double dexp<double>(double x) { return exp(x); }

template <class TC> __device__ __forceinline__ TC pos(TC a) { return a > TC(0) ? a : TC(0); }

__device__ __forceinline__ double todbl(double x) { return x; }
__device__ __forceinline__ double todbl(float x) { return (double)x; }
__device__ __forceinline__ double todbl(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
template <class T> __device__ __forceinline__ T fromdbl(double x);
template <> __device__ __forceinline__ double fromdbl<double>(double x) { return x; }
template <> __device__ __forceinline__ float fromdbl<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ __nv_bfloat16 fromdbl<__nv_bfloat16>(double x) {
    return __float2bfloat16_rn((float)x);
}

// ------------------------------------------------------------------ FP32 fast paths
// In the FP32/BF16 path the exponential and the reciprocal use the hardware approximations
// (__expf: 2 + 1.2|x| ulp; __fdividef: 2 ulp), well inside the storage rounding of the values they
// produce; the FP64 path uses the correctly rounded library functions.
template <class TC> __device__ __forceinline__ TC fexp(TC x);
template <> __device__ __forceinline__ float fexp<float>(float x) { return __expf(x); }
template <> __device__ __forceinline__ double fexp<double>(double x) { return exp(x); }
template <class TC> __device__ __forceinline__ TC frcp(TC x);
template <> __device__ __forceinline__ float frcp<float>(float x) { return __fdividef(1.0f, x); }
template <> __device__ __forceinline__ double frcp<double>(double x) { return 1.0 / x; }

// Double-float (hi + lo) value and its exact-error addition (two-sum), used to combine the
// compensated per-lane sums across a warp with FP32 instructions only.
struct DF { float hi, lo; };
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
    const float h = s + e;
    return DF{h, e - (h - s)};
}
__device__ __forceinline__ DF warp_sum_df(DF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = df_add(v, w);
    }
    return v;
}

// Per-lane sum, then warp total (same value on every lane, fixed order).
template <class TC> struct Sum;
template <> struct Sum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double total() const { return warp_sum(s); }
};
template <> struct Sum<float> {      // Kahan-compensated lane sum, double-float warp combine
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ float total() const {
        const DF d = warp_sum_df(DF{s, -c});
        return d.hi + d.lo;
    }
};

// Boundary class of a cell, fixed per warp: interior, wall row (j = 0), far-field row (j = nj-1),
// or both (a one-layer mesh).  Each class gets its own compiled loop so that interior cells, which
// are all but 2/nj of the mesh, carry no boundary logic.
enum { kInterior = 0, kWallCell = 1, kFarCell = 2, kWallFar = 3 };
constexpr int kBlockIters = 8 / DVM_CPL;   // stages summed in FP32 before one compensated add

// ------------------------------------------------------------------ tiled-TMA pipeline
// A block owns 8 radially adjacent cells (i, j0..j0+7), one warp per cell.  The distribution is a
// 3D tensor [nj][ni][16-byte chunks]; for each row of 32 chunks (32 lanes x 16 B) the block needs
// its column with one halo row on each side (rows j0-1..j0+8) and the columns i-1 and i+1 (rows
// j0..j0+7).  Three tiled TMA loads (cp.async.bulk.tensor) bring them into one pipeline stage:
// periodicity in i is a coordinate, rows outside [0, nj) are zero-filled and never used.  Thread 0
// issues the first kStages chunk rows; every warp waits on the stage's "full" mbarrier, computes
// and releases the stage, and the last warp to release it issues its next chunk row.  Every wait
// is bounded (kWaitNs by the global timer): a wait that runs out sets *err, the block stops, and
// each warp drains the copies it issued.
// Tile parameters: kCPL 16-byte chunks per lane per stage (a stage row is 32 kCPL chunks, one TMA
// box of 128 kCPL 32-bit elements, at most 256) and kStages stages per block.
constexpr int kCPL = DVM_CPL;
constexpr int kRowChunks = 32 * kCPL;
constexpr int kStages = DVM_STAGES;
static_assert(kCPL >= 1 && kCPL <= 2, "a TMA box row holds at most 256 elements");
constexpr int kPrimalRows = 26;      // column 10 rows + west 8 + east 8
constexpr int kAdjointRows = 34;     // phi column 10 + phi west 8 + phi east 8 + f 8
constexpr unsigned kSuspendNs = 1000000;                  // suspend-time hint of one try
constexpr unsigned long long kWaitNs = 2000000000ull;     // a wait gives up after 2 s ...
constexpr unsigned kWaitTries = 100000000u;               // ... or this many tries

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// The suspend hint is an upper bound only (a try may return much sooner), so the limit is kept in
// time: kWaitNs of %globaltimer, with a cap on the tries as a backstop.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned t = 0; t < kWaitTries; ++t) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Acquire-release increment of a shared-memory counter (block scope); returns the old value.
__device__ __forceinline__ unsigned atom_inc_acq_rel(unsigned* p) {
    unsigned old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;" : "=r"(old) : "r"(smem_u32(p)) : "memory");
    return old;
}

// Non-tensor bulk copy global -> shared (16-byte aligned, size a multiple of 16) on the same mbarrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"((unsigned long long)__cvta_generic_to_global(src)), "r"(bytes),
                 "r"(smem_u32(bar))
                 : "memory");
}

// A block's pipeline: stages, their "full" mbarriers and release counters.
struct Feed {
    const CUtensorMap* col;      // box 32 chunks x 1 cell x 10 rows (the value being swept)
    const CUtensorMap* side;     // box 32 chunks x 1 cell x 8 rows (the same buffer)
    const CUtensorMap* extra;    // box 32 chunks x 1 cell x 8 rows of a second buffer (adjoint: f), or null
    int i, im, ip, j0, rows;     // block column, its periodic neighbours, first row, rows per stage
    unsigned A;                  // warps that consume each stage
    const float4* vpa;           // paired velocity table, (vx, vx', vy, vy') per pair, or null
    const float4* vpb;           // (w, w', h, h') per pair
    unsigned vprow;              // velocity pairs per stage row (0: the table is not staged)
    unsigned stride;             // 16-byte units per stage: rows x kRowChunks chunks, then 2 vprow pairs
    uint4* stage;                // kStages x stride
    uint64_t* full;
    unsigned* released;          // per stage, warps that have released it so far (monotone)
    __device__ __forceinline__ void issue(unsigned it) const {
        const unsigned st = it % kStages;
        uint4* d = stage + (size_t)st * stride;
        const int x = (int)(it * kRowChunks * 4u);           // uint32 elements: 16-byte aligned
        mbar_expect_tx(&full[st], stride * 16u);
        tma_load_3d(d, col, x, i, j0 - 1, &full[st]);
        tma_load_3d(d + 10 * kRowChunks, side, x, im, j0, &full[st]);
        tma_load_3d(d + 18 * kRowChunks, side, x, ip, j0, &full[st]);
        if (extra) tma_load_3d(d + 26 * kRowChunks, extra, x, i, j0, &full[st]);
        if (vprow) {                 // the velocity pairs of this row: (vx, vy) block, then (w, h) block
            uint4* t = d + (size_t)rows * kRowChunks;
            bulk_load(t, vpa + (size_t)it * vprow, vprow * 16u, &full[st]);
            bulk_load(t + vprow, vpb + (size_t)it * vprow, vprow * 16u, &full[st]);
        }
    }
};

// 2^x by the hardware approximation (ex2.approx.ftz.f32: relative error 2^-22 on the fraction).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// g1 = n0 exp(-|v-u|^2/(2T)) written as 2^(t kA + kB) with t = |v|^2/2 - v.u (one FMA chain).
// FP64: exp(t kA + kB) with the natural-log constants.
template <class TC> struct Gauss;
template <> struct Gauss<float> {
    float kA, kB;
    __device__ __forceinline__ void setup(float rho, float u1, float u2, float T) {   // FP32 only
        constexpr float L2E = 1.44269504088896341f;
        const float iT = 1.0f / T;
        kA = -L2E * iT;
        kB = log2f(rho * iT * 0.159154943091895336f) - L2E * 0.5f * (u1 * u1 + u2 * u2) * iT;
    }
    __device__ __forceinline__ float eval(float t) const { return ex2_approx(fmaf(t, kA, kB)); }
};
template <> struct Gauss<double> {
    double kA, kB;
    __device__ __forceinline__ void setup(double rho, double u1, double u2, double T) {
        kA = -1.0 / T;
        kB = log(rho / (2.0 * kPi * T)) - 0.5 * (u1 * u1 + u2 * u2) / T;
    }
    __device__ __forceinline__ double eval(double t) const { return exp(fma(t, kA, kB)); }
};

// ------------------------------------------------------------------ paired FP32 arithmetic
// Two velocities at a time with the paired FP32 instructions of sm_100+ (round-to-nearest, one
// rounding per lane as in the scalar forms).  Broadcast operands are pairs of equal values.
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 inflow(float2 a) { return make_float2(fmaxf(-a.x, 0.f), fmaxf(-a.y, 0.f)); }
__device__ __forceinline__ float2 pex2(float2 a) { return make_float2(ex2_approx(a.x), ex2_approx(a.y)); }
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 prcp(float2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
template <int KV> __device__ __forceinline__ float2 pair_of(const float (&a)[KV], int p) {
    return make_float2(a[2 * p], a[2 * p + 1]);
}

// One pipeline step shared by both sweeps: wait for stage `it`, run `body` on it and release it.
// The warp whose release is the last one for this round of the stage refills it with chunk row
// it + kStages, so no warp ever waits for a stage to drain.  The acquire-release counter orders
// every warp's reads of the stage before that warp's copy into it (then the proxy fence orders
// them before the asynchronous write).  Returns false when a wait ran out.
template <class Body>
__device__ __forceinline__ bool pipeline_step(const Feed& F, unsigned it, unsigned niter, int lane, Body&& body) {
    const unsigned st = it % kStages, ph = (it / kStages) & 1u;
    const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(&F.full[st], ph));
    if (!got) return false;
    body(F.stage + (size_t)st * F.stride);
    __syncwarp();
    if (lane == 0) {
        // after round r of stage st its counter reaches (r + 1) A; the warp that brings it there is last
        const unsigned old = atom_inc_acq_rel(&F.released[st]);
        if (old + 1 == (it / kStages + 1) * F.A && it + kStages < niter) {
            fence_proxy_async();
            F.issue(it + kStages);
        }
    }
    return true;
}

// Resident blocks per SM (the register budget) of the FP32/BF16 sweeps; FP64 keeps 4 (primal) and
// 3 (adjoint).  DVM_PAIRED selects the paired FP32 arithmetic for FP32/BF16 storage.
#ifndef DVM_PRIMAL_BLOCKS
#define DVM_PRIMAL_BLOCKS 3
#endif
#ifndef DVM_ADJOINT_BLOCKS
#define DVM_ADJOINT_BLOCKS 3
#endif
#ifndef DVM_PAIRED
#define DVM_PAIRED 1
#endif
template <class TS> constexpr bool kPaired = DVM_PAIRED && std::is_same<typename Pack<TS>::TC, float>::value;
template <class TS> constexpr int kPrimalMinBlocks = std::is_same<typename Pack<TS>::TC, float>::value ? DVM_PRIMAL_BLOCKS : 4;
template <class TS> constexpr int kAdjointMinBlocks = std::is_same<typename Pack<TS>::TC, float>::value ? DVM_ADJOINT_BLOCKS : 3;

// ================================================================== primal sweep (K1)
// One point-implicit sweep of Eq. (numerpr_gov), first-order upwind, fused with the moments of
// the new state (Eq. macint_reduce), its wall density (Eq. formula_bgk_fdw), the drag partial of
// Eq. (numer_J) and (kRes) the residual R(f_old) = D (f_old - f_new).
// D = V/tau + sum_e max(a_e, 0) = V/tau + (1/2) sum_e |a_e| because the faces of a cell close
// (sum_e A_e n_e = 0); the inflow faces add -min(a_e, 0) F_up to the right-hand side.  The staged
// neighbour chunks are used whether or not a face is an inflow face (the factor min(a_e, 0) is 0),
// which keeps the loop free of per-velocity branches.
// FP32 / BF16 form of the sweep: the same update two velocities at a time.  D uses the inflow
// weights n_e = max(-a_e, 0): sum_e max(a_e, 0) = sum_e n_e on a closed cell.
//
// kLin (refinement, FP32 storage): the same sweep applied to a correction e of the state at a fixed
// linearisation point (prim_old): the relaxation source V/tau g of Eq. (numerpr_gov) is replaced by its
// linearisation in the moments dW of e_old (lagged like g itself),
//   V/tau dg + V d(1/tau) (g - f),   dg1/g1 = drho/rho + (v - u).du/T + (|v - u|^2/(2T^2) - 1/T) dT,
//   dg2 = (T/2) dg1 + (dT/2) g1,      d(1/tau)/(1/tau) = drho/rho + dT/(2T),
// the far field injects nothing, the wall re-emits (dF_rhow / D_l) gbar_w, and the right-hand side gains
// D s, with s the increment of one FP64 sweep of the full problem.  One such sweep is e <- s + e - (J e)/D
// with J the Jacobian of the steady residual, so at its fixed point J e = -R.
template <class TS, bool kRes, int kBnd, bool kDef, bool kLin, bool kShard, bool kRM>
__device__ __forceinline__ bool primal_cell_paired(const PrimalArgs<TS, float>& P, int c, int w, int lane,
                                                   const Feed& F) {
    using PK = Pack<TS>;
    constexpr int KV = PK::KV, NP = KV / 2;
    constexpr bool wall = (kBnd & kWallCell) != 0, far = (kBnd & kFarCell) != 0;
    const float2 S0 = P.S[4 * c], S1 = P.S[4 * c + 1], S2 = P.S[4 * c + 2], S3 = P.S[4 * c + 3];
    const double4 pr = P.prim_old[c], pm = P.maxw_old[c];   // moments (tau), Maxwellian parameters (g)
    const float rho = (float)pm.x, u1 = (float)pm.y, u2 = (float)pm.z, T = (float)pm.w;
    Gauss<float> G;
    G.setup(rho, u1, u2, T);
    const float Vt = P.V[c] * (float)pr.x * sqrtf((float)pr.w) * (float)P.inv_tau_inf;      // V / tau
    const float2 kA = bc(G.kA), kB = bc(G.kB), mu1 = bc(-u1), mu2 = bc(-u2), Vt2 = bc(Vt), hT = bc(0.5f * T);
    float2 lc0 = bc(0.f), lcx = lc0, lcy = lc0, lct = lc0, lhdT = lc0, lVk = lc0;
    if (kLin) {                      // linearised Maxwellian and relaxation rate from the moment sums of e_old
        const double4 dw = P.dW_old[c];
        const float drho = (float)dw.x, dmx = (float)dw.y, dmy = (float)dw.z, dE = (float)dw.w;
        const float ir = 1.f / rho, iT = 1.f / T, uu = 0.5f * (u1 * u1 + u2 * u2);
        const float dux = (dmx - u1 * drho) * ir, duy = (dmy - u2 * drho) * ir;
        const float dT = (2.f / 3.f) * ir * (dE - (u1 * dmx + u2 * dmy) + (uu - 1.5f * T) * drho);
        lcx = bc(dux * iT);
        lcy = bc(duy * iT);
        lct = bc(dT * iT * iT);
        lc0 = bc(drho * ir - (u1 * dux + u2 * duy) * iT + (uu * iT - 1.f) * iT * dT);
        lhdT = bc(0.5f * dT);
        lVk = bc(Vt * (drho * ir + 0.5f * dT * iT));
    }
    const float2 s0x = bc(S0.x), s0y = bc(S0.y), s1x = bc(S1.x), s1y = bc(S1.y);
    const float2 s2x = bc(S2.x), s2y = bc(S2.y), s3x = bc(S3.x), s3y = bc(S3.y);
    float2 cw1 = bc(0.f), cw2 = bc(0.f), dxy = bc(0.f), dyy = bc(0.f);
    float invA = 0.f;
    if (wall) {
        const float c1 = (float)P.Fw_old[c] / (float)P.wallD[c];
        cw1 = bc(c1);
        cw2 = bc(c1 * P.halfTw);
        dxy = bc(P.dirx);
        dyy = bc(P.diry);
        invA = 1.f / sqrtf(S3.x * S3.x + S3.y * S3.y);
    }
    uint4* fw = reinterpret_cast<uint4*>(P.f_new);
    const unsigned nq = (unsigned)P.nq, niter = (nq + kRowChunks - 1) / kRowChunks, oc = (unsigned)c * nq;

    Sum<float> m0, m1, m2, m3, fwa, ja, rs, q0, q1, q2, q3;
    constexpr bool rmom = kRes && kRM;               // moments of the residual (macroscopic prediction)
    bool ok = true;
    unsigned it = 0;
    while (it < niter && ok) {
        float2 bm0 = bc(0.f), bm1 = bm0, bm2 = bm0, bm3 = bm0, bfw = bm0, bj = bm0, brs = bm0;
        float2 bq0 = bm0, bq1 = bm0, bq2 = bm0, bq3 = bm0;
        for (int b = 0; b < kBlockIters && it < niter && ok; ++b, ++it) {
            ok = pipeline_step(F, it, niter, lane, [&](const uint4* d) {
#pragma unroll
              for (int cc = 0; cc < kCPL; ++cc) {
                const unsigned q = it * kRowChunks + cc * 32 + lane;
                if (q >= nq) break;
                const uint4* e = d + cc * 32 + lane;
                const uint4 ro = e[(w + 1) * kRowChunks];
                const uint4 r0 = e[(10 + w) * kRowChunks], r2 = e[(18 + w) * kRowChunks];
                const uint4 r1 = far ? ro : e[(w + 2) * kRowChunks];
                const uint4 r3 = wall ? ro : e[w * kRowChunks];
                float fo1[KV], fo2[KV], e01[KV], e02[KV], e11[KV], e12[KV], e21[KV], e22[KV], e31[KV], e32[KV];
                PK::unpack(ro, fo1, fo2);
                PK::unpack(r0, e01, e02);
                PK::unpack(r1, e11, e12);
                PK::unpack(r2, e21, e22);
                PK::unpack(r3, e31, e32);
                float dq1[KV], dq2[KV];
                if (kDef) PK::unpack(ldg16(reinterpret_cast<const uint4*>(P.defect) + oc + q), dq1, dq2);
                float ls1[KV], ls2[KV], lf1[KV], lf2[KV];
                if (kLin) {
                    PK::unpack(ldg16(reinterpret_cast<const uint4*>(P.lin_src) + oc + q), ls1, ls2);
                    PK::unpack(ldg16(reinterpret_cast<const uint4*>(P.lin_f) + oc + q), lf1, lf2);
                }
                float fn1[KV], fn2[KV];
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) {
                    const int kp = q * NP + pp;                  // velocity pair 2kp, 2kp+1
                    const int lp = (cc * 32 + lane) * NP + pp;   // its slot in the staged table
                    const float4* sA = reinterpret_cast<const float4*>(d + F.rows * kRowChunks);
                    const float4 A = sA[lp], B = sA[F.vprow + lp];
                    const float2 vx = make_float2(A.x, A.y), vy = make_float2(A.z, A.w);
                    const float2 wk = make_float2(B.x, B.y), hv = make_float2(B.z, B.w);
                    const float2 a0 = pfma(s0y, vy, pmul(s0x, vx)), a1 = pfma(s1y, vy, pmul(s1x, vx));
                    const float2 a2 = pfma(s2y, vy, pmul(s2x, vx)), a3 = pfma(s3y, vy, pmul(s3x, vx));
                    const float2 n0 = inflow(a0), n1 = inflow(a1), n2 = inflow(a2), n3 = inflow(a3);
                    float2 f11 = pair_of<KV>(e11, pp), f12 = pair_of<KV>(e12, pp);
                    float2 f31 = pair_of<KV>(e31, pp), f32 = pair_of<KV>(e32, pp);
                    if (far) {
                        if (kLin) {
                            f11 = bc(0.f);
                            f12 = bc(0.f);
                        } else {
                            const float4 g = *reinterpret_cast<const float4*>(P.fd + 2 * kp);   // (g1,g2) x 2
                            f11 = make_float2(g.x, g.z);
                            f12 = make_float2(g.y, g.w);
                        }
                    }
                    if (wall) {
                        const float2 gw = *reinterpret_cast<const float2*>(P.gw + 2 * kp);
                        f31 = pmul(cw1, gw);
                        f32 = pmul(cw2, gw);
                    }
                    const float2 D = padd(Vt2, padd(padd(n0, n1), padd(n2, n3)));
                    const float2 tt = pfma(vy, mu2, pfma(vx, mu1, hv));        // |v|^2/2 - v.u
                    const float2 g1 = pex2(pfma(tt, kA, kB));
                    float2 r1, r2;
                    if (kLin) {
                        const float2 A1 = pfma(tt, lct, pfma(vy, lcy, pfma(vx, lcx, lc0)));   // dg1 / g1
                        const float2 Vg = pmul(Vt2, g1);
                        r1 = pfma(D, pair_of<KV>(ls1, pp), pmul(Vg, A1));
                        r2 = pfma(D, pair_of<KV>(ls2, pp), pmul(Vg, pfma(A1, hT, lhdT)));
                        r1 = pfma(lVk, padd(g1, pmul(bc(-1.f), pair_of<KV>(lf1, pp))), r1);
                        r2 = pfma(lVk, pfma(hT, g1, pmul(bc(-1.f), pair_of<KV>(lf2, pp))), r2);
                    } else {
                        r1 = pmul(Vt2, g1);
                        r2 = pmul(hT, r1);
                    }
                    r1 = pfma(n0, pair_of<KV>(e01, pp), r1); r2 = pfma(n0, pair_of<KV>(e02, pp), r2);
                    r1 = pfma(n1, f11, r1);                  r2 = pfma(n1, f12, r2);
                    r1 = pfma(n2, pair_of<KV>(e21, pp), r1); r2 = pfma(n2, pair_of<KV>(e22, pp), r2);
                    r1 = pfma(n3, f31, r1);                  r2 = pfma(n3, f32, r2);
                    if (kDef) {
                        r1 = pfma(pair_of<KV>(dq1, pp), bc(-1.f), r1);
                        r2 = pfma(pair_of<KV>(dq2, pp), bc(-1.f), r2);
                    }
                    const float2 iD = prcp(D);
                    const float2 x1 = pmul(r1, iD), x2 = pmul(r2, iD);
                    fn1[2 * pp] = x1.x; fn1[2 * pp + 1] = x1.y;
                    fn2[2 * pp] = x2.x; fn2[2 * pp + 1] = x2.y;
                    if (kRes) {
                        const float2 R1 = pmul(D, pfma(x1, bc(-1.f), pair_of<KV>(fo1, pp)));
                        const float2 R2 = pmul(D, pfma(x2, bc(-1.f), pair_of<KV>(fo2, pp)));
                        brs = pfma(wk, pfma(R2, R2, pmul(R1, R1)), brs);
                        if (rmom) {
                            const float2 wR = pmul(wk, R1);
                            bq0 = padd(bq0, wR);
                            bq1 = pfma(wR, vx, bq1);
                            bq2 = pfma(wR, vy, bq2);
                            bq3 = pfma(wk, R2, pfma(wR, hv, bq3));
                        }
                    }
                    const float2 wf1 = pmul(wk, x1);
                    bm0 = padd(bm0, wf1);
                    bm1 = pfma(wf1, vx, bm1);
                    bm2 = pfma(wf1, vy, bm2);
                    bm3 = pfma(wk, x2, pfma(wf1, hv, bm3));
                    if (wall) {
                        const float2 wp = pmul(wf1, padd(a3, n3));      // w f1 max(a3, 0)
                        bfw = padd(bfw, wp);
                        bj = pfma(wp, pfma(dyy, vy, pmul(dxy, vx)), bj);
                    }
                }
                stg16(fw + oc + q, PK::pack(fn1, fn2));
              }
            });
        }
        m0.add(bm0.x + bm0.y); m1.add(bm1.x + bm1.y); m2.add(bm2.x + bm2.y); m3.add(bm3.x + bm3.y);
        if (kRes) rs.add(brs.x + brs.y);
        if (rmom) { q0.add(bq0.x + bq0.y); q1.add(bq1.x + bq1.y); q2.add(bq2.x + bq2.y); q3.add(bq3.x + bq3.y); }
        if (wall) { fwa.add(bfw.x + bfw.y); ja.add(bj.x + bj.y); }
    }
    if (!ok) return false;
    const float M0 = m0.total(), M1 = m1.total(), M2 = m2.total(), M3 = m3.total();
    float RS = 0.f, FW = 0.f, JA = 0.f;
    if (kRes) RS = rs.total();
    if (rmom) {
        const float Q0 = q0.total(), Q1 = q1.total(), Q2 = q2.total(), Q3 = q3.total();
        if (lane == 0) P.rW[c] = make_double4(Q0, Q1, Q2, Q3);
    }
    if (wall) { FW = fwa.total(); JA = ja.total(); }
    if (kShard && lane == 0) {           // velocity shard: raw sums of this slice
        const size_t nc = (size_t)P.ncell;
        reinterpret_cast<double4*>(P.part)[c] = make_double4(M0, M1, M2, M3);
        const float V = P.V[c];
        P.part[4 * nc + c] = kRes ? (double)(RS / (V * V)) : 0.0;
        if (wall) {
            P.part[5 * nc + c] = (double)(FW * invA);
            P.part[5 * nc + P.ni + c] = (double)JA;
        }
    } else if (lane == 0) {
        if (kLin) {
            P.dW_new[c] = make_double4(M0, M1, M2, M3);
        } else {
            const float ir = 1.f / M0;
            const float nu1 = M1 * ir, nu2 = M2 * ir;
            const float nT = (2.f / 3.f) * (M3 * ir - 0.5f * (nu1 * nu1 + nu2 * nu2));
            P.prim_new[c] = make_double4(M0, nu1, nu2, nT);
        }
        if (kRes) {
            const float V = P.V[c];
            P.respart[c] = (double)(RS / (V * V));
        }
        if (wall) {
            P.Fw_new[c] = (double)(FW * invA);
            P.Jpart[c] = (double)JA;
        }
    }
    return true;
}

template <class TS, bool kRes, int kBnd, bool kDef, bool kShard, bool kRM>
__device__ __forceinline__ bool primal_cell(const PrimalArgs<TS, typename Pack<TS>::TC>& P, int c, int w,
                                            int lane, const Feed& F) {   // no linearised form (FP32 only)
    using PK = Pack<TS>;
    using TC = typename PK::TC;
    using TC2 = typename Vec<TC>::v2;
    using TC4 = typename Vec<TC>::v4;
    constexpr int KV = PK::KV;
    constexpr bool wall = (kBnd & kWallCell) != 0, far = (kBnd & kFarCell) != 0;
    const TC2 S0 = P.S[4 * c], S1 = P.S[4 * c + 1], S2 = P.S[4 * c + 2], S3 = P.S[4 * c + 3];
    const double4 pr = P.prim_old[c], pm = P.maxw_old[c];   // moments (tau), Maxwellian parameters (g)
    const TC rho = (TC)pm.x, u1 = (TC)pm.y, u2 = (TC)pm.z, T = (TC)pm.w;
    Gauss<TC> G;
    G.setup(rho, u1, u2, T);
    const TC halfT = TC(0.5) * T;
    const TC Vt = P.V[c] * (TC)pr.x * sqrt((TC)pr.w) * (TC)P.inv_tau_inf;        // V / tau
    TC cw1 = TC(0), cw2 = TC(0), invA = TC(0);
    if (wall) {
        cw1 = (TC)P.Fw_old[c] / (TC)P.wallD[c];
        cw2 = cw1 * P.halfTw;
        invA = TC(1) / sqrt(S3.x * S3.x + S3.y * S3.y);
    }
    uint4* fw = reinterpret_cast<uint4*>(P.f_new);
    const unsigned nq = (unsigned)P.nq, niter = (nq + kRowChunks - 1) / kRowChunks, oc = (unsigned)c * nq;

    Sum<TC> m0, m1, m2, m3, fwa, ja, rs, q0, q1, q2, q3;
    constexpr bool rmom = kRes && kRM;               // moments of the residual (macroscopic prediction)
    bool ok = true;
    unsigned it = 0;
    while (it < niter && ok) {
        TC bm0 = TC(0), bm1 = TC(0), bm2 = TC(0), bm3 = TC(0), bfw = TC(0), bj = TC(0), brs = TC(0);
        TC bq0 = TC(0), bq1 = TC(0), bq2 = TC(0), bq3 = TC(0);
        for (int b = 0; b < kBlockIters && it < niter && ok; ++b, ++it) {
            ok = pipeline_step(F, it, niter, lane, [&](const uint4* d) {
#pragma unroll
              for (int cc = 0; cc < kCPL; ++cc) {
                const unsigned q = it * kRowChunks + cc * 32 + lane;
                if (q >= nq) break;
                const uint4* e = d + cc * 32 + lane;
                const uint4 ro = e[(w + 1) * kRowChunks];
                const uint4 r0 = e[(10 + w) * kRowChunks], r2 = e[(18 + w) * kRowChunks];
                const uint4 r1 = far ? ro : e[(w + 2) * kRowChunks];
                const uint4 r3 = wall ? ro : e[w * kRowChunks];
                TC fo1[KV], fo2[KV], e01[KV], e02[KV], e11[KV], e12[KV], e21[KV], e22[KV], e31[KV], e32[KV];
                PK::unpack(ro, fo1, fo2);
                PK::unpack(r0, e01, e02);
                PK::unpack(r1, e11, e12);
                PK::unpack(r2, e21, e22);
                PK::unpack(r3, e31, e32);
                TC dq1[KV], dq2[KV];
                if (kDef) PK::unpack(ldg16(reinterpret_cast<const uint4*>(P.defect) + oc + q), dq1, dq2);
                TC fn1[KV], fn2[KV];
#pragma unroll
                for (int kk = 0; kk < KV; ++kk) {
                    const int k = q * KV + kk;
                    const TC4 t = P.vt[k];
                    const TC vx = t.x, vy = t.y, wk = t.z, hv = t.w;
                    const TC a0 = S0.x * vx + S0.y * vy, a1 = S1.x * vx + S1.y * vy;
                    const TC a2 = S2.x * vx + S2.y * vy, a3 = S3.x * vx + S3.y * vy;
                    if (far) { const TC2 fd = P.fd[k]; e11[kk] = fd.x; e12[kk] = fd.y; }
                    if (wall) { const TC gw = P.gw[k]; e31[kk] = cw1 * gw; e32[kk] = cw2 * gw; }
                    const TC D = Vt + TC(0.5) * ((fabs(a0) + fabs(a1)) + (fabs(a2) + fabs(a3)));
                    const TC g1 = G.eval(fma(vy, -u2, fma(vx, -u1, hv)));
                    TC r1_ = Vt * g1;
                    TC r2_ = halfT * r1_;
                    const TC b0 = fmin(a0, TC(0)), b1 = fmin(a1, TC(0)), b2 = fmin(a2, TC(0)), b3 = fmin(a3, TC(0));
                    r1_ -= b0 * e01[kk]; r2_ -= b0 * e02[kk];
                    r1_ -= b1 * e11[kk]; r2_ -= b1 * e12[kk];
                    r1_ -= b2 * e21[kk]; r2_ -= b2 * e22[kk];
                    r1_ -= b3 * e31[kk]; r2_ -= b3 * e32[kk];
                    if (kDef) { r1_ -= dq1[kk]; r2_ -= dq2[kk]; }
                    const TC iD = frcp<TC>(D);
                    fn1[kk] = r1_ * iD;
                    fn2[kk] = r2_ * iD;
                    if (kRes) {
                        const TC R1 = D * (fo1[kk] - fn1[kk]), R2 = D * (fo2[kk] - fn2[kk]);
                        brs += wk * (R1 * R1 + R2 * R2);
                        if (rmom) {
                            const TC wR = wk * R1;
                            bq0 += wR; bq1 += wR * vx; bq2 += wR * vy; bq3 += wR * hv + wk * R2;
                        }
                    }
                    const TC wf1 = wk * fn1[kk];
                    bm0 += wf1;
                    bm1 += wf1 * vx;
                    bm2 += wf1 * vy;
                    bm3 += wf1 * hv + wk * fn2[kk];
                    if (wall) {
                        const TC p3 = a3 - b3;                   // max(a3, 0)
                        bfw += wf1 * p3;
                        bj += wf1 * p3 * (P.dirx * vx + P.diry * vy);
                    }
                }
                stg16(fw + oc + q, PK::pack(fn1, fn2));
              }
            });
        }
        m0.add(bm0); m1.add(bm1); m2.add(bm2); m3.add(bm3);
        if (kRes) rs.add(brs);
        if (rmom) { q0.add(bq0); q1.add(bq1); q2.add(bq2); q3.add(bq3); }
        if (wall) { fwa.add(bfw); ja.add(bj); }
    }
    if (!ok) return false;
    const TC M0 = m0.total(), M1 = m1.total(), M2 = m2.total(), M3 = m3.total();
    TC RS = TC(0), FW = TC(0), JA = TC(0);
    if (kRes) RS = rs.total();
    if (rmom) {
        const TC Q0 = q0.total(), Q1 = q1.total(), Q2 = q2.total(), Q3 = q3.total();
        if (lane == 0) P.rW[c] = make_double4(Q0, Q1, Q2, Q3);
    }
    if (wall) { FW = fwa.total(); JA = ja.total(); }
    if (kShard && lane == 0) {           // velocity shard: raw sums of this slice
        const size_t nc = (size_t)P.ncell;
        reinterpret_cast<double4*>(P.part)[c] = make_double4(M0, M1, M2, M3);
        const TC V = P.V[c];
        P.part[4 * nc + c] = kRes ? (double)(RS / (V * V)) : 0.0;
        if (wall) {
            P.part[5 * nc + c] = (double)(FW * invA);
            P.part[5 * nc + P.ni + c] = (double)JA;
        }
    } else if (lane == 0) {
        const TC ir = TC(1) / M0;
        const TC nu1 = M1 * ir, nu2 = M2 * ir;
        const TC nT = TC(2.0 / 3.0) * (M3 * ir - TC(0.5) * (nu1 * nu1 + nu2 * nu2));
        P.prim_new[c] = make_double4(M0, nu1, nu2, nT);
        if (kRes) {
            const TC V = P.V[c];
            P.respart[c] = (double)(RS / (V * V));
        }
        if (wall) {
            P.Fw_new[c] = (double)(FW * invA);
            P.Jpart[c] = (double)JA;
        }
    }
    return true;
}

// Velocity pairs per stage row staged with the distribution (paired FP32 arithmetic only).
template <class TS> constexpr unsigned kVpRow = kPaired<TS> ? kRowChunks * (Pack<TS>::KV / 2) : 0;
template <class TS> constexpr int primal_smem_bytes() {
    return kStages * (kPrimalRows * kRowChunks + 2 * kVpRow<TS>) * 16 + 2 * kStages * 8;
}
template <class TS> constexpr int adjoint_smem_bytes() {
    return kStages * (kAdjointRows * kRowChunks + 2 * kVpRow<TS>) * 16 + 2 * kStages * 8;
}

// Block prologue/epilogue shared by both sweeps: barriers, active warps, the first
// stages and, on exit, the drain of copies still in flight.
struct BlockPipe {
    Feed F;
    unsigned niter;
    int A;                        // active warps (cells j0 .. j0+A-1 exist)
};

__device__ __forceinline__ bool block_pipe_setup(BlockPipe& B, unsigned char* smem, int rows, int nj, int ni,
                                                 unsigned nq, const CUtensorMap* col, const CUtensorMap* side,
                                                 const CUtensorMap* extra, int i, int j0, const float4* vpa,
                                                 const float4* vpb, unsigned vprow) {
    B.A = min(kWarpsPerBlock, nj - j0);
    B.niter = (nq + kRowChunks - 1) / kRowChunks;
    B.F.col = col; B.F.side = side; B.F.extra = extra;
    B.F.i = i; B.F.im = (i - 1 + ni) % ni; B.F.ip = (i + 1) % ni; B.F.j0 = j0; B.F.rows = rows;
    B.F.A = (unsigned)B.A;
    B.F.vpa = vpa; B.F.vpb = vpb; B.F.vprow = vprow;
    B.F.stride = (unsigned)rows * kRowChunks + 2u * vprow;
    B.F.stage = reinterpret_cast<uint4*>(smem);
    B.F.full = reinterpret_cast<uint64_t*>(smem + (size_t)kStages * B.F.stride * 16);
    B.F.released = reinterpret_cast<unsigned*>(B.F.full + kStages);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&B.F.full[s], 1);
            B.F.released[s] = 0u;
        }
        fence_mbar_init();
        for (unsigned it = 0; it < min((unsigned)kStages, B.niter); ++it) B.F.issue(it);
    }
    __syncthreads();
    return (int)(threadIdx.x >> 5) < B.A;
}

// Drain after an aborted sweep: every warp waits (bounded) for the copies it may have issued.
__device__ __forceinline__ void block_pipe_drain(const BlockPipe& B) {
    for (int s = 0; s < kStages; ++s)
        for (unsigned ph = 0; ph < 2; ++ph) mbar_try_wait(&B.F.full[s], ph);
}

template <class TS, bool kRes, bool kDef, bool kLin = false, bool kShard = false, bool kRM = false>
__device__ __forceinline__ void primal_block(const PrimalArgs<TS, typename Pack<TS>::TC>& P, const CUtensorMap* m10,
                                             const CUtensorMap* m8, int i, int j0, unsigned char* smem) {
    BlockPipe B;
    if (!block_pipe_setup(B, smem, kPrimalRows, P.nj, P.ni, (unsigned)P.nq, m10, m8, nullptr, i, j0, P.vpa, P.vpb,
                          kVpRow<TS>))
        return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = j0 + w, c = j * P.ni + i;
    const int bnd = (j == 0 ? kWallCell : 0) | (j == P.nj - 1 ? kFarCell : 0);
    bool ok;
    if constexpr (kPaired<TS>) {
        switch (bnd) {
            case kInterior: ok = primal_cell_paired<TS, kRes, kInterior, kDef, kLin, kShard, kRM>(P, c, w, lane, B.F); break;
            case kWallCell: ok = primal_cell_paired<TS, kRes, kWallCell, kDef, kLin, kShard, kRM>(P, c, w, lane, B.F); break;
            case kFarCell: ok = primal_cell_paired<TS, kRes, kFarCell, kDef, kLin, kShard, kRM>(P, c, w, lane, B.F); break;
            default: ok = primal_cell_paired<TS, kRes, kWallFar, kDef, kLin, kShard, kRM>(P, c, w, lane, B.F); break;
        }
    } else {
        static_assert(!kLin, "the linearised sweep has the paired FP32 form only");
        switch (bnd) {
            case kInterior: ok = primal_cell<TS, kRes, kInterior, kDef, kShard, kRM>(P, c, w, lane, B.F); break;
            case kWallCell: ok = primal_cell<TS, kRes, kWallCell, kDef, kShard, kRM>(P, c, w, lane, B.F); break;
            case kFarCell: ok = primal_cell<TS, kRes, kFarCell, kDef, kShard, kRM>(P, c, w, lane, B.F); break;
            default: ok = primal_cell<TS, kRes, kWallFar, kDef, kShard, kRM>(P, c, w, lane, B.F); break;
        }
    }
    if (!ok && lane == 0) {
        atomicExch(P.err, 1);
        block_pipe_drain(B);
    }
}


template <class TS, bool kRes, bool kDef>
__global__ void __launch_bounds__(256, kPrimalMinBlocks<TS>) k_primal_sweep(const PrimalArgs<TS, typename Pack<TS>::TC> P,
                                                         const __grid_constant__ CUtensorMap m10,
                                                         const __grid_constant__ CUtensorMap m8) {
    extern __shared__ __align__(1024) unsigned char smem[];
    primal_block<TS, kRes, kDef>(P, &m10, &m8, blockIdx.x, blockIdx.y * kWarpsPerBlock, smem);
}

// Residual sweep of a prediction block: the same update, which also writes the moments of its input's
// residual, sum_k w Psi_k R_k, per cell to P.rW (see k_coarse_assemble).
template <class TS>
__global__ void __launch_bounds__(256, 2) k_primal_sweep_rm(const PrimalArgs<TS, typename Pack<TS>::TC> P,
                                                            const __grid_constant__ CUtensorMap m10,
                                                            const __grid_constant__ CUtensorMap m8) {
    extern __shared__ __align__(1024) unsigned char smem[];
    primal_block<TS, true, false, false, false, true>(P, &m10, &m8, blockIdx.x, blockIdx.y * kWarpsPerBlock, smem);
}

// Sweep of a velocity shard: the same update, with the raw velocity sums of the slice written to the
// shard buffer in place of the moments, wall density, drag and residual partials.
template <class TS, bool kRes>
__global__ void __launch_bounds__(256, 2) k_primal_shard_sweep(const PrimalArgs<TS, typename Pack<TS>::TC> P,
                                                               const __grid_constant__ CUtensorMap m10,
                                                               const __grid_constant__ CUtensorMap m8) {
    extern __shared__ __align__(1024) unsigned char smem[];
    primal_block<TS, kRes, false, false, true>(P, &m10, &m8, blockIdx.x, blockIdx.y * kWarpsPerBlock, smem);
}

// Linearised correction sweep of the refinement (FP32 storage; see primal_cell_paired).
template <bool kRes, bool kRM>
__global__ void __launch_bounds__(256, 2) k_primal_lin_sweep(const PrimalArgs<float, float> P,
                                                                const __grid_constant__ CUtensorMap m10,
                                                                const __grid_constant__ CUtensorMap m8) {
    extern __shared__ __align__(1024) unsigned char smem[];
    primal_block<float, kRes, false, true, false, kRM>(P, &m10, &m8, blockIdx.x, blockIdx.y * kWarpsPerBlock, smem);
}

// Make the tensor maps of a descriptor in global memory visible to the tensor-map proxy.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* m) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
}

// Batched primal sweep: block b runs work item items[b] = (request, i, j0) of the descriptor
// table; every request advances one sweep.  parity selects, per request, the buffer pair of this
// sweep (descriptor slot 0 reads the buffer current at the start of the tick).  The grid is the
// table's capacity and *count (device memory) the items in use, so one launch shape, and one captured
// graph, serves any admitted set that fits the capacity; blocks beyond the count return at once.
template <class TS, bool kRes>
__global__ void __launch_bounds__(256, kPrimalMinBlocks<TS>) k_primal_sweep_batch(const PrimalBatchDesc<TS>* __restrict__ descs,
                                                               const int4* __restrict__ items, const int* __restrict__ count,
                                                               int parity) {
    extern __shared__ __align__(1024) unsigned char smem[];
    if ((int)blockIdx.x >= *count) return;
    const int4 it = items[blockIdx.x];
    const PrimalBatchDesc<TS>* d = descs + it.x;
    if (threadIdx.x == 0) {
        tensormap_acquire(&d->maps[parity].col);
        tensormap_acquire(&d->maps[parity].side);
    }
    primal_block<TS, kRes, false>(d->args[parity], &d->maps[parity].col, &d->maps[parity].side, it.y, it.z, smem);
}

// ================================================================== adjoint sweep (K2)
// Transposed (downwind) point-implicit sweep of the discrete adjoint of Eq. (numerad_gov):
//   D phi = -dJ/df/w + sum_{a>0, interior} a phi_nb + Z . Psi - [wall, a>0] (v.n) Lambda
// Z = (V/tau) What - V rhohat' d(1/tau)/dW collects the linearised collision terms
// (Eq. adjoint_eqdefines / adjoint_macdefines) of the previous sweep; it is rebuilt here from
// the new phi: What = J_P^T Phat with Phat = sum_k w (phi1 dg1/dp + phi2 dg2/dp), p = (rho,u,T),
// and rhohat' = sum_k w phi . (f - g).  Lambda = sum_{a<=0} w a phi . gbar_w (Eq. formula_adjointbgk).
// Z with the conservative Maxwellian: the Maxwellian part p_g (derivatives with respect to the fitted
// parameters) maps to W through dp/dW = (dM/dp)^{-1} (K, row-major [q][m]), the relaxation-time part
// (a, b) = d/d(rho, T) of the physical moments through J_P.
__device__ __forceinline__ double4 z_fitted(const double* K, double g0, double g1, double g2, double g3,
                                            double a, double b, double j30, double j31, double j32, double j33) {
    double4 z;
    z.x = a + b * j30 + K[0] * g0 + K[4] * g1 + K[8] * g2 + K[12] * g3;
    z.y = b * j31 + K[1] * g0 + K[5] * g1 + K[9] * g2 + K[13] * g3;
    z.z = b * j32 + K[2] * g0 + K[6] * g1 + K[10] * g2 + K[14] * g3;
    z.w = b * j33 + K[3] * g0 + K[7] * g1 + K[11] * g2 + K[15] * g3;
    return z;
}

// The per-cell constants of the linearisation (Maxwellian parameters, V/tau, J_P, d(1/tau)/dp)
// come precomputed in AdjCell.  kUpdate = false: phi is not advanced; the couplings of phi_old are
// written to the *_new slots (used after an upload of phi or a change of the primal state).
// FP32 / BF16 form of the adjoint sweep, two velocities at a time.  D uses the outflow weights
// max(a_e, 0) directly; the Maxwellian is accumulated as exp(-c^2/2T) = 2^(c^2 kE) and its factor
// n0 applied to the block sums (every coupling is linear in g1).
template <class TS, bool kUpdate, bool kRes, int kBnd, bool kDef>
__device__ __forceinline__ bool adjoint_cell_paired(const AdjointArgs<TS, float>& P, int c, int w, int lane,
                                                    const Feed& F) {
    using PK = Pack<TS>;
    constexpr int KV = PK::KV, NP = KV / 2;
    constexpr bool wall = (kBnd & kWallCell) != 0, far = (kBnd & kFarCell) != 0;
    constexpr float L2E = 1.44269504088896341f;
    const float2 S0 = P.S[4 * c], S1 = P.S[4 * c + 1], S2 = P.S[4 * c + 2], S3 = P.S[4 * c + 3];
    const AdjCell<float>* ccp = P.cell + c;
    const float u1 = __ldg(&ccp->u1), u2 = __ldg(&ccp->u2), n0 = __ldg(&ccp->n0), inv2T = __ldg(&ccp->inv2T);
    const float halfT = __ldg(&ccp->halfT), Vt = __ldg(&ccp->Vt);
    const double4 Z = P.Z_old[c];
    const float2 z0 = bc((float)Z.x), z1 = bc((float)Z.y), z2 = bc((float)Z.z), z3 = bc((float)Z.w);
    const float2 mu1 = bc(-u1), mu2 = bc(-u2), hT = bc(halfT), Vt2 = bc(Vt);
    const float2 kE = bc(-inv2T * L2E);
    const float2 s0x = bc(S0.x), s0y = bc(S0.y), s1x = bc(S1.x), s1y = bc(S1.y);
    const float2 s2x = bc(S2.x), s2y = bc(S2.y), s3x = bc(S3.x), s3y = bc(S3.y);
    float2 ndx = bc(0.f), ndy = bc(0.f), nhc = bc(0.f), nsrc = bc(0.f), gbw = bc(0.f), hTw = bc(0.f);
    if (wall) {
        const float A = sqrtf(S3.x * S3.x + S3.y * S3.y);
        ndx = bc(-P.dirx);
        ndy = bc(-P.diry);
        nhc = bc(-P.heat);
        nsrc = bc(-(float)(P.wallM[c] + P.Lam_old[c]) / A);          // (M + Lambda)/A multiplies a3
        gbw = bc(1.f / (float)P.wallD[c]);
        hTw = bc(P.halfTw);
    }
    uint4* pw = reinterpret_cast<uint4*>(P.phi_new);
    const unsigned nq = (unsigned)P.nq, niter = (nq + kRowChunks - 1) / kRowChunks, oc = (unsigned)c * nq;

    Sum<float> sh, shx, shy, shc, sg2, sr, lam, rs;
    bool ok = true;
    unsigned it = 0;
    while (it < niter && ok) {
        float2 bh = bc(0.f), bhx = bh, bhy = bh, bhc = bh, bg2 = bh, bwf = bh, bl = bh, brs = bh;
        for (int b = 0; b < kBlockIters && it < niter && ok; ++b, ++it) {
            ok = pipeline_step(F, it, niter, lane, [&](const uint4* d) {
#pragma unroll
              for (int cc = 0; cc < kCPL; ++cc) {
                const unsigned q = it * kRowChunks + cc * 32 + lane;
                if (q >= nq) break;
                const uint4* e = d + cc * 32 + lane;
                const uint4 ro = e[(w + 1) * kRowChunks], rf = e[(26 + w) * kRowChunks];
                uint4 r0 = ro, r1 = ro, r2 = ro, r3 = ro;
                if (kUpdate) {
                    r0 = e[(10 + w) * kRowChunks];
                    r2 = e[(18 + w) * kRowChunks];
                    if (!far) r1 = e[(w + 2) * kRowChunks];
                    if (!wall) r3 = e[w * kRowChunks];
                }
                float po1[KV], po2[KV], f1[KV], f2[KV], e01[KV], e02[KV], e11[KV], e12[KV], e21[KV], e22[KV],
                    e31[KV], e32[KV];
                PK::unpack(ro, po1, po2);
                PK::unpack(rf, f1, f2);
                PK::unpack(r0, e01, e02);
                PK::unpack(r1, e11, e12);
                PK::unpack(r2, e21, e22);
                PK::unpack(r3, e31, e32);
                float dq1[KV], dq2[KV];
                if (kDef) PK::unpack(ldg16(reinterpret_cast<const uint4*>(P.defect) + oc + q), dq1, dq2);
                float pn1[KV], pn2[KV];
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) {
                    const int kp = q * NP + pp;
                    const int lp = (cc * 32 + lane) * NP + pp;
                    const float4* sA = reinterpret_cast<const float4*>(d + F.rows * kRowChunks);
                    const float4 A = sA[lp], B = sA[F.vprow + lp];
                    const float2 vx = make_float2(A.x, A.y), vy = make_float2(A.z, A.w);
                    const float2 wk = make_float2(B.x, B.y), hv = make_float2(B.z, B.w);
                    const float2 a3 = pfma(s3y, vy, pmul(s3x, vx));
                    float2 x1 = pair_of<KV>(po1, pp), x2 = pair_of<KV>(po2, pp);
                    if (kUpdate) {
                        const float2 a0 = pfma(s0y, vy, pmul(s0x, vx)), a1 = pfma(s1y, vy, pmul(s1x, vx));
                        const float2 a2 = pfma(s2y, vy, pmul(s2x, vx));
                        const float2 o0 = inflow(make_float2(-a0.x, -a0.y)), o1 = inflow(make_float2(-a1.x, -a1.y));
                        const float2 o2 = inflow(make_float2(-a2.x, -a2.y)), o3 = inflow(make_float2(-a3.x, -a3.y));
                        const float2 D = padd(Vt2, padd(padd(o0, o1), padd(o2, o3)));
                        float2 r1 = pfma(z3, hv, pfma(z2, vy, pfma(z1, vx, z0)));
                        float2 r2 = z3;
                        r1 = pfma(o0, pair_of<KV>(e01, pp), r1); r2 = pfma(o0, pair_of<KV>(e02, pp), r2);
                        r1 = pfma(o2, pair_of<KV>(e21, pp), r1); r2 = pfma(o2, pair_of<KV>(e22, pp), r2);
                        if (!far) { r1 = pfma(o1, pair_of<KV>(e11, pp), r1); r2 = pfma(o1, pair_of<KV>(e12, pp), r2); }
                        if (wall) r1 = pfma(o3, pfma(nhc, hv, pfma(ndy, vy, pfma(ndx, vx, nsrc))), r1);
                        else { r1 = pfma(o3, pair_of<KV>(e31, pp), r1); r2 = pfma(o3, pair_of<KV>(e32, pp), r2); }
                        if (kDef) {
                            r1 = pfma(pair_of<KV>(dq1, pp), bc(-1.f), r1);
                            r2 = pfma(pair_of<KV>(dq2, pp), bc(-1.f), r2);
                        }
                        const float2 iD = prcp(D);
                        const float2 y1 = pmul(r1, iD), y2 = pmul(r2, iD);
                        if (kRes) {
                            const float2 R1 = pmul(D, pfma(y1, bc(-1.f), x1));
                            const float2 R2 = pmul(D, pfma(y2, bc(-1.f), x2));
                            brs = pfma(wk, pfma(R2, R2, pmul(R1, R1)), brs);
                        }
                        x1 = y1;
                        x2 = y2;
                    }
                    pn1[2 * pp] = x1.x; pn1[2 * pp + 1] = x1.y;
                    pn2[2 * pp] = x2.x; pn2[2 * pp + 1] = x2.y;
                    // couplings of the next sweep, from the new phi
                    const float2 dx = padd(vx, mu1), dy = padd(vy, mu2);
                    const float2 c2 = pfma(dy, dy, pmul(dx, dx));
                    const float2 wg1 = pmul(wk, pex2(pmul(c2, kE)));          // g1 / n0
                    const float2 h = pmul(wg1, pfma(hT, x2, x1));
                    bh = padd(bh, h);
                    bhx = pfma(h, dx, bhx);
                    bhy = pfma(h, dy, bhy);
                    bhc = pfma(h, c2, bhc);
                    bg2 = pfma(wg1, x2, bg2);
                    bwf = pfma(wk, pfma(x2, pair_of<KV>(f2, pp), pmul(x1, pair_of<KV>(f1, pp))), bwf);
                    if (wall) {
                        const float2 gw = *reinterpret_cast<const float2*>(P.gw + 2 * kp);
                        const float2 in3 = inflow(a3);                       // -min(a3, 0)
                        bl = pfma(pmul(pmul(wk, in3), pmul(gw, gbw)), pfma(hTw, x2, x1), bl);
                    }
                }
                if (kUpdate) stg16(pw + oc + q, PK::pack(pn1, pn2));
              }
            });
        }
        const float bhs = n0 * (bh.x + bh.y);
        sh.add(bhs); shx.add(n0 * (bhx.x + bhx.y)); shy.add(n0 * (bhy.x + bhy.y)); shc.add(n0 * (bhc.x + bhc.y));
        sg2.add(n0 * (bg2.x + bg2.y)); sr.add((bwf.x + bwf.y) - bhs);
        if (kRes) rs.add(brs.x + brs.y);
        if (wall) lam.add(-(bl.x + bl.y));
    }
    if (!ok) return false;
    const float Sh = sh.total(), Shx = shx.total(), Shy = shy.total(), Shc = shc.total();
    const float Sg2 = sg2.total(), Sr = sr.total();
    float RS = 0.f, LAM = 0.f;
    if (kRes) RS = rs.total();
    if (wall) LAM = lam.total();
    if (lane == 0) {
        const AdjCell<float> cc = *ccp;
        const float ph0 = Sh * cc.irg, ph1 = Shx * cc.iT, ph2 = Shy * cc.iT;
        const float ph3 = Shc * cc.iT2h - Sh * cc.iT + 0.5f * Sg2;
        double4 zn;
        if (P.Kinv) {
            zn = z_fitted(P.Kinv + 16 * (size_t)c, Vt * ph0, Vt * ph1, Vt * ph2, Vt * ph3, -Sr * cc.c0,
                          -Sr * cc.c3, cc.j30, cc.j31, cc.j32, cc.j33);
        } else {
            const float p0 = Vt * ph0 - Sr * cc.c0, p1 = Vt * ph1, p2 = Vt * ph2, p3 = Vt * ph3 - Sr * cc.c3;
            zn.x = (double)(p0 - (p1 * u1 + p2 * u2) * cc.ir + p3 * cc.j30);
            zn.y = (double)(p1 * cc.ir + p3 * cc.j31);
            zn.z = (double)(p2 * cc.ir + p3 * cc.j32);
            zn.w = (double)(p3 * cc.j33);
        }
        P.Z_new[c] = zn;
        if (kRes) {
            const float V = P.V[c];
            P.respart[c] = (double)(RS / (V * V));
        }
        if (wall) P.Lam_new[c] = (double)LAM;
    }
    return true;
}

template <class TS, bool kUpdate, bool kRes, int kBnd, bool kDef>
__device__ __forceinline__ bool adjoint_cell(const AdjointArgs<TS, typename Pack<TS>::TC>& P, int c, int w,
                                             int lane, const Feed& F) {
    using PK = Pack<TS>;
    using TC = typename PK::TC;
    using TC2 = typename Vec<TC>::v2;
    using TC4 = typename Vec<TC>::v4;
    constexpr int KV = PK::KV;
    constexpr bool wall = (kBnd & kWallCell) != 0, far = (kBnd & kFarCell) != 0;
    const TC2 S0 = P.S[4 * c], S1 = P.S[4 * c + 1], S2 = P.S[4 * c + 2], S3 = P.S[4 * c + 3];
    const AdjCell<TC>* ccp = P.cell + c;
    const TC u1 = __ldg(&ccp->u1), u2 = __ldg(&ccp->u2), n0 = __ldg(&ccp->n0), inv2T = __ldg(&ccp->inv2T);
    const TC halfT = __ldg(&ccp->halfT), Vt = __ldg(&ccp->Vt);
    const double4 Z = P.Z_old[c];
    const TC z0 = (TC)Z.x, z1 = (TC)Z.y, z2 = (TC)Z.z, z3 = (TC)Z.w;
    TC gb1s = TC(0), srcB = TC(0);
    if (wall) {
        const TC A = sqrt(S3.x * S3.x + S3.y * S3.y);
        gb1s = TC(1) / (TC)P.wallD[c];
        srcB = (TC)((P.wallM[c] + P.Lam_old[c])) / A;             // (M + Lambda)/A multiplies a3
    }
    uint4* pw = reinterpret_cast<uint4*>(P.phi_new);
    const unsigned nq = (unsigned)P.nq, niter = (nq + kRowChunks - 1) / kRowChunks, oc = (unsigned)c * nq;

    Sum<TC> sh, shx, shy, shc, sg2, sr, lam, rs;
    bool ok = true;
    unsigned it = 0;
    while (it < niter && ok) {
        TC bh = TC(0), bhx = TC(0), bhy = TC(0), bhc = TC(0), bg2 = TC(0), br = TC(0), bl = TC(0), brs = TC(0);
        for (int b = 0; b < kBlockIters && it < niter && ok; ++b, ++it) {
            ok = pipeline_step(F, it, niter, lane, [&](const uint4* d) {
#pragma unroll
              for (int cc = 0; cc < kCPL; ++cc) {
                const unsigned q = it * kRowChunks + cc * 32 + lane;
                if (q >= nq) break;
                const uint4* e = d + cc * 32 + lane;
                const uint4 ro = e[(w + 1) * kRowChunks], rf = e[(26 + w) * kRowChunks];
                uint4 r0 = ro, r1 = ro, r2 = ro, r3 = ro;
                if (kUpdate) {
                    r0 = e[(10 + w) * kRowChunks];
                    r2 = e[(18 + w) * kRowChunks];
                    if (!far) r1 = e[(w + 2) * kRowChunks];
                    if (!wall) r3 = e[w * kRowChunks];
                }
                TC po1[KV], po2[KV], f1[KV], f2[KV], e01[KV], e02[KV], e11[KV], e12[KV], e21[KV], e22[KV],
                    e31[KV], e32[KV];
                PK::unpack(ro, po1, po2);
                PK::unpack(rf, f1, f2);
                PK::unpack(r0, e01, e02);
                PK::unpack(r1, e11, e12);
                PK::unpack(r2, e21, e22);
                PK::unpack(r3, e31, e32);
                TC dq1[KV], dq2[KV];
                if (kDef) PK::unpack(ldg16(reinterpret_cast<const uint4*>(P.defect) + oc + q), dq1, dq2);
                TC pn1[KV], pn2[KV];
#pragma unroll
                for (int kk = 0; kk < KV; ++kk) {
                    const int k = q * KV + kk;
                    const TC4 t = P.vt[k];
                    const TC vx = t.x, vy = t.y, wk = t.z, hv = t.w;
                    const TC a3 = S3.x * vx + S3.y * vy;
                    if (kUpdate) {
                        const TC a0 = S0.x * vx + S0.y * vy, a1 = S1.x * vx + S1.y * vy;
                        const TC a2 = S2.x * vx + S2.y * vy;
                        const TC D = Vt + TC(0.5) * ((fabs(a0) + fabs(a1)) + (fabs(a2) + fabs(a3)));
                        TC r1_ = z0 + z1 * vx + z2 * vy + z3 * hv;
                        TC r2_ = z3;
                        const TC p0 = fmax(a0, TC(0)), p2 = fmax(a2, TC(0)), p3 = fmax(a3, TC(0));
                        r1_ += p0 * e01[kk]; r2_ += p0 * e02[kk];
                        r1_ += p2 * e21[kk]; r2_ += p2 * e22[kk];
                        if (!far) { const TC p1 = fmax(a1, TC(0)); r1_ += p1 * e11[kk]; r2_ += p1 * e12[kk]; }
                        if (wall) r1_ -= p3 * (P.dirx * vx + P.diry * vy + P.heat * hv + srcB);
                        else { r1_ += p3 * e31[kk]; r2_ += p3 * e32[kk]; }
                        if (kDef) { r1_ -= dq1[kk]; r2_ -= dq2[kk]; }
                        const TC iD = frcp<TC>(D);
                        pn1[kk] = r1_ * iD;
                        pn2[kk] = r2_ * iD;
                        if (kRes) {
                            const TC R1 = D * (po1[kk] - pn1[kk]), R2 = D * (po2[kk] - pn2[kk]);
                            brs += wk * (R1 * R1 + R2 * R2);
                        }
                    } else {
                        pn1[kk] = po1[kk];
                        pn2[kk] = po2[kk];
                    }
                    // couplings of the next sweep, from the new phi
                    const TC dx = vx - u1, dy = vy - u2, c2 = dx * dx + dy * dy;
                    const TC wg1 = wk * n0 * fexp<TC>(-c2 * inv2T);
                    const TC h = wg1 * (pn1[kk] + halfT * pn2[kk]);
                    bh += h;
                    bhx += h * dx;
                    bhy += h * dy;
                    bhc += h * c2;
                    bg2 += wg1 * pn2[kk];
                    br += wk * (pn1[kk] * f1[kk] + pn2[kk] * f2[kk]) - h;     // w phi.(f - g)
                    if (wall) bl += wk * fmin(a3, TC(0)) * P.gw[k] * gb1s * (pn1[kk] + P.halfTw * pn2[kk]);
                }
                if (kUpdate) stg16(pw + oc + q, PK::pack(pn1, pn2));
              }
            });
        }
        sh.add(bh); shx.add(bhx); shy.add(bhy); shc.add(bhc); sg2.add(bg2); sr.add(br);
        if (kRes) rs.add(brs);
        if (wall) lam.add(bl);
    }
    if (!ok) return false;
    const TC Sh = sh.total(), Shx = shx.total(), Shy = shy.total(), Shc = shc.total();
    const TC Sg2 = sg2.total(), Sr = sr.total();
    TC RS = TC(0), LAM = TC(0);
    if (kRes) RS = rs.total();
    if (wall) LAM = lam.total();
    if (lane == 0) {
        const AdjCell<TC> cc = *ccp;   // epilogue-only constants, loaded after the loop
        // Phat in primitive variables, then p = (V/tau) Phat - V rhohat' d(1/tau)/dp, Z = J_P^T p
        const TC ph0 = Sh * cc.irg, ph1 = Shx * cc.iT, ph2 = Shy * cc.iT;
        const TC ph3 = Shc * cc.iT2h - Sh * cc.iT + TC(0.5) * Sg2;
        double4 zn;
        if (P.Kinv) {
            zn = z_fitted(P.Kinv + 16 * (size_t)c, Vt * ph0, Vt * ph1, Vt * ph2, Vt * ph3, -Sr * cc.c0,
                          -Sr * cc.c3, cc.j30, cc.j31, cc.j32, cc.j33);
        } else {
            const TC p0 = Vt * ph0 - Sr * cc.c0, p1 = Vt * ph1, p2 = Vt * ph2, p3 = Vt * ph3 - Sr * cc.c3;
            zn.x = (double)(p0 - (p1 * u1 + p2 * u2) * cc.ir + p3 * cc.j30);
            zn.y = (double)(p1 * cc.ir + p3 * cc.j31);
            zn.z = (double)(p2 * cc.ir + p3 * cc.j32);
            zn.w = (double)(p3 * cc.j33);
        }
        P.Z_new[c] = zn;
        if (kRes) {
            const TC V = P.V[c];
            P.respart[c] = (double)(RS / (V * V));
        }
        if (wall) P.Lam_new[c] = (double)LAM;
    }
    return true;
}

template <class TS, bool kUpdate, bool kRes, bool kDef>
__device__ __forceinline__ void adjoint_block(const AdjointArgs<TS, typename Pack<TS>::TC>& P, const CUtensorMap* m10,
                                              const CUtensorMap* m8, const CUtensorMap* mf8, int i, int j0,
                                              unsigned char* smem) {
    BlockPipe B;
    if (!block_pipe_setup(B, smem, kAdjointRows, P.nj, P.ni, (unsigned)P.nq, m10, m8, mf8, i, j0, P.vpa, P.vpb,
                          kVpRow<TS>))
        return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = j0 + w, c = j * P.ni + i;
    const int bnd = (j == 0 ? kWallCell : 0) | (j == P.nj - 1 ? kFarCell : 0);
    bool ok;
    if constexpr (kPaired<TS>) {
        switch (bnd) {
            case kInterior: ok = adjoint_cell_paired<TS, kUpdate, kRes, kInterior, kDef>(P, c, w, lane, B.F); break;
            case kWallCell: ok = adjoint_cell_paired<TS, kUpdate, kRes, kWallCell, kDef>(P, c, w, lane, B.F); break;
            case kFarCell: ok = adjoint_cell_paired<TS, kUpdate, kRes, kFarCell, kDef>(P, c, w, lane, B.F); break;
            default: ok = adjoint_cell_paired<TS, kUpdate, kRes, kWallFar, kDef>(P, c, w, lane, B.F); break;
        }
    } else {
        switch (bnd) {
            case kInterior: ok = adjoint_cell<TS, kUpdate, kRes, kInterior, kDef>(P, c, w, lane, B.F); break;
            case kWallCell: ok = adjoint_cell<TS, kUpdate, kRes, kWallCell, kDef>(P, c, w, lane, B.F); break;
            case kFarCell: ok = adjoint_cell<TS, kUpdate, kRes, kFarCell, kDef>(P, c, w, lane, B.F); break;
            default: ok = adjoint_cell<TS, kUpdate, kRes, kWallFar, kDef>(P, c, w, lane, B.F); break;
        }
    }
    if (!ok && lane == 0) {
        atomicExch(P.err, 1);
        block_pipe_drain(B);
    }
}

template <class TS, bool kUpdate, bool kRes, bool kDef>
__global__ void __launch_bounds__(256, kAdjointMinBlocks<TS>) k_adjoint_sweep(const AdjointArgs<TS, typename Pack<TS>::TC> P,
                                                          const __grid_constant__ CUtensorMap m10,
                                                          const __grid_constant__ CUtensorMap m8,
                                                          const __grid_constant__ CUtensorMap mf8) {
    extern __shared__ __align__(1024) unsigned char smem[];
    adjoint_block<TS, kUpdate, kRes, kDef>(P, &m10, &m8, &mf8, blockIdx.x, blockIdx.y * kWarpsPerBlock, smem);
}

template <class TS, bool kRes>
__global__ void __launch_bounds__(256, kAdjointMinBlocks<TS>) k_adjoint_sweep_batch(const AdjointBatchDesc<TS>* __restrict__ descs,
                                                                const int4* __restrict__ items, const int* __restrict__ count,
                                                                int parity) {
    extern __shared__ __align__(1024) unsigned char smem[];
    if ((int)blockIdx.x >= *count) return;
    const int4 it = items[blockIdx.x];
    const AdjointBatchDesc<TS>* d = descs + it.x;
    if (threadIdx.x == 0) {
        tensormap_acquire(&d->phi_maps[parity].col);
        tensormap_acquire(&d->phi_maps[parity].side);
        tensormap_acquire(&d->f_maps.side);
    }
    adjoint_block<TS, true, kRes, false>(d->args[parity], &d->phi_maps[parity].col, &d->phi_maps[parity].side,
                                  &d->f_maps.side, it.y, it.z, smem);
}

// Per-cell constants of the adjoint linearisation from the primal moments (fixed while the
// primal state does not change): Maxwellian parameters, V/tau, the Jacobian J_P = d(rho,u,T)/dW
// and V d(1/tau)/d(rho, T).
template <class TC>
__global__ void k_adjoint_cellconst(int ncell, const double4* prim, const double4* maxw, const double* V,
                                    double inv_tau_inf, AdjCell<TC>* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double4 p = prim[c], q = maxw[c];            // moments (tau, J_P); Maxwellian parameters (g)
    const double rho = p.x, u1 = p.y, u2 = p.z, T = p.w, sT = sqrt(T), ir = 1.0 / rho;
    const double iT = 1.0 / q.w;
    AdjCell<TC> a;
    a.n0 = (TC)(q.x * iT / (2.0 * kPi));
    a.inv2T = (TC)(0.5 * iT);
    a.halfT = (TC)(0.5 * q.w);
    a.Vt = (TC)(V[c] * rho * sT * inv_tau_inf);
    a.u1 = (TC)q.y;
    a.u2 = (TC)q.z;
    a.ir = (TC)ir;
    a.irg = (TC)(1.0 / q.x);
    a.iT = (TC)iT;
    a.iT2h = (TC)(0.5 * iT * iT);
    a.c0 = (TC)(V[c] * sT * inv_tau_inf);
    a.c3 = (TC)(V[c] * rho * inv_tau_inf / (2.0 * sT));
    a.j30 = (TC)((u1 * u1 + u2 * u2) / 3.0 - T) * (TC)ir;
    a.j31 = (TC)(-(2.0 / 3.0) * u1 * ir);
    a.j32 = (TC)(-(2.0 / 3.0) * u2 * ir);
    a.j33 = (TC)((2.0 / 3.0) * ir);
    out[c] = a;
}

// ================================================================== setup kernels
template <class TC>
__global__ void k_flow_tables(int nvp, const typename Vec<TC>::v4* vt, double u1, double u2, double Tw,
                              typename Vec<TC>::v2* fd, TC* gw) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nvp) return;
    const auto t = vt[k];
    const TC dx = t.x - (TC)u1, dy = t.y - (TC)u2;
    const TC g1 = (TC)(1.0 / (2.0 * kPi)) * dexp<TC>(-(dx * dx + dy * dy) * TC(0.5));
    fd[k].x = g1;
    fd[k].y = TC(0.5) * g1;
    gw[k] = (TC)(1.0 / (2.0 * kPi * Tw)) * dexp<TC>(-(t.x * t.x + t.y * t.y) * (TC)(0.5 / Tw));
}

// Per wall face l: D_l = -sum_{a<=0} w (v.n) g_M1(1,0,Tw) (the normaliser of Eq. barg) and
// M_l = sum_{a<=0} w (v.d) a g_M1 / D_l (the reflected part of J per unit F_rhow).
__global__ void k_wall_setup(int nvp, const double2* S, const double4* vd, const double* gw, MomentJ mj,
                             double* wallD, double* wallM, int raw) {
    const int l = blockIdx.x;
    const double2 s = S[4 * l + 3];
    const double A = sqrt(s.x * s.x + s.y * s.y);
    double d = 0.0, m = 0.0;
    for (int k = threadIdx.x; k < nvp; k += blockDim.x) {
        const double4 t = vd[k];
        const double a = s.x * t.x + s.y * t.y;
        if (!(a > 0.0)) {
            d -= t.z * (a / A) * gw[k];
            m += t.z * (mj.dx * t.x + mj.dy * t.y + mj.h * t.w) * a * gw[k];
        }
    }
    __shared__ double sd[32], sm[32];
    d = warp_sum(d);
    m = warp_sum(m);
    if ((threadIdx.x & 31) == 0) { sd[threadIdx.x >> 5] = d; sm[threadIdx.x >> 5] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double D = 0.0, M = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { D += sd[i]; M += sm[i]; }
        wallD[l] = D;
        wallM[l] = raw ? M : M / D;
    }
}

template <class TS>
__global__ void k_fill_freestream(TS* f, size_t n_pairs, int nvp,
                                  const typename Vec<typename Pack<TS>::TC>::v2* fd) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pairs) return;
    const auto d = fd[i % nvp];
    const size_t o = fpos<TS>(i / nvp, nvp, (int)(i % nvp));
    f[o] = fromdbl<TS>((double)d.x);
    f[o + kComp<TS>] = fromdbl<TS>((double)d.y);
}

// part != null (velocity shard): the raw sums and the wall density go to the shard buffer instead.
template <class TS>
__global__ void k_moments(const TS* f, int ncell, int nvp, const int4* nb, const double2* S, const double4* vd,
                          double4* prim, double* Fw, double* part, int ni) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= ncell) return;
    const bool wall = nb[c].w == kWall;
    const double2 s = S[4 * c + 3];
    double m0 = 0, m1 = 0, m2 = 0, m3 = 0, fw = 0;
    for (int k = lane; k < nvp; k += 32) {
        const double4 t = vd[k];
        const size_t o = fpos<TS>(c, nvp, k);
        const double f1 = todbl(f[o]), f2 = todbl(f[o + kComp<TS>]);
        m0 += t.z * f1;
        m1 += t.z * t.x * f1;
        m2 += t.z * t.y * f1;
        m3 += t.z * (t.w * f1 + f2);
        const double a = s.x * t.x + s.y * t.y;
        if (wall && a > 0.0) fw += t.z * a * f1;
    }
    m0 = warp_sum(m0); m1 = warp_sum(m1); m2 = warp_sum(m2); m3 = warp_sum(m3); fw = warp_sum(fw);
    if (lane == 0 && part) {
        reinterpret_cast<double4*>(part)[c] = make_double4(m0, m1, m2, m3);
        part[4 * (size_t)ncell + c] = 0.0;
        if (wall) {
            part[5 * (size_t)ncell + c] = fw / sqrt(s.x * s.x + s.y * s.y);
            part[5 * (size_t)ncell + ni + c] = 0.0;
        }
    } else if (lane == 0) {
        const double u1 = m1 / m0, u2 = m2 / m0;
        prim[c] = make_double4(m0, u1, u2, (2.0 / 3.0) * (m3 / m0 - 0.5 * (u1 * u1 + u2 * u2)));
        if (wall) Fw[c] = fw / sqrt(s.x * s.x + s.y * s.y);
    }
}

// ================================================================== conservative discrete Maxwellian
// The cell Maxwellian of the collision term with parameters p = (rho, u1, u2, T) chosen so that its
// discrete moments equal the cell's: M(p) = sum_k w_k Psi_k g_k(p) = W, Psi = (1, vx, vy, |v|^2/2) on g1
// and 1 on g2 = T g1 / 2 (the conservative discrete velocity schemes the paper builds on).  Newton's
// method, `iters` steps from the previous fit (warm) or from the primitive variables; with Kinv the
// inverse Jacobian dp/dW = (dM/dp)^{-1} at the final p (row-major [q][m]) for the adjoint.  One warp
// per cell: per-lane sums and a fixed xor butterfly, which leaves bitwise-equal totals in every lane,
// so every lane takes the same Newton step.
template <class T>
__device__ __forceinline__ bool lu4_solve(T A[4][4], T b[4], T x[4]) {
    int piv[4] = {0, 1, 2, 3};
#pragma unroll
    for (int col = 0; col < 4; ++col) {
        int best = col;
        for (int r = col + 1; r < 4; ++r)
            if (fabs(A[piv[r]][col]) > fabs(A[piv[best]][col])) best = r;
        const int t = piv[col]; piv[col] = piv[best]; piv[best] = t;
        if (A[piv[col]][col] == T(0)) return false;
        for (int r = col + 1; r < 4; ++r) {
            const T m = A[piv[r]][col] / A[piv[col]][col];
            for (int c2 = col; c2 < 4; ++c2) A[piv[r]][c2] -= m * A[piv[col]][c2];
            b[piv[r]] -= m * b[piv[col]];
        }
    }
    for (int col = 3; col >= 0; --col) {
        T acc = b[piv[col]];
        for (int c2 = col + 1; c2 < 4; ++c2) acc -= A[piv[col]][c2] * x[c2];
        x[col] = acc / A[piv[col]][col];
    }
    return true;
}

template <class T> __device__ __forceinline__ T warp_sum_t(T v);
template <> __device__ __forceinline__ double warp_sum_t<double>(double v) { return warp_sum(v); }
template <> __device__ __forceinline__ float warp_sum_t<float>(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The residual M - W decides where Newton's method stops, so M is summed in two levels (partial sums
// of 8 velocities) and reduced across the warp in FP64; the Jacobian only steers the steps and is summed and solved in the compute type
// (FP64 for the inverse Jacobian that the adjoint uses).
template <class TC>
__global__ void __launch_bounds__(256) k_maxwell_fit(int ncell, int nvp, const typename Vec<TC>::v4* __restrict__ vt,
                                                     const double4* __restrict__ prim, double4* __restrict__ fit,
                                                     int warm, int iters, double* __restrict__ Kinv) {
    const int lane = threadIdx.x & 31, c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= ncell) return;
    const double4 pr = prim[c];
    const double W[4] = {pr.x, pr.x * pr.y, pr.x * pr.z, pr.x * (0.5 * (pr.y * pr.y + pr.z * pr.z) + 1.5 * pr.w)};
    double4 p = warm ? fit[c] : pr;
    for (int it = 0; it <= iters; ++it) {
        const bool inverse = it == iters;
        if (inverse && !Kinv) break;
        const TC rho = (TC)p.x, u1 = (TC)p.y, u2 = (TC)p.z, T = (TC)p.w;
        const TC i2T = TC(0.5) / T, iT = TC(1) / T, ir = TC(1) / rho;
        const TC hT = TC(0.5) * T;
        Gauss<TC> G;                               // g1 exactly as the sweeps evaluate it
        G.setup(rho, u1, u2, T);
        // M_m = sum w psi_m g1, psi = (1, vx, vy, h + T/2) (g2 = T g1 / 2); J[m][q] = sum w psi_m dg1/dp_q,
        // dg1/dp = g1 (1/rho, cx/T, cy/T, c^2/(2T^2) - 1/T), plus sum w g1 / 2 in J[3][3] (dg2/dT).
        // M: partial sums of 8 velocities added into a second accumulator (no FP64 inside the loop)
        TC md[4] = {TC(0), TC(0), TC(0), TC(0)};
        TC mb[4] = {TC(0), TC(0), TC(0), TC(0)};
        TC sj[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) sj[i] = TC(0);
        int nb = 0;
#pragma unroll 4
        for (int k = lane; k < nvp; k += 32) {
            const auto t = vt[k];
            const TC vx = t.x, vy = t.y, w = t.z, h = t.w;
            const TC cx = vx - u1, cy = vy - u2, c2 = cx * cx + cy * cy;
            const TC wg = w * G.eval(fma(vy, -u2, fma(vx, -u1, h)));
            const TC d[4] = {ir, cx * iT, cy * iT, c2 * i2T * iT - iT};
            const TC psi[4] = {TC(1), vx, vy, h + hT};
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const TC wp = wg * psi[m];
                mb[m] += wp;
#pragma unroll
                for (int q = 0; q < 4; ++q) sj[4 * m + q] += wp * d[q];
            }
            sj[15] += TC(0.5) * wg;
            if (++nb == 8) {
#pragma unroll
                for (int m = 0; m < 4; ++m) { md[m] += mb[m]; mb[m] = TC(0); }
                nb = 0;
            }
        }
        double M[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) M[m] = warp_sum((double)md[m] + (double)mb[m]);
        if (inverse) {                             // dp/dW = J^{-1}, column by column, in FP64
            double A[4][4];
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int q = 0; q < 4; ++q) A[m][q] = warp_sum((double)sj[4 * m + q]);
            if (lane < 4) {                        // lane = column of the inverse
                double B[4][4], e[4] = {0.0, 0.0, 0.0, 0.0}, x[4];
                for (int m = 0; m < 4; ++m)
                    for (int q = 0; q < 4; ++q) B[m][q] = A[m][q];
                e[lane] = 1.0;
                if (!lu4_solve<double>(B, e, x)) x[0] = x[1] = x[2] = x[3] = 0.0;
                for (int q = 0; q < 4; ++q) Kinv[16 * (size_t)c + 4 * q + lane] = x[q];
            }
            break;
        }
        TC A[4][4], r[4], x[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            r[m] = (TC)(M[m] - W[m]);
#pragma unroll
            for (int q = 0; q < 4; ++q) A[m][q] = warp_sum_t<TC>(sj[4 * m + q]);
        }
        if (!lu4_solve<TC>(A, r, x)) break;
        p.x -= (double)x[0]; p.y -= (double)x[1]; p.z -= (double)x[2]; p.w -= (double)x[3];
    }
    if (lane == 0) fit[c] = p;
}

// ================================================================== failure path of the bounded waits
// One warp waits on an mbarrier that nothing completes, with the sweeps' bounded wait: after
// kWaitNs of the global timer the wait gives up, the kernel sets *err and returns (no fault, no
// hang), and the host reads the flag as DVM_ERR_TIMEOUT.
__global__ void k_wait_probe(int* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
}

// ================================================================== moment-space mixing
// Anderson mixing of the cell moments: W = (rho, rho u1, rho u2, rho E) of every cell as one FP64
// vector, and the shift that imposes mixed moments on f, f += g(W_mix) - g(W) per cell and velocity
// (both components), which keeps the non-equilibrium part of f and vanishes at a fixed point.  A cell
// whose mixed moments have no positive density and temperature is left as it is.
__global__ void k_prim_to_W(int ncell, const double4* __restrict__ prim, double* __restrict__ W) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double4 p = prim[c];
    W[4 * c] = p.x;
    W[4 * c + 1] = p.x * p.y;
    W[4 * c + 2] = p.x * p.z;
    W[4 * c + 3] = p.x * (0.5 * (p.y * p.y + p.z * p.z) + 1.5 * p.w);
}

template <class TS>
__global__ void __launch_bounds__(256) k_moment_shift(TS* __restrict__ f, int ncell, int nvp, const double4* __restrict__ vd,
                                                      const double4* __restrict__ prim, const double* __restrict__ W) {
    using TC = typename Pack<TS>::TC;
    const int lane = threadIdx.x & 31, c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= ncell) return;
    const double4 p = prim[c];
    const double r1 = W[4 * c], u1 = W[4 * c + 1] / r1, u2 = W[4 * c + 2] / r1;
    const double T1 = (2.0 / 3.0) * (W[4 * c + 3] / r1 - 0.5 * (u1 * u1 + u2 * u2));
    if (!(r1 > 0.0) || !(T1 > 0.0)) return;
    // g(W_mix) - g = g (exp(l) - 1) with l = ln(g(W_mix) / g) = l0 + l1 vx + l2 vy + l3 |v|^2/2, its
    // coefficients formed in FP64: the shift keeps its relative accuracy when it is small, where the
    // difference of two rounded Gaussians would not
    const double ia = 1.0 / T1, ib = 1.0 / p.w;
    const TC l0 = (TC)(log(r1 * ia / (p.x * ib)) - 0.5 * (u1 * u1 + u2 * u2) * ia + 0.5 * (p.y * p.y + p.z * p.z) * ib);
    const TC l1 = (TC)(u1 * ia - p.y * ib), l2 = (TC)(u2 * ia - p.z * ib), l3 = (TC)(ib - ia);
    Gauss<TC> Gb;
    Gb.setup((TC)p.x, (TC)p.y, (TC)p.z, (TC)p.w);
    const TC hA = (TC)(0.5 * T1), dh = (TC)(0.5 * (T1 - p.w));
    for (int k = lane; k < nvp; k += 32) {
        const double4 t = vd[k];
        const TC vx = (TC)t.x, vy = (TC)t.y, h = (TC)t.w;
        const TC gb = Gb.eval(h - vx * (TC)p.y - vy * (TC)p.z);
        const TC dg = gb * expm1(l0 + l1 * vx + l2 * vy + l3 * h);
        const size_t o = fpos<TS>(c, nvp, k);
        f[o] = fromdbl<TS>(todbl(f[o]) + (double)dg);
        f[o + kComp<TS>] = fromdbl<TS>(todbl(f[o + kComp<TS>]) + (double)(hA * dg + dh * gb));
    }
}

// ================================================================== macroscopic prediction (coarse correction)
// At small Kn the slow modes of the point-implicit sweeps are the cell moments: collisions relax f to
// the local Maxwellian within a sweep, and only transport moves the moments.  A prediction step solves
// for a moment correction dW per cell the moments of the linearised steady residual restricted to
// local Maxwellian perturbations,
//     sum_k w Psi_k [J (dg/dW) dW]_k = -sum_k w Psi_k R_k ,
// and shifts f by g(W + dW) - g(W).  For a Maxwellian perturbation the collision term cancels, so the
// operator is the discrete upwind transport of dg/dW in moment form (a kinetic flux-vector splitting of
// the linearised Euler equations on this velocity set): per cell c and face e the outflow block
//     OUT[c][e] = sum_{k: a_e,k > 0} w_k a_e,k Psi_k (dg_k/dW)(W_c)      (4 x 4)
// gives the diagonal block sum_e OUT[c][e] and, across face e, the neighbour's block -OUT[nb][e'] (its
// outflow through the shared face is this cell's inflow).  On the wall the re-emitted flux
// (dF_rhow / D_l) gbar_w adds the rank-one block u v^T (u = sum_{a<=0} w a Psi gbar_w / D_l, v = dF_rhow/dW);
// the far field injects nothing.  Psi = (1, vx, vy, |v|^2/2) on f1 and (0, 0, 0, 1) on f2.
template <class TC>
__global__ void __launch_bounds__(256, 1) k_coarse_assemble(int ncell, int nvp, const typename Vec<TC>::v4* __restrict__ vt,
                                                            const double2* __restrict__ S, const int4* __restrict__ nb,
                                                            const double4* __restrict__ prim, const TC* __restrict__ gw,
                                                            const double* __restrict__ wallD, double halfTw,
                                                            double* __restrict__ out, double* __restrict__ dinv) {
    const int lane = threadIdx.x & 31, c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= ncell) return;
    const double4 p = prim[c];
    const TC rho = (TC)p.x, u1 = (TC)p.y, u2 = (TC)p.z, T = (TC)p.w;
    Gauss<TC> G;
    G.setup(rho, u1, u2, T);
    const TC ir = TC(1) / rho, iT = TC(1) / T, hT = TC(0.5) * T, hTw = (TC)halfTw;
    TC sx[4], sy[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) { sx[e] = (TC)S[4 * c + e].x; sy[e] = (TC)S[4 * c + e].y; }
    const bool wall = nb[c].w == kWall;
    TC acc[4][16];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[e][i] = TC(0);
    TC wu[4] = {TC(0), TC(0), TC(0), TC(0)}, wv[4] = {TC(0), TC(0), TC(0), TC(0)};
    for (int k = lane; k < nvp; k += 32) {
        const auto t = vt[k];
        const TC vx = t.x, vy = t.y, w = t.z, h = t.w;
        const TC cx = vx - u1, cy = vy - u2;
        const TC g1 = G.eval(fma(vy, -u2, fma(vx, -u1, h)));
        const TC d[4] = {g1 * ir, g1 * cx * iT, g1 * cy * iT, g1 * ((cx * cx + cy * cy) * TC(0.5) * iT * iT - iT)};
        TC R[16];                               // row r of Psi . dg/dp: f1 rows 0..2, energy row 3 with f2
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            R[q] = d[q];
            R[4 + q] = vx * d[q];
            R[8 + q] = vy * d[q];
            R[12 + q] = (h + hT) * d[q];
        }
        R[15] += TC(0.5) * g1;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const TC a = sx[e] * vx + sy[e] * vy;
            const TC wa = a > TC(0) ? w * a : TC(0);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[e][i] = fma(wa, R[i], acc[e][i]);
        }
        if (wall) {
            const TC a = sx[3] * vx + sy[3] * vy;
            if (a > TC(0)) {
#pragma unroll
                for (int q = 0; q < 4; ++q) wv[q] = fma(w * a, d[q], wv[q]);
            } else {
                const TC wg = w * a * gw[k];
                wu[0] += wg; wu[1] += wg * vx; wu[2] += wg * vy; wu[3] += wg * (h + hTw);
            }
        }
    }
    // dp/dW for p = (rho, u1, u2, T), W = (rho, rho u, rho E), E = |u|^2/2 + 3T/2
    const double r = p.x, a1 = p.y, a2 = p.z, Tt = p.w, uu = 0.5 * (a1 * a1 + a2 * a2);
    const double Pm[4][4] = {{1.0, 0.0, 0.0, 0.0},
                             {-a1 / r, 1.0 / r, 0.0, 0.0},
                             {-a2 / r, 0.0, 1.0 / r, 0.0},
                             {(2.0 / 3.0) * (uu - 1.5 * Tt) / r, -(2.0 / 3.0) * a1 / r, -(2.0 / 3.0) * a2 / r, (2.0 / 3.0) / r}};
    // one face at a time: 16 warp sums, then lane 0 maps them to W and adds them to the diagonal block
    double Dg[4][4] = {{0}};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        double Ae[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) Ae[i] = warp_sum((double)acc[e][i]);
        if (lane == 0) {
            double* o = out + ((size_t)c * 4 + e) * 16;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const double v = Ae[4 * i] * Pm[0][j] + Ae[4 * i + 1] * Pm[1][j] + Ae[4 * i + 2] * Pm[2][j] +
                                     Ae[4 * i + 3] * Pm[3][j];
                    o[4 * i + j] = v;
                    Dg[i][j] += v;
                }
        }
    }
    double U[4] = {0, 0, 0, 0}, Vw[4] = {0, 0, 0, 0};
    if (wall) {
#pragma unroll
        for (int q = 0; q < 4; ++q) { U[q] = warp_sum((double)wu[q]); Vw[q] = warp_sum((double)wv[q]); }
    }
    if (lane != 0) return;
    if (wall) {                       // re-emission of the outgoing mass flux: (U / D_l) (Vw / A) P
        const double Aw = sqrt(S[4 * c + 3].x * S[4 * c + 3].x + S[4 * c + 3].y * S[4 * c + 3].y);
        double vW[4];
        for (int j = 0; j < 4; ++j) {
            vW[j] = 0.0;
            for (int q = 0; q < 4; ++q) vW[j] += Vw[q] * Pm[q][j];
            vW[j] /= Aw;
        }
        const double iD = 1.0 / wallD[c];
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) Dg[i][j] += U[i] * iD * vW[j];
    }
    double* di = dinv + (size_t)c * 16;
    for (int col = 0; col < 4; ++col) {           // inverse column by column
        double M[4][4], bb[4] = {0, 0, 0, 0}, x[4];
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) M[i][j] = Dg[i][j];
        bb[col] = 1.0;
        if (!lu4_solve(M, bb, x)) x[0] = x[1] = x[2] = x[3] = 0.0;
        for (int i = 0; i < 4; ++i) di[4 * i + col] = x[i];
    }
}

// Residual moments of a finished block from its last sweep's input and output, for paths whose sweeps do
// not accumulate them (the served batch): rW_c = sum_k w Psi_k R_k with R = D (f_old - f_new),
// D = V/tau(f_old) + sum_e max(-a_e, 0) as in the sweep, Psi = (1, vx, vy, |v|^2/2) on f1 and (0, 0, 0, 1)
// on f2.  The same moments as the sweep's own (k_primal_sweep_rm), summed in another order.
template <class TS, class TC>
__global__ void __launch_bounds__(256) k_primal_restrict(int ncell, int nvp, const typename Vec<TC>::v4* __restrict__ vt,
                                                         const double2* __restrict__ S, const double* __restrict__ V,
                                                         const double4* __restrict__ prim_old, double inv_tau_inf,
                                                         const TS* __restrict__ f_old, const TS* __restrict__ f_new,
                                                         double4* __restrict__ rW) {
    const int lane = threadIdx.x & 31, c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= ncell) return;
    const double4 p = prim_old[c];
    const TC Vt = (TC)(V[c] * p.x * sqrt(p.w) * inv_tau_inf);
    TC sx[4], sy[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) { sx[e] = (TC)S[4 * c + e].x; sy[e] = (TC)S[4 * c + e].y; }
    TC m0 = TC(0), m1 = TC(0), m2 = TC(0), m3 = TC(0);
    for (int k = lane; k < nvp; k += 32) {
        const auto t = vt[k];
        const TC vx = t.x, vy = t.y, w = t.z, h = t.w;
        TC D = Vt;
#pragma unroll
        for (int e = 0; e < 4; ++e) { const TC a = sx[e] * vx + sy[e] * vy; D += a < TC(0) ? -a : TC(0); }
        const size_t o = fpos<TS>(c, nvp, k);
        const TC R1 = D * (TC)(todbl(f_old[o]) - todbl(f_new[o]));
        const TC R2 = D * (TC)(todbl(f_old[o + kComp<TS>]) - todbl(f_new[o + kComp<TS>]));
        const TC wR = w * R1;
        m0 += wR;
        m1 = fma(wR, vx, m1);
        m2 = fma(wR, vy, m2);
        m3 = fma(wR, h, fma(w, R2, m3));
    }
    const double M0 = warp_sum((double)m0), M1 = warp_sum((double)m1), M2 = warp_sum((double)m2);
    const double M3 = warp_sum((double)m3);
    if (lane == 0) rW[c] = make_double4(M0, M1, M2, M3);
}

// Target moments of the prediction: W = W(prim) + s omega dW (conserved variables, [ncell][4]), with the
// largest s in [0, 1] (by bisection) that keeps the cell's density and temperature within a relative change
// `cap` and positive: far from the steady state the linear correction can overshoot.
__device__ __forceinline__ bool coarse_ok(double4 p, double r, double m1, double m2, double e, double cap) {
    if (!(r > 0.0)) return false;
    const double u1 = m1 / r, u2 = m2 / r, T = (2.0 / 3.0) * (e / r - 0.5 * (u1 * u1 + u2 * u2));
    return T > 0.0 && fabs(r - p.x) <= cap * p.x && fabs(T - p.w) <= cap * p.w;
}
__global__ void k_coarse_target(int ncell, const double4* __restrict__ prim, const double4* __restrict__ dW,
                                double omega, double cap, double* __restrict__ W) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double4 p = prim[c], d = dW[c];
    const double w0 = p.x, w1 = p.x * p.y, w2 = p.x * p.z, w3 = p.x * (0.5 * (p.y * p.y + p.z * p.z) + 1.5 * p.w);
    double sc = omega;
    if (!(isfinite(d.x) && isfinite(d.y) && isfinite(d.z) && isfinite(d.w))) {
        sc = 0.0;                                   // a coarse solution that ran away: no shift
    } else if (!coarse_ok(p, w0 + sc * d.x, w1 + sc * d.y, w2 + sc * d.z, w3 + sc * d.w, cap)) {
        double lo = 0.0, hi = omega;
        for (int i = 0; i < 24; ++i) {
            const double m = 0.5 * (lo + hi);
            if (coarse_ok(p, w0 + m * d.x, w1 + m * d.y, w2 + m * d.z, w3 + m * d.w, cap)) lo = m;
            else hi = m;
        }
        sc = lo;
    }
    W[4 * c] = sc > 0.0 ? w0 + sc * d.x : w0;
    W[4 * c + 1] = sc > 0.0 ? w1 + sc * d.y : w1;
    W[4 * c + 2] = sc > 0.0 ? w2 + sc * d.z : w2;
    W[4 * c + 3] = sc > 0.0 ? w3 + sc * d.w : w3;
}

// Prediction of the adjoint sweeps: the transposed coarse problem.  With the prolongation dW -> (dg/dW) dW
// and the restriction delta f -> sum_k w Psi_k delta f_k of the primal prediction, the adjoint (in the
// w-weighted product that the adjoint sweep uses) takes the prolongation lambda -> Psi . lambda and the
// restriction r -> sum_k w (dg_k/dW)^T r_k, and its coarse operator is A^T.  Residual restriction of the
// last adjoint sweep: R = D (phi_old - phi_new), D = V/tau + sum_e max(a_e, 0), at the primal moments.
template <class TS, class TC>
__global__ void __launch_bounds__(256) k_adjoint_restrict(int ncell, int nvp, const typename Vec<TC>::v4* __restrict__ vt,
                                                          const double2* __restrict__ S, const double* __restrict__ V,
                                                          const double4* __restrict__ prim, double inv_tau_inf,
                                                          const TS* __restrict__ phi_o, const TS* __restrict__ phi_n,
                                                          double4* __restrict__ rA) {
    const int lane = threadIdx.x & 31, c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= ncell) return;
    const double4 p = prim[c];
    const TC u1 = (TC)p.y, u2 = (TC)p.z, hT = (TC)(0.5 * p.w);
    const TC Vt = (TC)(V[c] * p.x * sqrt(p.w) * inv_tau_inf);
    Gauss<TC> G;
    G.setup((TC)p.x, u1, u2, (TC)p.w);
    TC sx[4], sy[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) { sx[e] = (TC)S[4 * c + e].x; sy[e] = (TC)S[4 * c + e].y; }
    TC q0 = TC(0), qx = TC(0), qy = TC(0), qc = TC(0), q2 = TC(0);
    for (int k = lane; k < nvp; k += 32) {
        const auto t = vt[k];
        const TC vx = t.x, vy = t.y, w = t.z, h = t.w;
        TC D = Vt;
#pragma unroll
        for (int e = 0; e < 4; ++e) { const TC a = sx[e] * vx + sy[e] * vy; D += a > TC(0) ? a : TC(0); }
        const size_t o = fpos<TS>(c, nvp, k);
        const TC R1 = D * (TC)(todbl(phi_o[o]) - todbl(phi_n[o]));
        const TC R2 = D * (TC)(todbl(phi_o[o + kComp<TS>]) - todbl(phi_n[o + kComp<TS>]));
        const TC cx = vx - u1, cy = vy - u2;
        const TC wg = w * G.eval(fma(vy, -u2, fma(vx, -u1, h)));
        const TC m = wg * fma(hT, R2, R1);
        q0 += m;
        qx = fma(m, cx, qx);
        qy = fma(m, cy, qy);
        qc = fma(m, TC(0.5) * (cx * cx + cy * cy), qc);
        q2 = fma(wg, R2, q2);
    }
    const double Q0 = warp_sum((double)q0), Qx = warp_sum((double)qx), Qy = warp_sum((double)qy);
    const double Qc = warp_sum((double)qc), Q2 = warp_sum((double)q2);
    if (lane != 0) return;
    // sum_k w (dg/dp)^T R, p = (rho, u1, u2, T), then (dp/dW)^T
    const double r = p.x, a1 = p.y, a2 = p.z, T = p.w, ir = 1.0 / r, iT = 1.0 / T;
    const double ph0 = Q0 * ir, ph1 = Qx * iT, ph2 = Qy * iT, ph3 = Qc * iT * iT - Q0 * iT + 0.5 * Q2;
    const double uu = 0.5 * (a1 * a1 + a2 * a2);
    rA[c] = make_double4(ph0 - (ph1 * a1 + ph2 * a2) * ir + ph3 * (2.0 / 3.0) * (uu - 1.5 * T) * ir,
                         (ph1 - (2.0 / 3.0) * a1 * ph3) * ir, (ph2 - (2.0 / 3.0) * a2 * ph3) * ir,
                         (2.0 / 3.0) * ph3 * ir);
}

// The adjoint prediction's update: phi1 += omega (l0 + l1 vx + l2 vy + l3 |v|^2/2), phi2 += omega l3 (the
// prolongation Psi . lambda); a cell whose lambda is not finite is left as it is.
template <class TS>
__global__ void __launch_bounds__(256) k_adjoint_shift(int ncell, int nvp, const double4* __restrict__ vd,
                                                       const double4* __restrict__ x, double omega, TS* __restrict__ phi) {
    const int lane = threadIdx.x & 31, c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= ncell) return;
    const double4 l = x[c];
    if (!(isfinite(l.x) && isfinite(l.y) && isfinite(l.z) && isfinite(l.w))) return;
    for (int k = lane; k < nvp; k += 32) {
        const double4 t = vd[k];
        const size_t o = fpos<TS>(c, nvp, k);
        phi[o] = fromdbl<TS>(todbl(phi[o]) + omega * (l.x + l.y * t.x + l.z * t.y + l.w * t.w));
        phi[o + kComp<TS>] = fromdbl<TS>(todbl(phi[o + kComp<TS>]) + omega * l.w);
    }
}

// Prediction of the refinement's linear correction e (FP32, state layout): e += (dg/dW)(prim) s omega x, the
// Maxwellian perturbation with conserved moments s omega x, then the moment sums of e and, on wall cells,
// its outgoing wall mass flux per unit area, which the next linearised sweep reads as its lagged dW and
// dF_rhow.  A correction is small against the state; s <= 1 keeps the density and temperature parts
// within `cap` of the state's (s = 0 for a non-finite x), so that a coarse solution that ran away (the
// block-Jacobi iteration is non-normal) cannot carry into e.
__global__ void __launch_bounds__(256) k_coarse_lin_shift(int ncell, int nvp, const double4* __restrict__ vd,
                                                          const double2* __restrict__ S, const int4* __restrict__ nb,
                                                          const double4* __restrict__ prim, const double4* __restrict__ x,
                                                          double omega, double cap, float* __restrict__ e,
                                                          double4* __restrict__ dW, double* __restrict__ dF) {
    const int lane = threadIdx.x & 31, c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= ncell) return;
    const double4 p = prim[c], xw = x[c];
    const double r = p.x, a1 = p.y, a2 = p.z, T = p.w, ir = 1.0 / r, iT = 1.0 / T;
    double x0 = omega * xw.x, x1 = omega * xw.y, x2 = omega * xw.z, x3 = omega * xw.w;
    double dT = (2.0 / 3.0) * ir * (x3 - (a1 * x1 + a2 * x2) + (0.5 * (a1 * a1 + a2 * a2) - 1.5 * T) * x0);
    double sc = 1.0;
    if (!(fabs(x0) <= cap * r) || !(fabs(dT) <= cap * T))
        sc = (isfinite(x0) && isfinite(dT)) ? fmin(cap * r / fabs(x0), cap * T / fabs(dT)) : 0.0;
    x0 *= sc; x1 *= sc; x2 *= sc; x3 *= sc; dT *= sc;
    const double du1 = (x1 - a1 * x0) * ir, du2 = (x2 - a2 * x0) * ir;
    // dg1 / g1 = k0 + k1 vx + k2 vy + k3 |v|^2/2 (the linearised Maxwellian in v, coefficients in FP64)
    const double k1 = du1 * iT - a1 * dT * iT * iT, k2 = du2 * iT - a2 * dT * iT * iT, k3 = dT * iT * iT;
    const double k0 = x0 * ir - (a1 * du1 + a2 * du2) * iT + (0.5 * (a1 * a1 + a2 * a2) * iT - 1.0) * iT * dT;
    const float fk0 = (float)k0, fk1 = (float)k1, fk2 = (float)k2, fk3 = (float)k3;
    const float hT = (float)(0.5 * T), hdT = (float)(0.5 * dT);
    Gauss<float> G;
    G.setup((float)r, (float)a1, (float)a2, (float)T);
    const bool wall = nb[c].w == kWall;
    const double2 s3 = S[4 * c + 3];
    double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0, fw = 0.0;
    for (int k = lane; k < nvp; k += 32) {
        const double4 t = vd[k];
        const float vx = (float)t.x, vy = (float)t.y, h = (float)t.w;
        const float g1 = G.eval(h - vx * (float)a1 - vy * (float)a2);
        const float d1 = g1 * (fk0 + fk1 * vx + fk2 * vy + fk3 * h);
        const size_t o = fpos<float>(c, nvp, k);
        const float e1 = e[o] + d1, e2 = e[o + kComp<float>] + (hT * d1 + hdT * g1);
        e[o] = e1;
        e[o + kComp<float>] = e2;
        const double we = t.z * (double)e1;
        m0 += we;
        m1 += we * t.x;
        m2 += we * t.y;
        m3 += we * t.w + t.z * (double)e2;
        if (wall) {
            const double a = s3.x * t.x + s3.y * t.y;
            if (a > 0.0) fw += we * a;
        }
    }
    m0 = warp_sum(m0); m1 = warp_sum(m1); m2 = warp_sum(m2); m3 = warp_sum(m3);
    if (wall) fw = warp_sum(fw);
    if (lane == 0) {
        dW[c] = make_double4(m0, m1, m2, m3);
        if (wall) dF[c] = fw / sqrt(s3.x * s3.x + s3.y * s3.y);
    }
}

// ================================================================== second order (reconstruction)
// Linear reconstruction of the upwind cell on interior faces, F_e = f_up + grad f_up . (x_e - x_up),
// with the unlimited Gauss gradient of Eq. (gaussgrad), grad f_c = (1/V_c) sum_e fbar_e A_e n_e: fbar_e
// is the face average (f_c + f_nb)/2 inside and the first-order face value on the far-field and wall
// faces (own f on an outflow face; the free stream, or the diffuse-wall Maxwellian (F_rhow/D) g_M, on
// an inflow face).  x_c is the mean of the four corners and x_e the midpoint of face e.  Boundary faces
// keep their first-order values, so the added flux is
//     dR_c = sum_{interior e} a_e grad f_up . (x_e - x_up),
// taken by the sweep as a defect of the previous state (the first-order diagonal D stays).  dR is
// affine in f; with lambda = w phi its transpose gathers, per cell u and interior face e with a_e > 0,
//     mu_u = sum_e a_e (phi_u - phi_nb) (x_e - x_u)          (the weight of grad f_u in sum lambda.dR)
// and then spreads s_{u,e} = A_e n_e . mu_u / V_u over the values fbar_{u,e} depends on: half to each
// side of an interior face, all to u on an outflow boundary face, and through F_rhow to the outgoing
// velocities of a wall cell.  Four kernels, each a warp per cell over 16-byte chunks.
__device__ __forceinline__ void so_points(const double2* X, int ni, int c, double2& xc, double2 (&xe)[4]) {
    const int i = c % ni, j = c / ni, ip = (i + 1) % ni;
    const double2 P[4] = {X[j * ni + i], X[(j + 1) * ni + i], X[(j + 1) * ni + ip], X[j * ni + ip]};
    xc = make_double2(0.25 * ((P[0].x + P[1].x) + (P[2].x + P[3].x)), 0.25 * ((P[0].y + P[1].y) + (P[2].y + P[3].y)));
#pragma unroll
    for (int e = 0; e < 4; ++e)
        xe[e] = make_double2(0.5 * (P[e].x + P[(e + 1) & 3].x), 0.5 * (P[e].y + P[(e + 1) & 3].y));
}

// Offsets x_e - x_c of the cell's faces and x_e - x_nb of its interior neighbours (0 on boundary faces).
template <class TC2>
__device__ __forceinline__ void so_offsets(const double2* X, int ni, int c, const int (&nb)[4], TC2 (&dc)[4],
                                           TC2 (&dn)[4]) {
    double2 xc, xe[4];
    so_points(X, ni, c, xc, xe);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        dc[e].x = xe[e].x - xc.x;
        dc[e].y = xe[e].y - xc.y;
        dn[e].x = 0;
        dn[e].y = 0;
        if (nb[e] >= 0) {
            double2 xm, xx[4];
            so_points(X, ni, nb[e], xm, xx);
            dn[e].x = xe[e].x - xm.x;
            dn[e].y = xe[e].y - xm.y;
        }
    }
}

template <class TS>
__global__ void __launch_bounds__(256, DVM_SO_BLOCKS) k_so_gradient(const SOArgs<TS, typename Pack<TS>::TC> A) {
    using PK = Pack<TS>;
    using TC = typename PK::TC;
    using TC2 = typename Vec<TC>::v2;
    using TC4 = typename Vec<TC>::v4;
    constexpr int KV = PK::KV;
    const int lane = threadIdx.x & 31, c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= A.ncell) return;
    const int4 n4 = A.nb[c];
    const int nb[4] = {n4.x, n4.y, n4.z, n4.w};
    TC2 S[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) S[e] = A.S[4 * c + e];
    const TC iV = TC(1) / A.V[c];
    TC cw1 = TC(0), cw2 = TC(0);
    if (nb[3] == kWall) {
        cw1 = (TC)(A.Fw[c] / A.wallD[c]);
        cw2 = cw1 * A.halfTw;
    }
    const size_t nq = (size_t)A.nq;
    const uint4* f = reinterpret_cast<const uint4*>(A.in);
    uint4* gx = reinterpret_cast<uint4*>(A.gx);
    uint4* gy = reinterpret_cast<uint4*>(A.gy);
    for (int q = lane; q < A.nq; q += 32) {
        TC o1[KV], o2[KV], m1[4][KV], m2[4][KV];
        PK::unpack(ldg16(f + c * nq + q), o1, o2);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (nb[e] >= 0) PK::unpack(ldg16(f + (size_t)nb[e] * nq + q), m1[e], m2[e]);
            else PK::unpack(make_uint4(0u, 0u, 0u, 0u), m1[e], m2[e]);
        }
        TC x1[KV], x2[KV], y1[KV], y2[KV];
#pragma unroll
        for (int kk = 0; kk < KV; ++kk) {
            const int k = q * KV + kk;
            const TC4 t = A.vt[k];
            TC sx1 = TC(0), sy1 = TC(0), sx2 = TC(0), sy2 = TC(0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                TC b1, b2;
                if (nb[e] >= 0) {
                    b1 = TC(0.5) * (o1[kk] + m1[e][kk]);
                    b2 = TC(0.5) * (o2[kk] + m2[e][kk]);
                } else if (S[e].x * t.x + S[e].y * t.y > TC(0)) {
                    b1 = o1[kk];
                    b2 = o2[kk];
                } else if (nb[e] == kFar) {
                    const TC2 g = A.fd[k];
                    b1 = g.x;
                    b2 = g.y;
                } else {
                    const TC g = A.gw[k];
                    b1 = cw1 * g;
                    b2 = cw2 * g;
                }
                sx1 += b1 * S[e].x; sy1 += b1 * S[e].y;
                sx2 += b2 * S[e].x; sy2 += b2 * S[e].y;
            }
            x1[kk] = sx1 * iV; y1[kk] = sy1 * iV;
            x2[kk] = sx2 * iV; y2[kk] = sy2 * iV;
        }
        gx[c * nq + q] = PK::pack(x1, x2);
        gy[c * nq + q] = PK::pack(y1, y2);
    }
}

template <class TS>
__global__ void __launch_bounds__(256, DVM_SO_BLOCKS) k_so_defect(const SOArgs<TS, typename Pack<TS>::TC> A) {
    using PK = Pack<TS>;
    using TC = typename PK::TC;
    using TC2 = typename Vec<TC>::v2;
    using TC4 = typename Vec<TC>::v4;
    constexpr int KV = PK::KV;
    const int lane = threadIdx.x & 31, c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= A.ncell) return;
    const int4 n4 = A.nb[c];
    const int nb[4] = {n4.x, n4.y, n4.z, n4.w};
    TC2 S[4], dc[4], dn[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) S[e] = A.S[4 * c + e];
    so_offsets(A.nodes, A.ni, c, nb, dc, dn);
    const size_t nq = (size_t)A.nq;
    const uint4* gx = reinterpret_cast<const uint4*>(A.gx);
    const uint4* gy = reinterpret_cast<const uint4*>(A.gy);
    uint4* out = reinterpret_cast<uint4*>(A.out);
    for (int q = lane; q < A.nq; q += 32) {
        TC ox1[KV], ox2[KV], oy1[KV], oy2[KV], nx1[4][KV], nx2[4][KV], ny1[4][KV], ny2[4][KV], av[4][KV];
        PK::unpack(ldg16(gx + c * nq + q), ox1, ox2);
        PK::unpack(ldg16(gy + c * nq + q), oy1, oy2);
#pragma unroll
        for (int kk = 0; kk < KV; ++kk) {
            const TC4 t = A.vt[q * KV + kk];
#pragma unroll
            for (int e = 0; e < 4; ++e) av[e][kk] = S[e].x * t.x + S[e].y * t.y;
        }
        // a neighbour's gradient enters only through its inflow faces (a <= 0): load it where needed
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            bool need = false;
#pragma unroll
            for (int kk = 0; kk < KV; ++kk) need |= av[e][kk] <= TC(0);
            uint4 qx = make_uint4(0u, 0u, 0u, 0u), qy = qx;
            if (need && nb[e] >= 0) {
                qx = ldg16(gx + (size_t)nb[e] * nq + q);
                qy = ldg16(gy + (size_t)nb[e] * nq + q);
            }
            PK::unpack(qx, nx1[e], nx2[e]);
            PK::unpack(qy, ny1[e], ny2[e]);
        }
        TC d1[KV], d2[KV];
#pragma unroll
        for (int kk = 0; kk < KV; ++kk) {
            TC r1 = TC(0), r2 = TC(0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (nb[e] < 0) continue;
                const TC a = av[e][kk];
                if (a > TC(0)) {
                    r1 += a * (ox1[kk] * dc[e].x + oy1[kk] * dc[e].y);
                    r2 += a * (ox2[kk] * dc[e].x + oy2[kk] * dc[e].y);
                } else {
                    r1 += a * (nx1[e][kk] * dn[e].x + ny1[e][kk] * dn[e].y);
                    r2 += a * (nx2[e][kk] * dn[e].x + ny2[e][kk] * dn[e].y);
                }
            }
            d1[kk] = r1;
            d2[kk] = r2;
        }
        out[c * nq + q] = PK::pack(d1, d2);
    }
}

// Node gradient of Lambda = sum_c lambda_c . dR_c (lambda = w phi) for the full discrete sensitivity
// of a second-order state.  With mu_u of the transposed reconstruction, Lambda = sum_u grad f_u . mu_u,
// and its geometric derivative gathers, per cell u, five terms: the volume in the Gauss gradient
// (-(grad f_u . mu_u) / V_u dV_u), its face vectors (fbar_e mu_u / V_u . dS_e), the wall inflow values'
// dependence on the wall face vector through F_rhow / D, the face weights a_e = S_e . v of mu_u
// ((grad f_u . d_e) (lambda_u - lambda_nb) v . dS_e on outflow faces) and the offsets d_e = x_e - x_u
// (a_e (lambda_u - lambda_nb) grad f_u . d(d_e)).  k_so_sens_cells writes each cell's share of the
// derivative at its four corners; k_so_sens_nodes adds, per node, the shares of the cells around it.
template <class TS>
__global__ void __launch_bounds__(256) k_so_sens_cells(const SOArgs<TS, typename Pack<TS>::TC> A, const TS* __restrict__ phi,
                                                       double2* __restrict__ corner) {
    using PK = Pack<TS>;
    using TC = typename PK::TC;
    using TC2 = typename Vec<TC>::v2;
    using TC4 = typename Vec<TC>::v4;
    constexpr int KV = PK::KV;
    const int lane = threadIdx.x & 31, c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= A.ncell) return;
    const int4 n4 = A.nb[c];
    const int nb[4] = {n4.x, n4.y, n4.z, n4.w};
    const bool wall = nb[3] == kWall;
    TC2 S[4], dc[4], dn[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) S[e] = A.S[4 * c + e];
    so_offsets(A.nodes, A.ni, c, nb, dc, dn);
    const TC iV = TC(1) / A.V[c];
    TC cw1 = TC(0), cw2 = TC(0);
    if (wall) {
        cw1 = (TC)(A.Fw[c] / A.wallD[c]);
        cw2 = cw1 * A.halfTw;
    }
    const size_t nq = (size_t)A.nq;
    const uint4* fq = reinterpret_cast<const uint4*>(A.in);
    const uint4* pq = reinterpret_cast<const uint4*>(phi);
    // sums: 0 sV; 1..8 T_e; 9..16 U_e; 17..24 Y_e (compensated, like the first-order face sums);
    // wall cells: 0 Lam2, 1 Fw, 2..3 dFw, 4 D, 5..6 dD in FP64, because the wall term takes the
    // difference (dFw D - Fw dD) / D^2 of them
    Acc<TC> s[25];
    double sw[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) sw[i] = 0.0;
    for (size_t q = lane; q < nq; q += 32) {
        TC o1[KV], o2[KV], m1[4][KV], m2[4][KV], l1[KV], l2[KV], k1[4][KV], k2[4][KV];
        PK::unpack(ldg16(fq + (size_t)c * nq + q), o1, o2);
        PK::unpack(ldg16(pq + (size_t)c * nq + q), l1, l2);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const size_t m = nb[e] >= 0 ? (size_t)nb[e] : (size_t)c;
            PK::unpack(ldg16(fq + m * nq + q), m1[e], m2[e]);
            PK::unpack(ldg16(pq + m * nq + q), k1[e], k2[e]);
        }
#pragma unroll
        for (int kk = 0; kk < KV; ++kk) {
            const int k = (int)q * KV + kk;
            const TC4 t = A.vt[k];
            const TC w = t.z;
            TC a[4], fb1[4], fb2[4];
            TC gx1 = TC(0), gy1 = TC(0), gx2 = TC(0), gy2 = TC(0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                a[e] = S[e].x * t.x + S[e].y * t.y;
                if (nb[e] >= 0) {
                    fb1[e] = TC(0.5) * (o1[kk] + m1[e][kk]);
                    fb2[e] = TC(0.5) * (o2[kk] + m2[e][kk]);
                } else if (a[e] > TC(0)) {
                    fb1[e] = o1[kk]; fb2[e] = o2[kk];
                } else if (nb[e] == kFar) {
                    const TC2 fd = A.fd[k]; fb1[e] = fd.x; fb2[e] = fd.y;
                } else {
                    const TC gk = A.gw[k]; fb1[e] = cw1 * gk; fb2[e] = cw2 * gk;
                }
                gx1 += fb1[e] * S[e].x; gy1 += fb1[e] * S[e].y;
                gx2 += fb2[e] * S[e].x; gy2 += fb2[e] * S[e].y;
            }
            gx1 *= iV; gy1 *= iV; gx2 *= iV; gy2 *= iV;
            // mu and the outflow-face terms, lambda = w phi
            TC mx1 = TC(0), my1 = TC(0), mx2 = TC(0), my2 = TC(0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (nb[e] < 0 || !(a[e] > TC(0))) continue;
                const TC dl1 = w * (l1[kk] - k1[e][kk]), dl2 = w * (l2[kk] - k2[e][kk]);
                const TC ad1 = a[e] * dl1, ad2 = a[e] * dl2;
                mx1 += ad1 * dc[e].x; my1 += ad1 * dc[e].y;
                mx2 += ad2 * dc[e].x; my2 += ad2 * dc[e].y;
                const TC gd = (gx1 * dc[e].x + gy1 * dc[e].y) * dl1 + (gx2 * dc[e].x + gy2 * dc[e].y) * dl2;
                s[9 + 2 * e].add(gd * t.x);
                s[10 + 2 * e].add(gd * t.y);
                s[17 + 2 * e].add(ad1 * gx1 + ad2 * gx2);
                s[18 + 2 * e].add(ad1 * gy1 + ad2 * gy2);
            }
            s[0].add(gx1 * mx1 + gy1 * my1 + gx2 * mx2 + gy2 * my2);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                s[1 + 2 * e].add((fb1[e] * mx1 + fb2[e] * mx2) * iV);
                s[2 + 2 * e].add((fb1[e] * my1 + fb2[e] * my2) * iV);
            }
            if (wall) {
                const double gk = (double)A.gw[k], wd = (double)w;
                if (a[3] > TC(0)) {
                    const double wo = wd * (double)o1[kk];
                    sw[1] += wo * (double)a[3];
                    sw[2] += wo * (double)t.x;
                    sw[3] += wo * (double)t.y;
                } else {
                    const TC sm1 = (S[3].x * mx1 + S[3].y * my1) * iV, sm2 = (S[3].x * mx2 + S[3].y * my2) * iV;
                    sw[0] += (double)(sm1 + sm2 * A.halfTw) * gk;
                    sw[4] -= wd * (double)a[3] * gk;
                    sw[5] -= wd * (double)t.x * gk;
                    sw[6] -= wd * (double)t.y * gk;
                }
            }
        }
    }
    double r[32];
#pragma unroll
    for (int i = 0; i < 25; ++i) r[i] = warp_sum(s[i].get());
#pragma unroll
    for (int i = 0; i < 7; ++i) r[25 + i] = warp_sum(sw[i]);
    if (lane != 0) return;
    const int ni = A.ni, i = c % ni, j = c / ni, ip = (i + 1) % ni;
    const double2 P[4] = {A.nodes[j * ni + i], A.nodes[(j + 1) * ni + i], A.nodes[(j + 1) * ni + ip], A.nodes[j * ni + ip]};
    const double V = (double)A.V[c];
    double2 C[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) C[q] = make_double2(0.0, 0.0);
    double X[4][2];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        X[e][0] = r[1 + 2 * e] + r[9 + 2 * e];
        X[e][1] = r[2 + 2 * e] + r[10 + 2 * e];
    }
    if (wall && r[29] != 0.0) {            // F_rhow / D as a function of the wall face vector
        const double Fw = r[26], D = r[29];
        X[3][0] += r[25] * (r[27] * D - Fw * r[30]) / (D * D);
        X[3][1] += r[25] * (r[28] * D - Fw * r[31]) / (D * D);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {          // S_e = (Qy - Py, -(Qx - Px)): d/dP = (X_y, -X_x), d/dQ = (-X_y, X_x)
        const int e1 = (e + 1) & 3;
        C[e].x += X[e][1]; C[e].y -= X[e][0];
        C[e1].x -= X[e][1]; C[e1].y += X[e][0];
    }
    const double kv = -r[0] / V;           // volume: dV/dP_e = ((P_{e+1} - P_{e-1})_y, (P_{e-1} - P_{e+1})_x) / 2
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const double2 Pn = P[(e + 1) & 3], Pp = P[(e + 3) & 3];
        C[e].x += kv * 0.5 * (Pn.y - Pp.y);
        C[e].y += kv * 0.5 * (Pp.x - Pn.x);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {          // d_e = x_e - x_u: x_e the midpoint of P_e P_{e+1}, x_u the corner mean
        const double yx = r[17 + 2 * e], yy = r[18 + 2 * e];
        const int e1 = (e + 1) & 3;
        C[e].x += 0.5 * yx; C[e].y += 0.5 * yy;
        C[e1].x += 0.5 * yx; C[e1].y += 0.5 * yy;
#pragma unroll
        for (int q = 0; q < 4; ++q) { C[q].x -= 0.25 * yx; C[q].y -= 0.25 * yy; }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) corner[4 * (size_t)c + q] = C[q];
}

// node (jj, ii) is corner 0 of cell (jj, ii), 1 of (jj-1, ii), 2 of (jj-1, ii-1) and 3 of (jj, ii-1)
__global__ void k_so_sens_nodes(int ni, int nj, const double2* __restrict__ corner, double2* __restrict__ node_grad) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (nj + 1) * ni) return;
    const int jj = id / ni, ii = id % ni, im = (ii - 1 + ni) % ni;
    double2 g = node_grad[id];
    if (jj < nj) {
        const double2 a = corner[4 * (size_t)(jj * ni + ii) + 0], b = corner[4 * (size_t)(jj * ni + im) + 3];
        g.x += a.x + b.x; g.y += a.y + b.y;
    }
    if (jj > 0) {
        const double2 a = corner[4 * (size_t)((jj - 1) * ni + ii) + 1], b = corner[4 * (size_t)((jj - 1) * ni + im) + 2];
        g.x += a.x + b.x; g.y += a.y + b.y;
    }
    node_grad[id] = g;
}

template <class TS>
__global__ void __launch_bounds__(256, DVM_SO_BLOCKS) k_so_adjoint_mu(const SOArgs<TS, typename Pack<TS>::TC> A) {
    using PK = Pack<TS>;
    using TC = typename PK::TC;
    using TC2 = typename Vec<TC>::v2;
    using TC4 = typename Vec<TC>::v4;
    constexpr int KV = PK::KV;
    const int lane = threadIdx.x & 31, c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= A.ncell) return;
    const int4 n4 = A.nb[c];
    const int nb[4] = {n4.x, n4.y, n4.z, n4.w};
    TC2 S[4], dc[4], dn[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) S[e] = A.S[4 * c + e];
    so_offsets(A.nodes, A.ni, c, nb, dc, dn);
    const size_t nq = (size_t)A.nq;
    const uint4* phi = reinterpret_cast<const uint4*>(A.in);
    uint4* gx = reinterpret_cast<uint4*>(A.gx);
    uint4* gy = reinterpret_cast<uint4*>(A.gy);
    for (int q = lane; q < A.nq; q += 32) {
        TC o1[KV], o2[KV], m1[4][KV], m2[4][KV], av[4][KV];
        PK::unpack(ldg16(phi + c * nq + q), o1, o2);
#pragma unroll
        for (int kk = 0; kk < KV; ++kk) {
            const TC4 t = A.vt[q * KV + kk];
#pragma unroll
            for (int e = 0; e < 4; ++e) av[e][kk] = S[e].x * t.x + S[e].y * t.y;
        }
        // only the outflow faces (a > 0) of u carry its reconstruction: load those neighbours
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            bool need = false;
#pragma unroll
            for (int kk = 0; kk < KV; ++kk) need |= av[e][kk] > TC(0);
            uint4 qm = make_uint4(0u, 0u, 0u, 0u);
            if (need && nb[e] >= 0) qm = ldg16(phi + (size_t)nb[e] * nq + q);
            PK::unpack(qm, m1[e], m2[e]);
        }
        TC x1[KV], x2[KV], y1[KV], y2[KV];
#pragma unroll
        for (int kk = 0; kk < KV; ++kk) {
            TC mx1 = TC(0), my1 = TC(0), mx2 = TC(0), my2 = TC(0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (nb[e] < 0) continue;
                const TC a = av[e][kk];
                if (a > TC(0)) {
                    const TC d1 = a * (o1[kk] - m1[e][kk]), d2 = a * (o2[kk] - m2[e][kk]);
                    mx1 += d1 * dc[e].x; my1 += d1 * dc[e].y;
                    mx2 += d2 * dc[e].x; my2 += d2 * dc[e].y;
                }
            }
            x1[kk] = mx1; y1[kk] = my1;
            x2[kk] = mx2; y2[kk] = my2;
        }
        gx[c * nq + q] = PK::pack(x1, x2);
        gy[c * nq + q] = PK::pack(y1, y2);
    }
}

template <class TS>
__global__ void __launch_bounds__(256, DVM_SO_BLOCKS) k_so_adjoint_defect(const SOArgs<TS, typename Pack<TS>::TC> A) {
    using PK = Pack<TS>;
    using TC = typename PK::TC;
    using TC2 = typename Vec<TC>::v2;
    using TC4 = typename Vec<TC>::v4;
    constexpr int KV = PK::KV;
    const int lane = threadIdx.x & 31, c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= A.ncell) return;
    const int4 n4 = A.nb[c];
    const int nb[4] = {n4.x, n4.y, n4.z, n4.w};
    TC2 S[4];
    TC iVn[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        S[e] = A.S[4 * c + e];
        iVn[e] = nb[e] >= 0 ? TC(1) / A.V[nb[e]] : TC(0);
    }
    const TC iV = TC(1) / A.V[c];
    const size_t nq = (size_t)A.nq;
    const uint4* gx = reinterpret_cast<const uint4*>(A.gx);
    const uint4* gy = reinterpret_cast<const uint4*>(A.gy);
    uint4* out = reinterpret_cast<uint4*>(A.out);
    // wall: the inflow values (F_rhow / D) g_M depend on f1 of the outgoing velocities through F_rhow
    TC wcoef = TC(0);
    if (nb[3] == kWall) {
        double lam = 0.0;
        for (int q = lane; q < A.nq; q += 32) {
            TC ox1[KV], ox2[KV], oy1[KV], oy2[KV];
            PK::unpack(ldg16(gx + c * nq + q), ox1, ox2);
            PK::unpack(ldg16(gy + c * nq + q), oy1, oy2);
#pragma unroll
            for (int kk = 0; kk < KV; ++kk) {
                const int k = q * KV + kk;
                const TC4 t = A.vt[k];
                if (S[3].x * t.x + S[3].y * t.y <= TC(0)) {
                    const TC s1 = (S[3].x * ox1[kk] + S[3].y * oy1[kk]) * iV;
                    const TC s2 = (S[3].x * ox2[kk] + S[3].y * oy2[kk]) * iV;
                    lam += (double)(t.z * A.gw[k] * (s1 + A.halfTw * s2));
                }
            }
        }
        lam = warp_sum(lam);
        const double area = sqrt((double)S[3].x * (double)S[3].x + (double)S[3].y * (double)S[3].y);
        wcoef = (TC)(lam / (A.wallD[c] * area));
    }
    for (int q = lane; q < A.nq; q += 32) {
        TC ox1[KV], ox2[KV], oy1[KV], oy2[KV], nx1[4][KV], nx2[4][KV], ny1[4][KV], ny2[4][KV];
        PK::unpack(ldg16(gx + c * nq + q), ox1, ox2);
        PK::unpack(ldg16(gy + c * nq + q), oy1, oy2);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const size_t m = nb[e] >= 0 ? (size_t)nb[e] : (size_t)c;
            PK::unpack(ldg16(gx + m * nq + q), nx1[e], nx2[e]);
            PK::unpack(ldg16(gy + m * nq + q), ny1[e], ny2[e]);
        }
        TC d1[KV], d2[KV];
#pragma unroll
        for (int kk = 0; kk < KV; ++kk) {
            const TC4 t = A.vt[q * KV + kk];
            TC r1 = TC(0), r2 = TC(0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const TC s1 = (S[e].x * ox1[kk] + S[e].y * oy1[kk]) * iV;
                const TC s2 = (S[e].x * ox2[kk] + S[e].y * oy2[kk]) * iV;
                if (nb[e] >= 0) {
                    // own share of the face average, and the neighbour's (its face vector is -S_e)
                    const TC u1 = (S[e].x * nx1[e][kk] + S[e].y * ny1[e][kk]) * iVn[e];
                    const TC u2 = (S[e].x * nx2[e][kk] + S[e].y * ny2[e][kk]) * iVn[e];
                    r1 += TC(0.5) * (s1 - u1);
                    r2 += TC(0.5) * (s2 - u2);
                } else if (S[e].x * t.x + S[e].y * t.y > TC(0)) {
                    r1 += s1;
                    r2 += s2;
                }
            }
            if (nb[3] == kWall) {
                const TC a3 = S[3].x * t.x + S[3].y * t.y;
                if (a3 > TC(0)) r1 += a3 * wcoef;
            }
            d1[kk] = r1;
            d2[kk] = r2;
        }
        out[c * nq + q] = PK::pack(d1, d2);
    }
}

// Deterministic single-block reduction: out[0] = sum respart, out[1] = sum_l (Jpart_l + Fw_l M_l).
__global__ void k_finalize(const double* respart, int ncell, const double* Jpart, const double* Fw,
                           const double* M, int ni, double* out) {
    __shared__ double s0[32], s1[32];
    double a = 0.0, b = 0.0;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) a += respart[c];
    if (Jpart)
        for (int l = threadIdx.x; l < ni; l += blockDim.x) b += Jpart[l] + (Fw ? Fw[l] * M[l] : 0.0);
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) { s0[threadIdx.x >> 5] = a; s1[threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { A += s0[i]; B += s1[i]; }
        out[0] = A;
        out[1] = B;
    }
}

// J = sum_l sum_k w m a f1_l  (Eq. numer_J) for an arbitrary direction; one block per wall face.
template <class TS>
__global__ void k_functional(const TS* f, int nvp, const double2* S, const double4* vd, const double* gw,
                             const double* wallD, const double* Fw, MomentJ mj, double* face_out) {
    const int l = blockIdx.x;
    const double2 s = S[4 * l + 3];
    const double cw = Fw[l] / wallD[l];
    double j = 0.0;
    for (int k = threadIdx.x; k < nvp; k += blockDim.x) {
        const double4 t = vd[k];
        const double a = s.x * t.x + s.y * t.y;
        const double f1 = a > 0.0 ? todbl(f[fpos<TS>(l, nvp, k)]) : cw * gw[k];
        j += t.z * (mj.dx * t.x + mj.dy * t.y + mj.h * t.w) * a * f1;
    }
    __shared__ double sj[32];
    j = warp_sum(j);
    if ((threadIdx.x & 31) == 0) sj[threadIdx.x >> 5] = j;
    __syncthreads();
    if (threadIdx.x == 0) {
        double J = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) J += sj[i];
        face_out[l] = J;
    }
}

template <class TA, class TB>
__global__ void k_convert(const TA* src, TB* dst, int ncell, int nv_src, int nv_dst) {
    // copies ncell x min(nv_src, nv_dst) pairs, zero-fills the rest of dst
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n = (size_t)ncell * nv_dst;
    if (i >= n) return;
    const size_t c = i / nv_dst, k = i % nv_dst;
    TB a = fromdbl<TB>(0.0), b = fromdbl<TB>(0.0);
    if ((int)k < nv_src) {
        const size_t o = fpos<TA>(c, nv_src, (int)k);
        a = fromdbl<TB>(todbl(src[o]));
        b = fromdbl<TB>(todbl(src[o + kComp<TA>]));
    }
    const size_t o = fpos<TB>(c, nv_dst, (int)k);
    dst[o] = a;
    dst[o + kComp<TB>] = b;
}

// ================================================================== paper sensitivity (K4a)
// Per wall element l (one block): Eq. (sens_J_itf) and (sens_B_itf) with the Gauss gradient of
// Eq. (gaussgrad) from the same interface values as the sweep, phi_w of Eq. (formula_adjointbgk).
// elem[l] = (dL/dA, dL/dx (2), dL/dn (2)).  Sums in FP64 (NI x nv work only).
template <class TS>
__global__ void k_sens_paper_elem(const TS* f, const TS* phi, int nvp, const int4* nb, const double2* S,
                                  const double* Vc, const double4* vd, const double2* fd, const double* gw,
                                  const double* wallD, const double* Fw, double halfTw, MomentJ mj,
                                  double* elem) {
    const int l = blockIdx.x;   // wall cell index (j = 0)
    const int4 n = nb[l];
    const double2 s[4] = {S[4 * l], S[4 * l + 1], S[4 * l + 2], S[4 * l + 3]};
    const double A = sqrt(s[3].x * s[3].x + s[3].y * s[3].y);
    const double nx = s[3].x / A, ny = s[3].y / A, iV = 1.0 / Vc[l];
    const double cw = Fw[l] / wallD[l];
    const int nbs[4] = {n.x, n.y, n.z, n.w};
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    // 0 dA | 1,2 X1 | 3,4 Gp | 5 Pg | 6,7 Vf | 8,9 N1
    for (int k = threadIdx.x; k < nvp; k += blockDim.x) {
        const double4 t = vd[k];
        const double vx = t.x, vy = t.y, w = t.z, m = mj.dx * vx + mj.dy * vy + mj.h * t.w;
        const size_t ol = fpos<TS>(l, nvp, k);
        const double fc1 = todbl(f[ol]), fc2 = todbl(f[ol + kComp<TS>]);
        double F1[4], F2[4];
        for (int e = 0; e < 4; ++e) {
            const double a = s[e].x * vx + s[e].y * vy;
            if (a > 0.0) { F1[e] = fc1; F2[e] = fc2; }
            else if (nbs[e] >= 0) {
                const size_t oe = fpos<TS>(nbs[e], nvp, k);
                F1[e] = todbl(f[oe]);
                F2[e] = todbl(f[oe + kComp<TS>]);
            } else if (nbs[e] == kFar) { F1[e] = fd[k].x; F2[e] = fd[k].y; }
            else { F1[e] = cw * gw[k]; F2[e] = cw * halfTw * gw[k]; }
        }
        double g1x = 0, g1y = 0, g2x = 0, g2y = 0;
        for (int e = 0; e < 4; ++e) {
            g1x += F1[e] * s[e].x; g1y += F1[e] * s[e].y;
            g2x += F2[e] * s[e].x; g2y += F2[e] * s[e].y;
        }
        g1x *= iV; g1y *= iV; g2x *= iV; g2y *= iV;
        const double vn = vx * nx + vy * ny, fl1 = F1[3];
        acc[0] += w * m * vn * fl1;
        acc[1] += w * m * vn * A * g1x;
        acc[2] += w * m * vn * A * g1y;
        acc[6] += w * vx * fl1;
        acc[7] += w * vy * fl1;
        acc[8] += w * m * vx * A * fl1;
        acc[9] += w * m * vy * A * fl1;
        if (vn > 0.0) {
            acc[3] += w * vn * g1x;
            acc[4] += w * vn * g1y;
        } else {
            const size_t op = fpos<TS>(l, nvp, k);
            const double p1 = todbl(phi[op]), p2 = todbl(phi[op + kComp<TS>]);
            const double pw1 = -vn * (p1 + m), pw2 = -vn * p2;
            const double gb1 = gw[k] / wallD[l];
            acc[1] += w * A * (pw1 * g1x + pw2 * g2x);
            acc[2] += w * A * (pw1 * g1y + pw2 * g2y);
            acc[5] += w * (pw1 * gb1 + pw2 * halfTw * gb1);
        }
    }
    __shared__ double sh[10][8];
    for (int i = 0; i < 10; ++i) {
        const double v = warp_sum(acc[i]);
        if ((threadIdx.x & 31) == 0) sh[i][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[10];
        for (int i = 0; i < 10; ++i) {
            r[i] = 0.0;
            for (int j = 0; j < (int)(blockDim.x >> 5); ++j) r[i] += sh[i][j];
        }
        elem[5 * l + 0] = r[0];
        elem[5 * l + 1] = r[1] - A * r[3] * r[5];
        elem[5 * l + 2] = r[2] - A * r[4] * r[5];
        elem[5 * l + 3] = r[8] - A * r[5] * r[6];
        elem[5 * l + 4] = r[9] - A * r[5] * r[7];
    }
}

// Element -> wall node (Eq. sens_nod): node m belongs to elements m-1 (as its first end X(0,m))
// and m (as its second end).  For an end x_a with the other end x_b: dA/dx_a = (x_a - x_b)/A,
// dx_l/dx_a = 1/2, dn/dx_a = sigma R90 n n^T / A, sigma = sign((x_a - x_b) x n).
__global__ void k_sens_paper_nodes(int ni, const double2* nodes, const double2* S, const double* elem,
                                   double* node_grad) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= ni) return;
    double gx = 0.0, gy = 0.0;
    for (int side = 0; side < 2; ++side) {
        // element l spans wall nodes l and l+1
        const int l = side == 0 ? (m - 1 + ni) % ni : m;
        const int ob = side == 0 ? (m - 1 + ni) % ni : (m + 1) % ni;
        const double2 xa = nodes[m], xb = nodes[ob];
        const double2 s = S[4 * l + 3];
        const double A = sqrt(s.x * s.x + s.y * s.y);
        const double nx = s.x / A, ny = s.y / A;
        const double ex = xa.x - xb.x, ey = xa.y - xb.y;
        const double cr = ex * ny - ey * nx;
        const double sg = cr > 0.0 ? 1.0 : (cr < 0.0 ? -1.0 : 0.0);
        const double* e = elem + 5 * l;
        // (dn/dx_a)^T dL/dn with dn/dx_a[r][c] = sg/A * (R90 n)_r n_c, R90 n = (-ny, nx)
        const double rn = sg / A * (-ny * e[3] + nx * e[4]);
        gx += e[0] * ex / A + 0.5 * e[1] + rn * nx;
        gy += e[0] * ey / A + 0.5 * e[2] + rn * ny;
    }
    node_grad[2 * m] = gx;
    node_grad[2 * m + 1] = gy;
}

// ================================================================== full-discrete sensitivity (K4b)
// dJ/dalpha = dJ/dalpha|_f + sum w phi . dR/dalpha|_f.  R depends on the geometry through the face
// vectors S_f (linear in their two end nodes), the volumes V_c and, on the wall, through n_l in
// F_rhow and gbar_w.  Per face f between L (owner) and R:
//   G_f = sum_k w v_k (phi_L - phi_R) . F_{f,k}   (F the upwind interface value)
// so that the face term is G_f . dS_f/dalpha; per cell vol_c = sum_k w phi . (f - g) / tau_c
// multiplies dV_c/dalpha; the wall face adds J's own S-dependence and the n-dependence
// (I - n n^T)/A * H * Vf with H = sum_{a<=0} w a (m gbar1 + phi . gbar), Vf = sum_k w v f1_l.
template <class TS>
__global__ void __launch_bounds__(256, 2) k_sens_faces(const TS* f, const TS* phi, int ncell, int nvp,
                                                    const int4* nb, const double2* S, const double* Vc,
                                                    const typename Vec<typename Pack<TS>::TC>::v4* vt,
                                                    const typename Vec<typename Pack<TS>::TC>::v2* fd,
                                                    const typename Pack<TS>::TC* gw, const double* wallD,
                                                    const double4* prim, const double4* maxw, const double* Fw,
                                                    double inv_tau_inf, double halfTw_d, MomentJ mj, double2* GN,
                                                    double2* GE, double2* GW, double* vol) {
    using TC = typename Pack<TS>::TC;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= ncell) return;
    const int4 n = nb[c];
    const double2 s1d = S[4 * c + 1], s2d = S[4 * c + 2], s3d = S[4 * c + 3];
    const TC s1x = (TC)s1d.x, s1y = (TC)s1d.y, s2x = (TC)s2d.x, s2y = (TC)s2d.y, s3x = (TC)s3d.x, s3y = (TC)s3d.y;
    const double4 pr = prim[c], pm = maxw[c];          // moments (tau); Maxwellian parameters (g)
    const TC u1 = (TC)pm.y, u2 = (TC)pm.z;
    const TC halfT = (TC)(0.5 * pm.w), halfTw = (TC)halfTw_d, dirx = (TC)mj.dx, diry = (TC)mj.dy, hcoef = (TC)mj.h;
    const bool wall = n.w == kWall;
    const TC cw = wall ? (TC)(Fw[c] / wallD[c]) : TC(0);
    const TC gbs = wall ? (TC)(1.0 / wallD[c]) : TC(0);
    Acc<TC> gnx, gny, gex, gey, gwx, gwy, H, vfx, vfy, vs;
    // 16-byte chunks of f and phi of the cell and of its north and east neighbours (coalesced, as in
    // the sweeps); the Maxwellian of the volume term evaluated as in the sweeps
    using PK = Pack<TS>;
    constexpr int KV = PK::KV;
    Gauss<TC> G;
    G.setup((TC)pm.x, u1, u2, (TC)pm.w);
    const size_t nq = (size_t)nvp / KV;
    const uint4* fq = reinterpret_cast<const uint4*>(f);
    const uint4* pq = reinterpret_cast<const uint4*>(phi);
    const size_t north = n.y >= 0 ? (size_t)n.y : (size_t)c;    // far field: own chunk, not used
    const size_t east = (size_t)n.z;
    const bool far = n.y < 0;
    // per-lane sums in plain TC over blocks of kSensBlock chunks, then one compensated add per block
    constexpr int kSensBlock = 4;
    TC b[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) b[i] = TC(0);
    auto flush = [&]() {
        gnx.add(b[0]); gny.add(b[1]); gex.add(b[2]); gey.add(b[3]); vs.add(b[4]);
        if (wall) { gwx.add(b[5]); gwy.add(b[6]); H.add(b[7]); vfx.add(b[8]); vfy.add(b[9]); }
#pragma unroll
        for (int i = 0; i < 10; ++i) b[i] = TC(0);
    };
    int nb_ = 0;
    for (size_t q = lane; q < nq; q += 32) {
        TC fc1[KV], fc2[KV], pc1[KV], pc2[KV], fn1[KV], fn2[KV], pn1[KV], pn2[KV], fe1[KV], fe2[KV], pe1[KV], pe2[KV];
        PK::unpack(ldg16(fq + (size_t)c * nq + q), fc1, fc2);
        PK::unpack(ldg16(pq + (size_t)c * nq + q), pc1, pc2);
        PK::unpack(ldg16(fq + north * nq + q), fn1, fn2);
        PK::unpack(ldg16(pq + north * nq + q), pn1, pn2);
        PK::unpack(ldg16(fq + east * nq + q), fe1, fe2);
        PK::unpack(ldg16(pq + east * nq + q), pe1, pe2);
#pragma unroll
        for (int kk = 0; kk < KV; ++kk) {
            const int k = (int)q * KV + kk;
            const auto t = vt[k];
            const TC vx = t.x, vy = t.y, w = t.z;
            {   // north face: upwind value (own cell on outflow, north cell or far field on inflow)
                const TC a = s1x * vx + s1y * vy;
                TC i1 = fn1[kk], i2 = fn2[kk], q1 = pn1[kk], q2 = pn2[kk];
                if (far) {
                    const auto d = fd[k];
                    i1 = d.x; i2 = d.y; q1 = TC(0); q2 = TC(0);
                }
                const bool out = a > TC(0);
                const TC F1 = out ? fc1[kk] : i1, F2 = out ? fc2[kk] : i2;
                const TC d = w * ((pc1[kk] - q1) * F1 + (pc2[kk] - q2) * F2);
                b[0] += d * vx; b[1] += d * vy;
            }
            {   // east face (always interior)
                const bool out = s2x * vx + s2y * vy > TC(0);
                const TC F1 = out ? fc1[kk] : fe1[kk], F2 = out ? fc2[kk] : fe2[kk];
                const TC d = w * ((pc1[kk] - pe1[kk]) * F1 + (pc2[kk] - pe2[kk]) * F2);
                b[2] += d * vx; b[3] += d * vy;
            }
            if (wall) {
                const TC a = s3x * vx + s3y * vy;
                const TC m = dirx * vx + diry * vy + hcoef * t.w;
                const bool out = a > TC(0);
                const TC gk = gw[k];
                const TC F1 = out ? fc1[kk] : cw * gk, F2 = out ? fc2[kk] : cw * halfTw * gk;
                if (!out) b[7] += w * a * (gk * gbs) * (m + pc1[kk] + halfTw * pc2[kk]);
                const TC d = w * (pc1[kk] * F1 + pc2[kk] * F2 + m * F1);
                b[5] += d * vx; b[6] += d * vy;
                b[8] += w * vx * F1; b[9] += w * vy * F1;
            }
            {   // volume term
                const TC g1 = G.eval(fma(vy, -u2, fma(vx, -u1, (TC)t.w)));
                b[4] += w * (pc1[kk] * (fc1[kk] - g1) + pc2[kk] * (fc2[kk] - halfT * g1));
            }
        }
        if (++nb_ == kSensBlock) { flush(); nb_ = 0; }
    }
    flush();
    const double GNX = warp_sum(gnx.get()), GNY = warp_sum(gny.get()), GEX = warp_sum(gex.get());
    const double GEY = warp_sum(gey.get()), VS = warp_sum(vs.get());
    double GWX = 0, GWY = 0, HH = 0, VFX = 0, VFY = 0;
    if (wall) {
        GWX = warp_sum(gwx.get()); GWY = warp_sum(gwy.get()); HH = warp_sum(H.get());
        VFX = warp_sum(vfx.get()); VFY = warp_sum(vfy.get());
    }
    if (lane == 0) {
        GN[c] = make_double2(GNX, GNY);
        GE[c] = make_double2(GEX, GEY);
        vol[c] = VS * pr.x * sqrt(pr.w) * inv_tau_inf;   // / tau
        if (wall) {
            const double A = sqrt(s3d.x * s3d.x + s3d.y * s3d.y);
            const double nx = s3d.x / A, ny = s3d.y / A;
            const double px = HH * VFX / A, py = HH * VFY / A;     // H Vf / A
            const double dn = px * nx + py * ny;                   // projected with (I - n n^T)
            GW[c] = make_double2(GWX + px - dn * nx, GWY + py - dn * ny);
        }
    }
}

// Node gradient of the full-discrete sensitivity: each node gathers the face and cell terms it
// belongs to (no atomics, fixed order).  Face vector S of an edge P->Q is (Q_y - P_y, P_x - Q_x), so
// d(S.G)/dP = (G_y, -G_x), d(S.G)/dQ = (-G_y, G_x).  Cell volume (CCW corners):
// dV/dP_e = ((P_{e+1} - P_{e-1})_y, (P_{e-1} - P_{e+1})_x) / 2.
__global__ void k_sens_nodes(int ni, int nj, const double2* X, const double2* GN, const double2* GE,
                             const double2* GW, const double* vol, double2* node_grad) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (nj + 1) * ni) return;
    const int j = id / ni, i = id % ni;
    const int im = (i - 1 + ni) % ni, ip = (i + 1) % ni;
    auto x = [&](int jj, int ii) { return X[jj * ni + ii]; };
    double gx = 0.0, gy = 0.0;
    // circumferential edge (j,i) -> (j,i+1)
    if (j >= 1) { const double2 G = GN[(j - 1) * ni + i]; gx += G.y; gy -= G.x; }       // node is P
    else { const double2 G = GW[i]; gx -= G.y; gy += G.x; }                                // wall: node is Q
    // circumferential edge (j,i-1) -> (j,i)
    if (j >= 1) { const double2 G = GN[(j - 1) * ni + im]; gx -= G.y; gy += G.x; }     // node is Q
    else { const double2 G = GW[im]; gx += G.y; gy -= G.x; }                               // wall: node is P
    // radial edges: east face of cell (j, i-1) runs X(j+1,i) -> X(j,i); of cell (j-1,i-1) X(j,i) -> X(j-1,i)
    if (j < nj) { const double2 G = GE[j * ni + im]; gx -= G.y; gy += G.x; }
    if (j >= 1) { const double2 G = GE[(j - 1) * ni + im]; gx += G.y; gy -= G.x; }
    // volumes of the (up to) four cells having this node as a corner
    if (j < nj) {
        double v = vol[j * ni + i];            // corner P0: next P1 = X(j+1,i), prev P3 = X(j,i+1)
        double2 nx = x(j + 1, i), pv = x(j, ip);
        gx += 0.5 * v * (nx.y - pv.y); gy += 0.5 * v * (pv.x - nx.x);
        v = vol[j * ni + im];                  // corner P3 of cell (j,i-1): next P0 = X(j,i-1), prev P2 = X(j+1,i)
        nx = x(j, im); pv = x(j + 1, i);
        gx += 0.5 * v * (nx.y - pv.y); gy += 0.5 * v * (pv.x - nx.x);
    }
    if (j >= 1) {
        double v = vol[(j - 1) * ni + i];      // corner P1 of cell (j-1,i): next P2 = X(j,i+1), prev P0 = X(j-1,i)
        double2 nx = x(j, ip), pv = x(j - 1, i);
        gx += 0.5 * v * (nx.y - pv.y); gy += 0.5 * v * (pv.x - nx.x);
        v = vol[(j - 1) * ni + im];            // corner P2 of cell (j-1,i-1): next P3 = X(j-1,i), prev P1 = X(j,i-1)
        nx = x(j - 1, i); pv = x(j, im);
        gx += 0.5 * v * (nx.y - pv.y); gy += 0.5 * v * (pv.x - nx.x);
    }
    node_grad[id] = make_double2(gx, gy);
}

// grad[p] = sum_{rows j, i} (1 - s_j) node_grad(j,i) . dwall[p][i]  (s_j == nullptr -> rows = 1, weight 1)
__global__ void k_contract(const double2* node_grad, int nrows, int ni, const double* s_j,
                           const double* dwall, double* grad) {
    const int p = blockIdx.x;
    double acc = 0.0;
    for (int id = threadIdx.x; id < nrows * ni; id += blockDim.x) {
        const int j = id / ni, i = id % ni;
        const double wgt = s_j ? 1.0 - s_j[j] : 1.0;
        const double2 g = node_grad[id];
        acc += wgt * (g.x * dwall[((size_t)p * ni + i) * 2] + g.y * dwall[((size_t)p * ni + i) * 2 + 1]);
    }
    __shared__ double sh[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
        grad[p] = s;
    }
}

// Volume constraint (Eq. formula_opt with n into the solid, D = 2): Q = V_min + (1/2) sum_l x_l . S_l
// over the wall elements (x_l the midpoint, S_l = A_l n_l), and dQ/dalpha_p = sum_m dQ/dx_m .
// dwall[p][m] with dQ/dx_m = (1/2)(S_{m-1} + S_m), Eq. (sens_con_nod).  One block.
__global__ void k_volume(int ni, const double2* S, const double2* nodes, double vmin, const double* dwall, int P,
                         double* out) {
    __shared__ double red[32];
    double q = 0.0;
    for (int l = threadIdx.x; l < ni; l += blockDim.x) {
        const double2 a = nodes[l], b = nodes[(l + 1) % ni], s = S[4 * l + 3];
        q += 0.25 * ((a.x + b.x) * s.x + (a.y + b.y) * s.y);
    }
    for (int p = -1; p < P; ++p) {
        double v = q;
        if (p >= 0) {
            v = 0.0;
            for (int m = threadIdx.x; m < ni; m += blockDim.x) {
                const double2 s0 = S[4 * ((m - 1 + ni) % ni) + 3], s1 = S[4 * m + 3];
                v += 0.5 * ((s0.x + s1.x) * dwall[((size_t)p * ni + m) * 2] + (s0.y + s1.y) * dwall[((size_t)p * ni + m) * 2 + 1]);
            }
        }
        v = warp_sum(v);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
            out[p + 1] = p < 0 ? t + vmin : t;
        }
    }
}

// ================================================================== Anderson mixing
// Convergence acceleration of the fixed-point sweeps (the discrete problem and its solution are
// unchanged): every accel_period sweeps map the iterate x to G(x); with r = G(x) - x and the last m
// differences dR, dG of r and G, the next iterate is G - dG gamma, gamma = argmin |r - dR gamma|.
// The vectors are the flat storage arrays (any layout: the operations are elementwise), held in
// TH = the arithmetic type (FP32, or FP64 for FP64 storage).
// ================================================================== refinement (elementwise)
// FP32 chunk i of a state holds (f1_k, f1_k+1, f2_k, f2_k+1) for k = 2 (i mod nvp/2) of cell i div (nvp/2);
// the same four values sit at 4i .. 4i+3 of the FP64 layout in the order (f1_k, f2_k, f1_k+1, f2_k+1).
__global__ void __launch_bounds__(256) k_refine_compose(const float4* __restrict__ fbar, const float4* __restrict__ delta,
                                                        double2* __restrict__ f64, size_t nchunk) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nchunk; i += (size_t)gridDim.x * blockDim.x) {
        const float4 a = fbar[i], d = delta[i];
        f64[2 * i] = make_double2((double)a.x + (double)d.x, (double)a.z + (double)d.z);
        f64[2 * i + 1] = make_double2((double)a.y + (double)d.y, (double)a.w + (double)d.w);
    }
}

__global__ void __launch_bounds__(256) k_refine_diff(const double2* __restrict__ fnew, const double2* __restrict__ fold,
                                                     float4* __restrict__ src, size_t nchunk) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nchunk; i += (size_t)gridDim.x * blockDim.x) {
        const double2 a0 = fnew[2 * i], a1 = fnew[2 * i + 1], b0 = fold[2 * i], b1 = fold[2 * i + 1];
        src[i] = make_float4((float)(a0.x - b0.x), (float)(a1.x - b1.x), (float)(a0.y - b0.y), (float)(a1.y - b1.y));
    }
}

// delta += e, then (fbar, delta) <- (fl(fbar + delta), exact remainder) by the two-sum of Knuth.
__device__ __forceinline__ void two_sum_into(float& a, float& b) {
    const float s = a + b, bb = s - a;
    b = (a - (s - bb)) + (b - bb);
    a = s;
}
__global__ void __launch_bounds__(256) k_refine_update(float4* __restrict__ fbar, float4* __restrict__ delta,
                                                       const float4* __restrict__ e, size_t n4) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        float4 a = fbar[i], d = delta[i];
        const float4 x = e[i];
        d.x += x.x; d.y += x.y; d.z += x.z; d.w += x.w;
        two_sum_into(a.x, d.x); two_sum_into(a.y, d.y); two_sum_into(a.z, d.z); two_sum_into(a.w, d.w);
        fbar[i] = a;
        delta[i] = d;
    }
}

constexpr int kAAMax = 8;             // deepest history
constexpr int kAABlocks = 1216;       // 152 SMs x 8 blocks of 256 threads, grid-stride

// Four consecutive elements (n is a multiple of 8: cells x padded velocities x 2).
template <class T> struct Quad;
template <> struct Quad<float> {
    template <class TH> __device__ static void ld(const float* p, TH (&v)[4]) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    template <class TH> __device__ static void st(float* p, const TH (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
    }
};
template <> struct Quad<double> {
    template <class TH> __device__ static void ld(const double* p, TH (&v)[4]) {
        const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
        v[0] = (TH)a.x; v[1] = (TH)a.y; v[2] = (TH)b.x; v[3] = (TH)b.y;
    }
    template <class TH> __device__ static void st(double* p, const TH (&v)[4]) {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
};
template <> struct Quad<__nv_bfloat16> {
    template <class TH> __device__ static void ld(const __nv_bfloat16* p, TH (&v)[4]) {
        const uint2 a = *reinterpret_cast<const uint2*>(p);
        v[0] = __uint_as_float(a.x << 16); v[1] = __uint_as_float(a.x & 0xffff0000u);
        v[2] = __uint_as_float(a.y << 16); v[3] = __uint_as_float(a.y & 0xffff0000u);
    }
    template <class TH> __device__ static void st(__nv_bfloat16* p, const TH (&v)[4]) {
        const __nv_bfloat162 h0 = __floats2bfloat162_rn((float)v[0], (float)v[1]);
        const __nv_bfloat162 h1 = __floats2bfloat162_rn((float)v[2], (float)v[3]);
        uint2 u;
        memcpy(&u.x, &h0, 4);
        memcpy(&u.y, &h1, 4);
        *reinterpret_cast<uint2*>(p) = u;
    }
};

template <class TS, class TH>
__global__ void __launch_bounds__(256) k_aa_load(size_t n, const TS* __restrict__ F, TH* __restrict__ X) {
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n / 4; q += (size_t)gridDim.x * blockDim.x) {
        TH v[4];
        Quad<TS>::ld(F + 4 * q, v);
        Quad<TH>::st(X + 4 * q, v);
    }
}

// r = G - X, the new differences (slot `slot` of the ring, unless first) and the dots
// dR_i . dR_slot (part[i]) and dR_i . r (part[m + i]) for the cnt columns in use, per block.  The
// dots of FP32 vectors are Kahan-compensated per thread: the least-squares problem of the mixing is
// ill-conditioned (its columns become nearly parallel as the iteration slows), and plain FP32 sums
// of a few hundred terms per thread are not accurate enough for it.
template <class TS, class TH>
__global__ void __launch_bounds__(256) k_aa_collect(size_t n, const TS* __restrict__ G, TH* __restrict__ X,
                                                    TH* __restrict__ Rp, TH* __restrict__ Gp, TH* __restrict__ dR,
                                                    TH* __restrict__ dG, int m, int cnt, int slot, int first,
                                                    double* __restrict__ part) {
    Acc<TH> acc[2 * kAAMax];
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n / 4; q += (size_t)gridDim.x * blockDim.x) {
        const size_t e = 4 * q;
        TH g[4], x[4], r[4];
        Quad<TS>::ld(G + e, g);
        Quad<TH>::ld(X + e, x);
#pragma unroll
        for (int u = 0; u < 4; ++u) r[u] = g[u] - x[u];
        if (first) {
            Quad<TH>::st(X + e, g);
        } else {
            TH rp[4], gp[4], dr[4], dg[4];
            Quad<TH>::ld(Rp + e, rp);
            Quad<TH>::ld(Gp + e, gp);
#pragma unroll
            for (int u = 0; u < 4; ++u) { dr[u] = r[u] - rp[u]; dg[u] = g[u] - gp[u]; }
            Quad<TH>::st(dR + (size_t)slot * n + e, dr);
            Quad<TH>::st(dG + (size_t)slot * n + e, dg);
#pragma unroll
            for (int i = 0; i < kAAMax; ++i) {
                if (i < cnt) {
                    TH c[4];
                    if (i == slot) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) c[u] = dr[u];
                    } else {
                        Quad<TH>::ld(dR + (size_t)i * n + e, c);
                    }
                    acc[i].add((c[0] * dr[0] + c[1] * dr[1]) + (c[2] * dr[2] + c[3] * dr[3]));
                    acc[kAAMax + i].add((c[0] * r[0] + c[1] * r[1]) + (c[2] * r[2] + c[3] * r[3]));
                }
            }
        }
        Quad<TH>::st(Rp + e, r);
        Quad<TH>::st(Gp + e, g);
    }
    if (first) return;
    __shared__ double red[8][2 * kAAMax];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 2 * kAAMax; ++i) {
        const double v = warp_sum(acc[i].get());
        if (lane == 0) red[wid][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * m) {
        const int i = threadIdx.x < m ? threadIdx.x : kAAMax + threadIdx.x - m;
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][i];
        part[(size_t)blockIdx.x * 2 * m + threadIdx.x] = t;
    }
}

// Fixed-order sum of the per-block dots: out[j] = sum_b part[b][j], j < 2m.
__global__ void k_aa_sum(const double* __restrict__ part, int nb, int m2, double* __restrict__ out) {
    const int j = threadIdx.x;
    if (j >= m2) return;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[(size_t)b * m2 + j];
    out[j] = t;
}

// x = G - sum_i gamma_i dG_i into the state (rounded to storage) and X (the stored value); with
// `positive` (a distribution), neg is set when any value turns negative.
template <class TS, class TH>
__global__ void __launch_bounds__(256) k_aa_mix(size_t n, TS* __restrict__ F, TH* __restrict__ X,
                                                const TH* __restrict__ Gp, const TH* __restrict__ dG, int cnt,
                                                const double* __restrict__ gamma, int positive,
                                                int* __restrict__ neg) {
    TH gam[kAAMax];
#pragma unroll
    for (int i = 0; i < kAAMax; ++i) gam[i] = i < cnt ? (TH)gamma[i] : TH(0);
    bool bad = false;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n / 4; q += (size_t)gridDim.x * blockDim.x) {
        const size_t e = 4 * q;
        TH x[4];
        Quad<TH>::ld(Gp + e, x);
#pragma unroll
        for (int i = 0; i < kAAMax; ++i) {
            if (i < cnt) {
                TH d[4];
                Quad<TH>::ld(dG + (size_t)i * n + e, d);
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] -= gam[i] * d[u];
            }
        }
        Quad<TS>::st(F + e, x);
        TH v[4];
        Quad<TS>::ld(F + e, v);                  // X holds the stored (rounded) value
        Quad<TH>::st(X + e, v);
#pragma unroll
        for (int u = 0; u < 4; ++u) bad |= positive && x[u] < TH(0);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(neg, 1);
}

// Undo a rejected mix: the state and X return to G.
template <class TS, class TH>
__global__ void __launch_bounds__(256) k_aa_restore(size_t n, TS* __restrict__ F, TH* __restrict__ X,
                                                    const TH* __restrict__ Gp) {
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n / 4; q += (size_t)gridDim.x * blockDim.x) {
        TH v[4];
        Quad<TH>::ld(Gp + 4 * q, v);
        Quad<TS>::st(F + 4 * q, v);
        Quad<TH>::st(X + 4 * q, v);
    }
}

inline int cdiv(size_t a, size_t b) { return (int)((a + b - 1) / b); }

}  // namespace

// ================================================================== launchers
size_t storage_bytes(int storage) { return storage == 0 ? 16 : (storage == 1 ? 8 : 4); }

cudaError_t launch_flow_tables(const DevGrid& g, DevFlow& fl, cudaStream_t s) {
    const int b = 256, n = cdiv(g.nvp, b);
    k_flow_tables<double><<<n, b, 0, s>>>(g.nvp, g.vd, fl.u1, fl.u2, fl.Tw, fl.fdd, fl.gwd);
    k_flow_tables<float><<<n, b, 0, s>>>(g.nvp, g.vf, fl.u1, fl.u2, fl.Tw, fl.fdf, fl.gwf);
    return cudaGetLastError();
}

cudaError_t launch_wall_setup(const DevMesh& m, const DevGrid& g, const DevFlow& fl, MomentJ mj,
                              double* wallD, double* wallM, cudaStream_t s, bool raw) {
    k_wall_setup<<<m.ni, 256, 0, s>>>(g.nvp, m.Sd, g.vd, fl.gwd, mj, wallD, wallM, raw ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_fill_freestream(int storage, void* f, int ncell, const DevGrid& g, const DevFlow& fl,
                                   cudaStream_t s) {
    const size_t n = (size_t)ncell * g.nvp;
    const int b = 256;
    if (storage == 0) k_fill_freestream<double><<<cdiv(n, b), b, 0, s>>>((double*)f, n, g.nvp, fl.fdd);
    else if (storage == 1) k_fill_freestream<float><<<cdiv(n, b), b, 0, s>>>((float*)f, n, g.nvp, fl.fdf);
    else k_fill_freestream<__nv_bfloat16><<<cdiv(n, b), b, 0, s>>>((__nv_bfloat16*)f, n, g.nvp, fl.fdf);
    return cudaGetLastError();
}

template <class TS, class TC>
void second_order_launch(const void* args, bool adjoint, cudaStream_t s) {
    const auto& a = *static_cast<const SOArgs<TS, TC>*>(args);
    const int nb = cdiv(a.ncell, kWarpsPerBlock);
    if (adjoint) {
        k_so_adjoint_mu<TS><<<nb, 256, 0, s>>>(a);
        k_so_adjoint_defect<TS><<<nb, 256, 0, s>>>(a);
    } else {
        k_so_gradient<TS><<<nb, 256, 0, s>>>(a);
        k_so_defect<TS><<<nb, 256, 0, s>>>(a);
    }
}

cudaError_t launch_so_sens(int storage, const void* args, const void* phi, double2* corner, int ni, int nj,
                           double2* node_grad, cudaStream_t s) {
    const int ncell = ni * nj, nb = cdiv(ncell, kWarpsPerBlock);
    if (storage == 0)
        k_so_sens_cells<double><<<nb, 256, 0, s>>>(*static_cast<const SOArgs<double, double>*>(args), (const double*)phi, corner);
    else if (storage == 1)
        k_so_sens_cells<float><<<nb, 256, 0, s>>>(*static_cast<const SOArgs<float, float>*>(args), (const float*)phi, corner);
    else
        k_so_sens_cells<__nv_bfloat16><<<nb, 256, 0, s>>>(*static_cast<const SOArgs<__nv_bfloat16, float>*>(args),
                                                           (const __nv_bfloat16*)phi, corner);
    const int nn = (nj + 1) * ni;
    k_so_sens_nodes<<<cdiv(nn, 256), 256, 0, s>>>(ni, nj, corner, node_grad);
    return cudaGetLastError();
}

cudaError_t launch_second_order(int storage, const void* args, bool adjoint, cudaStream_t s) {
    if (storage == 0) second_order_launch<double, double>(args, adjoint, s);
    else if (storage == 1) second_order_launch<float, float>(args, adjoint, s);
    else second_order_launch<__nv_bfloat16, float>(args, adjoint, s);
    return cudaGetLastError();
}

cudaError_t launch_wait_probe(int* err, cudaStream_t s) {
    k_wait_probe<<<1, 32, 0, s>>>(err);
    return cudaGetLastError();
}

cudaError_t launch_prim_to_W(int ncell, const double4* prim, double* W, cudaStream_t s) {
    k_prim_to_W<<<cdiv(ncell, 256), 256, 0, s>>>(ncell, prim, W);
    return cudaGetLastError();
}

cudaError_t launch_moment_shift(int storage, void* f, const DevMesh& m, const DevGrid& g, const double4* prim,
                                const double* W, cudaStream_t s) {
    const int nb = cdiv(m.ncell, kWarpsPerBlock);
    if (storage == 0) k_moment_shift<double><<<nb, 256, 0, s>>>((double*)f, m.ncell, g.nvp, g.vd, prim, W);
    else if (storage == 1) k_moment_shift<float><<<nb, 256, 0, s>>>((float*)f, m.ncell, g.nvp, g.vd, prim, W);
    else k_moment_shift<__nv_bfloat16><<<nb, 256, 0, s>>>((__nv_bfloat16*)f, m.ncell, g.nvp, g.vd, prim, W);
    return cudaGetLastError();
}

cudaError_t launch_coarse_assemble(int storage, const DevMesh& m, const DevGrid& g, const DevFlow& fl,
                                   const double4* prim, double* out, double* dinv, cudaStream_t s) {
    const int nb = cdiv(m.ncell, kWarpsPerBlock);
    if (storage == 0)
        k_coarse_assemble<double><<<nb, 256, 0, s>>>(m.ncell, g.nvp, g.vd, m.Sd, m.nb, prim, fl.gwd, fl.wallD, 0.5 * fl.Tw, out, dinv);
    else
        k_coarse_assemble<float><<<nb, 256, 0, s>>>(m.ncell, g.nvp, g.vf, m.Sd, m.nb, prim, fl.gwf, fl.wallD, 0.5 * fl.Tw, out, dinv);
    return cudaGetLastError();
}

cudaError_t launch_coarse_target(int ncell, const double4* prim, const double4* dW, double omega, double cap,
                                 double* W, cudaStream_t s) {
    k_coarse_target<<<cdiv(ncell, 256), 256, 0, s>>>(ncell, prim, dW, omega, cap, W);
    return cudaGetLastError();
}

cudaError_t launch_primal_restrict(int storage, const DevMesh& m, const DevGrid& g, const double4* prim_old,
                                   double inv_tau_inf, const void* f_old, const void* f_new, double4* rW,
                                   cudaStream_t s) {
    const int nb = cdiv(m.ncell, kWarpsPerBlock);
    if (storage == 0)
        k_primal_restrict<double, double><<<nb, 256, 0, s>>>(m.ncell, g.nvp, g.vd, m.Sd, m.Vd, prim_old, inv_tau_inf,
                                                             (const double*)f_old, (const double*)f_new, rW);
    else if (storage == 1)
        k_primal_restrict<float, float><<<nb, 256, 0, s>>>(m.ncell, g.nvp, g.vf, m.Sd, m.Vd, prim_old, inv_tau_inf,
                                                           (const float*)f_old, (const float*)f_new, rW);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_adjoint_restrict(int storage, const DevMesh& m, const DevGrid& g, const double4* prim,
                                    double inv_tau_inf, const void* phi_o, const void* phi_n, double4* rA,
                                    cudaStream_t s) {
    const int nb = cdiv(m.ncell, kWarpsPerBlock);
    if (storage == 0)
        k_adjoint_restrict<double, double><<<nb, 256, 0, s>>>(m.ncell, g.nvp, g.vd, m.Sd, m.Vd, prim, inv_tau_inf,
                                                              (const double*)phi_o, (const double*)phi_n, rA);
    else if (storage == 1)
        k_adjoint_restrict<float, float><<<nb, 256, 0, s>>>(m.ncell, g.nvp, g.vf, m.Sd, m.Vd, prim, inv_tau_inf,
                                                            (const float*)phi_o, (const float*)phi_n, rA);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_adjoint_shift(int storage, const DevMesh& m, const DevGrid& g, const double4* x, double omega,
                                 void* phi, cudaStream_t s) {
    const int nb = cdiv(m.ncell, kWarpsPerBlock);
    if (storage == 0) k_adjoint_shift<double><<<nb, 256, 0, s>>>(m.ncell, g.nvp, g.vd, x, omega, (double*)phi);
    else if (storage == 1) k_adjoint_shift<float><<<nb, 256, 0, s>>>(m.ncell, g.nvp, g.vd, x, omega, (float*)phi);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_coarse_lin_shift(const DevMesh& m, const DevGrid& g, const double4* prim, const double4* x,
                                    double omega, double cap, float* e, double4* dW, double* dF, cudaStream_t s) {
    k_coarse_lin_shift<<<cdiv(m.ncell, kWarpsPerBlock), 256, 0, s>>>(m.ncell, g.nvp, g.vd, m.Sd, m.nb, prim, x, omega,
                                                                      cap, e, dW, dF);
    return cudaGetLastError();
}

cudaError_t launch_maxwell_fit(int storage, const DevMesh& m, const DevGrid& g, const double4* prim, double4* fit,
                               bool warm, int iters, double* Kinv, cudaStream_t s) {
    const int nb = cdiv(m.ncell, kWarpsPerBlock);
    if (storage == 0) k_maxwell_fit<double><<<nb, 256, 0, s>>>(m.ncell, g.nvp, g.vd, prim, fit, warm, iters, Kinv);
    else k_maxwell_fit<float><<<nb, 256, 0, s>>>(m.ncell, g.nvp, g.vf, prim, fit, warm, iters, Kinv);
    return cudaGetLastError();
}

cudaError_t launch_moments(int storage, const void* f, const DevMesh& m, const DevGrid& g, double4* prim,
                           double* Fw, cudaStream_t s) {
    const int nb = cdiv(m.ncell, kWarpsPerBlock);
    if (storage == 0) k_moments<double><<<nb, 256, 0, s>>>((const double*)f, m.ncell, g.nvp, m.nb, m.Sd, g.vd, prim, Fw, nullptr, m.ni);
    else if (storage == 1) k_moments<float><<<nb, 256, 0, s>>>((const float*)f, m.ncell, g.nvp, m.nb, m.Sd, g.vd, prim, Fw, nullptr, m.ni);
    else k_moments<__nv_bfloat16><<<nb, 256, 0, s>>>((const __nv_bfloat16*)f, m.ncell, g.nvp, m.nb, m.Sd, g.vd, prim, Fw, nullptr, m.ni);
    return cudaGetLastError();
}

cudaError_t launch_shard_moments(int storage, const void* f, const DevMesh& m, const DevGrid& g, double* part,
                                 cudaStream_t s) {
    const int nb = cdiv(m.ncell, kWarpsPerBlock);
    if (storage == 0) k_moments<double><<<nb, 256, 0, s>>>((const double*)f, m.ncell, g.nvp, m.nb, m.Sd, g.vd, nullptr, nullptr, part, m.ni);
    else if (storage == 1) k_moments<float><<<nb, 256, 0, s>>>((const float*)f, m.ncell, g.nvp, m.nb, m.Sd, g.vd, nullptr, nullptr, part, m.ni);
    else k_moments<__nv_bfloat16><<<nb, 256, 0, s>>>((const __nv_bfloat16*)f, m.ncell, g.nvp, m.nb, m.Sd, g.vd, nullptr, nullptr, part, m.ni);
    return cudaGetLastError();
}

// The shards' summed buffer: primitives of the whole grid's moments (as the sweep's epilogue forms
// them), the residual and drag partials and the wall density for the finalize, and the wall
// normaliser D_l and M_l of the whole grid.
__global__ void k_shard_combine(int ncell, int ni, const double* __restrict__ t, double4* __restrict__ prim,
                                double* __restrict__ Fw, double* __restrict__ respart, double* __restrict__ Jpart,
                                double* __restrict__ wallD, double* __restrict__ wallM) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double4 W = reinterpret_cast<const double4*>(t)[c];
    const double u1 = W.y / W.x, u2 = W.z / W.x;
    prim[c] = make_double4(W.x, u1, u2, (2.0 / 3.0) * (W.w / W.x - 0.5 * (u1 * u1 + u2 * u2)));
    respart[c] = t[4 * (size_t)ncell + c];
    if (c < ni) {
        const size_t o = 5 * (size_t)ncell;
        Fw[c] = t[o + c];
        Jpart[c] = t[o + ni + c];
        const double D = t[o + 2 * ni + c];
        wallD[c] = D;
        wallM[c] = t[o + 3 * ni + c] / D;
    }
}

cudaError_t launch_shard_combine(const DevMesh& m, const double* total, double4* prim, double* Fw, double* respart,
                                 double* Jpart, double* wallD, double* wallM, cudaStream_t s) {
    k_shard_combine<<<cdiv(m.ncell, 256), 256, 0, s>>>(m.ncell, m.ni, total, prim, Fw, respart, Jpart, wallD, wallM);
    return cudaGetLastError();
}

template <class TS, class TC>
void primal_launch(const void* args, const TmaMaps& maps, bool res, cudaStream_t s) {
    const auto& a = *static_cast<const PrimalArgs<TS, TC>*>(args);
    const dim3 grid(a.ni, cdiv(a.nj, kWarpsPerBlock));
    constexpr int sm = primal_smem_bytes<TS>();
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        cudaFuncSetAttribute(k_primal_sweep<TS, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_primal_sweep<TS, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_primal_sweep<TS, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_primal_sweep<TS, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        attr[dev] = true;
    }
    if (a.defect) {
        if (res) k_primal_sweep<TS, true, true><<<grid, 256, sm, s>>>(a, maps.col, maps.side);
        else k_primal_sweep<TS, false, true><<<grid, 256, sm, s>>>(a, maps.col, maps.side);
    } else {
        if (res) k_primal_sweep<TS, true, false><<<grid, 256, sm, s>>>(a, maps.col, maps.side);
        else k_primal_sweep<TS, false, false><<<grid, 256, sm, s>>>(a, maps.col, maps.side);
    }
}

cudaError_t launch_primal_sweep(int storage, const void* args, const TmaMaps& maps, bool res, cudaStream_t s) {
    if (storage == 0) primal_launch<double, double>(args, maps, res, s);
    else if (storage == 1) primal_launch<float, float>(args, maps, res, s);
    else primal_launch<__nv_bfloat16, float>(args, maps, res, s);
    return cudaGetLastError();
}

cudaError_t launch_primal_lin_sweep(const void* args, const TmaMaps& maps, bool res, bool rm, cudaStream_t s) {
    const auto& a = *static_cast<const PrimalArgs<float, float>*>(args);
    if (!a.lin_src || !a.lin_f || !a.dW_old || !a.dW_new || (rm && (!res || !a.rW))) return cudaErrorInvalidValue;
    const dim3 grid(a.ni, cdiv(a.nj, kWarpsPerBlock));
    constexpr int sm = primal_smem_bytes<float>();
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        cudaFuncSetAttribute(k_primal_lin_sweep<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_primal_lin_sweep<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_primal_lin_sweep<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        attr[dev] = true;
    }
    if (rm) k_primal_lin_sweep<true, true><<<grid, 256, sm, s>>>(a, maps.col, maps.side);
    else if (res) k_primal_lin_sweep<true, false><<<grid, 256, sm, s>>>(a, maps.col, maps.side);
    else k_primal_lin_sweep<false, false><<<grid, 256, sm, s>>>(a, maps.col, maps.side);
    return cudaGetLastError();
}

template <class TS, class TC>
void shard_launch(const void* args, const TmaMaps& maps, bool res, cudaStream_t s) {
    const auto& a = *static_cast<const PrimalArgs<TS, TC>*>(args);
    const dim3 grid(a.ni, cdiv(a.nj, kWarpsPerBlock));
    constexpr int sm = primal_smem_bytes<TS>();
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        cudaFuncSetAttribute(k_primal_shard_sweep<TS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_primal_shard_sweep<TS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        attr[dev] = true;
    }
    if (res) k_primal_shard_sweep<TS, true><<<grid, 256, sm, s>>>(a, maps.col, maps.side);
    else k_primal_shard_sweep<TS, false><<<grid, 256, sm, s>>>(a, maps.col, maps.side);
}

template <class TS, class TC>
void rm_launch(const void* args, const TmaMaps& maps, cudaStream_t s) {
    const auto& a = *static_cast<const PrimalArgs<TS, TC>*>(args);
    const dim3 grid(a.ni, cdiv(a.nj, kWarpsPerBlock));
    constexpr int sm = primal_smem_bytes<TS>();
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        cudaFuncSetAttribute(k_primal_sweep_rm<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        attr[dev] = true;
    }
    k_primal_sweep_rm<TS><<<grid, 256, sm, s>>>(a, maps.col, maps.side);
}

cudaError_t launch_primal_sweep_rm(int storage, const void* args, const TmaMaps& maps, cudaStream_t s) {
    if (storage == 0) rm_launch<double, double>(args, maps, s);
    else if (storage == 1) rm_launch<float, float>(args, maps, s);
    else rm_launch<__nv_bfloat16, float>(args, maps, s);
    return cudaGetLastError();
}

cudaError_t launch_primal_shard_sweep(int storage, const void* args, const TmaMaps& maps, bool res, cudaStream_t s) {
    if (storage == 0) shard_launch<double, double>(args, maps, res, s);
    else if (storage == 1) shard_launch<float, float>(args, maps, res, s);
    else shard_launch<__nv_bfloat16, float>(args, maps, res, s);
    return cudaGetLastError();
}

cudaError_t launch_refine_compose(const float* fbar, const float* delta, double* f64, int ncell, int nvp,
                                  cudaStream_t s) {
    const size_t n = (size_t)ncell * nvp / 2;
    k_refine_compose<<<std::min<size_t>(cdiv(n, 256), 152 * 16), 256, 0, s>>>(
        reinterpret_cast<const float4*>(fbar), reinterpret_cast<const float4*>(delta), reinterpret_cast<double2*>(f64), n);
    return cudaGetLastError();
}

cudaError_t launch_refine_diff(const double* f64_new, const double* f64_old, float* src, int ncell, int nvp,
                               cudaStream_t s) {
    const size_t n = (size_t)ncell * nvp / 2;
    k_refine_diff<<<std::min<size_t>(cdiv(n, 256), 152 * 16), 256, 0, s>>>(
        reinterpret_cast<const double2*>(f64_new), reinterpret_cast<const double2*>(f64_old),
        reinterpret_cast<float4*>(src), n);
    return cudaGetLastError();
}

cudaError_t launch_refine_update(float* fbar, float* delta, const float* e, size_t n, cudaStream_t s) {
    const size_t n4 = n / 4;
    k_refine_update<<<std::min<size_t>(cdiv(n4, 256), 152 * 16), 256, 0, s>>>(
        reinterpret_cast<float4*>(fbar), reinterpret_cast<float4*>(delta), reinterpret_cast<const float4*>(e), n4);
    return cudaGetLastError();
}

template <class TS, class TC>
void adjoint_launch(const void* args, const TmaMaps& phi_maps, const TmaMaps& f_maps, bool update, bool res,
                    cudaStream_t s) {
    const auto& a = *static_cast<const AdjointArgs<TS, TC>*>(args);
    const dim3 grid(a.ni, cdiv(a.nj, kWarpsPerBlock));
    constexpr int sm = adjoint_smem_bytes<TS>();
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        cudaFuncSetAttribute(k_adjoint_sweep<TS, false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_adjoint_sweep<TS, true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_adjoint_sweep<TS, true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_adjoint_sweep<TS, true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_adjoint_sweep<TS, true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        attr[dev] = true;
    }
    const CUtensorMap &pc = phi_maps.col, &ps = phi_maps.side, &fs = f_maps.side;
    if (!update) k_adjoint_sweep<TS, false, false, false><<<grid, 256, sm, s>>>(a, pc, ps, fs);
    else if (a.defect) {
        if (res) k_adjoint_sweep<TS, true, true, true><<<grid, 256, sm, s>>>(a, pc, ps, fs);
        else k_adjoint_sweep<TS, true, false, true><<<grid, 256, sm, s>>>(a, pc, ps, fs);
    } else if (res) k_adjoint_sweep<TS, true, true, false><<<grid, 256, sm, s>>>(a, pc, ps, fs);
    else k_adjoint_sweep<TS, true, false, false><<<grid, 256, sm, s>>>(a, pc, ps, fs);
}

cudaError_t launch_adjoint_sweep(int storage, const void* args, const TmaMaps& phi_maps, const TmaMaps& f_maps,
                                 bool update, bool res, cudaStream_t s) {
    if (storage == 0) adjoint_launch<double, double>(args, phi_maps, f_maps, update, res, s);
    else if (storage == 1) adjoint_launch<float, float>(args, phi_maps, f_maps, update, res, s);
    else adjoint_launch<__nv_bfloat16, float>(args, phi_maps, f_maps, update, res, s);
    return cudaGetLastError();
}

// Tensor maps of one distribution buffer: [nj][ni][nq*4 uint32], boxes of 32 chunks x 1 cell x
// {10, 8} rows, zero fill outside the tensor.
cudaError_t make_tmamaps(void* base, int ni, int nj, int nq, TmaMaps* out) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)nq * 4, (cuuint64_t)ni, (cuuint64_t)nj};
    const cuuint64_t strides[2] = {(cuuint64_t)nq * 16, (cuuint64_t)nq * 16 * ni};
    const cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t box10[3] = {128u * kCPL, 1, 10}, box8[3] = {128u * kCPL, 1, 8};
    CUresult r = encode(&out->col, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, base, dims, strides, box10, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
        r = encode(&out->side, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, base, dims, strides, box8, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_adjoint_cellconst(int storage, const double4* prim, const double4* maxw, const DevMesh& m,
                                     double inv_tau_inf,
                                     void* out, cudaStream_t s) {
    const int b = 256;
    if (storage == 0) k_adjoint_cellconst<double><<<cdiv(m.ncell, b), b, 0, s>>>(m.ncell, prim, maxw, m.Vd, inv_tau_inf, (AdjCell<double>*)out);
    else k_adjoint_cellconst<float><<<cdiv(m.ncell, b), b, 0, s>>>(m.ncell, prim, maxw, m.Vd, inv_tau_inf, (AdjCell<float>*)out);
    return cudaGetLastError();
}

template <class TS, class TC>
void primal_batch_launch(const void* descs, const int4* items, int n_items, const int* count, int parity, bool res,
                         cudaStream_t s) {
    constexpr int sm = primal_smem_bytes<TS>();
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        cudaFuncSetAttribute(k_primal_sweep_batch<TS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_primal_sweep_batch<TS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        attr[dev] = true;
    }
    const auto* d = static_cast<const PrimalBatchDesc<TS>*>(descs);
    if (res) k_primal_sweep_batch<TS, true><<<n_items, 256, sm, s>>>(d, items, count, parity);
    else k_primal_sweep_batch<TS, false><<<n_items, 256, sm, s>>>(d, items, count, parity);
}

cudaError_t launch_primal_sweep_batch(int storage, const void* descs, const int4* items, int n_items, const int* count,
                                      int parity, bool res, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    if (storage == 0) primal_batch_launch<double, double>(descs, items, n_items, count, parity, res, s);
    else if (storage == 1) primal_batch_launch<float, float>(descs, items, n_items, count, parity, res, s);
    else primal_batch_launch<__nv_bfloat16, float>(descs, items, n_items, count, parity, res, s);
    return cudaGetLastError();
}

template <class TS, class TC>
void adjoint_batch_launch(const void* descs, const int4* items, int n_items, const int* count, int parity, bool res,
                          cudaStream_t s) {
    constexpr int sm = adjoint_smem_bytes<TS>();
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        cudaFuncSetAttribute(k_adjoint_sweep_batch<TS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_adjoint_sweep_batch<TS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        attr[dev] = true;
    }
    const auto* d = static_cast<const AdjointBatchDesc<TS>*>(descs);
    if (res) k_adjoint_sweep_batch<TS, true><<<n_items, 256, sm, s>>>(d, items, count, parity);
    else k_adjoint_sweep_batch<TS, false><<<n_items, 256, sm, s>>>(d, items, count, parity);
}

cudaError_t launch_adjoint_sweep_batch(int storage, const void* descs, const int4* items, int n_items, const int* count,
                                       int parity, bool res, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    if (storage == 0) adjoint_batch_launch<double, double>(descs, items, n_items, count, parity, res, s);
    else if (storage == 1) adjoint_batch_launch<float, float>(descs, items, n_items, count, parity, res, s);
    else adjoint_batch_launch<__nv_bfloat16, float>(descs, items, n_items, count, parity, res, s);
    return cudaGetLastError();
}

// One block per request: out[2r] = sum respart_r, out[2r+1] = sum_l Jpart_l + Fw_l M_l (as k_finalize).
// *count (device memory) requests are in use; the grid is the table's capacity.
__global__ void k_finalize_batch(const FinalizeDesc* __restrict__ fd, const int* __restrict__ count, double* out) {
    const int r = blockIdx.x;
    if (r >= *count) return;
    const FinalizeDesc d = fd[r];
    __shared__ double s0[32], s1[32];
    double a = 0.0, b = 0.0;
    for (int c = threadIdx.x; c < d.ncell; c += blockDim.x) a += d.respart[c];
    if (d.Jpart)
        for (int l = threadIdx.x; l < d.ni; l += blockDim.x) b += d.Jpart[l] + (d.Fw ? d.Fw[l] * d.M[l] : 0.0);
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) { s0[threadIdx.x >> 5] = a; s1[threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, Bsum = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { A += s0[i]; Bsum += s1[i]; }
        out[2 * r] = A;
        out[2 * r + 1] = Bsum;
    }
}

cudaError_t launch_finalize_batch(const FinalizeDesc* fd, int n, const int* count, double* out, cudaStream_t s) {
    if (n > 0) k_finalize_batch<<<n, 1024, 0, s>>>(fd, count, out);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* respart, int ncell, const double* Jpart, const double* Fw,
                            const double* M, int ni, double* out, cudaStream_t s) {
    k_finalize<<<1, 1024, 0, s>>>(respart, ncell, Jpart, Fw, M, ni, out);
    return cudaGetLastError();
}

cudaError_t launch_functional(int storage, const void* f, const DevMesh& m, const DevGrid& g, const DevFlow& fl,
                              const double* Fw, MomentJ mj, double* face_out, double* out,
                              cudaStream_t s) {
    if (storage == 0)
        k_functional<double><<<m.ni, 256, 0, s>>>((const double*)f, g.nvp, m.Sd, g.vd, fl.gwd, fl.wallD, Fw, mj, face_out);
    else if (storage == 1)
        k_functional<float><<<m.ni, 256, 0, s>>>((const float*)f, g.nvp, m.Sd, g.vd, fl.gwd, fl.wallD, Fw, mj, face_out);
    else
        k_functional<__nv_bfloat16><<<m.ni, 256, 0, s>>>((const __nv_bfloat16*)f, g.nvp, m.Sd, g.vd, fl.gwd, fl.wallD, Fw, mj, face_out);
    k_finalize<<<1, 1024, 0, s>>>(face_out, 0, face_out, nullptr, nullptr, m.ni, out);
    return cudaGetLastError();
}

cudaError_t launch_convert(int storage, int direction, const void* src, void* dst, int ncell, int nv, int nvp,
                           cudaStream_t s) {
    const int b = 256;
    if (direction == 0) {   // device storage (nvp) -> double (nv)
        const size_t n = (size_t)ncell * nv;
        if (storage == 0) k_convert<double, double><<<cdiv(n, b), b, 0, s>>>((const double*)src, (double*)dst, ncell, nvp, nv);
        else if (storage == 1) k_convert<float, double><<<cdiv(n, b), b, 0, s>>>((const float*)src, (double*)dst, ncell, nvp, nv);
        else k_convert<__nv_bfloat16, double><<<cdiv(n, b), b, 0, s>>>((const __nv_bfloat16*)src, (double*)dst, ncell, nvp, nv);
    } else {                 // double (nv) -> device storage (nvp)
        const size_t n = (size_t)ncell * nvp;
        if (storage == 0) k_convert<double, double><<<cdiv(n, b), b, 0, s>>>((const double*)src, (double*)dst, ncell, nv, nvp);
        else if (storage == 1) k_convert<double, float><<<cdiv(n, b), b, 0, s>>>((const double*)src, (float*)dst, ncell, nv, nvp);
        else k_convert<double, __nv_bfloat16><<<cdiv(n, b), b, 0, s>>>((const double*)src, (__nv_bfloat16*)dst, ncell, nv, nvp);
    }
    return cudaGetLastError();
}

cudaError_t launch_sens_paper(int storage, const DevMesh& m, const DevGrid& g, const DevFlow& fl, const void* f,
                              const void* phi, const double* Fw, MomentJ mj, double* elem,
                              double* node_grad, cudaStream_t s) {
    const double hT = 0.5 * fl.Tw;
    if (storage == 0)
        k_sens_paper_elem<double><<<m.ni, 256, 0, s>>>((const double*)f, (const double*)phi, g.nvp, m.nb, m.Sd, m.Vd, g.vd,
                                                       fl.fdd, fl.gwd, fl.wallD, Fw, hT, mj, elem);
    else if (storage == 1)
        k_sens_paper_elem<float><<<m.ni, 256, 0, s>>>((const float*)f, (const float*)phi, g.nvp, m.nb, m.Sd, m.Vd, g.vd,
                                                      fl.fdd, fl.gwd, fl.wallD, Fw, hT, mj, elem);
    else
        k_sens_paper_elem<__nv_bfloat16><<<m.ni, 256, 0, s>>>((const __nv_bfloat16*)f, (const __nv_bfloat16*)phi, g.nvp,
                                                              m.nb, m.Sd, m.Vd, g.vd, fl.fdd, fl.gwd, fl.wallD, Fw, hT,
                                                              mj, elem);
    k_sens_paper_nodes<<<cdiv(m.ni, 128), 128, 0, s>>>(m.ni, m.nodes, m.Sd, elem, node_grad);
    return cudaGetLastError();
}

cudaError_t launch_sens_full(int storage, const DevMesh& m, const DevGrid& g, const DevFlow& fl, const void* f,
                             const void* phi, const double4* prim, const double4* maxw, const double* Fw, MomentJ mj,
                             double2* GN, double2* GE, double2* GW, double* vol, double2* node_grad, cudaStream_t s) {
    const int nb = cdiv(m.ncell, kWarpsPerBlock);
    const double hT = 0.5 * fl.Tw, it = 1.0 / fl.tau_inf;
    if (storage == 0)
        k_sens_faces<double><<<nb, 256, 0, s>>>((const double*)f, (const double*)phi, m.ncell, g.nvp, m.nb, m.Sd, m.Vd,
                                                g.vd, fl.fdd, fl.gwd, fl.wallD, prim, maxw, Fw, it, hT, mj, GN, GE,
                                                GW, vol);
    else if (storage == 1)
        k_sens_faces<float><<<nb, 256, 0, s>>>((const float*)f, (const float*)phi, m.ncell, g.nvp, m.nb, m.Sd, m.Vd,
                                               g.vf, fl.fdf, fl.gwf, fl.wallD, prim, maxw, Fw, it, hT, mj, GN, GE,
                                               GW, vol);
    else
        k_sens_faces<__nv_bfloat16><<<nb, 256, 0, s>>>((const __nv_bfloat16*)f, (const __nv_bfloat16*)phi, m.ncell,
                                                       g.nvp, m.nb, m.Sd, m.Vd, g.vf, fl.fdf, fl.gwf, fl.wallD, prim,
                                                       maxw, Fw, it, hT, mj, GN, GE, GW, vol);
    const int nn = (m.nj + 1) * m.ni;
    k_sens_nodes<<<cdiv(nn, 256), 256, 0, s>>>(m.ni, m.nj, m.nodes, GN, GE, GW, vol, node_grad);
    return cudaGetLastError();
}

int aa_max_depth() { return kAAMax; }
int aa_blocks() { return kAABlocks; }

#define DVM_AA_DISPATCH(storage, CALL)                                                                   \
    switch (storage) {                                                                                   \
        case 0: { using TS = double; using TH = double; CALL; } break;                                   \
        case 1: { using TS = float; using TH = float; CALL; } break;                                     \
        default: { using TS = __nv_bfloat16; using TH = float; CALL; } break;                            \
    }

cudaError_t launch_aa_load(int storage, size_t n, const void* F, void* X, cudaStream_t s) {
    DVM_AA_DISPATCH(storage, (k_aa_load<TS, TH><<<kAABlocks, 256, 0, s>>>(n, (const TS*)F, (TH*)X)))
    return cudaGetLastError();
}

cudaError_t launch_aa_collect(int storage, size_t n, const void* G, void* X, void* Rp, void* Gp, void* dR, void* dG,
                              int m, int cnt, int slot, int first, double* part, double* out, cudaStream_t s) {
    DVM_AA_DISPATCH(storage, (k_aa_collect<TS, TH><<<kAABlocks, 256, 0, s>>>(n, (const TS*)G, (TH*)X, (TH*)Rp, (TH*)Gp,
                                                                          (TH*)dR, (TH*)dG, m, cnt, slot, first, part)))
    if (!first) k_aa_sum<<<1, 32, 0, s>>>(part, kAABlocks, 2 * m, out);
    return cudaGetLastError();
}

cudaError_t launch_aa_mix(int storage, size_t n, void* F, void* X, const void* Gp, const void* dG, int cnt,
                          const double* gamma, int positive, int* neg, cudaStream_t s) {
    DVM_AA_DISPATCH(storage, (k_aa_mix<TS, TH><<<kAABlocks, 256, 0, s>>>(n, (TS*)F, (TH*)X, (const TH*)Gp, (const TH*)dG,
                                                                      cnt, gamma, positive, neg)))
    return cudaGetLastError();
}

cudaError_t launch_aa_restore(int storage, size_t n, void* F, void* X, const void* Gp, cudaStream_t s) {
    DVM_AA_DISPATCH(storage, (k_aa_restore<TS, TH><<<kAABlocks, 256, 0, s>>>(n, (TS*)F, (TH*)X, (const TH*)Gp)))
    return cudaGetLastError();
}
#undef DVM_AA_DISPATCH

cudaError_t launch_volume(const DevMesh& m, double vmin, const double* dwall, int P, double* out, cudaStream_t s) {
    k_volume<<<1, 256, 0, s>>>(m.ni, m.Sd, m.nodes, vmin, dwall, P, out);
    return cudaGetLastError();
}

cudaError_t launch_contract(const double2* node_grad, int nrows, int ni, const double* s_j, const double* dwall,
                            int P, double* grad, cudaStream_t s) {
    if (P > 0) k_contract<<<P, 256, 0, s>>>(node_grad, nrows, ni, s_j, dwall, grad);
    return cudaGetLastError();
}

}  // namespace dvm
