// batch.cu -- batched kernels: every problem of a batch in one launch per step (batch.cuh).
//
// Each kernel takes the device array of (problem, level) items and a BLaunch listing the items
// that take part with their first blocks; a block binary-searches its slot, decodes its local
// block index in the item's own geometry and runs the same per-point or per-tile body as the
// single-problem kernels (setup_core.cuh, march.cuh, exp_core.cuh, jcg_core.cuh).
#include "batch.cuh"

#include <algorithm>

#include "../../include/ecmg.h"
#include "exp_core.cuh"
#include "jcg_core.cuh"
#include "march.cuh"
#include "march_fx.cuh"
#include "setup_core.cuh"
#include "stencil_core.cuh"

namespace ecmg {
namespace {

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

constexpr int FLAT_TPB = 256;                  // BG_FLAT: 256 threads x 4 vectors of 4 floats
constexpr int ROWS_PER_BLOCK = 32;             // BG_ROWS: 8 warps x 4 rows
constexpr int EXP_TPB = 128;

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---- block -> item ---------------------------------------------------------------------------
struct Slot {
    int item;   // index into the item array
    int lb;     // block index inside the item
    int nb;     // blocks of the item in this launch
};
__device__ __forceinline__ Slot find_slot(const BLaunch& L)
{
    const int b = blockIdx.x;
    int lo = 0, hi = L.n;  // L.start[lo] <= b < L.start[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (L.start[mid] <= b) lo = mid;
        else hi = mid;
    }
    return Slot{L.id[lo], b - L.start[lo], L.start[lo + 1] - L.start[lo]};
}

// Work of a BG_SPAN block: node planes k0 .. k1-1, in each the vectors [v0, v1) of the plane's
// span (4-element vectors from node (0, 0, k)).
struct SpanRange {
    int k0, k1, v0, v1;
};
__device__ __forceinline__ SpanRange span_of(const Grid& g, int lb)
{
    const int nv = span_v4(g), ppb = span_planes_per_block(g), cpp = span_chunks_per_plane(g);
    if (cpp == 1) return SpanRange{lb * ppb, min((lb + 1) * ppb, g.nz + 1), 0, nv};
    // a large plane in cpp chunks of (nearly) equal length
    const int k = lb / cpp, c = lb - k * cpp, len = (nv + cpp - 1) / cpp;
    return SpanRange{k, k + 1, c * len, min((c + 1) * len, nv)};
}
// The same for a BG_SPAN_FINE block: chunk c of at most SPAN_FINE_V4 vectors of plane k.
__device__ __forceinline__ SpanRange span_fine_of(const Grid& g, int lb)
{
    const int nv = span_v4(g), cpp = (nv + SPAN_FINE_V4 - 1) / SPAN_FINE_V4;
    const int k = lb / cpp, c = lb - k * cpp;
    return SpanRange{k, k + 1, c * SPAN_FINE_V4, min((c + 1) * SPAN_FINE_V4, nv)};
}
// Calls f(t) for the 4-element vector index t (from the start of the level vector) of every
// vector of the block's range, the threads of a one-dimensional block striding over it.
template <typename F>
__device__ __forceinline__ void span_for(const Grid& g, const SpanRange& sr, F f)
{
    for (int k = sr.k0; k < sr.k1; ++k) {
        const int64_t p4 = g.off(0, 0, k) / 4;
        for (int v = sr.v0 + (int)threadIdx.x; v < sr.v1; v += (int)blockDim.x) f(p4 + v);
    }
}

// ---- reductions --------------------------------------------------------------------------------
template <int NP>
__device__ __forceinline__ void bblock_sum(double (&v)[NP], double* sh)
{
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = (nthr + 31) >> 5;
#pragma unroll
    for (int c = 0; c < NP; ++c)
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    if (lane == 0)
        for (int c = 0; c < NP; ++c) sh[c * 32 + warp] = v[c];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < NP; ++c) {
            v[c] = (lane < nw) ? sh[c * 32 + lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
        }
    }
    __syncthreads();
}

// Max of m over a one-dimensional block into *dst (bit patterns of nonnegative doubles order
// like the values). Every thread of the block must call it.
__device__ __forceinline__ void block_max_to(unsigned long long m, unsigned long long* dst)
{
    __shared__ unsigned long long sh[32];
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, sh[w]);
        atomicMax(dst, m);
    }
}

// Sum v over the nb blocks of one item (fixed order: deterministic). True in thread 0 of the
// item's last block to arrive, which then holds the totals.
template <int NP>
__device__ bool item_sum(double (&v)[NP], double* partials, unsigned int* arrive, int lb, int nb)
{
    __shared__ double sh[NP * 32];
    __shared__ unsigned int ticket;
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    bblock_sum<NP>(v, sh);
    if (tid == 0) {
        for (int c = 0; c < NP; ++c) partials[lb * NP + c] = v[c];
        __threadfence();
        ticket = atomicAdd(arrive, 1u);
    }
    __syncthreads();
    if (ticket != (unsigned int)(nb - 1)) return false;
    __threadfence();
    for (int c = 0; c < NP; ++c) v[c] = 0.0;
    for (int b = tid; b < nb; b += nthr)
        for (int c = 0; c < NP; ++c) v[c] += __ldcg(&partials[b * NP + c]);
    bblock_sum<NP>(v, sh);
    if (tid == 0) *arrive = 0u;
    return tid == 0;
}

// The same over compensated FP32 pairs of 256-thread blocks, merged in FP32 (block_merge) and
// widened to FP64 once per total (out); partials hold a float2 per double slot.
template <int NP>
__device__ bool item_merge(CSum (&v)[NP], double* partials, unsigned int* arrive, int lb, int nb, double (&out)[NP])
{
    __shared__ float2 sh[NP * 8], tot[NP];
    __shared__ unsigned int ticket;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    float2* pp = reinterpret_cast<float2*>(partials);
    block_merge<NP>(v, sh, tot);
    if (tid == 0) {
        for (int c = 0; c < NP; ++c) pp[lb * NP + c] = tot[c];
        __threadfence();
        ticket = atomicAdd(arrive, 1u);
    }
    __syncthreads();
    if (ticket != (unsigned int)(nb - 1)) return false;
    __threadfence();
    for (int c = 0; c < NP; ++c) v[c] = CSum{0.f, 0.f};
    for (int b = tid; b < nb; b += FLAT_TPB)
#pragma unroll
        for (int c = 0; c < NP; ++c) {
            const float2 p = __ldcg(&pp[b * NP + c]);
            twosum_merge(v[c].s, v[c].c, p.x, p.y);
        }
    block_merge<NP>(v, sh, tot);
    if (tid != 0) return false;
    *arrive = 0u;
    for (int c = 0; c < NP; ++c) out[c] = (double)tot[c].x + (double)tot[c].y;
    return true;
}

// Launch-wide arrival, one per item: the item's last block after its epilogue, or block 0 of an
// item that had nothing to do. True in the thread that brings the count to the number of items
// of the launch -- every item epilogue of the launch is then written.
__device__ bool item_arrives(BCtl* ctl, int nitems)
{
    __threadfence();
    if (atomicAdd(&ctl->arrive, 1u) != (unsigned int)(nitems - 1)) return false;
    __threadfence();
    ctl->arrive = 0u;
    return true;
}

// Loop condition: some item of the launch still runs; replacement condition: some running item
// asked for an FP64 residual replacement.
__device__ void batch_conditions(const BItem* items, const BLaunch& L, CondHandles ch)
{
    unsigned int run = 0u, upd = 0u;
    for (int s = 0; s < L.n; ++s) {
        const SolveState* st = items[L.id[s]].st;
        if (!__ldcg(&st->done)) {
            run = 1u;
            if (__ldcg(&st->need_update)) upd = 1u;
        }
    }
    if (ch.use) {
        cudaGraphSetConditional(ch.loop, run);
        if (ch.use > 1) cudaGraphSetConditional(ch.update, upd);
    }
}

// Block-uniform run flag from thread 0.
__device__ __forceinline__ bool block_flag(bool v)
{
    __shared__ int f;
    if (threadIdx.x + threadIdx.y * blockDim.x == 0) f = v ? 1 : 0;
    __syncthreads();
    return f != 0;
}

// ---- set-up ---------------------------------------------------------------------------------------
// Element (i, j, k) of the item's grid for a BG_ELEMS block; false when outside.
__device__ __forceinline__ bool elem_of(const Grid& g, int lb, int& i, int& j, int& k)
{
    const int gx = (g.nx + mt::BX - 1) / mt::BX, gy = (g.ny + mt::BY - 1) / mt::BY;
    i = (lb % gx) * mt::BX + threadIdx.x;
    j = ((lb / gx) % gy) * mt::BY + threadIdx.y;
    k = lb / (gx * gy);
    return i < g.nx && j < g.ny;
}
// Node (i, j, k) for a BG_NODES block.
__device__ __forceinline__ bool node_of(const Grid& g, int lb, int& i, int& j, int& k)
{
    const int gx = (g.nx + mt::BX) / mt::BX, gy = (g.ny + mt::BY) / mt::BY;
    i = (lb % gx) * mt::BX + threadIdx.x;
    j = ((lb / gx) % gy) * mt::BY + threadIdx.y;
    k = lb / (gx * gy);
    return i <= g.nx && j <= g.ny;
}

// beta of the level: packed from the caller's finest array or averaged from the finer level,
// and its FP32 copy.
__global__ void __launch_bounds__(256) bk_setup_beta(const BItem* __restrict__ items, const __grid_constant__ BLaunch L)
{
    COUNT_LAUNCH();
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    int i, j, k;
    if (!elem_of(it.g, sl.lb, i, j, k)) return;
    const int64_t o = it.g.off(i, j, k);
    double v;
    if (it.depth > 0) v = coarse_beta_at(it.fbeta, it.gf, i, j, k);
    else if (it.pre_beta) v = it.beta[o];  // one beta, filled before
    else v = it.in_beta[i + (int64_t)it.g.nx * (j + (int64_t)it.g.ny * k)];
    it.beta[o] = v;
    it.beta32[o] = (float)v;
}

// f, g_D, g_R of the level (packed from the caller's arrays, or injected from the finer level)
// and the FP32 Jacobi diagonal.
__global__ void __launch_bounds__(256) bk_setup_nodes(const BItem* __restrict__ items, const __grid_constant__ BLaunch L)
{
    COUNT_LAUNCH();
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    int i, j, k;
    if (!node_of(it.g, sl.lb, i, j, k)) return;
    const Grid& g = it.g;
    const int64_t o = g.off(i, j, k);
    if (it.depth == 0) {
        const int64_t t = i + (int64_t)(g.nx + 1) * (j + (int64_t)(g.ny + 1) * k);
        // Gauss-point f is read by the load kernel; a prefilled load needs no f
        if (it.fmode != ECMG_F_GAUSS && !it.pre_load) it.f[o] = it.in_f[t];
        if (!it.pre_gD) it.gD[o] = it.in_gD ? it.in_gD[t] : 0.0;
        it.gR[o] = it.in_gR ? it.in_gR[t] : 0.0;
    } else {
        const int64_t of = it.gf.off(2 * i, 2 * j, 2 * k);
        if (it.fmode == ECMG_F_NODAL) it.f[o] = it.ff[of];
        it.gD[o] = it.fgD[of];
        it.gR[o] = it.fgR[of];
    }
    it.dinv32[o] = jacobi32_at(g, it.op, it.beta32, i, j, k, it.precond);
}

// The load vector: consistent mass of the nodal data (NODAL), or the caller's finest load
// functional and its restrictions P^T b (LOAD).
__global__ void __launch_bounds__(256) bk_setup_load(const BItem* __restrict__ items, const __grid_constant__ BLaunch L)
{
    COUNT_LAUNCH();
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    int i, j, k;
    if (!node_of(it.g, sl.lb, i, j, k)) return;
    const int64_t o = it.g.off(i, j, k);
    if (it.fmode == ECMG_F_NODAL) it.b[o] = nodal_load_at(it.g, it.op, it.f, it.gR, i, j, k);
    else if (it.depth > 0) it.b[o] = restrict_at(it.fb, it.gf, i, j, k);
    else if (it.pre_load) return;  // assembled before from separable f
    else if (it.fmode == ECMG_F_GAUSS) it.b[o] = gauss_load_at(it.g, it.op, it.in_f, it.in_gR ? it.gR : nullptr, i, j, k);
    else it.b[o] = it.f[o];
}

// ---- start of a level -------------------------------------------------------------------------
__global__ void bk_state_init(const BItem* __restrict__ items, const __grid_constant__ BLaunch L, double inner)
{
    COUNT_LAUNCH();
    if (threadIdx.x != 0) return;
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    SolveState s = {};
    s.rtol2 = it.rtol * it.rtol;
    s.inner2 = inner * inner;
    s.max_iters = it.max_iters;
    s.fixed = it.fixed;
    *it.st = s;
}

// x = g_D on Dirichlet nodes, 0 elsewhere.
__global__ void __launch_bounds__(256) bk_dirichlet_ext(const BItem* __restrict__ items, const __grid_constant__ BLaunch L)
{
    COUNT_LAUNCH();
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    int i, j, k;
    if (!node_of(it.g, sl.lb, i, j, k)) return;
    const int64_t o = it.g.off(i, j, k);
    it.U[o] = on_dirichlet(it.g, it.op, i, j, k) ? it.gD[o] : 0.0;
}

// ||f_h||^2 per item and the stopping threshold.
template <bool ROBIN, bool CUBE>
__global__ void __launch_bounds__(256) bk_fh2(const BItem* __restrict__ items, const __grid_constant__ BLaunch L)
{
    COUNT_LAUNCH();
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    const Grid& g = it.g;
    const Weights<double> wts(it.op);
    const int nrows = (g.ny + 1) * (g.nz + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Op& op = it.op;
    // nodes i that need the FP64 stencil of the Dirichlet lift in a row away from the y and z
    // faces: the free nodes within one step of a Dirichlet x face (fh_at is b elsewhere)
    const int xlo = op.bc[0] == 0 ? 2 : 0, xhi = op.bc[1] == 0 ? g.nx - 2 : g.nx;
    constexpr int R = ROWS_PER_BLOCK / 8;  // rows of a warp
    double ss = 0.0;
    for (int r = 0; r < R; ++r) {
        const int row = sl.lb * ROWS_PER_BLOCK + warp * R + r;
        if (row >= nrows) break;
        const int j = row % (g.ny + 1), k = row / (g.ny + 1);
        const int64_t orow = g.plane_base(k) + g.in_plane(0, j);
        const bool near_yz = (op.bc[2] == 0 && j <= 1) || (op.bc[3] == 0 && j >= g.ny - 1) ||
                             (op.bc[4] == 0 && k <= 1) || (op.bc[5] == 0 && k >= g.nz - 1);
        if (near_yz) {  // every free node of the row needs the stencil: no lane idles
            for (int i = lane; i <= g.nx; i += 32) {
                if (on_dirichlet(g, op, i, j, k)) continue;
                const double f = fh_at<ROBIN, CUBE>(g, op, wts, it.beta, it.U, it.b, orow + i, i, j, k);
                ss = fma(f, f, ss);
            }
        } else {  // the inner run streams b; its x ends follow below, all rows of the warp at once
            for (int i = xlo + lane; i <= xhi; i += 32) {
                const double f = it.b[orow + i];
                ss = fma(f, f, ss);
            }
        }
    }
    // the free nodes next to a Dirichlet x face in the warp's rows away from the y and z faces:
    // up to two per face and row, one lane each (a single pass of the FP64 stencil per warp)
    if (xlo > 0 || xhi < g.nx) {
        const int per = (xlo > 0 ? 1 : 0) + (xhi < g.nx ? 1 : 0);  // x-shell nodes per row
        for (int u = lane; u < R * per; u += 32) {
            const int row = sl.lb * ROWS_PER_BLOCK + warp * R + u / per;
            if (row >= nrows) continue;
            const int j = row % (g.ny + 1), k = row / (g.ny + 1);
            const bool near_yz = (op.bc[2] == 0 && j <= 1) || (op.bc[3] == 0 && j >= g.ny - 1) ||
                                 (op.bc[4] == 0 && k <= 1) || (op.bc[5] == 0 && k >= g.nz - 1);
            if (near_yz) continue;
            if (per == 2 && u % per == 1 && g.nx - 1 <= 1) continue;  // the node i = 1 counted once
            const int i = (xlo > 0 && u % per == 0) ? 1 : g.nx - 1;
            if (i < 0 || i > g.nx || on_dirichlet(g, op, i, j, k)) continue;
            const double f = fh_at<ROBIN, CUBE>(g, op, wts, it.beta, it.U, it.b,
                                                g.plane_base(k) + g.in_plane(i, j), i, j, k);
            ss = fma(f, f, ss);
        }
    }
    double v[1] = {ss};
    if (item_sum<1>(v, it.part, &it.st->arrive, sl.lb, sl.nb)) {
        it.st->fh2 = v[0];
        it.st->thresh2 = it.st->rtol2 * v[0];
    }
}

// ---- initial guesses ----------------------------------------------------------------------------
template <int VARIANT>
__global__ void __launch_bounds__(EXP_TPB) bk_exp_finite(const BItem* __restrict__ items, const __grid_constant__ BLaunch L)
{
    COUNT_LAUNCH();
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    const Grid& g0 = it.g0;
    const int t = sl.lb * EXP_TPB + threadIdx.x;
    if (t >= g0.nx * g0.ny * g0.nz) return;
    const int ex = t % g0.nx, ey = (t / g0.nx) % g0.ny, ez = t / (g0.nx * g0.ny);
    exp_finite_element<VARIANT>(it.g, it.op, it.g1, it.U1, g0, it.U0, it.U, it.W, ex, ey, ez);
}

// Zero the FP32 search directions and correction of every item; W = x on the direct levels.
__global__ void __launch_bounds__(FLAT_TPB) bk_flat_init(const BItem* __restrict__ items, const __grid_constant__ BLaunch L)
{
    COUNT_LAUNCH();
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    const int64_t base = (int64_t)sl.lb * BFLAT_ELEMS;
    const int64_t end = min(base + BFLAT_ELEMS, it.g.total);
    for (int64_t t = base + threadIdx.x; t < end; t += FLAT_TPB) {
        it.pA32[t] = 0.f;
        it.pB32[t] = 0.f;
        it.e32[t] = 0.f;
        if (it.q32B) {
            it.q32[t] = 0.f;
            it.q32B[t] = 0.f;
            it.r32B[t] = 0.f;
        }
        if (it.level < 2) it.W[t] = it.U[t];
    }
}

// ---- JCG ----------------------------------------------------------------------------------------
// Tile (bx, by, bz) of a BG_STENCIL block over the item's nodes off the Dirichlet faces (the
// JCG kernels leave r, p and q at 0 on Dirichlet nodes).
__device__ __forceinline__ void tile_of(const BItem& it, const NodeRange& rg, int lb, int& bx, int& by, int& bz)
{
    const int gx = range_tiles_x(rg), gy = range_tiles_y(rg);
    bx = lb % gx;
    by = (lb / gx) % gy;
    bz = lb / (gx * gy);
}

// r = b - A x (FP64), stored FP32; ||r||^2 and the compensated FP32 r.z.
template <bool ROBIN, bool CUBE>
__global__ void __launch_bounds__(mt::NT) bk_res(const BItem* __restrict__ items, const __grid_constant__ BLaunch L,
                                                int mode, BCtl* ctl, CondHandles ch, int r_to_b)
{
    COUNT_LAUNCH();
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    SolveState* st = it.st;
    const bool run = block_flag(!st->done && (mode != RES_REPLACE || st->need_update));
    if (run) {
        const NodeRange rg = free_nodes(it.g, it.op);
        int bx, by, bz;
        tile_of(it, rg, sl.lb, bx, by, bz);
        double rr = 0.0;
        Acc<float> rz;
        const double* x = it.U;
        float* __restrict__ r32 = r_to_b ? it.r32B : it.r32;
        auto body = [&](int, int, int, int64_t o, double Av) {
            const double rv = it.b[o] - Av;
            const float ro = (float)rv;
            r32[o] = ro;
            rr = fma(rv, rv, rr);
            rz.add_prod(ro, it.dinv32[o] * ro);
        };
        if constexpr (CUBE) {
            // exact integer element sums (march_fx.cuh) on the scale of max |x| (bk_absmax or
            // bk_fold just before)
            const fx::FixedFrame fr = fx::fixed_frame(st->xbits);
            if (fr.finite) march_range_fxv<ROBIN>(it.g, it.beta, x, rg, bx, by, bz, it.kz, fr, it.op, body);
            else if (sl.lb == 0 && threadIdx.x == 0 && threadIdx.y == 0) rr = nan("");  // the iterate is not finite
        } else {
            auto src = [&](int64_t o) -> double { return x[o]; };
            auto body6 = [&](int i, int j, int k, int64_t o, double Av, double) { body(i, j, k, o, Av); };
            march_range<ROBIN, CUBE, double, double>(it.g, it.op, it.beta, rg, bx, by, bz, it.kz, src, body6);
        }
        double v[2] = {rr, rz.value()};
        if (item_sum<2>(v, it.part, &st->arrive, sl.lb, sl.nb)) {
            st->xbits = 0ull;  // every block has read the scale; the next fold or bk_absmax takes it anew
            res_epilogue(st, v[0], v[1], mode, CondHandles{0, 0, 0});
            if (item_arrives(ctl, L.n)) batch_conditions(items, L, CondHandles{ch.loop, 0, ch.use ? 1 : 0});
        }
    } else if (sl.lb == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        if (item_arrives(ctl, L.n)) batch_conditions(items, L, CondHandles{ch.loop, 0, ch.use ? 1 : 0});
    }
}

// K2: r -= alpha q; z = D^-1 r; r.z and r.r (compensated FP32); the item's tests.
__global__ void __launch_bounds__(FLAT_TPB) bk_update(const BItem* __restrict__ items, const __grid_constant__ BLaunch L,
                                                     BCtl* ctl, CondHandles ch)
{
    COUNT_LAUNCH();
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    SolveState* st = it.st;
    if (block_flag(!st->done)) {
        const float a = (float)st->alpha;
        Acc<float> rz, rr;
        const SpanRange sr = span_of(it.g, sl.lb);
        float4* __restrict__ r4 = reinterpret_cast<float4*>(it.r32);
        const float4* __restrict__ q4 = reinterpret_cast<const float4*>(it.q32);
        const float4* __restrict__ d4 = reinterpret_cast<const float4*>(it.dinv32);
        span_for(it.g, sr, [&](int64_t t) {
            float4 rv = r4[t];
            const float4 qv = q4[t], dv = d4[t];
            rv.x -= a * qv.x;
            rv.y -= a * qv.y;
            rv.z -= a * qv.z;
            rv.w -= a * qv.w;
            rz.add_prod(rv.x, dv.x * rv.x);
            rz.add_prod(rv.y, dv.y * rv.y);
            rz.add_prod(rv.z, dv.z * rv.z);
            rz.add_prod(rv.w, dv.w * rv.w);
            rr.add_prod(rv.x, rv.x);
            rr.add_prod(rv.y, rv.y);
            rr.add_prod(rv.z, rv.z);
            rr.add_prod(rv.w, rv.w);
            r4[t] = rv;
        });
        CSum pr[2] = {rz.v, rr.v};
        double v[2];
        if (item_merge<2>(pr, it.part, &st->arrive, sl.lb, sl.nb, v)) {
            update_epilogue<true>(st, v[0], v[1]);
            if (item_arrives(ctl, L.n)) batch_conditions(items, L, CondHandles{ch.loop, ch.update, ch.use ? 2 : 0});
        }
    } else if (sl.lb == 0 && threadIdx.x == 0) {
        if (item_arrives(ctl, L.n)) batch_conditions(items, L, CondHandles{ch.loop, ch.update, ch.use ? 2 : 0});
    }
}

// x64 += e + alpha_prev p_new; e = 0 (items that asked for a replacement).
__global__ void __launch_bounds__(FLAT_TPB) bk_fold(const BItem* __restrict__ items, const __grid_constant__ BLaunch L,
                                                   int pnew_is_b)
{
    COUNT_LAUNCH();
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    const SolveState* st = it.st;
    if (st->done || !st->need_update) return;
    const float a = (float)st->alpha_prev;
    const float* __restrict__ p = pnew_is_b ? it.pB32 : it.pA32;
    const SpanRange sr = span_fine_of(it.g, sl.lb);
    unsigned long long m = 0ull;
    span_for(it.g, sr, [&](int64_t t4) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t t = 4 * t4 + c;
            // the FP32 correction combined in FP32, added with one FP64 operation (jcg.cu k_fold32)
            const double xn = it.U[t] + fx::widen(fmaf(a, p[t], it.e32[t]));
            it.U[t] = xn;
            it.e32[t] = 0.f;
            m = max(m, fx::abs_bits(xn));
        }
    });
    block_max_to(m, &it.st->xbits);  // the scale of the exact residual that follows
}

// max |x| of each item's iterate into its state (the scale of the initial exact residual).
__global__ void __launch_bounds__(FLAT_TPB) bk_absmax(const BItem* __restrict__ items, const __grid_constant__ BLaunch L)
{
    COUNT_LAUNCH();
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    if (it.st->done) return;
    const SpanRange sr = span_fine_of(it.g, sl.lb);
    unsigned long long m = 0ull;
    span_for(it.g, sr, [&](int64_t t4) {
#pragma unroll
        for (int c = 0; c < 4; ++c) m = max(m, fx::abs_bits(it.U[4 * t4 + c]));
    });
    block_max_to(m, &it.st->xbits);
}

// EXP_true for levels >= 2.
__global__ void __launch_bounds__(EXP_TPB) bk_exp_true(const BItem* __restrict__ items, const __grid_constant__ BLaunch L)
{
    COUNT_LAUNCH();
    const Slot sl = find_slot(L);
    const BItem& it = items[sl.item];
    const Grid& gc = it.g1;
    const int t = sl.lb * EXP_TPB + threadIdx.x;
    if (t >= gc.nx * gc.ny * gc.nz) return;
    const int ex = t % gc.nx, ey = (t / gc.nx) % gc.ny, ez = t / (gc.nx * gc.ny);
    exp_true_element(it.g, it.U, gc, it.U1, it.Ut, ex, ey, ez);
}

inline int nblocks(const BLaunch& L) { return L.start[L.n]; }

}  // namespace

int bgeom_blocks(BGeom geo, const BItem& it)
{
    const Grid& g = it.g;
    switch (geo) {
    case BG_STENCIL: {
        const NodeRange rg = free_nodes(g, it.op);
        return range_tiles_x(rg) * range_tiles_y(rg) * range_tiles_z(rg, it.kz);
    }
    case BG_FLAT: return cdiv(g.total, BFLAT_ELEMS);
    case BG_SPAN:
        return span_chunks_per_plane(g) == 1 ? cdiv(g.nz + 1, span_planes_per_block(g))
                                             : (g.nz + 1) * span_chunks_per_plane(g);
    case BG_SPAN_FINE: return (g.nz + 1) * cdiv(span_v4(g), SPAN_FINE_V4);
    case BG_NODES: return cdiv(g.nx + 1, mt::BX) * cdiv(g.ny + 1, mt::BY) * (g.nz + 1);
    case BG_ELEMS: return cdiv(g.nx, mt::BX) * cdiv(g.ny, mt::BY) * g.nz;
    case BG_EXPF: return cdiv((int64_t)it.g0.nx * it.g0.ny * it.g0.nz, EXP_TPB);
    case BG_EXPT: return cdiv((int64_t)it.g1.nx * it.g1.ny * it.g1.nz, EXP_TPB);
    case BG_ROWS: return cdiv((int64_t)(g.ny + 1) * (g.nz + 1), ROWS_PER_BLOCK);
    default: return 1;
    }
}

int bitem_partials(const BItem& it)
{
    int m = bk1_max_blocks(it);
    for (BGeom geo : {BG_STENCIL, BG_FLAT, BG_SPAN, BG_SPAN_FINE, BG_ROWS}) m = std::max(m, bgeom_blocks(geo, it));
    return m;
}

void blaunch_setup(const BItem* items, const BLaunch& nodes, const BLaunch& elems, cudaStream_t s)
{
    if (nblocks(elems) == 0) return;
    bk_setup_beta<<<nblocks(elems), dim3(mt::BX, mt::BY), 0, s>>>(items, elems);
    bk_setup_nodes<<<nblocks(nodes), dim3(mt::BX, mt::BY), 0, s>>>(items, nodes);
    bk_setup_load<<<nblocks(nodes), dim3(mt::BX, mt::BY), 0, s>>>(items, nodes);
}

void blaunch_level_start(const BItem* items, const BLaunch& one, const BLaunch& nodes, const BLaunch& rows,
                         int robin, int cube, double inner_rtol, cudaStream_t s)
{
    if (one.n == 0) return;
    bk_state_init<<<nblocks(one), 32, 0, s>>>(items, one, inner_rtol);
    bk_dirichlet_ext<<<nblocks(nodes), dim3(mt::BX, mt::BY), 0, s>>>(items, nodes);
    auto k = robin ? (cube ? bk_fh2<true, true> : bk_fh2<true, false>)
                   : (cube ? bk_fh2<false, true> : bk_fh2<false, false>);
    k<<<nblocks(rows), 256, 0, s>>>(items, rows);
}

void blaunch_guess(const BItem* items, const BLaunch& expf, const BLaunch& flat_all, int variant, cudaStream_t s)
{
    if (expf.n > 0) {
        if (variant == ECMG_EXP_LAGRANGE27) bk_exp_finite<1><<<nblocks(expf), EXP_TPB, 0, s>>>(items, expf);
        else bk_exp_finite<0><<<nblocks(expf), EXP_TPB, 0, s>>>(items, expf);
    }
    if (flat_all.n > 0) bk_flat_init<<<nblocks(flat_all), FLAT_TPB, 0, s>>>(items, flat_all);
}

void blaunch_res(const BItem* items, const BLaunch& stencil, int robin, int cube, ResMode mode, BCtl* ctl,
                 CondHandles ch, cudaStream_t s, int r_to_b)
{
    auto k = robin ? (cube ? bk_res<true, true> : bk_res<true, false>)
                   : (cube ? bk_res<false, true> : bk_res<false, false>);
    k<<<nblocks(stencil), dim3(mt::BX, mt::BY), 0, s>>>(items, stencil, (int)mode, ctl, ch, r_to_b);
}

void blaunch_update(const BItem* items, const BLaunch& flat, BCtl* ctl, CondHandles ch, cudaStream_t s)
{
    bk_update<<<nblocks(flat), FLAT_TPB, 0, s>>>(items, flat, ctl, ch);
}

void blaunch_absmax(const BItem* items, const BLaunch& flat, cudaStream_t s)
{
    bk_absmax<<<nblocks(flat), FLAT_TPB, 0, s>>>(items, flat);
}

void blaunch_fold(const BItem* items, const BLaunch& flat, int pnew_is_b, cudaStream_t s)
{
    bk_fold<<<nblocks(flat), FLAT_TPB, 0, s>>>(items, flat, pnew_is_b);
}

void blaunch_exp_true(const BItem* items, const BLaunch& expt, cudaStream_t s)
{
    if (expt.n > 0) bk_exp_true<<<nblocks(expt), EXP_TPB, 0, s>>>(items, expt);
}

unsigned long long launches_batch()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_launches, sizeof(v));
    return v;
}

}  // namespace ecmg
