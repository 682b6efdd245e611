// batch_tma.cu -- the TMA-staged FP32 JCG step kernels (body in k1_body.cuh) over all
// (problem, level) items of a batched stage in one launch: K1 of the two-pass step, and the
// single-pass step, which also applies the previous step's residual update and sets the loop's
// conditions.
//
// Every item carries its own tensor maps (in global memory, encoded on the host at creation)
// and its own planes per block (k1kz); the launch picks one row count per thread (RY) for all of
// its items. A block finds its item from the launch's block offsets, decodes its tile in that
// item's tile grid and runs the same body as the single-problem kernel: the staged z-march
// forming p = D^-1 r + beta p_old, q = A p, the deferred correction e += alpha_prev p_old and the
// item's p.q, whose last block sets the item's step alpha. Items that have finished return at
// once (their blocks still occupy the launch, for a few cycles).
#include <cuda.h>

#include "batch.cuh"
#include "k1_body.cuh"

namespace ecmg {
namespace {

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

struct BSlot {
    int item, lb, nb;  // item index, block index inside the item, the item's blocks
};
__device__ __forceinline__ BSlot bslot(const BLaunch& L)
{
    const int b = blockIdx.x;
    int lo = 0, hi = L.n;  // L.start[lo] <= b < L.start[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (L.start[mid] <= b) lo = mid;
        else hi = mid;
    }
    return BSlot{L.id[lo], b - L.start[lo], L.start[lo + 1] - L.start[lo]};
}

// Tiles of an item's K1 grid along x and y.
__host__ __device__ inline int k1_tiles_x(const Range& rg) { return (max(rg.ihi - rg.ilo + 1, 1) + TBX - 1) / TBX; }
__host__ __device__ inline int k1_tiles_y(const Range& rg, int ry)
{
    return (max(rg.jhi - rg.jlo + 1, 1) + TBY * ry - 1) / (TBY * ry);
}

template <bool ROBIN, bool CUBE, int RY>
__global__ void __launch_bounds__(NT, RY == 1 ? (ROBIN ? 3 : 4) : 2)
bk_pq_tma(const BItem* __restrict__ items, const PlaneMaps* __restrict__ maps, const __grid_constant__ BLaunch L,
          int pin_is_b, int pidx)
{
    COUNT_LAUNCH();
    const BSlot sl = bslot(L);
    const BItem& it = items[sl.item];
    SolveState* st = it.st;
    const K1Scalars sc{st->done, (float)st->beta, (float)st->alpha_prev, 0.f, 0.f};
    const Grid g = it.g;
    const Op op = it.op;
    const Range rg = k1_range(g, op);
    const int gx = k1_tiles_x(rg), gy = k1_tiles_y(rg, RY);
    const K1Block kb{sl.lb % gx, (sl.lb / gx) % gy, sl.lb / (gx * gy), sl.lb, sl.nb};
    constexpr int v = RY == 1 ? 0 : 1;
    const PlaneMaps& m = maps[sl.item];
    k1_body<ROBIN, CUBE, RY, false, false>(m.r[v], pin_is_b ? m.pB[v] : m.pA[v], m.dinv[v], m.beta[v], m.r[v], m.e[v],
                                           g, op, rg, pin_is_b ? it.pA32 : it.pB32, it.q32, nullptr, it.e32, st,
                                           it.part, pidx, CondHandles{0, 0, 0}, it.k1kz, nullptr, sc, kb);
}

// Loop condition: some item of the launch still runs; replacement condition: some running item
// asked for an FP64 residual replacement (the same rule as the batched K2 in batch.cu).
__device__ void step_conditions(const BItem* items, const BLaunch& L, CondHandles ch)
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
        cudaGraphSetConditional(ch.update, upd);
    }
}

// The single-pass step (ECMG_CG_SINGLE_PASS form; body in k1_body.cuh) for every item of a
// stage: r = r_in - alpha_prev q_in while staging, e += alpha_prev p_old, p = D^-1 r + beta p_old,
// q = A p, r, p and q stored into the other buffer set, and the dots whose expansion gives the
// next r.z and r.r (sp_epilogue, per item). in_b: the buffer set (A = r32, q32, pA32; B = r32B,
// q32B, pB32) the step reads. Every block then arrives once at the launch-wide counter, after
// its own item's epilogue when it was that item's last block; the launch's last block sets the
// graph conditions from all items. A block counter (rather than one arrival per item) keeps the
// count right whatever path a block took.
// Two blocks per SM for either row count: at three (one row per thread) the register cap of 80
// spills.
template <bool ROBIN, bool CUBE, int RY>
__global__ void __launch_bounds__(NT, 2)
bk_step_tma(const BItem* __restrict__ items, const PlaneMaps* __restrict__ maps, const __grid_constant__ BLaunch L,
            int in_b, int pidx, BCtl* ctl, CondHandles ch)
{
    COUNT_LAUNCH();
    const BSlot sl = bslot(L);
    const BItem& it = items[sl.item];
    SolveState* st = it.st;
    const K1Scalars sc{st->done, (float)st->beta, (float)st->alpha_prev, 0.f, 0.f};
    const Grid g = it.g;
    const Op op = it.op;
    const Range rg = k1_range(g, op);
    const int gx = k1_tiles_x(rg), gy = k1_tiles_y(rg, RY);
    const K1Block kb{sl.lb % gx, (sl.lb / gx) % gy, sl.lb / (gx * gy), sl.lb, sl.nb};
    constexpr int v = RY == 1 ? 0 : 1;
    const PlaneMaps& m = maps[sl.item];
    k1_body<ROBIN, CUBE, RY, false, true>(in_b ? m.rB[v] : m.r[v], in_b ? m.pB[v] : m.pA[v], m.dinv[v], m.beta[v],
                                          in_b ? m.qB[v] : m.qA[v], m.e[v], g, op, rg, in_b ? it.pA32 : it.pB32,
                                          in_b ? it.q32 : it.q32B, in_b ? it.r32 : it.r32B, it.e32, st, it.part,
                                          pidx, CondHandles{0, 0, 0}, it.k1kz, nullptr, sc, kb);
    if ((threadIdx.x | threadIdx.y) == 0) {
        __threadfence();
        if (atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1) {
            __threadfence();
            ctl->arrive = 0u;
            step_conditions(items, L, ch);
        }
    }
}

template <int RY>
using BKernel = void (*)(const BItem*, const PlaneMaps*, const BLaunch, int, int);
template <int RY>
using BStepKernel = void (*)(const BItem*, const PlaneMaps*, const BLaunch, int, int, BCtl*, CondHandles);

template <int RY>
BStepKernel<RY> pick_step(int robin, int cube)
{
    return robin ? (cube ? bk_step_tma<true, true, RY> : bk_step_tma<true, false, RY>)
                 : (cube ? bk_step_tma<false, true, RY> : bk_step_tma<false, false, RY>);
}

template <int RY>
BKernel<RY> pick(int robin, int cube)
{
    return robin ? (cube ? bk_pq_tma<true, true, RY> : bk_pq_tma<true, false, RY>)
                 : (cube ? bk_pq_tma<false, true, RY> : bk_pq_tma<false, false, RY>);
}

template <int RY>
cudaError_t prepare_ry()
{
    cudaError_t e = cudaSuccess;
    for (int robin = 0; robin < 2 && e == cudaSuccess; ++robin)
        for (int cube = 0; cube < 2 && e == cudaSuccess; ++cube)
            e = cudaFuncSetAttribute(pick<RY>(robin, cube), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)stage_smem<RY, false, false>());
    for (int robin = 0; robin < 2 && e == cudaSuccess; ++robin)
        for (int cube = 0; cube < 2 && e == cudaSuccess; ++cube)
            e = cudaFuncSetAttribute(pick_step<RY>(robin, cube), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)stage_smem<RY, false, true>());
    return e;
}

}  // namespace

int bk1_blocks(const BItem& it, int ry)
{
    const Range rg = k1_range(it.g, it.op);
    const int nk = max(rg.khi - rg.klo + 1, 1);
    return k1_tiles_x(rg) * k1_tiles_y(rg, ry) * ((nk + it.k1kz - 1) / it.k1kz);
}

int bk1_max_blocks(const BItem& it) { return max_tma_blocks(it.g); }

int64_t bk1_nodes(const BItem& it) { return k1_nodes(it.g, it.op); }

cudaError_t bk1_prepare()
{
    cudaError_t e = prepare_ry<1>();
    if (e == cudaSuccess) e = prepare_ry<2>();
    return e;
}

void blaunch_pq_tma(const BItem* items, const PlaneMaps* maps, const BLaunch& L, int ry, int robin, int cube,
                    int pin_is_b, int pidx, cudaStream_t s)
{
    const int nb = L.start[L.n];
    if (nb == 0) return;
    if (ry == 1)
        pick<1>(robin, cube)<<<nb, dim3(TBX, TBY), stage_smem<1, false, false>(), s>>>(items, maps, L, pin_is_b, pidx);
    else
        pick<2>(robin, cube)<<<nb, dim3(TBX, TBY), stage_smem<2, false, false>(), s>>>(items, maps, L, pin_is_b, pidx);
}

void blaunch_step_tma(const BItem* items, const PlaneMaps* maps, const BLaunch& L, int ry, int robin, int cube,
                      int in_b, int pidx, BCtl* ctl, CondHandles ch, cudaStream_t s)
{
    const int nb = L.start[L.n];
    if (nb == 0) return;
    if (ry == 1)
        pick_step<1>(robin, cube)<<<nb, dim3(TBX, TBY), stage_smem<1, false, true>(), s>>>(items, maps, L, in_b, pidx,
                                                                                          ctl, ch);
    else
        pick_step<2>(robin, cube)<<<nb, dim3(TBX, TBY), stage_smem<2, false, true>(), s>>>(items, maps, L, in_b, pidx,
                                                                                          ctl, ch);
}

unsigned long long launches_batch_tma()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_launches, sizeof(v));
    return v;
}

}  // namespace ecmg
